"""Pins of the spectrum-slicing oracle (Jackson-damped Chebyshev windows, per-slice RR).

Pinned to things other than the oracle itself:
  * the indicator coefficients against numerical quadrature of the Chebyshev projection
    mu_j = (2 - delta_j0) / pi * int_ta^tb T_j(t) / sqrt(1 - t^2) dt (scipy.integrate.quad),
    and the whole interval [-1, 1] giving the constant 1;
  * the Jackson-damped window stays inside [0, 1] everywhere (the Jackson kernel is a
    positive kernel) and approaches the indicator away from the slice edges;
  * the recurrence sum on exact eigenvectors of A: p(A~) x = p(t_lambda) x with p evaluated by
    the closed form T_j(t) = cos(j arccos t);
  * slice_solve against dense generalized diagonalisation: every eigenvalue inside a slice is
    a Ritz value of that slice's small Rayleigh-Ritz step.
"""
import math

import numpy as np
import pytest
import scipy.integrate
import scipy.linalg

from oracle import pw_oracle as O
from oracle import pw_slicing as SL
from paper_2604_11139_gb300 import workloads as W


def _problem(with_q=True):
    return W.make_problem("tiny_gamma_fp64", box=(12, 12, 12), ecut=2.0, nband=12, with_q=with_q)


def _bounds(H, S):
    lam = scipy.linalg.eigh(H, S, eigvals_only=True)
    return lam, lam[0] - 0.05, lam[-1] + 0.05


@pytest.mark.parametrize("ta,tb", [(-0.3, 0.45), (-0.95, -0.7), (0.1, 0.9)])
def test_indicator_coefficients_match_quadrature(ta, tb):
    mu = SL.indicator_coefficients(12, ta, tb)
    for j in range(13):
        q, _ = scipy.integrate.quad(lambda t: math.cos(j * math.acos(t)) / math.sqrt(1 - t * t), ta, tb,
                                    epsabs=1e-13, epsrel=1e-13, limit=200)
        assert abs(mu[j] - (1 if j == 0 else 2) / math.pi * q) < 1e-11, j


def test_whole_interval_is_the_constant_one():
    mu = SL.indicator_coefficients(20, -1.0, 1.0)
    assert abs(mu[0] - 1.0) < 1e-15 and np.abs(mu[1:]).max() < 1e-14
    g = SL.jackson_damping(20)
    assert g[0] == pytest.approx(1.0, abs=1e-15)
    assert np.all(np.diff(g) < 0) and g[-1] > 0


@pytest.mark.parametrize("degree", [40, 200])
def test_damped_window_is_bounded_and_approaches_the_indicator(degree):
    lo, hi = -2.0, 6.0
    a, b = -0.5, 1.0
    coef = SL.window_coefficients(degree, a, b, lo, hi)
    lam = np.linspace(lo, hi, 4001)
    t = (lam - 0.5 * (hi + lo)) / (0.5 * (hi - lo))
    p = SL.window_value(coef, t)
    assert p.min() > -1e-12 and p.max() < 1 + 1e-12
    if degree == 200:
        inside = (lam > a + 0.4) & (lam < b - 0.4)
        outside = (lam < a - 0.4) | (lam > b + 0.4)
        assert np.abs(p[inside] - 1).max() < 0.02
        assert p[outside].max() < 0.02


def test_recurrence_sum_on_exact_eigenvectors():
    prob = _problem(True)
    ham = O.Hamiltonian.from_problem(prob)
    H, S = ham.dense()
    lam, lo, hi = _bounds(H, S)
    _, X = scipy.linalg.eigh(H, S)
    V = X[:, [0, 5, 40, 100]].T
    coef = SL.window_coefficients(30, lam[2], lam[9], lo, hi)
    Y = SL.chebyshev_sum(ham.apply_a, V, coef, lo, hi)
    t = (lam[[0, 5, 40, 100]] - 0.5 * (hi + lo)) / (0.5 * (hi - lo))
    ref = SL.window_value(coef, t)[:, None] * V
    assert np.abs(Y - ref).max() < 1e-11 * np.abs(V).max()


def test_slice_solve_finds_the_eigenvalues_of_each_slice():
    prob = _problem(True)
    ham = O.Hamiltonian.from_problem(prob)
    H, S = ham.dense()
    lam, lo, hi = _bounds(H, S)
    # cuts in the middle of the wide gaps at the bottom of the spectrum (2 and 3 eigenvalues),
    # 5 vectors per slice, two passes of the window
    cuts = [lo, 0.5 * (lam[1] + lam[2]), 0.5 * (lam[4] + lam[5])]
    X = W.psi0(prob.seed, ham.npw, 10)
    eig, V, res = SL.slice_solve(ham, X, 2, 200, lo, hi, cuts, passes=2)
    for s, count in ((0, 2), (1, 3)):
        inside = lam[(lam > cuts[s]) & (lam < cuts[s + 1])]
        assert len(inside) == count
        for l in inside:
            i = np.argmin(np.abs(eig[s] - l))
            assert abs(eig[s][i] - l) < 1e-9 and res[s][i] < 1e-4, (s, l)
