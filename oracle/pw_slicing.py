"""Plain FP64 CPU oracle of spectrum slicing with Jackson-damped Chebyshev windows.

TEST INFRASTRUCTURE ONLY.  Only ``tests/`` may import this module; the CUDA library never
calls it and shares no code with it.

The paper's closing section proposes spectrum slicing (Schofield, Chelikowsky & Saad 2012;
Liou et al. 2020) for large band counts: the wanted part of the spectrum is cut into
slices, each slice gets its own block of vectors filtered by a high-degree polynomial that
passes only that slice, and each slice is then solved by a small, independent Rayleigh-Ritz
step instead of one global one.  The paper gives no formulas; the readings here are the
standard ones of that literature:

  * spectrum mapping: A = S^-1 H with spectrum inside [lo, hi]; t = (lambda - c) / e,
    c = (hi + lo) / 2, e = (hi - lo) / 2, so the spectrum maps into [-1, 1];
  * window of a slice [a, b] (mapped to [ta, tb]): the Chebyshev expansion of its indicator
    function, mu_0 = (arccos ta - arccos tb) / pi, mu_j = 2 (sin(j arccos ta) - sin(j arccos tb))
    / (j pi), damped by the Jackson factors of degree d (Di Napoli, Polizzi & Saad 2016),
    g_j = [(1 - j/(d+2)) sin(a_d) cos(j a_d) + cos(a_d) sin(j a_d) / (d+2)] / sin(a_d),
    a_d = pi / (d+2):  p(t) = sum_{j<=d} g_j mu_j T_j(t);
  * filtered block Y = p(A~) X, A~ = (A - c)/e, with T_j(A~) X from the three-term
    recurrence T_0 X = X, T_1 X = A~ X, T_{j+1} X = 2 A~ T_j X - T_{j-1} X;
  * per slice: two S-Ortho passes (Alg. 9) and the Rayleigh-Ritz step (Alg. 5) on its block;
    the window may be applied several times (subspace iteration per slice), each block made
    S-orthonormal in between.

Arrays hold bands as rows (shape (m, N)).  Pins: tests/test_oracle_slicing.py.
"""
from __future__ import annotations

import math

import numpy as np

from . import pw_oracle as O


def jackson_damping(degree: int) -> np.ndarray:
    """g_j, j = 0..degree."""
    j = np.arange(degree + 1, dtype=float)
    a = math.pi / (degree + 2)
    return ((1.0 - j / (degree + 2)) * math.sin(a) * np.cos(j * a) + math.cos(a) * np.sin(j * a) / (degree + 2)) \
        / math.sin(a)


def indicator_coefficients(degree: int, ta: float, tb: float) -> np.ndarray:
    """Chebyshev coefficients mu_j of the indicator of [ta, tb] inside [-1, 1]."""
    tha, thb = math.acos(ta), math.acos(tb)
    mu = np.empty(degree + 1)
    mu[0] = (tha - thb) / math.pi
    j = np.arange(1, degree + 1, dtype=float)
    mu[1:] = 2.0 * (np.sin(j * tha) - np.sin(j * thb)) / (j * math.pi)
    return mu


def window_coefficients(degree: int, a: float, b: float, lo: float, hi: float) -> np.ndarray:
    """g_j mu_j of the slice [a, b] for a spectrum inside [lo, hi] (the slice clipped to it)."""
    c, e = 0.5 * (hi + lo), 0.5 * (hi - lo)
    ta = min(max((a - c) / e, -1.0), 1.0)
    tb = min(max((b - c) / e, -1.0), 1.0)
    return jackson_damping(degree) * indicator_coefficients(degree, ta, tb)


def window_value(coef: np.ndarray, t: np.ndarray) -> np.ndarray:
    """p(t) = sum_j coef_j T_j(t) on [-1, 1] by T_j(t) = cos(j arccos t)."""
    th = np.arccos(np.clip(t, -1.0, 1.0))
    return np.cos(np.outer(th, np.arange(len(coef)))) @ coef


def chebyshev_sum(apply_a, X: np.ndarray, coef: np.ndarray, lo: float, hi: float) -> np.ndarray:
    """sum_j coef_j T_j(A~) X, A~ = (A - c)/e, through the three-term recurrence."""
    c, e = 0.5 * (hi + lo), 0.5 * (hi - lo)
    T0 = X
    acc = coef[0] * T0
    if len(coef) == 1:
        return acc
    T1 = (apply_a(X) - c * X) / e
    acc = acc + coef[1] * T1
    for j in range(2, len(coef)):
        T0, T1 = T1, 2.0 * (apply_a(T1) - c * T1) / e - T0
        acc = acc + coef[j] * T1
    return acc


def slice_filter(ham: "O.Hamiltonian", X: np.ndarray, nslice: int, degree: int, lo: float, hi: float, cuts):
    """Each block of X (nslice blocks of equal size) through the window of its slice."""
    nper = X.shape[0] // nslice
    out = np.empty_like(X, dtype=complex)
    for s in range(nslice):
        coef = window_coefficients(degree, cuts[s], cuts[s + 1], lo, hi)
        out[s * nper:(s + 1) * nper] = chebyshev_sum(ham.apply_a, X[s * nper:(s + 1) * nper], coef, lo, hi)
    return out


def slice_solve(ham: "O.Hamiltonian", X: np.ndarray, nslice: int, degree: int, lo: float, hi: float, cuts,
                passes: int = 1):
    """slice_filter (``passes`` times, each block S-orthonormalised between passes), then per
    slice two S-Ortho passes and Rayleigh-Ritz.  Returns the Ritz values (nslice, nper), the
    Ritz vectors (band rows, slice by slice) and residual norms."""
    nper = X.shape[0] // nslice
    Y = X
    for p in range(passes):
        if p > 0:
            for s in range(nslice):
                B = Y[s * nper:(s + 1) * nper]
                Y[s * nper:(s + 1) * nper], _ = O.s_ortho(B, ham.apply_s(B))
        Y = slice_filter(ham, Y, nslice, degree, lo, hi, cuts)
    eig = np.empty((nslice, nper))
    res = np.empty((nslice, nper))
    V = np.empty_like(Y)
    for s in range(nslice):
        B = Y[s * nper:(s + 1) * nper]
        for _ in range(2):
            B, _ = O.s_ortho(B, ham.apply_s(B))
        lam, B, HB, SB, _ = O.rayleigh_ritz(B, ham.apply_h(B), ham.apply_s(B))
        eig[s] = lam
        res[s] = O.residual_norms(lam, HB, SB)
        V[s * nper:(s + 1) * nper] = B
    return eig, V, res
