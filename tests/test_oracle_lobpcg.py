"""Pins of the LOBPCG oracle (Alg. 11 with S-Deflate, S-Ortho and RR, Alg. 8-10).

Pinned to things other than the oracle itself:
  * the Teter-Payne-Allan preconditioner against values of its rational form worked by hand
    (K(0) = 1, K(1) = 65/81, K(2) = 175/431) and its large-x limit 1/(2x);
  * S-Deflate: the output is S-orthogonal to the deflating block and differs from the input
    by an element of that block's span (deflating twice changes nothing);
  * S-Ortho: the output is S-orthonormal and spans the input (X = X_new U, U upper triangular);
  * the whole solver against dense generalized diagonalisation (scipy.linalg.eigh(H, S)) of
    the oracle's dense H and S, one block and several blocks, with and without S;
  * the minimisation property: a block's Ritz values never increase from one line
    minimisation to the next (the RR subspace contains the previous block);
  * an exact invariant subspace as the start: zero residual, no line minimisation, exact
    eigenvalues.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import pw_oracle as O
from oracle import pw_lobpcg as L
from paper_2604_11139_gb300 import workloads as W


def _problem(with_q, nband=8, box=(12, 12, 12), ecut=2.0):
    return W.make_problem("tiny_gamma_fp64", box=box, ecut=ecut, nband=nband, with_q=with_q)


def _dense(prob):
    ham = O.Hamiltonian.from_problem(prob)
    H, S = ham.dense()
    lam, X = scipy.linalg.eigh(H, S)
    return ham, H, S, lam, X


def test_tpa_preconditioner_values():
    assert L.tpa_preconditioner(np.array([0.0]), 1.0)[0] == 1.0
    np.testing.assert_allclose(L.tpa_preconditioner(np.array([1.0, 2.0]), 1.0), [65 / 81, 175 / 431], rtol=1e-15)
    # x = t / E_kin: scaling both leaves K unchanged
    np.testing.assert_allclose(L.tpa_preconditioner(np.array([6.0]), 3.0), [175 / 431], rtol=1e-15)
    x = np.array([1e3, 1e4])
    np.testing.assert_allclose(L.tpa_preconditioner(x, 1.0) * 2 * x, 1.0, rtol=2e-3)
    k = L.tpa_preconditioner(np.linspace(0, 50, 200), 1.0)
    assert np.all(np.diff(k) < 0) and np.all(k > 0)


def test_band_kinetic_of_single_plane_waves():
    kin = np.array([0.0, 0.5, 2.0, 3.0])
    X = np.eye(4, dtype=complex)[[1, 3]] * (2 - 1j)
    np.testing.assert_allclose(L.band_kinetic(X, kin), [0.5, 3.0], rtol=1e-15)


@pytest.mark.parametrize("with_q", [False, True])
def test_s_deflate_is_the_s_orthogonal_projection(with_q):
    prob = _problem(with_q)
    ham = O.Hamiltonian.from_problem(prob)
    Y0 = W.random_block(11, ham.npw, 3)
    Y0, _, SY0 = L.s_ortho3(Y0, Y0, ham.apply_s(Y0))
    X = W.random_block(12, ham.npw, 4)
    Xd = L.s_deflate(X, Y0, SY0)
    assert np.abs(SY0.conj() @ Xd.T).max() < 1e-13
    # X - Xd lies in span(Y0): least squares against Y0 leaves no remainder
    D = (X - Xd).T
    coef, *_ = np.linalg.lstsq(Y0.T, D, rcond=None)
    assert np.abs(Y0.T @ coef - D).max() < 1e-12
    np.testing.assert_allclose(L.s_deflate(Xd, Y0, SY0), Xd, atol=1e-13)


@pytest.mark.parametrize("with_q", [False, True])
def test_s_ortho_is_s_orthonormal_with_the_same_span(with_q):
    prob = _problem(with_q)
    ham = O.Hamiltonian.from_problem(prob)
    X = W.random_block(13, ham.npw, 6)
    HX, SX = ham.apply_h(X), ham.apply_s(X)
    Xn, HXn, SXn = L.s_ortho3(X, HX, SX)
    np.testing.assert_allclose(Xn.conj() @ ham.apply_s(Xn).T, np.eye(6), atol=1e-12)
    np.testing.assert_allclose(HXn, ham.apply_h(Xn), atol=1e-11)
    np.testing.assert_allclose(SXn, ham.apply_s(Xn), atol=1e-12)
    # X = Xn U with U upper triangular (band rows: X = U^T Xn)
    U = Xn.conj() @ ham.apply_s(X).T
    assert np.abs(np.tril(U, -1)).max() < 1e-12
    np.testing.assert_allclose(U.T @ Xn, X, atol=1e-12)


# 4 bands end in a gap of the spectrum (about 0.11 Ha to the fifth state): convergence to
# rounding; 8 bands end next to a near-degenerate pair (1.4e-3 Ha apart), which converges slowly
@pytest.mark.parametrize("with_q,nband,nblocks,atol", [(False, 4, 1, 1e-12), (True, 4, 1, 1e-12),
                                                       (False, 4, 2, 1e-12), (True, 4, 2, 1e-12),
                                                       (False, 8, 4, 1e-9), (True, 8, 4, 1e-9)])
def test_lobpcg_converges_to_the_dense_eigenpairs(with_q, nband, nblocks, atol):
    prob = _problem(with_q, nband=nband)
    ham, H, S, lam_d, _ = _dense(prob)
    psi0 = W.psi0(prob.seed, ham.npw, prob.nband)
    lam, Y, res, its = L.lobpcg(ham, psi0, nblocks, 30, tol=1e-7)
    np.testing.assert_allclose(lam, lam_d[:prob.nband], atol=atol)
    assert res.max() < (1e-7 if nband == 4 else 1e-5)
    # the residuals returned are the definition's: ||H y - lambda S y||
    np.testing.assert_allclose(res, np.linalg.norm(ham.apply_h(Y) - lam[:, None] * ham.apply_s(Y), axis=1),
                               rtol=1e-6, atol=1e-12)
    np.testing.assert_allclose(Y.conj() @ ham.apply_s(Y).T, np.eye(prob.nband), atol=1e-10)


@pytest.mark.parametrize("with_q", [False, True])
def test_ritz_values_never_increase(with_q):
    prob = _problem(with_q)
    ham = O.Hamiltonian.from_problem(prob)
    psi0 = W.psi0(prob.seed, ham.npw, prob.nband)
    hist = []
    L.lobpcg(ham, psi0, 2, 6, tol=0.0, history=hist)
    for blk in (0, 1):
        seq = [h[2] for h in hist if h[0] == blk]
        assert len(seq) == 6
        for a, b in zip(seq, seq[1:]):
            assert np.all(b <= a + 1e-12)


def test_exact_invariant_subspace_needs_no_line_minimisation():
    prob = _problem(True)
    ham, H, S, lam_d, X = _dense(prob)
    psi0 = X[:, :prob.nband].T.copy()
    lam, Y, res, its = L.lobpcg(ham, psi0, 2, 5, tol=1e-9)
    assert its == [0, 0]
    np.testing.assert_allclose(lam, lam_d[:prob.nband], atol=1e-11)
    assert res.max() < 1e-9
