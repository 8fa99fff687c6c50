"""Pins of the FP64 oracle against what the physics and the mathematics fix.

No value here comes from the CUDA path.  Each test states what pins which part:
a dropped term, a wrong sign, index or transposed operand anywhere in the oracle
breaks at least one of them (tests/test_oracle_mutations.py plants such mistakes).
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg

from oracle import pw_oracle as O
from paper_2604_11139_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def load_r3():
    rows = [l.split() for l in open(os.path.join(GOLD, "r3_counts.txt")) if l.strip() and not l.startswith("#")]
    return {int(a): int(b) for a, b in rows}


def small_problem(with_q=False, box=(16, 16, 16), ecut=3.0, nband=8, kpt=None, seed=None):
    return W.make_problem("tiny_gamma_fp64", box=box, ecut=ecut, nband=nband, with_q=with_q,
                          kpt=kpt, seed=seed)


# --- a1: sphere and kinetic diagonal ---------------------------------------------------

def test_r3_fixture_matches_theta_cubed():
    """The golden r_3 table equals the coefficients of theta(q)^3 (independent route)."""
    r3 = load_r3()
    n = max(r3) + 1
    th = np.zeros(n, dtype=np.int64)
    for k in range(-10, 11):
        if k * k < n:
            th[k * k] += 1
    t3 = np.convolve(np.convolve(th, th)[:n], th)[:n]
    assert [r3[i] for i in range(n)] == list(t3)


@pytest.mark.parametrize("R2", [0, 1, 2, 5, 9, 14, 24, 33, 38])
def test_sphere_counts_free_electron(R2):
    """Cubic cell, Gamma: #G with |G|^2 <= (2 pi/a)^2 R2 equals sum r_3(n), n <= R2, and the
    sorted kinetic energies are the shells (2pi/a)^2 n / 2 with degeneracy r_3(n)."""
    r3 = load_r3()
    a = 10.0
    unit = 0.5 * (2 * math.pi / a) ** 2
    ecut = unit * (R2 + 0.5)
    m, kin = O.g_sphere(np.diag([a, a, a]), [0, 0, 0], ecut, (24, 24, 24))
    assert m.shape[0] == sum(r3[n] for n in range(R2 + 1))
    expect = np.concatenate([np.full(r3[n], unit * n) for n in range(R2 + 1)])
    np.testing.assert_allclose(np.sort(kin), expect, rtol=1e-14, atol=1e-14)


def test_sphere_shift_by_reciprocal_vector():
    """The sphere at k + b1 is the sphere at k shifted by (-1, 0, 0), same kinetic energies."""
    lat = np.diag([10.0, 11.0, 12.0])
    k = np.array([0.125, -0.25, 0.375])
    m1, t1 = O.g_sphere(lat, k, 3.0, (24, 24, 24))
    m2, t2 = O.g_sphere(lat, k + np.array([1.0, 0, 0]), 3.0, (24, 24, 24))
    assert m1.shape == m2.shape
    np.testing.assert_array_equal(m1, m2 + np.array([1, 0, 0]))
    np.testing.assert_allclose(t1, t2, rtol=1e-13)


def test_sphere_order_and_gamma_inversion():
    m, _ = O.g_sphere(np.diag([10.0] * 3), [0, 0, 0], 7.6, (24, 24, 24))
    key = [tuple(r) for r in m]
    assert key == sorted(key)
    s = set(key)
    assert all((-a, -b, -c) in s for a, b, c in key)


def test_sphere_rejects_box_too_small():
    with pytest.raises(ValueError):
        O.g_sphere(np.diag([10.0] * 3), [0, 0, 0], 7.6, (12, 12, 12))


# --- H-apply: free electron, constant potential, Hermiticity, three routes agree -------

def test_free_electron_spectrum():
    p = small_problem()
    h = O.Hamiltonian(p.lattice, p.kpt, p.ecut, p.box, np.zeros(p.box), p.tau, p.sigmas,
                      np.zeros_like(p.D))
    H, S = h.dense()
    ev = np.linalg.eigvalsh(H)
    np.testing.assert_allclose(ev, np.sort(h.kin), atol=1e-13)
    np.testing.assert_allclose(S, np.eye(h.npw), atol=0)


def test_constant_potential_shift():
    p = small_problem()
    V0 = -0.731
    h = O.Hamiltonian(p.lattice, p.kpt, p.ecut, p.box, np.full(p.box, V0), p.tau, p.sigmas,
                      np.zeros_like(p.D))
    H, _ = h.dense()
    np.testing.assert_allclose(np.linalg.eigvalsh(H), np.sort(h.kin) + V0, atol=1e-12)
    g = np.array([[0, 0, 0], [1, 0, 0], [0, 2, -1], [3, 1, 5]])
    vt = O.vtilde(np.full(p.box, V0), g)
    np.testing.assert_allclose(vt, [V0, 0, 0, 0], atol=1e-14)
    # matrix-free route gives the same shift on a random block
    C = W.random_block(3, h.npw, 3)
    np.testing.assert_allclose(O.apply_local(h.vloc, h.miller, C), V0 * C, atol=1e-13)


@pytest.mark.parametrize("with_q", [False, True])
def test_hermiticity(with_q):
    p = small_problem(with_q=with_q, kpt=[0.1, -0.2, 0.3])
    h = O.Hamiltonian.from_problem(p)
    phi = W.random_block(11, h.npw, 1)[0]
    psi = W.random_block(12, h.npw, 1)[0]
    for op in (h.apply_h, h.apply_s):
        l = np.vdot(phi, op(psi[None])[0])
        r = np.conj(np.vdot(psi, op(phi[None])[0]))
        assert abs(l - r) <= 1e-13 * abs(l)


@pytest.mark.parametrize("with_q", [False, True])
def test_dense_equals_matrix_free(with_q):
    p = small_problem(with_q=with_q, kpt=[0.25, 0.0, -0.125])
    h = O.Hamiltonian.from_problem(p)
    H, S = h.dense()
    C = W.random_block(5, h.npw, 4)
    np.testing.assert_allclose(h.apply_h(C), C @ H.T, rtol=0, atol=1e-12 * np.abs(C @ H.T).max())
    np.testing.assert_allclose(h.apply_s(C), C @ S.T, rtol=0, atol=1e-13)
    np.testing.assert_allclose(H, H.conj().T, atol=1e-13)


def test_local_matches_numpy_fft():
    """Library check: the direct separable DFT route equals numpy.fft on the box."""
    p = small_problem(box=(12, 16, 18), ecut=2.0, kpt=[0.1, 0.2, 0.3])
    h = O.Hamiltonian.from_problem(p)
    C = W.random_block(7, h.npw, 3)
    F = O.to_box(C, h.miller, p.box)
    n = float(np.prod(p.box))
    psi_r = np.fft.ifftn(F, axes=(1, 2, 3)) * n
    ref = O.from_box(np.fft.fftn(psi_r * h.vloc[None], axes=(1, 2, 3)) / n, h.miller, p.box)
    np.testing.assert_allclose(O.apply_local(h.vloc, h.miller, C), ref, atol=1e-13)


def test_woodbury_inverse():
    p = small_problem(with_q=True)
    h = O.Hamiltonian.from_problem(p)
    x = W.random_block(9, h.npw, 3)
    np.testing.assert_allclose(h.apply_s(h.apply_sinv(x)), x, atol=1e-13)
    np.testing.assert_allclose(h.apply_sinv(h.apply_s(x)), x, atol=1e-13)


def test_projector_symmetries():
    lat = np.diag([10.0] * 3)
    m, _ = O.g_sphere(lat, [0, 0, 0], 3.0, (16, 16, 16))
    P0 = O.projectors(lat, [0, 0, 0], m, np.zeros((1, 3)), [0.9])
    np.testing.assert_allclose(np.linalg.norm(P0, axis=0), 1.0, rtol=1e-14)
    # atom at the origin, Gamma: s even, p odd under G -> -G, so <s|p> = 0
    G = np.abs(P0.conj().T @ P0)
    assert G[0, 1:].max() < 1e-14
    idx = {tuple(r): i for i, r in enumerate(m)}
    neg = np.array([idx[(-a, -b, -c)] for a, b, c in m])
    np.testing.assert_allclose(P0[neg, 0], P0[:, 0], atol=1e-15)
    np.testing.assert_allclose(P0[neg, 1:], -P0[:, 1:], atol=1e-15)
    # p_x is proportional to q_x: zero on the h = 0 plane
    assert np.abs(P0[m[:, 0] == 0, 1]).max() == 0
    # lattice translation multiplies by exp(-i k.L) (k = 0.3 b1)
    k = np.array([0.3, 0.0, 0.0])
    mk, _ = O.g_sphere(lat, k, 3.0, (16, 16, 16))
    R = np.array([[1.2, -0.7, 2.5]])
    Pa = O.projectors(lat, k, mk, R, [0.8])
    Pb = O.projectors(lat, k, mk, R + lat[0], [0.8])
    np.testing.assert_allclose(Pb, Pa * np.exp(-1j * 2 * math.pi * 0.3), atol=1e-14)


# --- filter, bounds, Rayleigh-Ritz -------------------------------------------------

@pytest.mark.parametrize("with_q", [False, True])
def test_chebyshev_scaling_of_eigenvectors(with_q):
    """Exact eigenvectors x of A = S^{-1}H come out as T_m((lambda - c)/e) x."""
    p = small_problem(with_q=with_q)
    h = O.Hamiltonian.from_problem(p)
    H, S = h.dense()
    lam, X = scipy.linalg.eigh(H, S)
    a, b, m = lam[5] + 0.01, lam[-1] + 0.5, 7
    c, e = 0.5 * (a + b), 0.5 * (b - a)
    pick = [0, 3, 6, 40, len(lam) - 1]
    Y0 = X[:, pick].T.copy()
    Y = O.chebyshev_filter(h.apply_a, Y0, m, a, b)
    T = O.chebyshev_t(m, (lam[pick] - c) / e)
    np.testing.assert_allclose(Y, T[:, None] * Y0, rtol=0, atol=1e-10 * np.abs(T).max())


def test_chebyshev_closed_form_recurrence_values():
    # T_m(cos t) = cos(m t), T_2 = 2x^2 - 1, T_3 = 4x^3 - 3x
    x = np.array([-3.0, -1.0, -0.3, 0.2, 1.0, 2.5])
    np.testing.assert_allclose(O.chebyshev_t(2, x), 2 * x ** 2 - 1, rtol=1e-13)
    np.testing.assert_allclose(O.chebyshev_t(3, x), 4 * x ** 3 - 3 * x, rtol=1e-13)


def test_lanczos_upper_bound():
    p = small_problem(with_q=True)
    h = O.Hamiltonian.from_problem(p)
    H, S = h.dense()
    lmax_h = np.linalg.eigvalsh(H).max()
    lmax_pencil = scipy.linalg.eigh(H, S, eigvals_only=True).max()
    v0 = W.lanczos_v0(1, h.npw)
    up, theta = O.lanczos_upper(h.apply_h, v0, 10)
    assert theta <= lmax_h + 1e-12
    assert up >= lmax_h - 1e-12
    assert up >= lmax_pencil
    assert up <= lmax_h + 5.0


def test_rayleigh_ritz_matches_generalized_eigh():
    p = small_problem(with_q=True)
    h = O.Hamiltonian.from_problem(p)
    Y = W.random_block(21, h.npw, 6)
    HY, SY = h.apply_h(Y), h.apply_s(Y)
    lam, Yr, HYr, SYr, X = O.rayleigh_ritz(Y, HY, SY)
    Hs = Y.conj() @ HY.T
    Ss = Y.conj() @ SY.T
    ref = scipy.linalg.eigh(0.5 * (Hs + Hs.conj().T), 0.5 * (Ss + Ss.conj().T), eigvals_only=True)
    np.testing.assert_allclose(lam, ref, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(Yr.conj() @ SYr.T, np.eye(6), atol=1e-12)
    np.testing.assert_allclose(Yr.conj() @ HYr.T, np.diag(lam), atol=1e-11)
    np.testing.assert_allclose(HYr, h.apply_h(Yr), atol=1e-11)


def test_s_ortho():
    p = small_problem(with_q=True)
    h = O.Hamiltonian.from_problem(p)
    Y = W.random_block(22, h.npw, 5)
    Yn, SYn = O.s_ortho(Y, h.apply_s(Y))
    np.testing.assert_allclose(Yn.conj() @ SYn.T, np.eye(5), atol=1e-12)
    np.testing.assert_allclose(SYn, h.apply_s(Yn), atol=1e-12)
    # same span: Y = R Yn for some R
    R = np.linalg.lstsq(Yn.T, Y.T, rcond=None)[0]
    np.testing.assert_allclose(Yn.T @ R, Y.T, atol=1e-11)


@pytest.mark.parametrize("with_q", [False, True])
def test_one_s_ortho_pass_before_rr_gives_the_same_ritz_pairs(with_q):
    """How the GPU path orthonormalises before Rayleigh-Ritz: one Cholesky-QR pass, then Alg. 5 (whose Cholesky of
    S_Psi is the second pass), against the oracle's two passes then Alg. 5, on a filtered
    (ill-conditioned) block; and Ritz values do not depend on the basis of the span."""
    p = small_problem(with_q=with_q, nband=8)
    h = O.Hamiltonian.from_problem(p)
    Y0 = W.random_block(23, h.npw, 8)
    Y = O.chebyshev_filter(h.apply_a, Y0, 24, 0.0, 2.0 * p.ecut + 3.0)
    s = np.linalg.svd(Y, compute_uv=False)
    assert s[0] / s[-1] > 1e6                 # the case the second pass is there for
    y2 = Y
    for _ in range(2):
        y2, _ = O.s_ortho(y2, h.apply_s(y2))
    lam2, Yr2, *_ = O.rayleigh_ritz(y2, h.apply_h(y2), h.apply_s(y2))
    y1, _ = O.s_ortho(Y, h.apply_s(Y))
    lam1, Yr1, HYr1, SYr1, _ = O.rayleigh_ritz(y1, h.apply_h(y1), h.apply_s(y1))
    np.testing.assert_allclose(lam1, lam2, rtol=0, atol=1e-11)
    np.testing.assert_allclose(Yr1.conj() @ SYr1.T, np.eye(8), atol=1e-12)
    np.testing.assert_allclose(Yr1.conj() @ HYr1.T, np.diag(lam1), atol=1e-11)
    # another basis of the same span (of a well-conditioned block)
    B = W.random_block(24, 8, 8) + 3.0 * np.eye(8)
    ritz = []
    for Z in (Y0, B @ Y0):
        z, _ = O.s_ortho(Z, h.apply_s(Z))
        ritz.append(O.rayleigh_ritz(z, h.apply_h(z), h.apply_s(z))[0])
    np.testing.assert_allclose(ritz[1], ritz[0], rtol=0, atol=1e-12)


def _exact_pairs(with_q, nvec=6):
    """Lowest generalized eigenpairs of the dense pencil (H, S) by LAPACK: S-orthonormal
    columns V (V^dagger S V = I), H V = S V diag(lam).  Returned as band rows."""
    p = small_problem(with_q=with_q)
    h = O.Hamiltonian.from_problem(p)
    H, S = h.dense()
    lam, V = scipy.linalg.eigh(H, S)
    return H, S, lam[:nvec], V[:, :nvec].T.copy()


@pytest.mark.parametrize("with_q", [False, True])
def test_rayleigh_quotients_of_exact_and_mixed_vectors(with_q):
    """Alg. 12's Rayleigh quotients.  (i) Exact eigenvectors of the pencil give their
    eigenvalues.  (ii) x = v_i + d v_j (v S-orthonormal eigenvectors, complex d) has the
    closed form (lam_i + |d|^2 lam_j) / (1 + |d|^2), whatever the scale of x: the
    numerator is x^dagger H x and the denominator x^dagger S x (not |x|^2 when Q != 0)."""
    H, S, lam, V = _exact_pairs(with_q)
    rq = O.rayleigh_quotients(V, V @ H.T, V @ S.T)
    assert np.isrealobj(rq)
    np.testing.assert_allclose(rq, lam, rtol=1e-12, atol=1e-12)
    pairs = [(0, 3, 0.3 + 0.4j), (1, 5, -0.7j), (2, 4, 1.5 - 0.2j), (5, 0, 0.05)]
    X = np.stack([(2.5 - 1j) * (V[i] + d * V[j]) for i, j, d in pairs])
    expect = np.array([(lam[i] + abs(d) ** 2 * lam[j]) / (1 + abs(d) ** 2) for i, j, d in pairs])
    rq = O.rayleigh_quotients(X, X @ H.T, X @ S.T)
    np.testing.assert_allclose(rq, expect, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("with_q", [False, True])
def test_residual_norms_of_exact_and_perturbed_pairs(with_q):
    """Alg. 12's residual ||H psi_i - lambda_i S psi_i||.  (i) Exact pencil eigenpairs give
    ~0 (relative to the scale of H psi).  (ii) For x = v_i + d v_j and lambda = lam_i the
    residual is d (lam_j - lam_i) S v_j, so its norm is |d| |lam_j - lam_i| ||S v_j||; with
    S = I, ||S v_j|| = 1 and the value is closed-form.  A residual that omits S fails (i)
    when Q != 0; one that returns zeros fails (ii)."""
    H, S, lam, V = _exact_pairs(with_q)
    r = O.residual_norms(lam, V @ H.T, V @ S.T)
    scale = np.linalg.norm(V @ H.T, axis=1)
    assert np.all(r <= 1e-10 * scale)
    pairs = [(0, 3, 0.3 + 0.4j), (1, 5, -0.7j), (4, 2, 0.01)]
    X = np.stack([V[i] + d * V[j] for i, j, d in pairs])
    lam_x = np.array([lam[i] for i, _, _ in pairs])
    r = O.residual_norms(lam_x, X @ H.T, X @ S.T)
    if with_q:
        svj = np.array([np.linalg.norm(S @ V[j]) for _, j, _ in pairs])
        assert np.all(np.abs(svj - 1.0) > 1e-3)      # S v_j is not a unit vector here
    else:
        svj = np.ones(len(pairs))
    expect = np.array([abs(d) * abs(lam[j] - lam[i]) for i, j, d in pairs]) * svj
    np.testing.assert_allclose(r, expect, rtol=1e-10, atol=1e-13)


@pytest.mark.parametrize("with_q", [False, True])
def test_chebfi_residuals_match_dense_pencil(with_q):
    """The residuals ChebFi reports (Alg. 12) are ||H y_i - lambda_i S y_i|| of the Ritz
    pairs it returns, with H and S the dense matrices built entrywise."""
    p = small_problem(with_q=with_q, nband=8)
    h = O.Hamiltonian.from_problem(p)
    H, S = h.dense()
    Y0 = W.psi0(p.seed, h.npw, p.nband)
    v0 = W.lanczos_v0(p.seed, h.npw)
    lam, Y, res, _ = O.chebfi(h, Y0, v0, degree=6, cycles=2)
    ref = np.linalg.norm(Y @ H.T - lam[:, None] * (Y @ S.T), axis=1)
    assert ref.min() > 1e-6                      # not yet converged: the values mean something
    np.testing.assert_allclose(res, ref, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("with_q", [False, True])
def test_chebfi_converges_to_dense(with_q):
    """Brute force: ChebFi eigenvalues -> lowest dense (generalized) eigenvalues."""
    p = small_problem(with_q=with_q, box=(16, 16, 16), ecut=3.0, nband=10)
    h = O.Hamiltonian.from_problem(p)
    H, S = h.dense()
    ref = scipy.linalg.eigh(H, S, eigvals_only=True)[:p.nband]
    Y0 = W.psi0(p.seed, h.npw, p.nband)
    v0 = W.lanczos_v0(p.seed, h.npw)
    lam, Y, res, up = O.chebfi(h, Y0, v0, degree=10, cycles=12)
    np.testing.assert_allclose(lam[:7], ref[:7], atol=1e-9)
    assert res[:7].max() < 1e-5


@pytest.mark.slow
def test_chebfi_tiny_config_vs_dense():
    """The tiny 24^3 / ~1000 plane-wave Gamma problem against dense diagonalisation."""
    p = W.make_problem("tiny_gamma_fp64")
    h = O.Hamiltonian.from_problem(p)
    assert 950 < h.npw < 1100
    H, _ = h.dense()
    ref = np.linalg.eigvalsh(H)[:p.nband]
    Y0 = W.psi0(p.seed, h.npw, p.nband)
    v0 = W.lanczos_v0(p.seed, h.npw)
    lam, Y, res, up = O.chebfi(h, Y0, v0, degree=p.degree, cycles=20)
    np.testing.assert_allclose(lam[:10], ref[:10], atol=1e-8)


# --- density -----------------------------------------------------------------------

def test_density_parseval_and_positivity():
    p = small_problem(box=(12, 12, 16), ecut=2.0)
    h = O.Hamiltonian.from_problem(p)
    C = W.random_block(31, h.npw, 4)
    w = np.array([2.0, 1.0, 0.5, 0.25])
    rho = O.density_grad(C, None, w, h.miller, p.box)
    n = np.prod(p.box)
    np.testing.assert_allclose(rho.sum(), n * np.sum(w * np.linalg.norm(C, axis=1) ** 2), rtol=1e-13)
    assert rho.min() >= 0
    # cross term is symmetric in its real part
    D = W.random_block(32, h.npw, 4)
    g1 = O.density_grad(C, D, w, h.miller, p.box)
    g2 = O.density_grad(D, C, w, h.miller, p.box)
    np.testing.assert_allclose(g1, g2, atol=1e-12)
    # Hellmann-Feynman: d<psi|V|psi>/dV(r_j) = |psi(r_j)|^2 / n for the unnormalised psi(r)
    j = (3, 5, 7)
    c0 = C[:1]
    V = np.zeros(p.box)
    V[j] = 1.0
    e = np.vdot(c0[0], O.apply_local(V, h.miller, c0)[0]).real
    np.testing.assert_allclose(e, O.density_grad(c0, None, [1.0], h.miller, p.box)[j] / n, rtol=1e-12)
