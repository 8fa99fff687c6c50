"""Plain FP64 CPU oracle of the Chebyshev-filtered plane-wave H-apply.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  The CUDA library never
calls it and shares no code with it.

Every function is the plain definition (or the algorithm's steps in the paper's
order) in numpy float64/complex128, with no blocking, fusion or reordering beyond
what the definition states.  Library primitives used as steps: matrix products,
``numpy.linalg.cholesky``/``eigh``, ``scipy.linalg.solve_triangular``.

Conventions (the paper is silent on them; these are the readings this oracle takes):
  * bands are stored as rows of an (M, N) array, i.e. the N x M wave-function
    matrix Psi of Sec. 3.1 in column-major order;
  * psi(r) = sum_G c_G exp(i (k+G).r); the inverse DFT is unnormalised (+i),
    the forward DFT (-i) is divided by n1 n2 n3; the exp(i k.r) factor cancels
    in V_loc psi;
  * G components are taken modulo the box when placed on the grid, so the
    local term is H_loc[G, G'] = Vt(G - G' mod n) exactly.

Pins (tests marked ``not gpu`` in tests/test_oracle_pins.py): free-electron
spectrum and shell degeneracies (tests/golden/r3_counts.txt), constant-potential
shift, Hermiticity, dense == matrix-free == numpy.fft, Woodbury identity,
Chebyshev scaling of exact eigenvectors against the closed form of T_m, Lanczos
bound >= lambda_max, Rayleigh quotients and residual norms of exact and perturbed
pencil eigenpairs against closed forms, Rayleigh-Ritz against scipy's generalized
eigensolver, ChebFi convergence to dense diagonalisation, Parseval for the
density, projector symmetries, adjoint against finite differences.
"""
from __future__ import annotations

import math
from typing import Callable, Optional, Tuple

import numpy as np
import scipy.linalg


# ---------------------------------------------------------------------------
# a1: plane-wave sphere (Sec. 3.1 problem setup; E_cut fixes N and the box, Sec. 4.2)
# ---------------------------------------------------------------------------

def reciprocal(lattice: np.ndarray) -> np.ndarray:
    """Rows b_i with a_i . b_j = 2 pi delta_ij."""
    return 2.0 * math.pi * np.linalg.inv(np.asarray(lattice, float)).T


def g_sphere(lattice, kpt, ecut, box) -> Tuple[np.ndarray, np.ndarray]:
    """All integer G = (h, k, l) with |k + G|^2 / 2 <= ecut.

    Returns (miller (N, 3) int32 sorted by (h, k, l) ascending, kinetic (N,)).
    Raises if the sphere does not fit in the box without aliasing."""
    B = reciprocal(lattice)
    kc = np.asarray(kpt, float) @ B
    gmax = math.sqrt(2.0 * ecut)
    # bound each Miller index by |h| <= (gmax + |k|) |a_i| / (2 pi)
    A = np.asarray(lattice, float)
    lim = [int(math.ceil((gmax + np.linalg.norm(kc)) * np.linalg.norm(A[i]) / (2 * math.pi))) + 1
           for i in range(3)]
    rng = [np.arange(-l, l + 1) for l in lim]
    H, K, L = np.meshgrid(*rng, indexing="ij")
    m = np.stack([H.ravel(), K.ravel(), L.ravel()], axis=1)
    q = m @ B + kc
    kin = 0.5 * np.einsum("ij,ij->i", q, q)
    keep = kin <= ecut
    m = m[keep]
    kin = kin[keep]
    order = np.lexsort((m[:, 2], m[:, 1], m[:, 0]))
    m = m[order].astype(np.int32)
    kin = kin[order]
    for i in range(3):
        if m.shape[0] and (m[:, i].max() - m[:, i].min()) >= box[i]:
            raise ValueError("plane-wave sphere does not fit in the FFT box")
    return m, kin


# ---------------------------------------------------------------------------
# a2: projectors P = <G|p_i^R> (Sec. 4.2, nonlocal operator)
# ---------------------------------------------------------------------------

def projectors(lattice, kpt, miller, tau, sigmas) -> np.ndarray:
    """N x N_projs projector matrix (complex128), columns ordered atom-major,
    then channel, then (s, p_x, p_y, p_z).

    s:   exp(-q^2 s^2 / 2);  p_a: (-i) q_a s exp(-q^2 s^2 / 2);  q = k + G;
    each column carries the structure phase exp(-i q.R) and is scaled to unit
    2-norm over the sphere."""
    B = reciprocal(lattice)
    q = miller.astype(float) @ B + np.asarray(kpt, float) @ B
    q2 = np.einsum("ij,ij->i", q, q)
    cols = []
    for R in np.asarray(tau, float):
        phase = np.exp(-1j * (q @ R))
        for s in sigmas:
            g = np.exp(-0.5 * q2 * s * s)
            cols.append(g * phase)
            for a in range(3):
                cols.append(-1j * q[:, a] * s * g * phase)
    if not cols:                  # no atoms: no nonlocal term
        return np.zeros((miller.shape[0], 0), dtype=np.complex128)
    P = np.stack(cols, axis=1)
    P /= np.linalg.norm(P, axis=0, keepdims=True)
    return P


# ---------------------------------------------------------------------------
# local potential (Sec. 2.1, Alg. 2; Sec. 3.2 matrix-free H-apply)
# ---------------------------------------------------------------------------

def _dft_matrix(n: int, sign: int) -> np.ndarray:
    j = np.arange(n)
    return np.exp(sign * 2j * math.pi * np.outer(j, j) / n)


def vtilde(vloc: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Vt(g) = (1 / n1n2n3) sum_r V(r) exp(-i g.r) for integer g (rows), by a
    separable direct sum (no FFT)."""
    n1, n2, n3 = vloc.shape
    e1 = np.exp(-2j * math.pi * np.outer(g[:, 0], np.arange(n1)) / n1)
    e2 = np.exp(-2j * math.pi * np.outer(g[:, 1], np.arange(n2)) / n2)
    e3 = np.exp(-2j * math.pi * np.outer(g[:, 2], np.arange(n3)) / n3)
    t = np.einsum("gk,ijk->gij", e3, vloc.astype(complex))
    t = np.einsum("gj,gij->gi", e2, t)
    return np.einsum("gi,gi->g", e1, t) / (n1 * n2 * n3)


def to_box(C: np.ndarray, miller: np.ndarray, box) -> np.ndarray:
    """Scatter sphere coefficients (M, N) onto the box (M, n1, n2, n3), G taken mod n."""
    M = C.shape[0]
    out = np.zeros((M,) + tuple(box), dtype=np.complex128)
    idx = tuple((miller[:, i] % box[i]) for i in range(3))
    out[(slice(None),) + idx] = C
    return out


def from_box(F: np.ndarray, miller: np.ndarray, box) -> np.ndarray:
    idx = tuple((miller[:, i] % box[i]) for i in range(3))
    return F[(slice(None),) + idx]


def inverse_dft_direct(C: np.ndarray, miller: np.ndarray, box) -> np.ndarray:
    """psi(r_j) = sum_G c_G exp(+2 pi i G.j/n), unnormalised, separable direct DFT."""
    F = to_box(C, miller, box)
    for ax in range(3):
        W = _dft_matrix(box[ax], +1)
        F = np.moveaxis(np.tensordot(F, W, axes=([ax + 1], [1])), -1, ax + 1)
    return F


def forward_dft_direct(F: np.ndarray) -> np.ndarray:
    """(1/n1n2n3) sum_j f(r_j) exp(-2 pi i G.j/n) on the whole box, separable direct DFT."""
    box = F.shape[1:]
    for ax in range(3):
        W = _dft_matrix(box[ax], -1)
        F = np.moveaxis(np.tensordot(F, W, axes=([ax + 1], [1])), -1, ax + 1)
    return F / float(np.prod(box))


def apply_local(vloc: np.ndarray, miller: np.ndarray, C: np.ndarray) -> np.ndarray:
    """V_loc C: scatter to box, inverse DFT, multiply by V(r), forward DFT, gather."""
    box = vloc.shape
    psi_r = inverse_dft_direct(C, miller, box)
    return from_box(forward_dft_direct(psi_r * vloc[None]), miller, box)


# ---------------------------------------------------------------------------
# Hamiltonian / overlap (Sec. 3.1, 3.2; HX / HX_SX / Sinv of Sec. 3.3)
# ---------------------------------------------------------------------------

class Hamiltonian:
    """H = T + V_loc + P D P^dagger,  S = I + P Q P^dagger  (Q None => S = I)."""

    def __init__(self, lattice, kpt, ecut, box, vloc, tau, sigmas, D, Q=None, P=None):
        self.lattice = np.asarray(lattice, float)
        self.kpt = np.asarray(kpt, float)
        self.box = tuple(box)
        self.vloc = np.asarray(vloc, float)
        self.miller, self.kin = g_sphere(lattice, kpt, ecut, box)
        self.P = projectors(lattice, kpt, self.miller, tau, sigmas) if P is None else P
        self.D = np.asarray(D, float)
        self.Q = None if Q is None else np.asarray(Q, float)
        self._K = None

    @classmethod
    def from_problem(cls, prob, kpt=None, ecut=None):
        return cls(prob.lattice, prob.kpt if kpt is None else kpt,
                   prob.ecut if ecut is None else ecut, prob.box, prob.vloc,
                   prob.tau, prob.sigmas, prob.D, prob.Q)

    @property
    def npw(self) -> int:
        return self.miller.shape[0]

    def project(self, C):
        """C_proj = <p|psi> = P^dagger psi, returned as (M, N_projs)."""
        return C @ self.P.conj()

    def apply_h(self, C: np.ndarray) -> np.ndarray:
        C = np.atleast_2d(C)
        out = C * self.kin[None, :]
        out = out + apply_local(self.vloc, self.miller, C)
        out = out + (self.project(C) @ self.D.T) @ self.P.T
        return out

    def apply_s(self, C: np.ndarray) -> np.ndarray:
        C = np.atleast_2d(C)
        if self.Q is None:
            return C.copy()
        return C + (self.project(C) @ self.Q.T) @ self.P.T

    def woodbury_k(self) -> np.ndarray:
        """K = (Q^{-1} + P^dagger P)^{-1} (Woodbury form of S^{-1}, Sec. 3.3 Sinv)."""
        if self._K is None:
            self._K = np.linalg.inv(np.linalg.inv(self.Q) + self.P.conj().T @ self.P)
        return self._K

    def apply_sinv(self, C: np.ndarray) -> np.ndarray:
        """S^{-1} C = C - P K P^dagger C."""
        C = np.atleast_2d(C)
        if self.Q is None:
            return C.copy()
        K = self.woodbury_k()
        return C - (self.project(C) @ K.T) @ self.P.T

    def apply_a(self, C: np.ndarray) -> np.ndarray:
        """A = S^{-1} H, the operator whose spectrum the filter shapes (Alg. 12)."""
        return self.apply_sinv(self.apply_h(C))

    def dense(self) -> Tuple[np.ndarray, np.ndarray]:
        """Dense H and S, entrywise (small N only)."""
        m = self.miller
        dg = m[:, None, :] - m[None, :, :]
        N = m.shape[0]
        flat = dg.reshape(-1, 3)
        uniq, inv = np.unique(flat, axis=0, return_inverse=True)
        vt = vtilde(self.vloc, uniq)
        H = vt[inv.reshape(-1)].reshape(N, N)
        H = H + np.diag(self.kin)
        H = H + self.P @ self.D @ self.P.conj().T
        S = np.eye(N, dtype=complex)
        if self.Q is not None:
            S = S + self.P @ self.Q @ self.P.conj().T
        return H, S


# ---------------------------------------------------------------------------
# Chebyshev filter (Alg. 7 / Alg. 12; three-term recurrence of Zhou et al.)
# ---------------------------------------------------------------------------

def chebyshev_filter(apply_a: Callable, Y0: np.ndarray, degree: int, a: float, b: float) -> np.ndarray:
    """Y_m with c=(b+a)/2, e=(b-a)/2, Y_1=(A-c)Y_0/e, Y_{k+1}=(2/e)(A-c)Y_k - Y_{k-1}."""
    c = 0.5 * (b + a)
    e = 0.5 * (b - a)
    Yprev = Y0
    Y = (apply_a(Y0) - c * Y0) / e
    for _ in range(1, degree):
        Ynew = (2.0 / e) * (apply_a(Y) - c * Y) - Yprev
        Yprev, Y = Y, Ynew
    return Y


def chebyshev_t(m: int, x: np.ndarray) -> np.ndarray:
    """T_m(x) by its closed form: cos(m arccos x) on [-1,1], sign^m cosh(m arccosh|x|) outside."""
    x = np.asarray(x, float)
    out = np.empty_like(x)
    inside = np.abs(x) <= 1
    out[inside] = np.cos(m * np.arccos(x[inside]))
    xo = x[~inside]
    out[~inside] = np.sign(xo) ** m * np.cosh(m * np.arccosh(np.abs(xo)))
    return out


# ---------------------------------------------------------------------------
# spectrum bounds (Alg. 12 lines on Rayleigh quotients; upper bound by Lanczos)
# ---------------------------------------------------------------------------

def rayleigh_quotients(C, HC, SC) -> np.ndarray:
    """lambda_i = (H psi_i)^dagger psi_i / ((S psi_i)^dagger psi_i)."""
    num = np.real(np.einsum("ij,ij->i", C.conj(), HC))
    den = np.real(np.einsum("ij,ij->i", C.conj(), SC))
    return num / den


def lanczos_upper(apply_h: Callable, v0: np.ndarray, steps: int) -> Tuple[float, float]:
    """k-step Lanczos on H from v0; returns (theta_max + |beta_k|, theta_max)."""
    v = v0 / np.linalg.norm(v0)
    vprev = np.zeros_like(v)
    alphas, betas = [], []
    beta = 0.0
    for j in range(steps):
        w = apply_h(v[None])[0]
        alpha = float(np.real(np.vdot(v, w)))
        w = w - alpha * v - beta * vprev
        beta = float(np.linalg.norm(w))
        alphas.append(alpha)
        betas.append(beta)
        vprev, v = v, w / beta
    T = np.diag(alphas) + np.diag(betas[:-1], 1) + np.diag(betas[:-1], -1)
    theta = float(np.linalg.eigvalsh(T).max())
    return theta + abs(betas[-1]), theta


# ---------------------------------------------------------------------------
# S-orthonormalisation (Alg. 9) and Rayleigh-Ritz (Alg. 5)
# ---------------------------------------------------------------------------

def s_ortho(Y: np.ndarray, SY: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """S_Psi = Psi^dagger (S Psi) = U^dagger U (Cholesky); Psi <- Psi U^{-1}; S Psi <- (S Psi) U^{-1}."""
    G = Y.conj() @ SY.T                       # G[i, j] = <y_i | S y_j>
    G = 0.5 * (G + G.conj().T)
    Lc = np.linalg.cholesky(G)                # G = L L^dagger, U = L^dagger
    U = Lc.conj().T
    # Psi (column-major N x M) times U^{-1}: rows of our arrays are columns of Psi
    Yn = scipy.linalg.solve_triangular(U, Y, trans="T", lower=False)
    SYn = scipy.linalg.solve_triangular(U, SY, trans="T", lower=False)
    return Yn, SYn


def rayleigh_ritz(Y, HY, SY):
    """H_Psi = Psi^dagger(H Psi), S_Psi = Psi^dagger(S Psi); H_Psi X = Lambda S_Psi X
    by Cholesky reduction and a standard Hermitian eigensolve; Psi <- Psi X,
    H Psi <- (H Psi) X, S Psi <- (S Psi) X.  Eigenvalues ascending."""
    Hs = Y.conj() @ HY.T
    Ss = Y.conj() @ SY.T
    Hs = 0.5 * (Hs + Hs.conj().T)
    Ss = 0.5 * (Ss + Ss.conj().T)
    L = np.linalg.cholesky(Ss)
    Li = scipy.linalg.solve_triangular(L, np.eye(L.shape[0]), lower=True)
    Cm = Li @ Hs @ Li.conj().T
    Cm = 0.5 * (Cm + Cm.conj().T)
    lam, U = np.linalg.eigh(Cm)
    X = Li.conj().T @ U
    # column-major Psi X  <=>  (band-row arrays)  X^T @ Y
    return lam, X.T @ Y, X.T @ HY, X.T @ SY, X


def residual_norms(lam, HY, SY) -> np.ndarray:
    """r_i = || H psi_i - lambda_i S psi_i || (Alg. 12 residual)."""
    return np.linalg.norm(HY - lam[:, None] * SY, axis=1)


def chebfi(ham: Hamiltonian, Y0: np.ndarray, v0: np.ndarray, degree: int, cycles: int,
           lanczos_steps: int = 10, return_history: bool = False):
    """Chebyshev-filtered subspace iteration (Alg. 7 / Alg. 12).  Where the paper is
    silent this oracle reads it as follows (the filter bounds are not written out in
    the paper; the Lanczos bound is the Zhou-Li estimate, and S >= I makes H's bound
    valid for S^{-1}H):

      b = theta_max + |beta_k| from Lanczos on H (spectrum of S^{-1}H is below it);
      cycle 1 cut a = max Rayleigh quotient of Psi_0; later a = largest Ritz value;
      each cycle: filter with A = S^{-1}H  ->  S-orthonormalise twice (Alg. 9)
                  ->  H Psi, S Psi  ->  Rayleigh-Ritz (Alg. 5)  ->  residuals.
    """
    upper, _ = lanczos_upper(ham.apply_h, v0, lanczos_steps)
    HY = ham.apply_h(Y0)
    SY = ham.apply_s(Y0)
    a = float(rayleigh_quotients(Y0, HY, SY).max())
    Y = Y0
    hist = []
    lam = res = None
    for _ in range(cycles):
        Y = chebyshev_filter(ham.apply_a, Y, degree, a, upper)
        for _rep in range(2):
            Y, _ = s_ortho(Y, ham.apply_s(Y))
        HY = ham.apply_h(Y)
        SY = ham.apply_s(Y)
        lam, Y, HY, SY, _ = rayleigh_ritz(Y, HY, SY)
        res = residual_norms(lam, HY, SY)
        hist.append((lam.copy(), res.copy(), a))
        a = float(lam.max())
    if return_history:
        return lam, Y, res, upper, hist
    return lam, Y, res, upper


# ---------------------------------------------------------------------------
# density / gradient contraction (Alg. 3 density step; dL/dV_loc contraction)
# ---------------------------------------------------------------------------

def density_grad(Ca: np.ndarray, Cb: Optional[np.ndarray], w: np.ndarray, miller, box) -> np.ndarray:
    """g(r_j) = sum_i w_i Re[conj(a_i(r_j)) b_i(r_j)], a_i(r), b_i(r) the
    unnormalised inverse DFTs of the sphere blocks.  Cb None => b = a (density)."""
    ar = inverse_dft_direct(Ca, miller, box)
    br = ar if Cb is None else inverse_dft_direct(Cb, miller, box)
    return np.einsum("i,ijkl->jkl", np.asarray(w, float), np.real(ar.conj() * br))
