"""Plain FP64 CPU oracle of LOBPCG with b blocks and k line minimizations (Alg. 11).

TEST INFRASTRUCTURE ONLY.  Only ``tests/`` may import this module; the CUDA library never
calls it and shares no code with it.

The steps follow the parallel LOBPCG of the paper's appendix (Alg. 11, with Alg. 8 S-Deflate,
Alg. 9 S-Ortho and Alg. 10 RR as its building blocks), in its order:

  for each block Psi_i of M/b bands:
    if i > 1: Psi_i <- S-Deflate(Psi_i) against the finished blocks Psi_1..Psi_{i-1}
    H Psi_i, S Psi_i;  S-Ortho(Psi_i);  RR(Psi_i)          (Rayleigh quotients initialisation)
    for n = 1..k:
      W_i <- (H - Lambda_i S) Psi_i;  stop when every residual norm is below tol
      W_i <- K W_i                                          (diagonal preconditioner)
      if i > 1: W_i <- S-Deflate(W_i)
      H W_i, S W_i
      n == 1: S-Ortho + RR on [Psi_i, W_i];  n > 1: on [Psi_i, W_i, P_i]
      the RR keeps the M/b lowest Ritz pairs: Psi_i <- (Psi part), P_i <- (W, P parts),
      then Psi_i <- Psi_i + P_i (with H Psi_i, S Psi_i alike)
  if b > 1: S-Ortho + RR on the whole Psi

Readings where the paper is silent:
  * K: the paper calls it a diagonal preconditioner without a formula.  Reading: the
    Teter-Payne-Allan preconditioner (Teter, Payne & Allan, Phys. Rev. B 40, 12255 (1989)),
    diagonal in G for each band: K_G = p(x) / (p(x) + 16 x^4), p(x) = 27 + 18 x + 12 x^2 + 8 x^3,
    x = t_G / E_kin, with t_G = |k+G|^2/2 and E_kin the kinetic energy of the band
    (sum_G t_G |psi_G|^2 / sum_G |psi_G|^2).
  * "exit if block is converged": the line loop of a block ends before the n-th
    minimisation when max_i ||W_i|| < tol (the residual of Alg. 12, ||H psi - lambda S psi||).
  * P after the RR of the basis Z = [Psi, W(, P)] (made S-orthonormal by S-Ortho, so the
    first M/b columns span Psi): with C the kept eigenvector coefficients, P = Z[W, P part]
    C[W, P rows] and Psi = Z[Psi part] C[Psi rows] + P.
  * Blocks are formed from consecutive bands of the starting block; M must be a multiple of b.

Arrays hold bands as rows (shape (m, N)), i.e. the transpose of the paper's column-major Psi.
Pins: tests/test_oracle_lobpcg.py.
"""
from __future__ import annotations

from typing import List, Optional, Tuple

import numpy as np
import scipy.linalg

from . import pw_oracle as O


def tpa_preconditioner(kin: np.ndarray, ekin: float) -> np.ndarray:
    """K_G = p(x) / (p(x) + 16 x^4), p(x) = 27 + 18 x + 12 x^2 + 8 x^3, x = t_G / E_kin."""
    x = np.asarray(kin, float) / ekin
    p = 27.0 + 18.0 * x + 12.0 * x ** 2 + 8.0 * x ** 3
    return p / (p + 16.0 * x ** 4)


def band_kinetic(X: np.ndarray, kin: np.ndarray) -> np.ndarray:
    """E_kin of each band: sum_G t_G |x_G|^2 / sum_G |x_G|^2."""
    a = np.abs(X) ** 2
    return (a @ np.asarray(kin, float)) / a.sum(axis=1)


def s_deflate(X: np.ndarray, Y0: np.ndarray, SY0: np.ndarray) -> np.ndarray:
    """Alg. 8: S_{Psi0,Psi} = (S Psi0)^dagger Psi; Psi <- Psi - Psi0 S_{Psi0,Psi}."""
    C = SY0.conj() @ X.T                      # (m', k): C[j, i] = <S y_j | x_i>
    return X - C.T @ Y0


def s_ortho3(X, HX, SX) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Alg. 9: S_Psi = Psi^dagger (S Psi) = U^dagger U; Psi, H Psi, S Psi <- (.) U^{-1}."""
    G = X.conj() @ SX.T
    G = 0.5 * (G + G.conj().T)
    U = np.linalg.cholesky(G).conj().T
    solve = lambda B: scipy.linalg.solve_triangular(U, B, trans="T", lower=False)
    return solve(X), solve(HX), solve(SX)


def residuals(lam, HX, SX) -> np.ndarray:
    """Rows of W = (H - Lambda S) Psi."""
    return HX - lam[:, None] * SX


def lobpcg(ham: "O.Hamiltonian", psi0: np.ndarray, nblocks: int, nline: int, tol: float = 0.0,
           history: Optional[List] = None):
    """Alg. 11 on the oracle Hamiltonian.  Returns (eig (M,), Psi (M, N), residual norms (M,),
    line minimisations done per block).  ``history`` (optional list) receives, per block and
    per line minimisation, the block's Ritz values after the RR."""
    M = psi0.shape[0]
    if nblocks < 1 or M % nblocks:
        raise ValueError("M must be a positive multiple of the block count")
    bs = M // nblocks
    kin = ham.kin
    Ys, HYs, SYs = [], [], []                 # finished blocks
    lams, its = [], []
    for i in range(nblocks):
        X = np.array(psi0[i * bs:(i + 1) * bs], dtype=complex)
        if i > 0:
            X = s_deflate(X, np.concatenate(Ys), np.concatenate(SYs))
        HX, SX = ham.apply_h(X), ham.apply_s(X)
        X, HX, SX = s_ortho3(X, HX, SX)
        lam, X, HX, SX, _ = O.rayleigh_ritz(X, HX, SX)
        P = HP = SP = None
        done = 0
        for n in range(nline):
            W = residuals(lam, HX, SX)
            if np.linalg.norm(W, axis=1).max() < tol:
                break
            W = W * np.stack([tpa_preconditioner(kin, e) for e in band_kinetic(X, kin)])
            if i > 0:
                W = s_deflate(W, np.concatenate(Ys), np.concatenate(SYs))
            HW, SW = ham.apply_h(W), ham.apply_s(W)
            if P is None:
                Z, HZ, SZ = (np.concatenate(t) for t in ((X, W), (HX, HW), (SX, SW)))
            else:
                Z, HZ, SZ = (np.concatenate(t) for t in ((X, W, P), (HX, HW, HP), (SX, SW, SP)))
            Z, HZ, SZ = s_ortho3(Z, HZ, SZ)
            lz, _, _, _, C = O.rayleigh_ritz(Z, HZ, SZ)
            Ck = C[:, :bs]                    # the bs lowest Ritz pairs
            lam = lz[:bs]
            P, HP, SP = (Ck[bs:].T @ A[bs:] for A in (Z, HZ, SZ))
            X, HX, SX = (Ck[:bs].T @ A[:bs] + B for A, B in ((Z, P), (HZ, HP), (SZ, SP)))
            done = n + 1
            if history is not None:
                history.append((i, n, lam.copy()))
        Ys.append(X)
        HYs.append(HX)
        SYs.append(SX)
        lams.append(lam)
        its.append(done)
    Y, HY, SY = np.concatenate(Ys), np.concatenate(HYs), np.concatenate(SYs)
    lam = np.concatenate(lams)
    if nblocks > 1:
        Y, HY, SY = s_ortho3(Y, HY, SY)
        lam, Y, HY, SY, _ = O.rayleigh_ritz(Y, HY, SY)
    res = np.linalg.norm(residuals(lam, HY, SY), axis=1)
    return lam, Y, res, its
