"""Plain FP64 reverse-mode adjoint of the ChebFi cycle (filter + S-Ortho + Rayleigh-Ritz)
with respect to V_loc(r) and D, for S = I.

TEST INFRASTRUCTURE ONLY (same rules as oracle/pw_oracle.py): imported by tests/,
__graft_entry__.smoke() and the CPU legs of bench.py, never by the CUDA library.

Gradient convention (PyTorch's for complex tensors): the adjoint of a complex block Z is
Zbar = dL/dRe(Z) + i dL/dIm(Z), so that dL = Re tr(Zbar^H dZ).  Blocks are (M, N)
band-row arrays like everywhere in the oracle; the formulas below are written for the
column-major N x M matrices they represent.

Pinned in tests/test_oracle_adjoint.py against central finite differences of the
forward below and against the Hellmann-Feynman theorem at convergence.

Forward (per cycle; a = previous largest Ritz value and the Lanczos bound b are held
fixed, i.e. not differentiated):
    Y_1 = (H - c) Y_0 / e,  Y_{k+1} = (2/e)(H - c) Y_k - Y_{k-1}     (Chebyshev filter)
    Y_m = Q R                                                      (two Cholesky-QR passes)
    A = Q^H H Q = X diag(lam) X^H,   Psi = Q X                      (Rayleigh-Ritz)
Backward, given lambar and Psibar:
    Qbar = Psibar X^H,  Xbar = Q^H Psibar
    Abar = Herm( X (diag(lambar) + F o (X^H Xbar)) X^H ),  F_ji = 1/(lam_i - lam_j), i != j
           (pairs among which the later computation is rotation invariant may be dropped:
            all pairs of earlier cycles, and pairs inside the occupied / inside the empty
            bands for a loss built from occupied eigenvalues and the occupied density)
    Qbar += 2 H Q Abar;   Vbar += (1/n) sum_j Re[conj((Q Abar)_j(r)) Q_j(r)];
    Dbar += Re[conj(P^H Q Abar) (P^H Q)^T]
    Ybar_m = (I - Q Q^H) Qbar R^{-H}          (the cycle depends on Y_m only through its span)
    Z_m = Ybar_m, Z_k = alpha_k (H - c) Z_{k+1} - beta_{k+1} Z_{k+2}    (adjoint recurrence)
    Vbar += alpha_k (1/n) sum_j Re[conj(Z_{k+1,j}(r)) Y_{k,j}(r)],  Dbar += alpha_k Re[conj(P^H Z_{k+1})(P^H Y_k)^T]
    Psibar of the previous cycle = Z_0.
"""
from __future__ import annotations

import numpy as np

from . import pw_oracle as O


def _apply_h_minus_c(ham, Y, c):
    return ham.apply_h(Y) - c * Y


def filter_with_tape(ham, Y0, degree, a, b):
    """Chebyshev filter keeping every iterate Y_0 .. Y_m (band-row arrays)."""
    c, e = 0.5 * (b + a), 0.5 * (b - a)
    Ys = [Y0]
    Ys.append(_apply_h_minus_c(ham, Y0, c) / e)
    for k in range(1, degree):
        Ys.append((2.0 / e) * _apply_h_minus_c(ham, Ys[k], c) - Ys[k - 1])
    return Ys, c, e


def cycle_forward(ham, Y0, degree, a, b):
    Ys, c, e = filter_with_tape(ham, Y0, degree, a, b)
    Ym = Ys[-1]
    Q = Ym
    for _ in range(2):
        Q, _ = O.s_ortho(Q, ham.apply_s(Q))
    HQ = ham.apply_h(Q)
    A = Q.conj() @ HQ.T                    # A[i, j] = q_i^H H q_j
    A = 0.5 * (A + A.conj().T)
    lam, X = np.linalg.eigh(A)
    Psi = X.T @ Q                          # column-major Q X
    R = Q.conj() @ Ym.T                    # column-major Q^H Y_m (upper triangular)
    return dict(Ys=Ys, c=c, e=e, Q=Q, HQ=HQ, X=X, lam=lam, R=R, Psi=Psi, a=a, b=b)


def chebfi_diff_forward(ham, Y0, v0, degree, cycles, lanczos_steps=10, bounds=None):
    """ChebFi cycles keeping the tape.  The cuts are stop-gradient: ``bounds`` =
    (upper, [a_1 .. a_cycles]) replays given ones (finite differences need this);
    None computes them as the plain solver does (Lanczos upper bound; cycle 1 cut the
    largest Rayleigh quotient of Y0, later the largest Ritz value)."""
    if bounds is None:
        upper, _ = O.lanczos_upper(ham.apply_h, v0, lanczos_steps)
        HY = ham.apply_h(Y0)
        a = float(O.rayleigh_quotients(Y0, HY, ham.apply_s(Y0)).max())
        cuts = None
    else:
        upper, cuts = bounds[0], list(bounds[1])
        a = cuts[0]
    Y = Y0
    tape = []
    used = []
    for cyc in range(cycles):
        if cuts is not None:
            a = cuts[cyc]
        used.append(a)
        t = cycle_forward(ham, Y, degree, a, upper)
        tape.append(t)
        Y = t["Psi"]
        a = float(t["lam"].max())
    return tape[-1]["lam"], tape[-1]["Psi"], tape, (upper, used)


def _param_contract(ham, Zbar_rows, Y_rows, weight, vbar, dbar):
    """vbar += weight (1/n) sum_j Re[conj(z_j(r)) y_j(r)];  dbar += weight Re[conj(P^H z)(P^H y)^T]."""
    n = float(np.prod(ham.box))
    w = np.full(Zbar_rows.shape[0], weight / n)
    vbar += O.density_grad(Zbar_rows, Y_rows, w, ham.miller, ham.box)
    Cz = ham.project(Zbar_rows)            # (M, np): Cz[j, a] = (P^H z_j)_a
    Cy = ham.project(Y_rows)
    dbar += weight * np.real(Cz.conj().T @ Cy)


def cycle_backward(ham, t, lambar, Psibar, vbar, dbar, keep):
    """One cycle's adjoint; returns the adjoint of its input block Y_0.  keep(i, j) says
    whether the eigenvector-coupling term of the band pair (i, j) is taken."""
    Q, HQ, X, lam, R = t["Q"], t["HQ"], t["X"], t["lam"], t["R"]
    M = lam.shape[0]
    Qc = Q.T                               # N x M column-major views
    HQc = HQ.T
    Pb = Psibar.T
    Qbar = Pb @ X.conj().T
    Xbar = Qc.conj().T @ Pb
    K = X.conj().T @ Xbar
    F = np.zeros((M, M))
    for i in range(M):
        for j in range(M):
            if i != j and keep(i, j):
                F[j, i] = 1.0 / (lam[i] - lam[j])
    G = F * K + np.diag(lambar)
    Abar = X @ G @ X.conj().T
    Abar = 0.5 * (Abar + Abar.conj().T)
    Qbar = Qbar + 2.0 * HQc @ Abar
    QA = Qc @ Abar
    _param_contract(ham, QA.T, Q, 1.0, vbar, dbar)
    # Y_m = Q R: the cycle depends on span(Y_m) only
    Ybar = Qbar - Qc @ (Qc.conj().T @ Qbar)
    Ybar = np.linalg.solve(R.conj(), Ybar.T).T   # Ybar R^{-H}
    # adjoint Chebyshev recurrence
    Ys, c, e = t["Ys"], t["c"], t["e"]
    m = len(Ys) - 1
    Z = {m: Ybar.T}                         # band-row arrays
    Z[m + 1] = np.zeros_like(Ys[0])
    for k in range(m - 1, -1, -1):
        alpha = 1.0 / e if k == 0 else 2.0 / e
        beta_next = 0.0 if k + 1 == 0 else 1.0   # beta_{k+1} (= 1 for k + 1 >= 1)
        _param_contract(ham, Z[k + 1], Ys[k], alpha, vbar, dbar)
        Z[k] = alpha * _apply_h_minus_c(ham, Z[k + 1], c) - (beta_next * Z[k + 2] if k + 2 <= m else 0.0)
    return Z[0]


def chebfi_diff_backward(ham, tape, lambar, Psibar, split=None):
    """dL/dV (grid, PyTorch real-gradient convention) and the unsymmetrised dL/dD matrix G
    (dL = sum_ab G_ab dD_ab) for lambar, Psibar of the last cycle.

    split: None keeps every band pair of the last cycle's eigenvector coupling; an integer s
    keeps only pairs with one band below s and one at or above it, which is exact for a loss
    unchanged by rotations among bands [0, s) and among bands [s, M) (the occupied-band sum
    and density loss with s = number of occupied bands) and avoids dividing by small gaps.
    Earlier cycles keep no pair: the next cycle sees their Ritz vectors only through their
    span (the filter acts column by column and Rayleigh-Ritz depends on the span alone)."""
    vbar = np.zeros(ham.box)
    dbar = np.zeros_like(ham.D)
    lb, pb = np.asarray(lambar, float), Psibar
    if split is None:
        keep_last = lambda i, j: True
    else:
        keep_last = lambda i, j: (i < split) != (j < split)
    keep = keep_last
    for t in reversed(tape):
        pb = cycle_backward(ham, t, lb, pb, vbar, dbar, keep)
        lb = np.zeros_like(lb)
        keep = lambda i, j: False
    return vbar, dbar


# ---------------------------------------------------------------------------
# the loss of the differentiation workload
# ---------------------------------------------------------------------------

def density(ham, Psi_occ, omega):
    """rho(r) = (1/Omega) sum_i |psi_i(r)|^2 for unit-norm coefficient vectors."""
    w = np.full(Psi_occ.shape[0], 1.0 / omega)
    return O.density_grad(Psi_occ, None, w, ham.miller, ham.box)


def target_density(ham, Y0, nocc, omega, field, amp=0.05):
    """rho_t = rho of the starting block's first nocc columns, each scaled to unit norm,
    times (1 + amp * field): the seeded target of the differentiation loss."""
    Yn = Y0[:nocc] / np.linalg.norm(Y0[:nocc], axis=1, keepdims=True)
    return density(ham, Yn, omega) * (1.0 + amp * field)


def loss(ham, lam, Psi, nocc, rho_t, omega):
    """L = sum_{i<nocc} lam_i + (Omega/n) sum_r (rho(r) - rho_t(r))^2."""
    n = float(np.prod(ham.box))
    rho = density(ham, Psi[:nocc], omega)
    return float(lam[:nocc].sum() + (omega / n) * np.sum((rho - rho_t) ** 2))


def loss_adjoint(ham, lam, Psi, nocc, rho_t, omega):
    """lambar and Psibar of the loss: lambar_i = 1 (i < nocc); Psibar_i = 4 V_{rho - rho_t} psi_i."""
    M = lam.shape[0]
    lambar = np.zeros(M)
    lambar[:nocc] = 1.0
    rho = density(ham, Psi[:nocc], omega)
    Psibar = np.zeros_like(Psi)
    Psibar[:nocc] = 4.0 * O.apply_local(rho - rho_t, ham.miller, Psi[:nocc])
    return lambar, Psibar
