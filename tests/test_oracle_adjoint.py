"""Pins of the oracle's reverse-mode adjoint (ChebFi cycle -> dL/dV_loc(r), dL/dD).

The adjoint is checked against central finite differences of the oracle's own forward
(which is pinned in test_oracle_pins.py), against the Hellmann-Feynman theorem at
convergence, and for the invariances that justify dropping eigenvector-coupling terms.
"""
import numpy as np
import pytest

from paper_2604_11139_gb300 import workloads as W
from oracle import pw_oracle as O
from oracle import pw_adjoint as A

H_FD = 1e-5


@pytest.fixture(scope="module")
def tiny():
    prob = W.make_problem("differentiation", box=(12, 12, 12), natom=2, ecut=1.5, nband=8)
    ham = O.Hamiltonian.from_problem(prob)
    N = ham.npw
    Y0 = W.psi0(prob.seed, N, prob.nband)
    v0 = W.lanczos_v0(prob.seed, N)
    omega = abs(np.linalg.det(prob.lattice))
    nocc, deg, cyc = 4, 4, 2
    field = W.smooth_field(prob.seed, prob.lattice, prob.box)
    rho_t = A.target_density(ham, Y0, nocc, omega, field)
    lam, Psi, tape, bounds = A.chebfi_diff_forward(ham, Y0, v0, deg, cyc)
    return dict(prob=prob, ham=ham, Y0=Y0, v0=v0, omega=omega, nocc=nocc, deg=deg, cyc=cyc,
                rho_t=rho_t, lam=lam, Psi=Psi, tape=tape, bounds=bounds)


def _loss_at(t, ham):
    lam, Psi, _, _ = A.chebfi_diff_forward(ham, t["Y0"], t["v0"], t["deg"], t["cyc"], bounds=t["bounds"])
    return A.loss(ham, lam, Psi, t["nocc"], t["rho_t"], t["omega"])


def _grads(t, split="occ"):
    ham = t["ham"]
    lb, pb = A.loss_adjoint(ham, t["lam"], t["Psi"], t["nocc"], t["rho_t"], t["omega"])
    return A.chebfi_diff_backward(ham, t["tape"], lb, pb, split=t["nocc"] if split == "occ" else split)


def _fd_v(t, idx):
    ham = t["ham"]
    ham.vloc[idx] += H_FD
    lp = _loss_at(t, ham)
    ham.vloc[idx] -= 2 * H_FD
    lm = _loss_at(t, ham)
    ham.vloc[idx] += H_FD
    return (lp - lm) / (2 * H_FD)


def _fd_d(t, a, b):
    ham = t["ham"]
    pairs = [(a, b)] if a == b else [(a, b), (b, a)]
    for p in pairs:
        ham.D[p] += H_FD
    lp = _loss_at(t, ham)
    for p in pairs:
        ham.D[p] -= 2 * H_FD
    lm = _loss_at(t, ham)
    for p in pairs:
        ham.D[p] += H_FD
    return (lp - lm) / (2 * H_FD)


def _v_points(t, count=8):
    rng = np.random.default_rng(t["prob"].seed + 5)
    box = t["ham"].box
    return [tuple(int(rng.integers(0, box[ax])) for ax in range(3)) for _ in range(count)]


D_ENTRIES = [(0, 0), (0, 1), (2, 5), (3, 3), (9, 10), (12, 15)]


def test_adjoint_dv_matches_central_differences(tiny):
    vbar, _ = _grads(tiny)
    pts = _v_points(tiny)
    fd = np.array([_fd_v(tiny, p) for p in pts])
    ad = np.array([vbar[p] for p in pts])
    assert np.abs(fd - ad).max() <= 1e-6 * np.abs(fd).max()


def test_adjoint_dd_matches_central_differences(tiny):
    _, dbar = _grads(tiny)
    fd = np.array([_fd_d(tiny, a, b) for a, b in D_ENTRIES])
    ad = np.array([dbar[a, b] + dbar[b, a] if a != b else dbar[a, a] for a, b in D_ENTRIES])
    assert np.abs(fd - ad).max() <= 1e-6 * np.abs(fd).max()


def test_dropped_pairs_are_exact(tiny):
    """Rotations among occupied (and among empty) bands leave the loss unchanged, and
    earlier cycles act through their span: dropping those coupling terms changes nothing."""
    v_occ, d_occ = _grads(tiny, split="occ")
    v_all, d_all = _grads(tiny, split=None)
    assert np.abs(v_occ - v_all).max() <= 1e-9 * np.abs(v_all).max()
    assert np.abs(d_occ - d_all).max() <= 1e-9 * np.abs(d_all).max()


def test_planted_mistake_is_caught(tiny, monkeypatch):
    """Dropping the Rayleigh-Ritz matrix's direct V/D term (a plausible slip) fails the FD pin."""
    orig = A._param_contract

    def skip_rr(ham, Z, Y, weight, vbar, dbar):
        if weight == 1.0:
            return
        orig(ham, Z, Y, weight, vbar, dbar)

    monkeypatch.setattr(A, "_param_contract", skip_rr)
    vbar, _ = _grads(tiny)
    pts = _v_points(tiny)[:3]
    fd = np.array([_fd_v(tiny, p) for p in pts])
    ad = np.array([vbar[p] for p in pts])
    assert np.abs(fd - ad).max() > 1e-3 * np.abs(fd).max()


def test_forward_replays_the_solver(tiny):
    """The taped forward is the plain ChebFi solve: same eigenvalues and cuts."""
    t = tiny
    lam, Y, res, upper, hist = O.chebfi(t["ham"], t["Y0"], t["v0"], t["deg"], t["cyc"], return_history=True)
    assert np.abs(lam - t["lam"]).max() < 1e-11
    assert abs(upper - t["bounds"][0]) < 1e-12
    assert np.allclose([h[2] for h in hist], t["bounds"][1], rtol=0, atol=1e-12)


def test_hellmann_feynman_at_convergence():
    """For converged eigenvectors d(sum_occ lambda_i)/dV(r) = (1/n) sum_occ |psi_i(r)|^2 and
    d(sum lambda)/dD_ab = sum_i Re(conj(C_ia) C_ib) (Hellmann-Feynman)."""
    prob = W.make_problem("differentiation", box=(10, 10, 10), natom=2, ecut=1.2, nband=6)
    ham = O.Hamiltonian.from_problem(prob)
    N = ham.npw
    Y0 = W.psi0(prob.seed, N, prob.nband)
    v0 = W.lanczos_v0(prob.seed, N)
    nocc = 3
    lam, Psi, tape, _ = A.chebfi_diff_forward(ham, Y0, v0, 10, 12)
    res = O.residual_norms(lam, ham.apply_h(Psi), Psi)
    assert res[:nocc].max() < 1e-9
    lb = np.zeros(prob.nband)
    lb[:nocc] = 1.0
    vbar, dbar = A.chebfi_diff_backward(ham, tape, lb, np.zeros_like(Psi))
    n = float(np.prod(ham.box))
    hf_v = O.density_grad(Psi[:nocc], None, np.full(nocc, 1.0 / n), ham.miller, ham.box)
    C = ham.project(Psi[:nocc])
    hf_d = np.real(C.conj().T @ C)
    assert np.abs(vbar - hf_v).max() <= 1e-7 * np.abs(hf_v).max()
    assert np.abs(dbar - hf_d).max() <= 1e-7 * np.abs(hf_d).max()
