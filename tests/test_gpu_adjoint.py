"""Differentiation form on the GPU (through the C ABI) against the oracle's adjoint,
against central finite differences of the GPU forward, and the c64 adjoint against the
FP64 one.

Tolerances: FP64 gradients against the oracle adjoint, 1e-8 relative in max-norm (the
adjoint divides by eigenvalue gaps and sums ~m + 1 contractions per cycle, each exact to
~1e-13); against central differences (h = 1e-5), 1e-6 relative in max-norm (the
target of the method); complex64 filter adjoint against FP64, 1e-5 relative in
max-norm (FP32 rounding of ~1e-7 per step of the recurrence and its adjoint; the
Rayleigh-Ritz adjoint, which carries most of the gradient, is FP64 in both forms;
measured 3e-8 on this case).
"""
import numpy as np
import pytest

from oracle import pw_oracle as O
from oracle import pw_adjoint as A
from paper_2604_11139_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - the marker deselects these on CPU
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2604_11139_gb300 import pwlib  # noqa: E402
from paper_2604_11139_gb300 import autograd as AG  # noqa: E402

NOCC, DEG, CYC = 6, 4, 2


@pytest.fixture(scope="module")
def case():
    prob = W.make_problem("differentiation", box=(18, 20, 24), natom=3, ecut=2.2, nband=12)
    ham = O.Hamiltonian.from_problem(prob)
    N = ham.npw
    Y0 = W.psi0(prob.seed, N, prob.nband)
    v0 = W.lanczos_v0(prob.seed, N)
    omega = abs(np.linalg.det(prob.lattice))
    field = W.smooth_field(prob.seed, prob.lattice, prob.box)
    rho_t = A.target_density(ham, Y0, NOCC, omega, field)
    lam, Psi, tape, bounds = A.chebfi_diff_forward(ham, Y0, v0, DEG, CYC)
    lb, pb = A.loss_adjoint(ham, lam, Psi, NOCC, rho_t, omega)
    vbar, dbar = A.chebfi_diff_backward(ham, tape, lb, pb, split=NOCC)
    return dict(prob=prob, ham=ham, Y0=Y0, v0=v0, omega=omega, rho_t=rho_t, lam=lam, bounds=bounds,
                vbar=vbar, dbar=dbar, field=field)


def dev(x, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dtype).cuda()


def gpu_grads(c, precision=pwlib.PW_FP64, ckpt=2, bounds=None):
    """The loss of the differentiation workload through the autograd front ends."""
    prob = c["prob"]
    ctx = pwlib.Context.from_problem(prob)
    handle = pwlib.Diff(ctx, prob.nband, DEG, CYC, ckpt=ckpt, precision=precision)
    V = torch.from_numpy(prob.vloc.copy()).cuda().requires_grad_(True)
    D = torch.from_numpy(prob.D.copy()).cuda().requires_grad_(True)
    psi0 = dev(c["Y0"])
    v0 = dev(c["v0"][None])
    eig, psi = AG.chebfi_rr(V, D, handle, psi0, v0=v0, bounds=c["bounds"] if bounds is None else bounds,
                            split=NOCC)
    rho = AG.density(psi[:NOCC], 1.0 / c["omega"], ctx)
    n = float(np.prod(prob.box))
    rho_t = torch.from_numpy(c["rho_t"]).cuda()
    L = eig[:NOCC].sum() + (c["omega"] / n) * ((rho - rho_t) ** 2).sum()
    L.backward()
    out = dict(L=float(L.detach()), eig=eig.detach().cpu().numpy(), dV=V.grad.cpu().numpy(), dD=D.grad.cpu().numpy(),
               handle=handle, ctx=ctx)
    return out


def maxrel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def test_local_apply_matches_oracle(case):
    prob, ham = case["prob"], case["ham"]
    ctx = pwlib.Context.from_problem(prob)
    v = case["field"] - 0.3
    psi = W.random_block(7, ham.npw, 5)
    ref = 1.7 * O.apply_local(v, ham.miller, psi)
    for prec, tol in ((pwlib.PW_FP64, 1e-11), (pwlib.PW_MIXED, 2e-5)):
        dt = torch.complex128 if prec == pwlib.PW_FP64 else torch.complex64
        out = ctx.local_apply(torch.from_numpy(v).cuda(), dev(psi, dt), alpha=1.7, precision=prec)
        got = out.cpu().numpy().astype(np.complex128)
        assert (np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)).max() < tol


def test_set_parameters_match_oracle(case):
    prob, ham = case["prob"], case["ham"]
    ctx = pwlib.Context.from_problem(prob)
    V2 = prob.vloc * 0.8 + 0.05 * case["field"]
    D2 = prob.D * 1.3
    ctx.set_vloc(torch.from_numpy(V2).cuda())
    ctx.set_D(D2)
    ham2 = O.Hamiltonian(prob.lattice, prob.kpt, prob.ecut, prob.box, V2, prob.tau, prob.sigmas, D2)
    psi = W.random_block(9, ham.npw, 4)
    h = torch.zeros((4, ham.npw), dtype=torch.complex128, device="cuda")
    ctx.hamiltonian_apply(dev(psi), h)
    ref = ham2.apply_h(psi)
    assert (np.linalg.norm(h.cpu().numpy() - ref, axis=1) / np.linalg.norm(ref, axis=1)).max() < 1e-11
    bad = D2.copy()
    bad[0, 9] = bad[9, 0] = 0.1      # couples two atoms' blocks
    with pytest.raises(pwlib.PWError):
        ctx.set_D(bad)


def test_forward_matches_oracle_and_solver(case):
    prob = case["prob"]
    ctx = pwlib.Context.from_problem(prob)
    handle = pwlib.Diff(ctx, prob.nband, DEG, CYC)
    psi = dev(case["Y0"])
    eig, bnd = handle.forward(psi, v0=dev(case["v0"][None]), lanczos_steps=10)
    assert abs(bnd[0] - case["bounds"][0]) < 1e-9
    assert np.abs(bnd[1:] - np.asarray(case["bounds"][1])).max() < 1e-9
    assert np.abs(eig - case["lam"]).max() < 1e-10
    psi2 = dev(case["Y0"])
    eig2, _, _ = ctx.chebfi_solve(psi2, DEG, CYC, dev(case["v0"][None]))
    assert np.abs(eig - eig2).max() < 1e-12


def test_adjoint_fp64_matches_oracle(case):
    g = gpu_grads(case)
    assert maxrel(g["dV"], case["vbar"]) < 1e-8
    assert maxrel(g["dD"], case["dbar"]) < 1e-8


def test_adjoint_fp64_matches_central_differences(case):
    prob = case["prob"]
    g = gpu_grads(case)
    ctx, handle = g["ctx"], g["handle"]
    # The central differences of the forward use the DFMA GEMMs: the digit-sliced tensor-core
    # GEMMs (the default FP64 form, error ~2^-44 of the row and column maxima per product) do
    # not vary smoothly at the 1e-15 level, and a step h = 1e-5 at one grid point divides that
    # noise by h.  The gradient under test above was computed with the default GEMMs.
    ctx.fp64_config(0)
    rng = np.random.default_rng(prob.seed + 11)
    n = float(np.prod(prob.box))
    rho_t = torch.from_numpy(case["rho_t"]).cuda()
    h = 1e-5

    def loss(V, D):
        ctx.set_vloc(V)
        ctx.set_D(D)
        psi = dev(case["Y0"])
        eig, _ = handle.forward(psi, bounds=case["bounds"])
        rho = ctx.density_grad(psi[:NOCC], [1.0 / case["omega"]] * NOCC)
        return eig[:NOCC].sum() + (case["omega"] / n) * float(((rho - rho_t) ** 2).sum())

    pts = [tuple(int(rng.integers(0, prob.box[a])) for a in range(3)) for _ in range(8)]
    fd, ad = [], []
    for p in pts:
        Vp, Vm = prob.vloc.copy(), prob.vloc.copy()
        Vp[p] += h
        Vm[p] -= h
        fd.append((loss(Vp, prob.D) - loss(Vm, prob.D)) / (2 * h))
        ad.append(g["dV"][p])
    assert maxrel(np.array(ad), np.array(fd)) < 1e-6
    fd, ad = [], []
    for a, b in [(0, 0), (1, 2), (5, 7), (8, 8), (10, 13), (17, 22)]:
        Dp, Dm = prob.D.copy(), prob.D.copy()
        for (i, j) in {(a, b), (b, a)}:
            Dp[i, j] += h
            Dm[i, j] -= h
        fd.append((loss(prob.vloc, Dp) - loss(prob.vloc, Dm)) / (2 * h))
        ad.append(g["dD"][a, b] + (g["dD"][b, a] if a != b else 0.0))
    assert maxrel(np.array(ad), np.array(fd)) < 1e-6


@pytest.mark.parametrize("ckpt", [1, 3, DEG])
def test_checkpointing_gives_the_same_gradients(case, ckpt):
    ref = gpu_grads(case, ckpt=2)
    g = gpu_grads(case, ckpt=ckpt)
    assert maxrel(g["dV"], ref["dV"]) < 1e-13
    assert maxrel(g["dD"], ref["dD"]) < 1e-13
    if ckpt > 2:
        assert g["handle"].tape_bytes() < ref["handle"].tape_bytes()


def test_adjoint_c64_against_fp64(case):
    g64 = gpu_grads(case)
    g32 = gpu_grads(case, precision=pwlib.PW_MIXED)
    e_v, e_d = maxrel(g32["dV"], g64["dV"]), maxrel(g32["dD"], g64["dD"])
    print(f"c64 adjoint vs FP64: dV {e_v:.2e}, dD {e_d:.2e}")
    assert e_v < 1e-5 and e_d < 1e-5


def test_errors(case):
    prob = case["prob"]
    ctx = pwlib.Context.from_problem(prob)
    handle = pwlib.Diff(ctx, prob.nband, DEG, CYC)
    with pytest.raises(pwlib.PWError):
        handle.backward(eig_bar=np.ones(prob.nband))          # no tape yet
    psi = dev(case["Y0"])
    handle.forward(psi, bounds=case["bounds"])
    ctx.set_vloc(prob.vloc)                                   # parameters replaced after the forward
    with pytest.raises(pwlib.PWError):
        handle.backward(eig_bar=np.ones(prob.nband))
    with pytest.raises(pwlib.PWError):
        handle.forward(psi, bounds=[1.0] + [2.0] * CYC)       # upper below the cut
    pq = W.make_problem("differentiation", box=(18, 20, 24), natom=3, ecut=2.2, nband=12, with_q=True)
    cq = pwlib.Context.from_problem(pq)
    with pytest.raises(pwlib.PWError):
        pwlib.Diff(cq, 4, DEG, CYC)


def test_full_size_differentiation_workload():
    """The differentiation workload at full size (64^3 box, 16 atoms / 128 projectors, 128
    bands of which 64 occupied, degree 10, 3 cycles): the FP64 adjoint against central
    differences of the FP64 forward at 32 seeded grid points and 16 entries of the D blocks,
    and the complex64 adjoint against the FP64 one."""
    prob = W.make_problem("differentiation")
    M, m, C, nocc = prob.nband, prob.degree, prob.cycles, 64
    ctx = pwlib.Context.from_problem(prob)
    omega = abs(float(np.linalg.det(prob.lattice)))
    n = float(np.prod(prob.box))
    y0 = dev(W.psi0(prob.seed, ctx.npw, M))
    v0 = dev(W.lanczos_v0(prob.seed, ctx.npw)[None])
    yn = y0[:nocc] / torch.linalg.vector_norm(y0[:nocc], dim=1, keepdim=True)
    field = torch.from_numpy(W.smooth_field(prob.seed, prob.lattice, prob.box)).cuda()
    rho_t = (AG.density(yn, 1.0 / omega, ctx) * (1.0 + 0.05 * field)).detach()
    h64 = pwlib.Diff(ctx, M, m, C, ckpt=2, precision=pwlib.PW_FP64)
    bounds = h64.forward(y0.clone(), v0=v0)[1]

    def grads(handle):
        V = torch.from_numpy(prob.vloc.copy()).cuda().requires_grad_(True)
        D = torch.from_numpy(prob.D.copy()).cuda().requires_grad_(True)
        eig, psi = AG.chebfi_rr(V, D, handle, y0, bounds=bounds, split=nocc)
        rho = AG.density(psi[:nocc], 1.0 / omega, ctx)
        L = eig[:nocc].sum() + (omega / n) * ((rho - rho_t) ** 2).sum()
        L.backward()
        return V.grad.cpu().numpy(), D.grad.cpu().numpy()

    gV, gD = grads(h64)
    ctx.fp64_config(0)   # central differences of the DFMA forward (see the small-box test)

    def loss(V, D):
        ctx.set_vloc(V)
        ctx.set_D(D)
        psi = y0.clone()
        eig, _ = h64.forward(psi, bounds=bounds)
        rho = ctx.density_grad(psi[:nocc], [1.0 / omega] * nocc)
        return eig[:nocc].sum() + (omega / n) * float(((rho - rho_t) ** 2).sum())

    # Central-difference steps: a step h in V(r_j) at one grid point moves H by only
    # h / (n1 n2 n3) = h / 262144, so with h = 1e-5 the change of L (~1e-9) is within a few
    # thousand roundings of L itself (measured FD error 2.8e-6 there); h_V = 1e-3 keeps the
    # operator step (4e-9) well below D's (1e-5) while the truncation error, of order
    # (h/n)^2, stays negligible.
    h, hv = 1e-5, 1e-3
    rng = np.random.default_rng(prob.seed + 23)
    fd, ad = [], []
    for _ in range(32):
        p = tuple(int(rng.integers(0, prob.box[a])) for a in range(3))
        Vp, Vm = prob.vloc.copy(), prob.vloc.copy()
        Vp[p] += hv
        Vm[p] -= hv
        fd.append((loss(Vp, prob.D) - loss(Vm, prob.D)) / (2 * hv))
        ad.append(gV[p])
    err_v = maxrel(np.array(ad), np.array(fd))
    fd, ad = [], []
    blk = 4 * len(prob.sigmas)
    for _ in range(16):
        at = int(rng.integers(0, prob.natom))
        a, b = (at * blk + int(x) for x in rng.integers(0, blk, 2))
        Dp, Dm = prob.D.copy(), prob.D.copy()
        for (i, j) in {(a, b), (b, a)}:
            Dp[i, j] += h
            Dm[i, j] -= h
        fd.append((loss(prob.vloc, Dp) - loss(prob.vloc, Dm)) / (2 * h))
        ad.append(gD[a, b] + (gD[b, a] if a != b else 0.0))
    err_d = maxrel(np.array(ad), np.array(fd))
    ctx.set_vloc(prob.vloc)
    ctx.set_D(prob.D)
    ctx.fp64_config(1)
    h32 = pwlib.Diff(ctx, M, m, C, ckpt=2, precision=pwlib.PW_MIXED)
    gV32, gD32 = grads(h32)
    e32v, e32d = maxrel(gV32, gV), maxrel(gD32, gD)
    print(f"full size: FD dV {err_v:.2e}, FD dD {err_d:.2e}; c64 vs FP64 dV {e32v:.2e}, dD {e32d:.2e}")
    assert err_v < 1e-6 and err_d < 1e-6
    assert e32v < 1e-5 and e32d < 1e-5
