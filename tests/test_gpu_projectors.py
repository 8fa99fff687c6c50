"""Explicit projectors at the C ABI (Sec. 4.2: the nonlocal operator takes the projector
functions <k+G|p_i^R> as data; Sec. 3.3 HX_SX and Sinv use the same P).

The descriptor's `proj` field replaces the generated Gaussian s/p projectors.  Checked
against the oracle built with the same P: (i) the oracle's own projector matrix passed
in explicitly, (ii) a seeded random unit-norm P with a projector count that is not a
multiple of 4 or of a GEMM tile, a dense random symmetric D and (with S) a random SPD Q.
Tolerances are those of the other parity tests: FP64 H|psi> 1e-11 relative per band,
S|psi> 1e-12, FP64 filter 1e-10; complex64 H|psi> 1e-5, mixed filter 1e-4.
"""
import numpy as np
import pytest

from oracle import pw_oracle as O
from paper_2604_11139_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2604_11139_gb300 import pwlib  # noqa: E402


def rel(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.linalg.norm(b, axis=-1)


def random_projectors(seed, npw, nproj):
    rng = np.random.default_rng(seed)
    P = rng.standard_normal((npw, nproj)) + 1j * rng.standard_normal((npw, nproj))
    return P / np.linalg.norm(P, axis=0, keepdims=True)


def random_coupling(seed, nproj, spd=False):
    rng = np.random.default_rng(seed)
    if spd:
        U, _ = np.linalg.qr(rng.standard_normal((nproj, nproj)))
        return (U * rng.uniform(0.05, 0.3, nproj)) @ U.T
    B = rng.uniform(-0.5, 0.5, (nproj, nproj))
    return 0.5 * (B + B.T)


def cases():
    out = []
    # (i) the oracle's projector matrix passed explicitly, S = I and S != I
    for with_q, kpt in ((False, [0.125, 0.375, -0.25]), (True, None)):
        prob = W.make_problem("tiny_gamma_fp64", box=(16, 16, 16), ecut=3.0, nband=7, with_q=with_q, kpt=kpt)
        m, _ = O.g_sphere(prob.lattice, prob.kpt, prob.ecut, prob.box)
        P = O.projectors(prob.lattice, prob.kpt, m, prob.tau, prob.sigmas)
        out.append((f"oracle_P_q{int(with_q)}", prob, P, prob.D, prob.Q))
    # (ii) random unit-norm P, 13 projectors, dense D, SPD Q
    for with_q in (False, True):
        prob = W.make_problem("differentiation", box=(20, 24, 30), ecut=3.0, natom=2, nband=9,
                              kpt=[0.0, 0.5, 0.25])
        m, _ = O.g_sphere(prob.lattice, prob.kpt, prob.ecut, prob.box)
        P = random_projectors(77, m.shape[0], 13)
        out.append((f"random_P13_q{int(with_q)}", prob, P, random_coupling(78, 13),
                    random_coupling(79, 13, spd=True) if with_q else None))
    return out


CASES = cases()


def oracle_for(prob, P, D, Q):
    return O.Hamiltonian(prob.lattice, prob.kpt, prob.ecut, prob.box, prob.vloc, prob.tau, prob.sigmas, D, Q, P=P)


def context_for(prob, P, D, Q):
    return pwlib.Context(prob.lattice, prob.kpt, prob.ecut, prob.box, prob.vloc, np.zeros((0, 3)), [], D, Q, P=P)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_explicit_projectors_fp64(case):
    _, prob, P, D, Q = case
    ham = oracle_for(prob, P, D, Q)
    with context_for(prob, P, D, Q) as ctx:
        assert ctx.nproj == P.shape[1] and ctx.npw == P.shape[0]
        np.testing.assert_array_equal(ctx.projectors().cpu().numpy().T, P)
        psi = W.random_block(300, ctx.npw, prob.nband)
        t = torch.from_numpy(psi).cuda()
        h, s = torch.zeros_like(t), torch.zeros_like(t)
        ctx.hamiltonian_apply(t, h, s)
        torch.cuda.synchronize()
        assert rel(h.cpu().numpy(), ham.apply_h(psi)).max() < 1e-11
        assert rel(s.cpu().numpy(), ham.apply_s(psi)).max() < 1e-12
        a, b = -0.5, 2.0 * prob.ecut + 3.0
        for degree in (1, 4):
            y = t.clone()
            ctx.chebyshev_filter(y, degree, a, b)
            torch.cuda.synchronize()
            ref = O.chebyshev_filter(ham.apply_a, psi, degree, a, b)
            assert rel(y.cpu().numpy(), ref).max() < 1e-10, degree


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_explicit_projectors_mixed(case):
    _, prob, P, D, Q = case
    ham = oracle_for(prob, P, D, Q)
    with context_for(prob, P, D, Q) as ctx:
        psi = W.random_block(301, ctx.npw, prob.nband)
        p32 = psi.astype(np.complex64).astype(np.complex128)
        t = torch.from_numpy(psi).to(torch.complex64).cuda()
        h = torch.zeros_like(t)
        ctx.hamiltonian_apply(t, h, precision=pwlib.PW_MIXED)
        torch.cuda.synchronize()
        assert rel(h.cpu().numpy().astype(np.complex128), ham.apply_h(p32)).max() < 1e-5
        a, b = 0.0, 2.0 * prob.ecut + 3.0
        ctx.chebyshev_filter(t, 5, a, b, precision=pwlib.PW_MIXED)
        torch.cuda.synchronize()
        ref = O.chebyshev_filter(ham.apply_a, p32, 5, a, b)
        assert rel(t.cpu().numpy().astype(np.complex128), ref).max() < 1e-4


def test_explicit_projectors_rayleigh_ritz():
    """Rayleigh-Ritz with the random P and Q: eigenvalues against the oracle's pencil
    reduction (one S-Ortho pass on the GPU, two in the oracle, the same span) to 1e-10 Ha."""
    _, prob, P, D, Q = CASES[3]
    ham = oracle_for(prob, P, D, Q)
    with context_for(prob, P, D, Q) as ctx:
        psi = W.random_block(302, ctx.npw, prob.nband)
        t = torch.from_numpy(psi).cuda()
        eig, _ = ctx.rayleigh_ritz(t)
        y = psi
        for _ in range(2):
            y, _ = O.s_ortho(y, ham.apply_s(y))
        lam, *_ = O.rayleigh_ritz(y, ham.apply_h(y), ham.apply_s(y))
        assert np.abs(eig - lam).max() < 1e-10
