"""Parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (FP64 path, from the target of the method): H|psi> relative 1e-11 per
band; eigenvalues 1e-10 Ha.  Mixed precision (complex64 FFT, FP32 accumulation):
relative 1e-5 per band on H|psi> (FP32 rounding of ~1e-7 per operation over a few
hundred accumulated terms).
"""
import numpy as np
import pytest

from oracle import pw_oracle as O
from paper_2604_11139_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - the marker deselects these on CPU
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2604_11139_gb300 import pwlib  # noqa: E402

SMALL = {
    "cubic16_q": dict(name="tiny_gamma_fp64", box=(16, 16, 16), ecut=3.0, nband=7, with_q=True),
    "ortho_k_ragged": dict(name="batched_kpoints", box=(18, 18, 20), ecut=2.5, natom=3, nband=5,
                           kpt=[0.125, 0.375, -0.25]),
    "box_2_3_5": dict(name="differentiation", box=(20, 24, 30), ecut=3.0, natom=4, nband=9, with_q=True,
                      kpt=[0.0, 0.5, 0.25]),
    "tiny_24_aliasing": dict(name="tiny_gamma_fp64", nband=16),
    # radix plans 8 x 8 (64) and 16 x 8 (128): line groups of 8 threads
    "box_64_tl8": dict(name="differentiation", box=(64, 64, 64), ecut=1.5, natom=2, nband=6),
    "box_128_x": dict(name="differentiation", box=(128, 20, 64), ecut=1.5, natom=2, nband=5,
                      kpt=[0.25, 0.0, 0.5]),
}


def make(key):
    kw = dict(SMALL[key])
    name = kw.pop("name")
    return W.make_problem(name, **kw)


_cache = {}


def setup(key):
    if key not in _cache:
        prob = make(key)
        _cache[key] = (prob, O.Hamiltonian.from_problem(prob))
    prob, ham = _cache[key]
    return prob, ham, pwlib.Context.from_problem(prob)


def to_dev(x, dtype=torch.complex128, ld=None):
    x = np.asarray(x)
    m, n = x.shape
    ld = n if ld is None else ld
    buf = torch.zeros((m, ld), dtype=dtype, device="cuda")
    buf[:, :n] = torch.from_numpy(x).to(dtype)
    return buf


def rel(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.linalg.norm(b, axis=-1)


@pytest.mark.parametrize("key", list(SMALL))
def test_sphere_and_projectors_match_oracle(key):
    prob, ham, ctx = setup(key)
    with ctx:
        m, kin = ctx.gvectors()
        np.testing.assert_array_equal(m, ham.miller)
        np.testing.assert_allclose(kin, ham.kin, rtol=1e-14, atol=1e-14)
        assert ctx.nproj == ham.P.shape[1]
        P = ctx.projectors().cpu().numpy().T
        np.testing.assert_allclose(P, ham.P, atol=1e-13)


@pytest.mark.parametrize("key", list(SMALL))
def test_hamiltonian_apply_fp64(key):
    prob, ham, ctx = setup(key)
    with ctx:
        psi = W.random_block(100, ctx.npw, prob.nband)
        t = to_dev(psi, ld=ctx.npw + 3)      # ragged leading dimension
        h = torch.zeros_like(t)
        s = torch.zeros_like(t)
        ctx.hamiltonian_apply(t, h, s)
        torch.cuda.synchronize()
        assert rel(h.cpu().numpy()[:, :ctx.npw], ham.apply_h(psi)).max() < 1e-11
        assert rel(s.cpu().numpy()[:, :ctx.npw], ham.apply_s(psi)).max() < 1e-12
        # padding beyond npw untouched
        assert torch.count_nonzero(h[:, ctx.npw:]) == 0


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 16, 19, 32, 35, 36, 38, 39, 40, 41, 42, 48, 51, 52, 54, 55, 58, 67, 71, 83, 87, 99, 103])
@pytest.mark.parametrize("key", ["cubic16_q", "ortho_k_ragged", "tiny_24_aliasing", "box_64_tl8"])
def test_hamiltonian_apply_mixed(key, variant):
    """The complex64 FFT pass kernel forms (variant = x-line form + 16 * plane form: line
    groups; one thread per line; warp groups with compile-time or table twiddles), the
    non-zero forms used where the box lengths have two-stage radix plans (the 24^3 and 64^3
    cases)."""
    prob, ham, ctx = setup(key)
    with ctx:
        ctx.fft_config(pwlib.PW_MIXED, variant=variant)
        psi = W.random_block(101, ctx.npw, prob.nband)
        t = to_dev(psi, torch.complex64)
        h = torch.zeros_like(t)
        ctx.hamiltonian_apply(t, h, precision=pwlib.PW_MIXED)
        torch.cuda.synchronize()
        ref = ham.apply_h(psi.astype(np.complex64).astype(np.complex128))
        assert rel(h.cpu().numpy().astype(np.complex128), ref).max() < 1e-5


@pytest.mark.parametrize("key", list(SMALL))
def test_filter_fp64(key):
    prob, ham, ctx = setup(key)
    with ctx:
        psi = W.random_block(102, ctx.npw, prob.nband)
        H, S = (None, None)
        a, b = -0.5, 2.0 * prob.ecut + 3.0
        for degree in (1, 2, 3, 5):
            t = to_dev(psi, ld=ctx.npw + 1)
            ctx.chebyshev_filter(t, degree, a, b)
            torch.cuda.synchronize()
            ref = O.chebyshev_filter(ham.apply_a, psi, degree, a, b)
            assert rel(t.cpu().numpy()[:, :ctx.npw], ref).max() < 1e-10, degree


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 16, 19, 32, 35, 36, 38, 39, 40, 41, 42, 48, 51, 52, 54, 55, 58, 67, 71, 83, 87, 99, 103])
@pytest.mark.parametrize("key", ["cubic16_q", "tiny_24_aliasing", "box_64_tl8"])
def test_filter_mixed(key, variant):
    prob, ham, ctx = setup(key)
    with ctx:
        ctx.fft_config(pwlib.PW_MIXED, variant=variant)
        psi = W.random_block(103, ctx.npw, prob.nband)
        a, b = 0.0, 2.0 * prob.ecut + 3.0
        t = to_dev(psi, torch.complex64)
        ctx.chebyshev_filter(t, 6, a, b, precision=pwlib.PW_MIXED)
        torch.cuda.synchronize()
        ref = O.chebyshev_filter(ham.apply_a, psi.astype(np.complex64).astype(np.complex128), 6, a, b)
        assert rel(t.cpu().numpy().astype(np.complex128), ref).max() < 1e-4


@pytest.mark.parametrize("key", list(SMALL))
def test_rayleigh_ritz(key):
    prob, ham, ctx = setup(key)
    with ctx:
        psi = W.random_block(104, ctx.npw, prob.nband)
        t = to_dev(psi)
        hp = torch.zeros_like(t)
        eig, res = ctx.rayleigh_ritz(t, hp)
        y = psi
        for _ in range(2):
            y, _ = O.s_ortho(y, ham.apply_s(y))
        lam, Yr, HYr, SYr, _ = O.rayleigh_ritz(y, ham.apply_h(y), ham.apply_s(y))
        np.testing.assert_allclose(eig, lam, atol=1e-10, rtol=0)
        np.testing.assert_allclose(res, O.residual_norms(lam, HYr, SYr), atol=1e-9, rtol=1e-8)
        Y = t.cpu().numpy()
        # Ritz vectors are S-orthonormal and reproduce the eigenvalues; H psi output is H of them
        np.testing.assert_allclose(Y.conj() @ ham.apply_s(Y).T, np.eye(prob.nband), atol=1e-11)
        np.testing.assert_allclose(np.real(np.einsum("ij,ij->i", Y.conj(), ham.apply_h(Y))), eig, atol=1e-10)
        assert rel(hp.cpu().numpy(), ham.apply_h(Y)).max() < 1e-11


@pytest.mark.parametrize("key", ["cubic16_q", "ortho_k_ragged"])
def test_spectrum_bounds(key):
    prob, ham, ctx = setup(key)
    with ctx:
        psi = W.random_block(105, ctx.npw, prob.nband)
        v0 = W.lanczos_v0(prob.seed, ctx.npw)
        lo, hi, up = ctx.spectrum_bounds(to_dev(psi), 10, to_dev(v0[None]))
        rq = O.rayleigh_quotients(psi, ham.apply_h(psi), ham.apply_s(psi))
        np.testing.assert_allclose([lo, hi], [rq.min(), rq.max()], rtol=1e-12)
        ref_up, _ = O.lanczos_upper(ham.apply_h, v0, 10)
        np.testing.assert_allclose(up, ref_up, rtol=1e-10)


@pytest.mark.parametrize("key", ["cubic16_q", "tiny_24_aliasing"])
def test_chebfi_solve_fp64_matches_oracle(key):
    prob, ham, ctx = setup(key)
    cycles = 4
    with ctx:
        psi0 = W.psi0(prob.seed, ctx.npw, prob.nband)
        v0 = W.lanczos_v0(prob.seed, ctx.npw)
        t = to_dev(psi0)
        eig, res, bnd = ctx.chebfi_solve(t, prob.degree, cycles, to_dev(v0[None]))
        lam, Y, rr, up = O.chebfi(ham, psi0, v0, prob.degree, cycles)
        np.testing.assert_allclose(bnd[0], up, rtol=1e-10)
        np.testing.assert_allclose(eig, lam, atol=1e-10, rtol=0)


@pytest.mark.parametrize("pieces", [3, 2])
def test_chebfi_solve_mixed_close_to_fp64(pieces):
    """Mixed-precision ChebFi within 1e-6 Ha of FP64, with 3 and with 2 bf16 pieces per
    GEMM operand."""
    prob, ham, ctx = setup("tiny_24_aliasing")
    with ctx:
        ctx.tc_config(pieces)
        psi0 = W.psi0(prob.seed, ctx.npw, prob.nband)
        v0 = to_dev(W.lanczos_v0(prob.seed, ctx.npw)[None])
        e64, _, _ = ctx.chebfi_solve(to_dev(psi0), prob.degree, prob.cycles, v0)
        emx, _, _ = ctx.chebfi_solve(to_dev(psi0), prob.degree, prob.cycles, v0, precision=pwlib.PW_MIXED)
        assert np.abs(emx - e64).max() < 1e-6


@pytest.mark.parametrize("key", ["ortho_k_ragged", "box_2_3_5", "tiny_24_aliasing", "box_64_tl8"])
def test_density_grad(key):
    prob, ham, ctx = setup(key)
    with ctx:
        a = W.random_block(106, ctx.npw, prob.nband)
        b = W.random_block(107, ctx.npw, prob.nband)
        w = np.linspace(0.5, 2.0, prob.nband)
        g1 = ctx.density_grad(to_dev(a), w).cpu().numpy()
        r1 = O.density_grad(a, None, w, ham.miller, prob.box)
        np.testing.assert_allclose(g1, r1, rtol=0, atol=1e-12 * np.abs(r1).max())
        g2 = ctx.density_grad(to_dev(a), w, b=to_dev(b)).cpu().numpy()
        r2 = O.density_grad(a, b, w, ham.miller, prob.box)
        np.testing.assert_allclose(g2, r2, rtol=0, atol=1e-12 * np.abs(r2).max())
        out = torch.from_numpy(g1).cuda()
        ctx.density_grad(to_dev(a), w, out=out, accumulate=True)
        np.testing.assert_allclose(out.cpu().numpy(), 2 * r1, rtol=0, atol=1e-12 * np.abs(r1).max())


# ---------------------------------------------------------------------------- edge cases

def test_edge_cases_and_errors():
    prob, ham, ctx = setup("cubic16_q")
    with ctx:
        # zero bands: a no-op that succeeds
        t = torch.zeros((1, ctx.npw), dtype=torch.complex128, device="cuda")
        lib = pwlib.load()
        assert lib.pw_hamiltonian_apply(ctx._h, None, ctx.npw, 0, None, None, ctx.npw, 0) == 0
        assert lib.pw_chebyshev_filter(ctx._h, None, ctx.npw, 0, 4, 0.0, 1.0, 0) == 0
        # ld < npw
        assert lib.pw_hamiltonian_apply(ctx._h, t.data_ptr(), ctx.npw - 1, 1, t.data_ptr(), None, ctx.npw, 0) == -1
        # aliasing input/output
        assert lib.pw_hamiltonian_apply(ctx._h, t.data_ptr(), ctx.npw, 1, t.data_ptr(), None, ctx.npw, 0) == -1
        # degenerate filter interval
        with pytest.raises(pwlib.PWError):
            ctx.chebyshev_filter(t, 3, 2.0, 1.0)
        # single band
        psi = W.random_block(108, ctx.npw, 1)
        h = torch.zeros_like(t)
        ctx.hamiltonian_apply(to_dev(psi), h)
        torch.cuda.synchronize()
        assert rel(h.cpu().numpy(), ham.apply_h(psi)).max() < 1e-11
    # FFT length with a factor 7
    p = W.make_problem("tiny_gamma_fp64", box=(14, 16, 16), ecut=1.0)
    with pytest.raises(pwlib.PWError) as e:
        pwlib.Context.from_problem(p)
    assert e.value.status == -7
    # sphere larger than the box
    p = W.make_problem("tiny_gamma_fp64", box=(12, 12, 12), ecut=7.6)
    with pytest.raises(pwlib.PWError) as e:
        pwlib.Context.from_problem(p)
    assert e.value.status == -1
    # overlap coefficients that are not positive definite
    p = W.make_problem("tiny_gamma_fp64", box=(16, 16, 16), ecut=3.0, with_q=True)
    p.Q = -p.Q
    with pytest.raises(pwlib.PWError) as e:
        pwlib.Context.from_problem(p)
    assert e.value.status == -4


# ------------------------------------------------------------- full-size sampled parity

def test_full_size_fp64_at_scale_sampled_bands():
    """96^3 box, ~55k plane waves, 512 projectors: 3 sampled bands against the oracle."""
    prob = W.make_problem("fp64_at_scale")
    ham = O.Hamiltonian.from_problem(prob)
    with pwlib.Context.from_problem(prob) as ctx:
        assert ctx.npw == ham.npw and 50000 < ctx.npw < 60000 and ctx.nproj == 512
        psi = W.psi0(prob.seed, ctx.npw, 3)
        t = to_dev(psi, ld=ctx.npw + 7)
        h = torch.zeros_like(t)
        ctx.hamiltonian_apply(t, h)
        torch.cuda.synchronize()
        ref = ham.apply_h(psi)
        assert rel(h.cpu().numpy()[:, :ctx.npw], ref).max() < 1e-11
        ctx.fft_config(pwlib.PW_FP64, variant=48)   # complex128 row-slice plane kernels
        h.zero_()
        ctx.hamiltonian_apply(t, h)
        torch.cuda.synchronize()
        assert rel(h.cpu().numpy()[:, :ctx.npw], ref).max() < 1e-11
        ctx.fft_config(pwlib.PW_FP64, variant=0)
        for variant in (0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 16, 19, 32, 35, 36, 38, 39, 40, 41, 42, 48, 51, 52, 54, 55, 58, 67, 71, 83, 87, 99, 103):
            ctx.fft_config(pwlib.PW_MIXED, variant=variant)
            t32 = to_dev(psi, torch.complex64)
            h32 = torch.zeros_like(t32)
            ctx.hamiltonian_apply(t32, h32, precision=pwlib.PW_MIXED)
            torch.cuda.synchronize()
            assert rel(h32.cpu().numpy().astype(np.complex128), ref).max() < 1e-5


FULL_SIZE = {
    "differentiation_64": dict(name="differentiation"),
    "batched_kpoints_72x72x90": dict(name="batched_kpoints", kpt_index=5),
    "paw_precision_120": dict(name="paw_precision"),
}


@pytest.mark.parametrize("key", list(FULL_SIZE))
def test_full_size_other_boxes_sampled_bands(key):
    """The full-size boxes of the other workloads (64^3: radix plan 8 x 8; 72 x 72 x 90:
    9 x 8 and 10 x 9; 120^3: 12 x 10, with Q): 2 sampled bands of H psi (and S psi) against
    the oracle, FP64 and mixed."""
    kw = dict(FULL_SIZE[key])
    prob = W.make_problem(kw.pop("name"))
    kpt, ecut = None, None
    if "kpt_index" in kw:
        i = kw.pop("kpt_index")
        kpt = W.mp_kpoints()[i]
        ecut = W.ecut_jitter(prob.seed, len(W.mp_kpoints()), prob.ecut)[i]
    ham = O.Hamiltonian.from_problem(prob, kpt=kpt, ecut=ecut)
    with pwlib.Context.from_problem(prob, kpt=kpt, ecut=ecut) as ctx:
        assert ctx.npw == ham.npw
        psi = W.psi0(prob.seed, ctx.npw, 2)
        t = to_dev(psi, ld=ctx.npw + 5)
        h = torch.zeros_like(t)
        sp = torch.zeros_like(t) if prob.Q is not None else None
        ctx.hamiltonian_apply(t, h, sp)
        torch.cuda.synchronize()
        ref = ham.apply_h(psi)
        err = rel(h.cpu().numpy()[:, :ctx.npw], ref).max()
        print(f"{key}: H psi FP64 rel err {err:.2e}")
        assert err < 1e-11
        ctx.fft_config(pwlib.PW_FP64, variant=48)   # complex128 row-slice plane kernels
        h48 = torch.zeros_like(t)
        ctx.hamiltonian_apply(t, h48)
        torch.cuda.synchronize()
        assert rel(h48.cpu().numpy()[:, :ctx.npw], ref).max() < 1e-11
        ctx.fft_config(pwlib.PW_FP64, variant=0)
        if sp is not None:
            assert rel(sp.cpu().numpy()[:, :ctx.npw], ham.apply_s(psi)).max() < 1e-12
        for variant in (0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 16, 19, 32, 35, 36, 38, 39, 40, 41, 42, 48, 51, 52, 54, 55, 58, 67, 71, 83, 87, 99, 103):
            ctx.fft_config(pwlib.PW_MIXED, variant=variant)
            t32 = to_dev(psi, torch.complex64)
            h32 = torch.zeros_like(t32)
            ctx.hamiltonian_apply(t32, h32, precision=pwlib.PW_MIXED)
            torch.cuda.synchronize()
            assert rel(h32.cpu().numpy().astype(np.complex128), ref).max() < 1e-5


@pytest.mark.parametrize("key", ["cubic16_q", "ortho_k_ragged"])
def test_few_bands_matrix_vector_forms(key):
    """1-4 bands take the matrix-vector forms of the projector products (P^dagger psi reads P
    once per column, P Z one row per thread, the recurrence epilogue included); 5 bands the
    tiled GEMM."""
    prob, ham, ctx = setup(key)
    with ctx:
        a, b = -0.5, 2.0 * prob.ecut + 3.0
        for nb in (1, 2, 3, 4, 5):
            psi = W.random_block(110 + nb, ctx.npw, nb)
            t = to_dev(psi, ld=ctx.npw + 2)
            h = torch.zeros_like(t)
            ctx.hamiltonian_apply(t, h)
            torch.cuda.synchronize()
            assert rel(h.cpu().numpy()[:, :ctx.npw], ham.apply_h(psi)).max() < 1e-11, nb
            ctx.chebyshev_filter(t, 3, a, b)
            torch.cuda.synchronize()
            ref = O.chebyshev_filter(ham.apply_a, psi, 3, a, b)
            assert rel(t.cpu().numpy()[:, :ctx.npw], ref).max() < 1e-10, nb


def test_rayleigh_ritz_ill_conditioned_block():
    """Columns scaled over four decades and mixed (condition number ~1e4, as after a filter):
    the Ritz values of the span do not depend on the basis, and the single Cholesky-QR pass
    before the Rayleigh-Ritz reduction keeps them at the FP64 level."""
    prob, ham, ctx = setup("tiny_24_aliasing")
    with ctx:
        psi = W.random_block(120, ctx.npw, prob.nband)
        mix = np.linalg.qr(W.random_block(121, prob.nband, prob.nband))[0]
        Y = (psi.T @ np.diag(np.geomspace(1.0, 1e-4, prob.nband)) @ mix).T
        t = to_dev(Y)
        eig, _ = ctx.rayleigh_ritz(t)
        y = psi
        for _ in range(2):
            y, _ = O.s_ortho(y, ham.apply_s(y))
        lam, *_ = O.rayleigh_ritz(y, ham.apply_h(y), ham.apply_s(y))
        np.testing.assert_allclose(eig, lam, atol=1e-9, rtol=0)
        R = t.cpu().numpy()
        np.testing.assert_allclose(R.conj() @ R.T, np.eye(prob.nband), atol=1e-11)


def test_rayleigh_ritz_many_bands():
    """Jacobi eigensolver on a 200 x 200 reduced problem (odd pairing rounds, many sweeps)."""
    prob = W.make_problem("tiny_gamma_fp64", nband=200)
    ham = O.Hamiltonian.from_problem(prob)
    with pwlib.Context.from_problem(prob) as ctx:
        psi = W.random_block(109, ctx.npw, 199)   # odd band count: one idle slot per pairing round
        t = to_dev(psi)
        eig, res = ctx.rayleigh_ritz(t)
        y = psi
        for _ in range(2):
            y, _ = O.s_ortho(y, ham.apply_s(y))
        lam, *_ = O.rayleigh_ritz(y, ham.apply_h(y), ham.apply_s(y))
        np.testing.assert_allclose(eig, lam, atol=1e-10, rtol=0)


@pytest.mark.parametrize("key", ["cubic16_q", "box_2_3_5", "tiny_24_aliasing"])
def test_fp64_digit_gemms_agree_with_dfma(key):
    """The FP64 GEMMs in their two forms (digit-sliced tensor-core GEMMs, the default, and
    DFMA): H|psi>, S|psi>, the filter and the Ritz values agree far below the oracle
    tolerances (error of a digit-sliced product below 2^-44 of the row and column maxima)."""
    prob, ham, ctx = setup(key)
    with ctx:
        psi = W.random_block(150, ctx.npw, prob.nband)
        out = {}
        for mode in (1, 0):
            ctx.fp64_config(mode)
            t = to_dev(psi)
            h, s = torch.zeros_like(t), torch.zeros_like(t)
            ctx.hamiltonian_apply(t, h, s)
            y = t.clone()
            ctx.chebyshev_filter(y, 5, -0.5, 2.0 * prob.ecut + 3.0)
            eig, _ = ctx.rayleigh_ritz(y)
            out[mode] = (h.cpu().numpy(), s.cpu().numpy(), y.cpu().numpy(), eig)
        assert ctx.fp64_config() == 0
        assert rel(out[1][0], out[0][0]).max() < 1e-13
        assert rel(out[1][1], out[0][1]).max() < 1e-13
        assert np.abs(out[1][3] - out[0][3]).max() < 1e-12


def test_fft_config_accepts_the_documented_forms_only():
    """complex64: x-line forms 0-10, plane forms 0-6 (variant = x + 16 p); complex128: plane
    forms 0 and 3 only (variants 0 and 48); everything else PW_EINVAL."""
    prob = W.make_problem("tiny_gamma_fp64", box=(16, 16, 16), ecut=3.0, nband=4)
    with pwlib.Context.from_problem(prob) as ctx:
        for v in (0, 10, 16, 48, 64, 74, 80, 90, 96, 106):
            assert ctx.fft_config(pwlib.PW_MIXED, variant=v)[1] == v
        for v in (11, 15, 107, 112):
            with pytest.raises(pwlib.PWError):
                ctx.fft_config(pwlib.PW_MIXED, variant=v)
        for v in (0, 48):
            assert ctx.fft_config(pwlib.PW_FP64, variant=v)[1] == v
        for v in (3, 32, 64):
            with pytest.raises(pwlib.PWError):
                ctx.fft_config(pwlib.PW_FP64, variant=v)
