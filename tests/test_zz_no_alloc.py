"""The allocation-free H-apply entry point (pw_hamiltonian_apply_noalloc).

It serves callers that must not allocate device memory when they apply H (their
framework's allocator owns the device, a memory cap, or a loop that cannot take
cudaFree's synchronisation).  Checked against pw_hamiltonian_apply on the same
inputs, on two calls in a row (the static scratch keeps the previous call's
contents), to the FP64 tolerance of the other parity tests (1e-11 relative per
band).  This file sorts last so that a stop-at-first-failure run has run every
other test before it.
"""
import numpy as np
import pytest

from paper_2604_11139_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2604_11139_gb300 import pwlib  # noqa: E402


def rel(a, b):
    return (torch.linalg.vector_norm(a - b, dim=1) / torch.linalg.vector_norm(b, dim=1)).max().item()


# tiny: one chunk; 96^3: chunks of 4 bands (matrix-vector GEMM forms); 64^3 with 40 bands:
# chunks of 17, 17 and 6 bands, so the tiled split-K GEMM reuses the partials and the C/Z
# regions of the scratch from one chunk to the next
@pytest.mark.parametrize("kw", [dict(name="tiny_gamma_fp64", nband=16),
                                dict(name="fp64_at_scale", nband=24),
                                dict(name="differentiation", nband=40)])
def test_noalloc_matches_hamiltonian_apply_twice(kw):
    kw = dict(kw)
    prob = W.make_problem(kw.pop("name"), **kw)
    with pwlib.Context.from_problem(prob) as ctx:
        for call, seed in enumerate((201, 202)):
            psi = torch.from_numpy(W.random_block(seed, ctx.npw, prob.nband)).cuda()
            ref = torch.zeros_like(psi)
            ctx.hamiltonian_apply(psi, ref)
            out = torch.full_like(psi, complex(np.nan, np.nan))
            ctx.hamiltonian_apply_noalloc(psi, out)
            torch.cuda.synchronize()
            assert rel(out, ref) < 1e-11, call


def test_noalloc_rejects_a_box_beyond_the_static_scratch():
    # 180^3 box, sphere of radius 40 grid units (81 x-planes): one band's half-box
    # planes alone take 81 * 180 * 180 * 16 bytes = 42 MB > 32 MiB
    prob = W.make_problem("tiny_gamma_fp64", box=(180, 180, 180), ecut=316.0, natom=1, nband=1)
    with pwlib.Context.from_problem(prob) as ctx:
        psi = torch.zeros((1, ctx.npw), dtype=torch.complex128, device="cuda")
        out = torch.zeros_like(psi)
        with pytest.raises(pwlib.PWError) as e:
            ctx.hamiltonian_apply_noalloc(psi, out)
        assert e.value.status == -1 and "static scratch" in str(e.value)
