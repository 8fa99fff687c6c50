"""Parity in the launch configuration the benchmark times.

The 96^3 workload (55,179 plane waves, 512 projectors) with all 256 bands in one call,
the FFT forms and band batch the autotuner picks for 256 bands, and 2 bf16 pieces per
projector-GEMM operand, as `bench.py` runs it.  The oracle computes three sampled bands
one by one: H psi and the degree-10 filter act on each band independently, so the sampled
rows of the 256-band result must equal the oracle's result for those rows alone.

Tolerances: FP64 H psi 1e-11 relative per band; mixed H psi 1e-4 and mixed filter 1e-3
relative per band (2 bf16 pieces give products with ~2^-16 relative error; an indexing or
batching slip gives errors of order 1).
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

SAMPLE = [0, 101, 255]


def rel(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.linalg.norm(b, axis=-1)


def test_bench_launch_configuration_sampled_bands():
    prob = W.make_problem("fp64_at_scale")
    M, m = prob.nband, prob.degree
    assert M == 256
    ham = O.Hamiltonian.from_problem(prob)
    with pwlib.Context.from_problem(prob) as ctx:
        psi = W.psi0(prob.seed, ctx.npw, M)
        v0 = torch.from_numpy(W.lanczos_v0(prob.seed, ctx.npw)[None]).cuda()
        Y0 = torch.from_numpy(psi).cuda()
        _, a, b = ctx.spectrum_bounds(Y0, 10, v0)
        ctx.tc_config(2)
        ctx.autotune(M, pwlib.PW_MIXED)

        # FP64 H psi of the whole block
        h64 = torch.zeros_like(Y0)
        ctx.hamiltonian_apply(Y0, h64)
        torch.cuda.synchronize()
        ref = ham.apply_h(psi[SAMPLE])
        assert rel(h64.cpu().numpy()[SAMPLE], ref).max() < 1e-11

        # mixed H psi and mixed filter of the whole block
        psi32 = psi.astype(np.complex64).astype(np.complex128)
        Y32 = Y0.to(torch.complex64)
        h32 = torch.zeros_like(Y32)
        ctx.hamiltonian_apply(Y32, h32, precision=pwlib.PW_MIXED)
        torch.cuda.synchronize()
        ref32 = ham.apply_h(psi32[SAMPLE])
        assert rel(h32.cpu().numpy()[SAMPLE].astype(np.complex128), ref32).max() < 1e-4

        ctx.chebyshev_filter(Y32, m, a, b, precision=pwlib.PW_MIXED)
        torch.cuda.synchronize()
        reff = O.chebyshev_filter(ham.apply_a, psi32[SAMPLE], m, a, b)
        assert rel(Y32.cpu().numpy()[SAMPLE].astype(np.complex128), reff).max() < 1e-3
