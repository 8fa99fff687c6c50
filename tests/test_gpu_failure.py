"""Failure detection without a device fault.

Every wait of the tensor-core kernels (the mixed-precision projector GEMM and the FP64
digit-sliced GEMM) is bounded.  The test hook pw_ctx_test_wait_expiry makes the next GEMM
issue no copies, so its first wait runs out: the kernel records the failing stage, waits
for what it issued, releases tensor memory and returns.  The host then reports
PW_ETIMEDOUT at the next synchronising call and poisons the context; a fresh context on
the same GPU still computes H|psi> to the FP64 parity bar (1e-11 relative per band).
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


def problem():
    return W.make_problem("tiny_gamma_fp64", box=(16, 16, 16), ecut=3.0, nband=8)


@pytest.mark.parametrize("precision", [pwlib.PW_MIXED, pwlib.PW_FP64], ids=["mixed_gemm", "fp64_digit_gemm"])
def test_expired_wait_is_reported_and_the_gpu_stays_usable(precision):
    prob = problem()
    dt = torch.complex64 if precision == pwlib.PW_MIXED else torch.complex128
    ctx = pwlib.Context.from_problem(prob)
    psi = torch.from_numpy(W.random_block(401, ctx.npw, prob.nband)).to(dt).cuda()
    h = torch.zeros_like(psi)
    ctx.hamiltonian_apply(psi, h, precision=precision)     # a normal call first
    ctx.sync()
    ctx.test_wait_expiry()
    ctx.hamiltonian_apply(psi, h, precision=precision)     # queued; the GEMM's wait expires
    with pytest.raises(pwlib.PWError) as e:
        ctx.sync()
    assert e.value.status == -5 and "expired" in str(e.value)
    with pytest.raises(pwlib.PWError) as e:
        ctx.hamiltonian_apply(psi, h, precision=precision)
    assert e.value.status == -3                             # poisoned
    ctx.close()
    torch.cuda.synchronize()                                # the device itself is healthy
    ham = O.Hamiltonian.from_problem(prob)
    with pwlib.Context.from_problem(prob) as ctx2:
        x = W.random_block(402, ctx2.npw, prob.nband)
        t = torch.from_numpy(x).cuda()
        hh = torch.zeros_like(t)
        ctx2.hamiltonian_apply(t, hh)
        ctx2.sync()
        ref = ham.apply_h(x)
        err = np.linalg.norm(hh.cpu().numpy() - ref, axis=1) / np.linalg.norm(ref, axis=1)
        assert err.max() < 1e-11
