"""k-point batching (ragged plane-wave spheres, one captured graph) against per-k calls
and the oracle."""
import numpy as np
import pytest

from oracle import pw_oracle as O
from paper_2604_11139_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2604_11139_gb300 import pwlib  # noqa: E402

KPTS = np.array([[0.125, 0.125, 0.25], [0.375, -0.125, 0.25], [-0.375, 0.375, -0.25]])


def problem(box=(24, 24, 30)):
    return W.make_problem("batched_kpoints", box=box, ecut=3.0, natom=3, nband=6)


def contexts(prob, ecuts, variant=None):
    ctxs = [pwlib.Context.from_problem(prob, kpt=k, ecut=e) for k, e in zip(KPTS, ecuts)]
    if variant is not None:
        for c in ctxs:
            c.fft_config(pwlib.PW_MIXED, variant=variant)
    return ctxs


# variant 35 on a 24^3 box: warp-group FFT kernels with the recurrence fused into pass 3
@pytest.mark.parametrize("precision,variant,box", [(pwlib.PW_FP64, None, (24, 24, 30)),
                                                   (pwlib.PW_MIXED, None, (24, 24, 30)),
                                                   (pwlib.PW_MIXED, 35, (24, 24, 24))])
def test_batch_filter_equals_per_k_filter(precision, variant, box):
    prob = problem(box)
    ecuts = W.ecut_jitter(prob.seed, len(KPTS), prob.ecut)
    ctxs = contexts(prob, ecuts, variant)
    assert len({c.npw for c in ctxs}) == len(ctxs)   # ragged spheres
    dt = torch.complex128 if precision == pwlib.PW_FP64 else torch.complex64
    with pwlib.Batch(ctxs) as bt:
        blocks = [torch.from_numpy(W.random_block(300 + i, c.npw, prob.nband)).to(dt).cuda()
                  for i, c in enumerate(ctxs)]
        for call, (a, b) in enumerate([(0.5, 9.0), (1.0, 12.0), (0.2, 7.5)]):
            ys = [x.clone() for x in blocks]
            bt.filter(ys, 5, [a] * len(ctxs), [b + 0.1 * i for i in range(len(ctxs))], precision)
            for i, (c, x) in enumerate(zip(ctxs, blocks)):
                ref = x.clone()
                c.chebyshev_filter(ref, 5, a, b + 0.1 * i, precision)
                torch.cuda.synchronize()
                err = (torch.linalg.vector_norm(ys[i] - ref) / torch.linalg.vector_norm(ref)).item()
                assert err < 1e-12, (call, i, err)
    for c in ctxs:
        c.close()


def test_batch_chebfi_matches_oracle():
    prob = problem()
    ecuts = W.ecut_jitter(prob.seed, len(KPTS), prob.ecut)
    ctxs = contexts(prob, ecuts)
    psis, v0s, refs = [], [], []
    for i, (c, k, e) in enumerate(zip(ctxs, KPTS, ecuts)):
        ham = O.Hamiltonian.from_problem(prob, kpt=k, ecut=e)
        assert ham.npw == c.npw
        y0 = W.psi0(prob.seed + i, c.npw, prob.nband)
        v0 = W.lanczos_v0(prob.seed + i, c.npw)
        lam, *_ = O.chebfi(ham, y0, v0, 6, 3)
        refs.append(lam)
        psis.append(torch.from_numpy(y0).cuda())
        v0s.append(torch.from_numpy(v0[None]).cuda())
    with pwlib.Batch(ctxs) as bt:
        eig, res = bt.chebfi_solve(psis, 6, 3, v0s)
    np.testing.assert_allclose(eig, np.array(refs), atol=1e-10, rtol=0)
    for c in ctxs:
        c.close()
