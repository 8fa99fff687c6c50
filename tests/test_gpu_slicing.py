"""Spectrum slicing through the C ABI against the oracle's slicing.

The batched window filter (all slices in one recurrence, per-slice coefficients) against the
oracle's slice-by-slice Chebyshev sums: FP64 to 1e-10 of each band's norm, complex64 to
1e-4 (x degree / 40 beyond degree 40);
with and without S, at Gamma and at a general k-point, degrees from 1 to 120.  The full solve
(filter + per-slice Rayleigh-Ritz): the Ritz values of each slice equal the oracle's to 1e-9
and, for slices cut in spectral gaps, the dense eigenvalues inside each slice to 1e-8.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import pw_oracle as O
from oracle import pw_slicing as SL
from paper_2604_11139_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2604_11139_gb300 import pwlib  # noqa: E402

PROBS = {
    "gamma_q": dict(name="tiny_gamma_fp64", box=(12, 12, 12), ecut=2.0, nband=12, with_q=True),
    "gamma": dict(name="tiny_gamma_fp64", box=(16, 16, 16), ecut=3.0, nband=12, with_q=False),
    "kpoint": dict(name="batched_kpoints", box=(18, 18, 20), ecut=2.5, natom=3, nband=12,
                   kpt=[0.125, 0.375, -0.25]),
}


def _setup(key):
    kw = dict(PROBS[key])
    prob = W.make_problem(kw.pop("name"), **kw)
    ham = O.Hamiltonian.from_problem(prob)
    H, S = ham.dense()
    lam = scipy.linalg.eigh(H, S, eigvals_only=True)
    return prob, ham, lam, lam[0] - 0.05, lam[-1] + 0.05


@pytest.mark.parametrize("key", list(PROBS))
@pytest.mark.parametrize("degree", [1, 7, 40, 120])
def test_slice_filter_matches_oracle(key, degree):
    prob, ham, lam, lo, hi = _setup(key)
    cuts = [lam[0] - 0.01, lam[3], lam[7] + 0.02, lam[15]]
    X = W.random_block(77, ham.npw, 12)
    ref = SL.slice_filter(ham, X, 3, degree, lo, hi, cuts)
    scale = np.linalg.norm(X, axis=1)
    with pwlib.Context.from_problem(prob) as ctx:
        t = torch.zeros((12, ctx.npw + 5), dtype=torch.complex128, device="cuda")
        t[:, :ctx.npw] = torch.from_numpy(X)
        ctx.slice_filter(t, 3, degree, lo, hi, cuts)
        y = t[:, :ctx.npw].cpu().numpy()
        assert torch.count_nonzero(t[:, ctx.npw:]) == 0
        assert (np.linalg.norm(y - ref, axis=1) / scale).max() < 1e-10
        t32 = torch.from_numpy(X.astype(np.complex64)).cuda()
        ctx.slice_filter(t32, 3, degree, lo, hi, cuts, precision=pwlib.PW_MIXED)
        y32 = t32.cpu().numpy().astype(np.complex128)
        assert (np.linalg.norm(y32 - ref, axis=1) / scale).max() < 1e-4 * max(1.0, degree / 40)


@pytest.mark.parametrize("key", ["gamma_q", "kpoint"])
def test_spectrum_slice_matches_oracle_and_dense(key):
    prob, ham, lam, lo, hi = _setup(key)
    # cuts in the middle of gaps at the bottom of the spectrum
    gaps = np.argsort(-np.diff(lam[:8]))[:2] + 1        # two widest gaps among the lowest 8
    g1, g2 = sorted(gaps)
    cuts = [lo, 0.5 * (lam[g1 - 1] + lam[g1]), 0.5 * (lam[g2 - 1] + lam[g2])]
    nper = max(g1, g2 - g1) + 3
    X = W.psi0(prob.seed, ham.npw, 2 * nper)
    eig_o, V_o, res_o = SL.slice_solve(ham, X, 2, 200, lo, hi, cuts)
    with pwlib.Context.from_problem(prob) as ctx:
        t = torch.from_numpy(X).cuda()
        eig, res = ctx.spectrum_slice(t, 2, 200, lo, hi, cuts)
    np.testing.assert_allclose(eig, eig_o, atol=1e-9, rtol=0)
    for s in range(2):
        inside = lam[(lam > cuts[s]) & (lam < cuts[s + 1])]
        assert len(inside) >= 1
        for l in inside:
            assert np.abs(eig[s] - l).min() < 1e-8, (s, l)


def test_slicing_rejects_bad_cuts():
    prob, ham, lam, lo, hi = _setup("gamma")
    with pwlib.Context.from_problem(prob) as ctx:
        t = torch.from_numpy(W.random_block(3, ctx.npw, 4)).cuda()
        with pytest.raises(pwlib.PWError) as e:
            ctx.slice_filter(t, 2, 10, lo, hi, [0.0, 0.5, 0.2])
        assert e.value.status == -1
        with pytest.raises(pwlib.PWError):
            ctx.slice_filter(t, 2, 10, hi, lo, [0.0, 0.1, 0.2])
