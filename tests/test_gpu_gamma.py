"""Gamma-point pairing of r-space-real bands (time-reversal symmetry at k = 0).

Checked: symmetrize / pack / unpack round trips to rounding (1e-15 relative in FP64); the
filter of m packed bands, unpacked, equals the filter of the 2m bands it carries (FP64 1e-10
relative per band, with S = I and with the Woodbury S^-1; complex64 1e-4) and the oracle's
filter of those bands (FP64 1e-10); the Ritz values of the paired filter + Rayleigh-Ritz equal
the oracle's (1e-10 Ha); contexts away from k = 0 are refused.
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


def symmetric_part(x):
    """(x(G) + conj x(-G)) / 2 with -G at index npw - 1 - i (canonical order at k = 0)."""
    return 0.5 * (x + np.conj(x[:, ::-1]))


@pytest.mark.parametrize("with_q", [False, True])
def test_pairing_round_trip_and_filter(with_q):
    prob = W.make_problem("tiny_gamma_fp64", box=(16, 16, 16), ecut=3.0, nband=8, with_q=with_q)
    ham = O.Hamiltonian.from_problem(prob)
    # the canonical order at k = 0 is symmetric: row npw - 1 - i is -G_i
    assert np.array_equal(ham.miller[::-1], -ham.miller)
    with pwlib.Context.from_problem(prob) as ctx:
        x = W.random_block(500, ctx.npw, prob.nband)
        xs = symmetric_part(x)
        t = torch.from_numpy(x).cuda()
        ctx.gamma_symmetrize(t)
        np.testing.assert_allclose(t.cpu().numpy(), xs, rtol=0, atol=1e-15)
        c = ctx.gamma_pack(t)
        back = ctx.gamma_unpack(c)
        np.testing.assert_allclose(back.cpu().numpy(), xs, rtol=0, atol=1e-15)
        a, b = -0.5, 2.0 * prob.ecut + 3.0
        ctx.chebyshev_filter(c, 5, a, b)
        yp = ctx.gamma_unpack(c).cpu().numpy()
        full = t.clone()
        ctx.chebyshev_filter(full, 5, a, b)
        ref = O.chebyshev_filter(ham.apply_a, xs, 5, a, b)
        assert rel(yp, full.cpu().numpy()).max() < 1e-10
        assert rel(yp, ref).max() < 1e-10
        # the filtered bands stay real in r-space
        assert np.abs(yp - symmetric_part(yp)).max() < 1e-10 * np.abs(yp).max()
        # Ritz values of the paired filter against the oracle's
        eig, _ = ctx.rayleigh_ritz(torch.from_numpy(yp).cuda())
        lam, *_ = O.rayleigh_ritz(ref, ham.apply_h(ref), ham.apply_s(ref))
        assert np.abs(eig - lam).max() < 1e-10
        # complex64 filter of the packed bands
        c32 = ctx.gamma_pack(t.to(torch.complex64), precision=pwlib.PW_MIXED)
        ctx.chebyshev_filter(c32, 5, a, b, precision=pwlib.PW_MIXED)
        y32 = ctx.gamma_unpack(c32, precision=pwlib.PW_MIXED).cpu().numpy().astype(np.complex128)
        assert rel(y32, ref).max() < 1e-4


def test_pairing_needs_gamma_and_even_bands():
    prob = W.make_problem("batched_kpoints", box=(18, 18, 20), ecut=2.5, natom=3, nband=4,
                          kpt=[0.125, 0.375, -0.25])
    with pwlib.Context.from_problem(prob) as ctx:
        t = torch.zeros((4, ctx.npw), dtype=torch.complex128, device="cuda")
        with pytest.raises(pwlib.PWError) as e:
            ctx.gamma_pack(t)
        assert e.value.status == -1
    prob = W.make_problem("tiny_gamma_fp64", box=(16, 16, 16), ecut=3.0, nband=3)
    with pwlib.Context.from_problem(prob) as ctx:
        t = torch.zeros((3, ctx.npw), dtype=torch.complex128, device="cuda")
        with pytest.raises(pwlib.PWError):
            ctx.gamma_pack(t)
