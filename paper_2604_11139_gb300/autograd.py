"""torch.autograd.Function front ends of the differentiation form.

``ChebFiRR`` maps the parameters of H (V_loc(r) on the FFT grid and D) to the Ritz
values and Ritz vectors of a ChebFi solve; ``Density`` maps a block of bands to
rho(r) = w sum_i |psi_i(r)|^2.  Both only marshal arguments: the forward passes, the
tape and the adjoints all run in the CUDA library (pw_diff_*, pw_density_grad,
pw_local_apply).
"""
from __future__ import annotations

import torch

from . import pwlib


class ChebFiRR(torch.autograd.Function):
    """(V_loc, D) -> (eigenvalues, Ritz vectors) of `cycles` ChebFi cycles from psi0.

    The filter interval (Lanczos upper bound and per-cycle cuts) is held fixed in the
    backward; pass ``bounds`` to replay a previous run's interval.  ``split`` is the
    band split of pw_diff_backward (-1: every eigenvector-coupling pair).  One handle
    holds one tape: call backward before the next forward on the same handle."""

    @staticmethod
    def forward(fctx, vloc, D, handle: pwlib.Diff, psi0, v0, bounds, split):
        ctx = handle.context
        ctx.set_vloc(vloc)
        ctx.set_D(D)
        psi = psi0.detach().clone()
        eig, bnd = handle.forward(psi, v0=v0, bounds=bounds)
        fctx.handle = handle
        fctx.split = int(split)
        fctx.bounds = bnd
        return torch.as_tensor(eig, dtype=torch.float64, device=psi.device), psi

    @staticmethod
    def backward(fctx, eig_bar, psi_bar):
        eb = None if eig_bar is None else eig_bar.detach().double().cpu().numpy()
        pb = None if psi_bar is None else psi_bar.detach().to(torch.complex128).contiguous()
        dV, dD = fctx.handle.backward(eig_bar=eb, psi_bar=pb, split=fctx.split)
        return dV, dD, None, None, None, None, None


class Density(torch.autograd.Function):
    """psi (complex128, bands x npw) -> rho(r) = w sum_i |psi_i(r)|^2 on the n1 x n2 x n3 grid,
    psi_i(r) the unnormalised inverse DFT of band i (Alg. 3 density step)."""

    @staticmethod
    def forward(fctx, psi, w, ctx: pwlib.Context):
        psi = psi.detach().contiguous()
        rho = ctx.density_grad(psi, [float(w)] * psi.shape[0])
        fctx.save_for_backward(psi)
        fctx.w = float(w)
        fctx.ctx = ctx
        return rho

    @staticmethod
    def backward(fctx, rho_bar):
        (psi,) = fctx.saved_tensors
        ctx = fctx.ctx
        n = float(ctx.box[0] * ctx.box[1] * ctx.box[2])
        out = ctx.local_apply(rho_bar.detach().contiguous(), psi, alpha=2.0 * fctx.w * n)
        return out, None, None


def chebfi_rr(vloc, D, handle, psi0, v0=None, bounds=None, split=-1):
    return ChebFiRR.apply(vloc, D, handle, psi0, v0, bounds, split)


def density(psi, w, ctx):
    return Density.apply(psi, w, ctx)
