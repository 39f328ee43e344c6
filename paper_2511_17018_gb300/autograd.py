"""torch.autograd.Function over the library's fit and its hand-written adjoint.

chi2 = TpcFit.apply(alignment, seeds, fitter, dev) runs tpcfit_fit with
checkpoint recording; backward calls tpcfit_fit_backward with grad_chi2 =
dL/dchi2 and returns dL/dalignment [36,152,2] and dL/dseeds [5,N].  Tracks
that fail (ndf <= 0) have chi2 = NaN in the output; mask them before summing.
"""
from __future__ import annotations

import torch

from . import tpcfit as tf


class TpcFit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, alignment, seeds, fitter, dev):
        fitter.set_alignment(alignment.detach().contiguous())
        fitter.set_record(True)
        d = dict(dev)
        d["seeds"] = seeds.detach().contiguous()
        out = fitter.fit(d)
        ctx.fitter, ctx.dev, ctx.out = fitter, d, out
        ctx.mark_non_differentiable(out["ndf"])
        return out["chi2"], out["params"], out["ndf"]

    @staticmethod
    def backward(ctx, g_chi2, g_params, g_ndf):
        g = torch.nan_to_num(g_chi2, nan=0.0).contiguous() if g_chi2 is not None else \
            torch.zeros_like(ctx.out["chi2"])
        if g_params is not None and torch.any(g_params != 0):
            raise NotImplementedError("gradients through the fitted parameters are not provided")
        ga, gs = ctx.fitter.backward(ctx.dev, ctx.out, g)
        return ga, gs, None, None


def fit_chi2(alignment, seeds, fitter, dev):
    """(chi2[N], params[5,N], ndf[N]) with gradients w.r.t. alignment and seeds."""
    return TpcFit.apply(alignment, seeds, fitter, dev)
