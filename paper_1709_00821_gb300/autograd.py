"""torch.autograd bridge for the RKETD adjoint: spectra as a differentiable function of the
per-cell plasma frequency squared and collision frequency.

Forward: rketd_set_medium + rketd_forward_ckpt + rketd_get_spectra_device (CUDA kernels).
Backward: rketd_adjoint with dL/dX from autograd. Marshalling only; no numerics here.
"""
from __future__ import annotations

import torch

from . import rketd as rk


class SpectraFunction(torch.autograd.Function):
    """(wp2, nu) [total cells] FP64 CUDA -> (X_re, X_im) [slabs, probes, freq] FP64 CUDA."""

    @staticmethod
    def forward(fctx, wp2, nu, engine):
        engine.ctx.set_medium(wp2.contiguous(), nu.contiguous())
        engine.ctx.forward_ckpt(engine.steps, engine.ckpt_every)
        shape = (engine.ctx.n_slabs, engine.ctx.n_probes, len(engine.ctx.freq))
        xr = torch.empty(shape, dtype=torch.float64, device=wp2.device)
        xi = torch.empty(shape, dtype=torch.float64, device=wp2.device)
        engine.ctx.spectra_device(xr.data_ptr(), xi.data_ptr())
        fctx.engine = engine
        fctx.n = wp2.numel()
        return xr, xi

    @staticmethod
    def backward(fctx, gxr, gxi):
        e = fctx.engine
        gw = torch.empty(fctx.n, dtype=torch.float64, device=gxr.device)
        gn = torch.empty(fctx.n, dtype=torch.float64, device=gxr.device)
        e.ctx.adjoint(gxr.contiguous(), gxi.contiguous(), e.w_lo, e.w_hi, gw, gn)
        return gw, gn, None


class SpectraEngine:
    """A context for a batch of slabs with a fixed run length, checkpoint interval and
    trainable window [w_lo, w_hi); call it with CUDA FP64 (wp2, nu) of all cells."""

    def __init__(self, slabs, prec="f32", steps=None, ckpt_every=512, window=(2048, 6144), options=None):
        self.ctx = rk.Context(slabs, prec, options=options)
        s0 = slabs[0] if isinstance(slabs, (list, tuple)) else slabs
        self.steps = s0.steps if steps is None else steps
        self.ckpt_every = ckpt_every
        self.w_lo, self.w_hi = window

    def __call__(self, wp2, nu):
        return SpectraFunction.apply(wp2, nu, self)

    def close(self):
        self.ctx.close()
