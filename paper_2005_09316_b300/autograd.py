"""torch.autograd.Function for fitting sky models in visibility space.

``peel_loss(ctx, obs, sky_tensors, gains, data, model=None)`` returns L = sum |D - g1 conj(g2) V(sky)|^2
and, on backward, the gradients of L with respect to every differentiable sky tensor (flux, alpha, l,
m, Gaussian axes and position angles, shapelet beta1, beta2, position angle and coefficients).  The
loss and all gradients come from one call of the library's adjoint (wn_predict_grad): phasors are
recomputed, not stored.  The structural arrays (counts, n_max, offsets, orders, nu_ref) are not
differentiable.  With ``model`` (a resident model of the same structure, e.g. from ``ctx.upload`` of
the starting sky) the forward re-packs that model in place from the current parameter values
(wn_sky_update) instead of uploading and freeing a model on every call, so a fitting loop allocates
nothing per step.
"""
from __future__ import annotations

import torch

from . import GRAD_FIELDS, Context, DeviceObs

DIFF_FIELDS = ("l", "m", "flux", "alpha", "g_maj", "g_min", "g_pa", "s_beta1", "s_beta2", "s_pa", "s_coeff")


class _PeelLoss(torch.autograd.Function):
    @staticmethod
    def forward(fctx, wctx: Context, obs: DeviceObs, structure: dict, gains, data, resident, *params):
        sky = dict(structure)
        for name, t in zip(DIFF_FIELDS, params):
            sky[name] = t.detach().contiguous().to(torch.float64)
        if resident is not None:
            resident.update(sky)
            out = wctx.predict_grad(obs, resident, gains, data)
        else:
            model = wctx.upload(sky)
            try:
                out = wctx.predict_grad(obs, model, gains, data)
            finally:
                model.free()
        fctx.grads = [out[name] for name in DIFF_FIELDS]
        return out["loss"][0].clone()

    @staticmethod
    def backward(fctx, g):
        return (None, None, None, None, None, None) + tuple(g * t for t in fctx.grads)


def peel_loss(wctx: Context, obs: DeviceObs, sky: dict, gains, data, model=None):
    """Differentiable loss of a device sky dict (keys as in paper_2005_09316_b300.sky_to_device); with
    model, that resident model is updated in place instead of a model being uploaded per call."""
    structure = {k: v for k, v in sky.items() if k not in DIFF_FIELDS}
    return _PeelLoss.apply(wctx, obs, structure, gains, data, model, *[sky[k] for k in DIFF_FIELDS])


__all__ = ["peel_loss", "DIFF_FIELDS", "GRAD_FIELDS"]
