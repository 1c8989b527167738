"""torch.autograd.Function around one KPM pass (argument marshalling only).

forward:  fields (26*N float64, CUDA) -> (obs 26*N, omega 1) via kpm_observables
backward: (dL/dobs, dL/domega) -> dL/dfields via kpm_backward (App. B backward
          recursion, rescaling held fixed)

Real-valued torch tensors in the library's layouts; complex entries are
stored as (re, im) pairs, so torch's real gradients are exactly the
(dL/dRe, dL/dIm) convention of the C ABI.
"""
from __future__ import annotations

import torch

from . import kpm


class KPMObservables(torch.autograd.Function):
    @staticmethod
    def forward(ctx, fields, ab, kctx, model, opts, ckpt_every):
        N = model.nx * model.ny
        obs = torch.empty(26 * N, dtype=torch.float64, device=fields.device)
        omega = torch.empty(1, dtype=torch.float64, device=fields.device)
        kpm.kpm_observables(kctx, model, opts, fields.detach().contiguous(), ab, obs, omega)
        ctx.save_for_backward(fields, ab)
        ctx.kctx, ctx.model, ctx.opts, ctx.ckpt = kctx, model, opts, ckpt_every
        return obs, omega

    @staticmethod
    def backward(ctx, g_obs, g_omega):
        fields, ab = ctx.saved_tensors
        N = ctx.model.nx * ctx.model.ny
        if g_obs is None:
            g_obs = torch.zeros(26 * N, dtype=torch.float64, device=fields.device)
        gom = float(g_omega.sum().item()) if g_omega is not None else 0.0
        grad = torch.empty_like(fields)
        kpm.kpm_backward(ctx.kctx, ctx.model, ctx.opts, fields.detach().contiguous(), ab,
                         g_obs.contiguous(), gom, grad, ckpt_every=ctx.ckpt)
        return grad, None, None, None, None, None


def observables(kctx, model, opts, fields, ab, ckpt_every=0):
    """Differentiable KPM observables and grand potential of the Nambu matrix
    built from `fields` (ab = spectral rescale, not differentiated)."""
    return KPMObservables.apply(fields, ab, kctx, model, opts, ckpt_every)
