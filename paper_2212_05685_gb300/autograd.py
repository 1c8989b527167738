"""torch.autograd.Function around one KPM pass (argument marshalling only).

forward:  fields (26*N float64, CUDA) -> (obs 26*N, omega 1) via kpm_observables
backward: (dL/dobs, dL/domega) -> dL/dfields via kpm_backward (App. B backward
          recursion, rescaling held fixed)

By default (ckpt_every = KPM_REGENERATE) the forward pass keeps the last two
recursion vectors of every slab (KPM_FLAG_KEEP_TAIL) and the backward pass
regenerates the earlier ones by running the recursion backwards, so it needs
no checkpoints and no forward sweep of its own; ckpt_every >= 0 selects the
checkpointing backward pass instead.

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
        fo = kpm.kpm_opts.from_buffer_copy(opts)
        if ckpt_every == kpm.KPM_REGENERATE:
            fo.flags |= kpm.KPM_FLAG_KEEP_TAIL
        kpm.kpm_observables(kctx, model, fo, fields.detach().contiguous(), ab, obs, omega)
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


def observables(kctx, model, opts, fields, ab, ckpt_every=kpm.KPM_REGENERATE):
    """Differentiable KPM observables and grand potential of the Nambu matrix
    built from `fields` (ab = spectral rescale, not differentiated)."""
    return KPMObservables.apply(fields, ab, kctx, model, opts, ckpt_every)
