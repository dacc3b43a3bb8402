"""Gradients of a trajectory loss through the library's discrete adjoint.

Loss: L = sum over steps n of sum over probe nodes p of (v_n[p] - target_n[p])^2,
v_n the state at the end of step n.  Parameters: the per-node conductivity
scale s (it enters K through element means) and the Aliev-Panfilov parameters
(k, a) with ga = gs = k.

The forward pass keeps the state every `checkpoint_every` steps.  The reverse
pass re-runs each segment from its checkpoint recording a tape per step (the
recomputation is bitwise identical, so it selects the forward's active sets),
then walks the segment backwards through sdc_step_adjoint.  Every step of the
method runs in the library's kernels; this module only moves device pointers
and adds the loss terms.
"""

from __future__ import annotations

import numpy as np
import torch

from .binding import SDC_TAPE_RECORD, SDC_TAPE_REPLAY


def _set_params(ctx, wl, scale, k, a):
    ctx.set_dof_scale(scale.detach().cpu().numpy())
    ion = dict(wl.ionic)
    ion["ga"] = float(k)
    ion["gs"] = float(k)
    ion["a"] = float(a)
    ctx.set_ionic(ion)


def trajectory_loss(ctx, wl, v0, w0, steps, probes, targets, checkpoint_every=20):
    """Forward pass: loss and the checkpoints (list of (step, v, w))."""
    v, w = v0.clone(), w0.clone()
    ckpts = []
    loss = 0.0
    for n in range(steps):
        if n % checkpoint_every == 0:
            ckpts.append((n, v.clone(), w.clone()))
        ctx.step(v, w, n * wl.dt, wl.dt, wl.sweeps, wl.tol, want_stats=False)
        d = v[probes] - targets[n]
        loss += float(torch.dot(d, d))
    return loss, ckpts


def trajectory_grad(ctx, wl, ckpts, steps, probes, targets, device):
    """Reverse pass: dL/ds (device, per node) and dL/d(ga, gs, a) (numpy[3])."""
    N = ctx.n
    grad_s = torch.zeros(N, dtype=torch.float64, device=device)
    grad_ion = np.zeros(3)
    lam_v = torch.zeros(N, dtype=torch.float64, device=device)
    lam_w = torch.zeros_like(lam_v)
    lam_v0 = torch.zeros_like(lam_v)
    lam_w0 = torch.zeros_like(lam_v)
    bounds = [c[0] for c in ckpts] + [steps]
    for seg in range(len(ckpts) - 1, -1, -1):
        n0, n1 = bounds[seg], bounds[seg + 1]
        v, w = ckpts[seg][1].clone(), ckpts[seg][2].clone()
        tapes, inputs, outputs = [], [], []
        for n in range(n0, n1):
            inputs.append((v.clone(), w.clone()))
            tp = ctx.new_tape(wl.sweeps, device)
            ctx.step_taped(v, w, n * wl.dt, wl.dt, wl.sweeps, wl.tol, tp, SDC_TAPE_RECORD)
            tapes.append(tp)
            outputs.append(v[probes].clone())
        for i in range(n1 - n0 - 1, -1, -1):
            n = n0 + i
            lam_v[probes] += 2.0 * (outputs[i] - targets[n])
            ctx.adjoint(tapes[i], inputs[i][0], inputs[i][1], wl.dt, lam_v, lam_w, lam_v0, lam_w0,
                        grad_scale=grad_s, grad_ionic=grad_ion)
            lam_v.copy_(lam_v0)
            lam_w.copy_(lam_w0)
        del tapes
    return grad_s, grad_ion


def replayed_loss(ctx, wl, v0, w0, steps, probes, targets, tapes):
    """Loss of a run that replays recorded active sets (for finite differences)."""
    v, w = v0.clone(), w0.clone()
    loss = 0.0
    for n in range(steps):
        ctx.step_taped(v, w, n * wl.dt, wl.dt, wl.sweeps, wl.tol, tapes[n], SDC_TAPE_REPLAY)
        d = v[probes] - targets[n]
        loss += float(torch.dot(d, d))
    return loss


class TrajectoryLoss(torch.autograd.Function):
    """L(s, k, a) for a context, a workload and probe targets, differentiated by
    the discrete adjoint with checkpoints every `checkpoint_every` steps.

    The context's parameters may change between forward and backward (another
    application of this function, a finite-difference probe): backward sets the
    forward's (s, k, a) for its recomputation and adjoint, then puts back the
    parameters the context held when backward started."""

    @staticmethod
    def forward(fctx, scale, ka, ctx, wl, steps, probes, targets, checkpoint_every):
        device = scale.device
        k, a = ka[0].item(), ka[1].item()
        _set_params(ctx, wl, scale, k, a)
        v0 = torch.tensor(wl.v0, dtype=torch.float64, device=device)
        w0 = torch.tensor(wl.w0, dtype=torch.float64, device=device)
        loss, ckpts = trajectory_loss(ctx, wl, v0, w0, steps, probes, targets, checkpoint_every)
        fctx.save = (ctx, wl, ckpts, steps, probes, targets, device)
        fctx.params = (scale.detach().clone(), k, a)
        return torch.tensor(loss, dtype=torch.float64, device=device)

    @staticmethod
    def backward(fctx, gout):
        ctx, wl, ckpts, steps, probes, targets, device = fctx.save
        prev_scale, prev_ionic = ctx.dof_scale, ctx.ionic
        _set_params(ctx, wl, *fctx.params)
        try:
            gs, gi = trajectory_grad(ctx, wl, ckpts, steps, probes, targets, device)
        finally:
            ctx.set_dof_scale(prev_scale)
            if prev_ionic is not None:
                ctx.set_ionic(prev_ionic)
        gka = torch.tensor([gi[0] + gi[1], gi[2]], dtype=torch.float64, device=device)
        return gout * gs, gout * gka, None, None, None, None, None, None
