"""torch.autograd front end of the reverse-mode gradient of the C ABI.

``electron_ke_after_run(pos0, vel0, ...)`` returns the electron kinetic energy
after a run of the split-step push (Sec. 2) with TREE forces (Sec. 3) as a
tensor whose gradient with respect to ``pos0`` and ``vel0`` comes from
``ucp_grad_ke_electrons`` (discrete adjoint, checkpointed recomputation).
``tree_accel(pos, ...)`` returns the TREE accelerations at ``pos`` with a
backward pass through ``ucp_accel_vjp`` (the tree held fixed).
"""
from __future__ import annotations

import torch

from .ucp import Context


class _ElectronKE(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos0, vel0, context, species, dt_e, k, n_steps, theta, eps, ckpt):
        dev = pos0.device
        p = pos0.detach().to(torch.float64).contiguous()
        v = vel0.detach().to(torch.float64).contiguous()
        s = species.to(dev).to(torch.int8).contiguous()
        context.set_state(p, v, s)
        gx = torch.empty_like(p)
        gv = torch.empty_like(v)
        loss, _, _ = context.grad_ke_electrons(dt_e, k, n_steps, theta, eps, ckpt, gx, gv)
        ctx.save_for_backward(gx, gv)
        return torch.tensor(loss, dtype=torch.float64, device=dev)

    @staticmethod
    def backward(ctx, g):
        gx, gv = ctx.saved_tensors
        return g * gx, g * gv, None, None, None, None, None, None, None, None


def electron_ke_after_run(pos0, vel0, species, context: Context, dt_e, ion_substep_ratio,
                          n_steps, theta, eps, checkpoint_every=None):
    """Electron kinetic energy after ``n_steps`` electron substeps, differentiable
    in the initial positions and velocities (CUDA tensors, N x 3 float64)."""
    ck = n_steps if checkpoint_every is None else checkpoint_every
    return _ElectronKE.apply(pos0, vel0, context, species, dt_e, ion_substep_ratio, n_steps,
                             theta, eps, ck)


class _TreeAccel(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos, context, species, theta, eps):
        p = pos.detach().to(torch.float64).contiguous()
        v = torch.zeros_like(p)
        s = species.to(p.device).to(torch.int8).contiguous()
        context.set_state(p, v, s)
        acc = torch.empty_like(p)
        context.tree_force(theta, eps, acc)
        ctx.save_for_backward(p, s)
        ctx.context, ctx.theta, ctx.eps = context, theta, eps
        return acc

    @staticmethod
    def backward(ctx, g):
        p, s = ctx.saved_tensors
        # the context may have moved on since the forward pass: put its state back
        ctx.context.set_state(p, torch.zeros_like(p), s)
        lam = g.detach().to(torch.float64).contiguous()
        mu = ctx.context.accel_vjp(ctx.theta, ctx.eps, lam)
        return mu, None, None, None, None


def tree_accel(pos, species, context: Context, theta, eps):
    """Accelerations a = q E / m of the TREE walk at ``pos`` (CUDA tensor N x 3,
    float64), differentiable in ``pos`` with the tree held fixed.  The context's
    state is replaced by (pos, zero velocities, species)."""
    return _TreeAccel.apply(pos, context, species, theta, eps)
