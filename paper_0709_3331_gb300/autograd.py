"""torch.autograd front end of the reverse-mode gradient of the C ABI.

``electron_ke_after_run(pos0, vel0, ...)`` returns the electron kinetic energy
after a run of the split-step push (Sec. 2) with TREE forces (Sec. 3) as a
tensor whose gradient with respect to ``pos0`` and ``vel0`` comes from
``ucp_grad_ke_electrons`` (discrete adjoint, checkpointed recomputation).
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
