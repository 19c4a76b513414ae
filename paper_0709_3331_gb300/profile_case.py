"""Run one named workload through the C ABI a fixed number of times, for a
profiler to capture (``ncu ... python -m paper_0709_3331_gb300.profile_case``).

``--what force`` runs ``ucp_tree_force`` (build + one walk over every
particle); ``--what step`` runs ``ucp_step`` blocks; ``--what grad`` runs
``ucp_grad_ke_electrons`` over one block (checkpoint at its end).
"""
from __future__ import annotations

import argparse

import torch

from . import UCP_FP32C, UCP_FP64, Context
from .inputs import WORKLOADS, gaussian_cloud


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="precision_n524288", choices=sorted(WORKLOADS))
    ap.add_argument("--n", type=int, default=0, help="override the particle count")
    ap.add_argument("--precision", default="fp32c", choices=["fp32c", "fp64"])
    ap.add_argument("--theta", type=float, default=0.5)
    ap.add_argument("--eps", type=float, default=0.01)
    ap.add_argument("--leaf-cap", type=int, default=16)
    ap.add_argument("--what", default="force", choices=["force", "step", "grad"])
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--shape", type=int, default=0, help="FP32C walk launch shape")
    a = ap.parse_args()
    w = dict(WORKLOADS[a.workload])
    if a.n:
        w["n"] = a.n
    c = gaussian_cloud(**w)
    dev = torch.device("cuda")
    prec = UCP_FP32C if a.precision == "fp32c" else UCP_FP64
    ctx = Context(c.n, c.q, c.m, leaf_cap=a.leaf_cap, precision=prec)
    ctx.set_state(torch.from_numpy(c.pos).to(dev), torch.from_numpy(c.vel).to(dev),
                  torch.from_numpy(c.species).to(dev))
    if prec == UCP_FP32C:
        ctx.set_walk_shape(a.shape)
    acc = torch.empty((c.n, 3), dtype=torch.float64, device=dev)
    phi = torch.empty(c.n, dtype=torch.float64, device=dev)
    for _ in range(a.repeat):
        if a.what == "force":
            ctx.tree_force(a.theta, a.eps, acc, phi)
        elif a.what == "grad":
            gx = torch.empty((c.n, 3), dtype=torch.float64, device=dev)
            gv = torch.empty_like(gx)
            ctx.grad_ke_electrons(1e-3, 10, 10, a.theta, a.eps, 10, gx, gv)
        else:
            ctx.step(1e-3, 10, 10, a.theta, a.eps)
    torch.cuda.synchronize()
    st = ctx.stats()
    print(f"n={c.n} walks={st[3]} p2p={st[0]} m2p={st[1]} boxes={st[4]} depth={st[5]}")
    ctx.close()


if __name__ == "__main__":
    main()
