#!/usr/bin/env python3
"""Benchmark of the TREE hot path (arXiv 0709.3331, Sec. 2-3) on one GB300.

One bench step = one block of the split-step push: k = 10 electron substeps of
dt_e = 1e-3 (each: kick, drift, tree build, walk over the electrons; the tenth
walks every particle), the ion kicks, and the energy/momentum reduction.
Workload: N = 524,288 (262,144 ions, 262,144 electrons), Gaussian cloud
sigma = 8, m_i/m_e = 1000, T_e = 1, T_i = 0.01, eps = 0.01, theta = 0.5,
leaf_cap = 32, FP32 node-relative walk with compensated sums and FP64 state.

Prints one JSON line.  ``value`` = tree-force interactions/s (direct pairs +
multipole evaluations) over the timed steps, device-timed with CUDA events on
the context's stream, L2 flushed before every step.  ``e2e`` is the same
metric through the public API with host buffers: state copied in from pinned
memory, advanced, energy and state copied back, every step.

``--impl reference`` times the FP64 CPU oracle (the slow, plain reference
implementation) on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(name="precision_n524288", n=524288, sigma=8.0, seed=3, theta=0.5, eps=0.01,
                leaf_cap=32, dt_e=1e-3, k=10)
METRIC = "tree-force interactions/s at N=524288 (FP32 compensated walk, FP64 state)"
UNIT = "interactions/s"
# Flops charged per interaction by the roofline (counted from the FP32C kernel's
# arithmetic, FMA = 2, rsqrt = 1): direct pair 20, multipole through quadrupole
# order 64 (R and |R|^2 come from the opening criterion and are not charged).
FLOP_P2P = 20
FLOP_M2P = 64
FP32_LANES_PER_SM = 128


def sm_peak_tflops(nsm, mhz):
    return nsm * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None
        self.skip = 0

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        # the timed region starts once the sampler is producing rows (at most 3 s)
        t0 = time.time()
        while time.time() - t0 < 3.0 and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.02)
        self.skip = sum(1 for _ in open(self.path))

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows, before = [], []
        for k, line in enumerate(open(self.path)):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                (rows if k >= getattr(self, "skip", 0) else before).append(parts)
        in_region = len(rows)
        if not rows:    # a region shorter than one sampling interval
            rows = before[-1:]
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4)
                          if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows), "samples_in_timed_region": in_region}


def reduce_over_ranks(ms, count, device="cpu"):
    """Replicas run independently; the job's time is the slowest rank's and its
    work is the sum over ranks (weak scaling).  Single process: unchanged."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms), float(count)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    c = torch.tensor([float(count)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), float(c.item())


def git_rev():
    try:
        return subprocess.run(["git", "-C", ROOT, "rev-parse", "--short", "HEAD"],
                              capture_output=True, text=True, timeout=5).stdout.strip() or None
    except Exception:
        return None


# --------------------------------------------------------------------- oracle
def oracle_sample(cloud, n_targets, nthreads, seed=0):
    """Oracle tree build over all particles + walk over a seeded target sample.
    Returns (seconds, interactions)."""
    from oracle import oracle as O
    rng = np.random.default_rng(seed)
    tl = np.sort(rng.choice(cloud.n, size=n_targets, replace=False))
    t0 = time.perf_counter()
    T = O.Tree(cloud.pos, cloud.species, cloud.q, leaf_cap=WORKLOAD["leaf_cap"])
    _, _, npp, nmp = T.force(WORKLOAD["theta"], WORKLOAD["eps"], targets=tl, nthreads=nthreads,
                             counts=True)
    dt = time.perf_counter() - t0
    return dt, int(npp.sum() + nmp.sum())


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def cpu_baseline(cloud, budget_s=12.0):
    """The oracle as it stands on the host cores: tree build + walk of every
    particle, repeated until about budget_s seconds of CPU work; and the same
    oracle on one core (tree build + walk of a seeded eighth of the targets)."""
    from oracle import oracle as O
    O.build()
    cores = os.cpu_count() or 1
    nthreads = cores if O.has_openmp() else 1
    tot_t, tot_i, reps = 0.0, 0, 0
    nt = cloud.n
    while tot_t < budget_s and reps < 20:
        dt, inter = oracle_sample(cloud, nt, nthreads, seed=reps)
        tot_t += dt
        tot_i += inter
        reps += 1
        if reps == 1 and dt > budget_s:
            break
    t1, i1 = oracle_sample(cloud, cloud.n // 8, 1, seed=77)
    return {"value": tot_i / tot_t, "unit": UNIT, "cores": nthreads, "kind": "oracle",
            "cpu_model": cpu_model(), "host_cores": cores,
            "sample": f"FP64 serial-tree oracle, {reps} x (tree build over all {cloud.n} "
                      f"particles + walk of all {nt} targets, theta {WORKLOAD['theta']}, "
                      f"leaf_cap {WORKLOAD['leaf_cap']}), OpenMP over targets, {tot_t:.1f} s",
            "one_core": {"value": i1 / t1, "unit": UNIT, "cores": 1,
                         "sample": f"tree build over all {cloud.n} particles + walk of "
                                   f"{cloud.n // 8} seeded targets on one thread, {t1:.1f} s"}}


def oracle_accuracy(cloud, tl, gpu, nthreads):
    """Force and potential errors on the seeded targets tl: the GPU tree (given,
    per theta) and the oracle tree against the direct sum (Sec. 2.1 Eq. 1-2), and
    the GPU tree against the oracle tree, all at the workload's initial state."""
    from oracle import oracle as O
    c = cloud
    qm = (c.q[c.species[tl]] / c.m[c.species[tl]])[:, None]
    Ed, pd = O.direct(c.pos, c.species, c.q, WORKLOAD["eps"], targets=tl, nthreads=nthreads)
    ad = Ed * qm
    T = O.Tree(c.pos, c.species, c.q, leaf_cap=WORKLOAD["leaf_cap"])

    def rr(a, b):
        return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))

    out = {}
    for th, (ga, gp) in gpu.items():
        Et, pt = T.force(float(th), WORKLOAD["eps"], targets=tl, nthreads=nthreads)
        at = Et * qm
        out[th] = {"gpu_tree_vs_direct": {"force": rr(ga, ad), "potential": rr(gp, pd)},
                   "oracle_tree_vs_direct": {"force": rr(at, ad), "potential": rr(pt, pd)},
                   "gpu_vs_oracle_tree": {"force": rr(ga, at), "potential": rr(gp, pt)}}
    return out


def oracle_drift_c1(steps, nthreads):
    """Total-energy drift of the oracle at the plain FP64 workload (N = 131072,
    sigma 4, theta 0.5, eps 0.01, dt_e 1e-3, k = 10) over a short span."""
    from oracle import oracle as O
    from paper_0709_3331_gb300.inputs import gaussian_cloud
    c1 = gaussian_cloud(131072, 4.0, 2)
    lc, th, eps, dt, k = WORKLOAD["leaf_cap"], 0.5, WORKLOAD["eps"], 1e-3, 10
    e0 = O.energy(c1.pos, c1.vel, c1.species, c1.q, c1.m, th, eps, leaf_cap=lc, nthreads=nthreads)
    t0 = time.perf_counter()
    p, v, _ = O.run(c1.pos, c1.vel, c1.species, c1.q, c1.m, dt, k, steps // k, th, eps,
                    leaf_cap=lc, nthreads=nthreads)
    t = time.perf_counter() - t0
    e1 = O.energy(p, v, c1.species, c1.q, c1.m, th, eps, leaf_cap=lc, nthreads=nthreads)
    return abs(e1[3] - e0[3]) / (e0[0] + e0[1] + abs(e0[2])), t


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_0709_3331_gb300.inputs import gaussian_cloud
    from oracle import oracle as O
    O.build()
    c = gaussian_cloud(WORKLOAD["n"], WORKLOAD["sigma"], WORKLOAD["seed"])
    cores = os.cpu_count() or 1
    nthreads = cores if O.has_openmp() else 1
    # a step: one tree build over every particle and a walk over an eighth of them
    # (a substep builds once and walks the N/2 electrons)
    nt = WORKLOAD["n"] // 8
    for _ in range(args.warmup):
        oracle_sample(c, 512, nthreads)
    tot_t, tot_i = 0.0, 0
    for s in range(args.steps):
        dt, inter = oracle_sample(c, nt, nthreads, seed=100 + s)
        tot_t += dt
        tot_i += inter
    v = tot_i / tot_t
    sample = (f"per step: FP64 oracle tree build over all {c.n} particles + walk of {nt} "
              f"seeded targets, OpenMP over targets on {nthreads} threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD["name"], "n": c.n,
                                        "theta": WORKLOAD["theta"], "eps": WORKLOAD["eps"],
                                        "leaf_cap": WORKLOAD["leaf_cap"]},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": nthreads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))
    return 0


# --------------------------------------------------------------------- GPU arm
def traffic_record():
    """DRAM bytes per walk launch of a block step (one walk over every particle,
    nine over the electrons) from the committed ncu summary, valid only while the
    walk source and the leaf population are those of the capture."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "walk_fp32c_traffic.txt")
    src = os.path.join(ROOT, "paper_0709_3331_gb300", "csrc", "ucp_walk.cu")
    if not os.path.exists(path):
        return None
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    rec = {}
    for line in open(path):
        if ":" in line:
            k, v = line.split(":", 1)
            rec[k.strip()] = v.strip()
    if rec.get("walk_source_sha256_16") != h or rec.get("leaf_cap") != str(WORKLOAD["leaf_cap"]):
        return None
    try:
        full = float(rec["dram_bytes_per_full_walk"])
        elec = float(rec["dram_bytes_per_electron_walk"])
    except (KeyError, ValueError):
        return None
    return (full + (WORKLOAD["k"] - 1) * elec) / WORKLOAD["k"]


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_0709_3331_gb300 import UCP_FP32C, UCP_FP64, Context
    from paper_0709_3331_gb300 import build as B
    from paper_0709_3331_gb300.ucp import WALK_SHAPE_TABLE
    from paper_0709_3331_gb300.inputs import gaussian_cloud

    ws, rank, local = dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    if rank == 0 or not B.up_to_date():
        B.build()
    if ws > 1:
        dist.barrier()
    dev = torch.device("cuda", torch.cuda.current_device())
    W = WORKLOAD
    c = gaussian_cloud(W["n"], W["sigma"], W["seed"])
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)

    pos_d = torch.from_numpy(c.pos).to(dev)
    vel_d = torch.from_numpy(c.vel).to(dev)
    sp_d = torch.from_numpy(c.species).to(dev)

    def timed_steps(ctx, steps, energy=True, profile=True):
        ctx.stats(reset=True)
        ctx.profile(profile)
        ctx.profile_read()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        energies = []
        for i in range(steps):
            flush.zero_()
            starts[i].record(stream)
            ctx.step(W["dt_e"], W["k"], W["k"], W["theta"], W["eps"])
            if energy:
                energies.append(ctx.energy(W["theta"], W["eps"]))
            ends[i].record(stream)
        torch.cuda.synchronize()
        ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
        walk_ms, walk_n = ctx.profile_read()
        ctx.profile(False)
        st = ctx.stats(reset=True)
        return ms, st, walk_ms, walk_n, energies

    # ---------------- FP32C headline
    ctx = Context(c.n, c.q, c.m, leaf_cap=W["leaf_cap"], precision=UCP_FP32C)
    ctx.set_state(pos_d, vel_d, sp_d)
    # one-time launch-shape choice of the walk (outside the timed region)
    shape, shape_ms = ctx.autotune(W["theta"], W["eps"])
    # every block step replays a captured CUDA graph (the warm-up steps capture it;
    # the walks inside it are timed by event-record nodes of the graph)
    ctx.set_graphs(True)
    ctx.stats(reset=True)
    ctx.profile(True)              # the timed steps replay the profiled capture
    for _ in range(args.warmup):
        ctx.step(W["dt_e"], W["k"], W["k"], W["theta"], W["eps"])
        ctx.energy(W["theta"], W["eps"])
    ctx.profile_read()
    ctx.profile(False)
    torch.cuda.synchronize()
    clk = Clocks(local)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk.start()
    t_wall0 = time.perf_counter()
    ms, st, walk_ms, walk_n, energies = timed_steps(ctx, args.steps)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    clocks = clk.stop()
    inter = int(st[0] + st[1])
    launches = int(st[6])
    ms_all, inter_all = reduce_over_ranks(ms, inter, dev)
    value = inter_all / (ms_all / 1e3)
    pst = W["n"] * W["k"] * args.steps * ws / (ms_all / 1e3)

    # roofline of the dominant kernel (the FP32C walk), flops per launch / launch time
    flops = FLOP_P2P * float(st[0]) + FLOP_M2P * float(st[1])
    achieved = flops / (walk_ms / 1e3) / 1e12 if walk_ms > 0 else None
    peak_mhz = 2070.0
    peak = sm_peak_tflops(nsm, peak_mhz)
    traffic = traffic_record()
    from paper_0709_3331_gb300.ucp import measure_peaks
    mpk = measure_peaks(stream.cuda_stream)
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": (achieved / peak) if achieved else None,
                "traffic": traffic, "kernel": "k_walk_fp32c",
                "peak_basis": f"FP32 pipe: {nsm} SMs x 128 lanes x 2 flop x {peak_mhz:.0f} MHz "
                              "(max SM clock); flops = 20 per direct pair + 64 per multipole",
                "measured_peaks": mpk,
                "frac_of_measured_fp32_fma": (achieved / mpk["fp32_fma_tflops"]) if achieved
                else None,
                "walk_ms_per_launch": walk_ms / max(walk_n, 1), "walk_launches": walk_n,
                "walk_share_of_step": walk_ms / ms if ms > 0 else None}

    # forces of the initial state on seeded targets, for the accuracy figures
    ACC_TARGETS = 8192
    tl = np.sort(np.random.default_rng(2024).choice(W["n"], ACC_TARGETS, replace=False))
    acc_d = torch.empty((W["n"], 3), dtype=torch.float64, device=dev)
    phi_d = torch.empty(W["n"], dtype=torch.float64, device=dev)
    ctx.set_state(pos_d, vel_d, sp_d)
    ctx.tree_force(W["theta"], W["eps"], acc_d, phi_d)
    gpu_samples = {str(W["theta"]): (acc_d.cpu().numpy()[tl], phi_d.cpu().numpy()[tl])}

    # ---------------- e2e through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(c, W, args, ws, dev, flush, Context, UCP_FP32C)

    # ---------------- FP64 walk and theta sweep (context lines, fewer steps)
    extra = {}
    if not args.quick:
        extra = run_extras(c, W, ws, pos_d, vel_d, sp_d, Context, UCP_FP32C, UCP_FP64,
                           timed_steps, flush, stream, peak, ms / args.steps, tl, gpu_samples,
                           mpk)

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_all / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 walk (compensated), f64 state",
        "data": "synthetic",
        "config": {"workload": W["name"], "n": W["n"], "sigma": W["sigma"], "theta": W["theta"],
                   "eps": W["eps"], "leaf_cap": W["leaf_cap"], "dt_e": W["dt_e"],
                   "ion_substep_ratio": W["k"],
                   "step": "one block of 10 electron substeps, replayed as a captured CUDA graph",
                   "parallelism": f"replicas x{ws}", "l2": "flushed (256 MB write) before "
                                                         "every timed step",
                   "walk_shape": {"index": shape, "threads": WALK_SHAPE_TABLE[shape][0],
                                  "blocks_per_sm": WALK_SHAPE_TABLE[shape][1],
                                  "staged_leaf_sources": bool(WALK_SHAPE_TABLE[shape][2]),
                                  "autotune_ms_walks_per_block": shape_ms}},
        "particle_steps_per_s": pst,
        "p2p_pairs_per_s": float(st[0]) * ws / (ms_all / 1e3),
        "m2p_evals_per_s": float(st[1]) * ws / (ms_all / 1e3),
        "interactions_per_target_walk": {"p2p": float(st[0]) / max(int(st[2]), 1),
                                         "m2p": float(st[1]) / max(int(st[2]), 1)},
        "roofline": roofline,
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": launches,
        "energy_last": energies[-1].tolist() if energies else None,
        "wall_s_timed_region": t_wall,
        "git": git_rev(),
    }
    out.update(extra)
    ctx.close()
    if rank == 0 and not args.no_cpu_baseline:
        # the oracle leg: host-core timings, the direct-sum accuracy reference and
        # the oracle's own drift at the plain workload
        out["cpu_baseline"] = cpu_baseline(c)
        from oracle import oracle as O
        nthr = (os.cpu_count() or 1) if O.has_openmp() else 1
        accs = oracle_accuracy(c, tl, gpu_samples, nthr)
        a0 = accs[str(W["theta"])]
        out["accuracy"] = {
            "force_rel_rms_vs_direct": a0["gpu_tree_vs_direct"]["force"],
            "potential_rel_rms_vs_direct": a0["gpu_tree_vs_direct"]["potential"],
            "oracle_tree_force_rel_rms_vs_direct": a0["oracle_tree_vs_direct"]["force"],
            "force_rel_rms_vs_oracle_tree": a0["gpu_vs_oracle_tree"]["force"],
            "theta": W["theta"], "leaf_cap": W["leaf_cap"], "targets": int(tl.size),
            "particle_steps_per_s": pst,
            "state": "initial state of the workload; FP32C tree forces against the FP64 direct "
                     "sum on seeded targets (oracle)",
            "note": "particle-steps/s at this force error compares leaf populations; "
                    "interactions/s counts a direct pair like a multipole"}
        for th, a in accs.items():
            if "theta_sweep" in out and th in out["theta_sweep"]:
                out["theta_sweep"][th]["accuracy"] = a
        if "plain_fp64_n131072" in out:
            d_orc, t_orc = oracle_drift_c1(10, nthr)
            out["plain_fp64_n131072"]["drift_10_substeps"] = {
                "gpu": out["plain_fp64_n131072"].pop("drift_10_substeps_gpu"), "oracle": d_orc,
                "oracle_s": t_orc,
                "note": "one block of 10 electron substeps from the same state, GPU FP64 walk "
                        "vs the FP64 CPU oracle"}
    if rank == 0:
        print(json.dumps(out))
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_e2e(c, W, args, ws, dev, flush, Context, UCP_FP32C):
    import torch
    import torch.distributed as dist
    pin_pos = torch.from_numpy(c.pos).pin_memory()
    pin_vel = torch.from_numpy(c.vel).pin_memory()
    pin_sp = torch.from_numpy(c.species).pin_memory()
    out_pos = torch.empty((c.n, 3), dtype=torch.float64).pin_memory()
    out_vel = torch.empty((c.n, 3), dtype=torch.float64).pin_memory()
    ctx_h = Context(c.n, c.q, c.m, leaf_cap=W["leaf_cap"], precision=UCP_FP32C)
    np_pos, np_vel, np_sp = pin_pos.numpy(), pin_vel.numpy(), pin_sp.numpy()
    np_opos, np_ovel = out_pos.numpy(), out_vel.numpy()
    ctx_h.set_state(np_pos, np_vel, np_sp)
    ctx_h.autotune(W["theta"], W["eps"])
    ctx_h.set_graphs(True)
    for _ in range(max(1, args.warmup)):
        ctx_h.set_state(np_pos, np_vel, np_sp)
        ctx_h.step(W["dt_e"], W["k"], W["k"], W["theta"], W["eps"])
        ctx_h.energy(W["theta"], W["eps"])
        ctx_h.get_state(np_opos, np_ovel)
    ctx_h.stats(reset=True)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    e0 = time.perf_counter()
    e_steps = max(1, args.steps)
    for _ in range(e_steps):
        flush.zero_()
        ctx_h.set_state(np_pos, np_vel, np_sp)
        ctx_h.step(W["dt_e"], W["k"], W["k"], W["theta"], W["eps"])
        ctx_h.energy(W["theta"], W["eps"])
        ctx_h.get_state(np_opos, np_ovel)
    torch.cuda.synchronize()
    e_t = time.perf_counter() - e0
    st_h = ctx_h.stats(reset=True)
    e_t_all, e_cnt = reduce_over_ranks(e_t, float(st_h[0] + st_h[1]), dev)
    e_val = e_cnt / e_t_all
    e2e = {"value": e_val, "unit": UNIT,
           "h2d_bytes_per_step": int(c.pos.nbytes + c.vel.nbytes + c.species.nbytes),
           "d2h_bytes_per_step": int(c.pos.nbytes + c.vel.nbytes + 6 * 8),
           "note": "per step: set_state from pinned host arrays (forces recomputed from the "
                   "copied state), one block step (a captured graph replay), energy, get_state "
                   "to host"}
    ctx_h.close()
    return e2e


def run_extras(c, W, ws, pos_d, vel_d, sp_d, Context, UCP_FP32C, UCP_FP64, timed_steps, flush,
               stream, peak, ms_step32, tl, gpu_samples, mpk):
    import torch
    extra = {}
    ctx64 = Context(c.n, c.q, c.m, leaf_cap=W["leaf_cap"], precision=UCP_FP64)
    ctx64.set_state(pos_d, vel_d, sp_d)
    ctx64.set_graphs(True)     # like the headline: blocks replay a profiled capture
    ctx64.profile(True)
    ctx64.step(W["dt_e"], W["k"], W["k"], W["theta"], W["eps"])
    torch.cuda.synchronize()
    ms64, st64, wms64, wn64, _ = timed_steps(ctx64, 1)
    fl64 = FLOP_P2P * float(st64[0]) + FLOP_M2P * float(st64[1])
    extra["fp64"] = {"value": float(st64[0] + st64[1]) / (ms64 / 1e3), "unit": UNIT,
                     "ms_per_step": ms64, "walk_ms_per_launch": wms64 / max(wn64, 1),
                     "speedup_fp32c_over_fp64": ms64 / ms_step32,
                     "walk_frac_fp64_peak": fl64 / (wms64 / 1e3) / 1e12 / mpk["fp64_fma_tflops"]
                     if wms64 > 0 else None,
                     "note": "walk_frac_fp64_peak: the same flop counts over the FP64 FMA rate "
                             "measured on this GPU (ucp_measure_peaks)"}
    ctx64.close()
    sweep = {}
    for th in (0.3, 0.5, 0.7):
        cs = Context(c.n, c.q, c.m, leaf_cap=W["leaf_cap"], precision=UCP_FP32C)
        cs.set_state(pos_d, vel_d, sp_d)
        if str(th) not in gpu_samples:
            a_s, p_s = cs.tree_force(th, W["eps"], torch.empty((c.n, 3), dtype=torch.float64,
                                                              device=pos_d.device),
                                     torch.empty(c.n, dtype=torch.float64, device=pos_d.device))
            gpu_samples[str(th)] = (a_s.cpu().numpy()[tl], p_s.cpu().numpy()[tl])
        cs.set_graphs(True)
        cs.profile(True)
        cs.step(W["dt_e"], W["k"], W["k"], th, W["eps"])
        torch.cuda.synchronize()
        cs.stats(reset=True)
        cs.profile(True)
        cs.profile_read()
        e_a = torch.cuda.Event(enable_timing=True)
        e_b = torch.cuda.Event(enable_timing=True)
        flush.zero_()
        e_a.record(stream)
        cs.step(W["dt_e"], W["k"], W["k"], th, W["eps"])
        e_b.record(stream)
        torch.cuda.synchronize()
        m1 = e_a.elapsed_time(e_b)
        wm, wn = cs.profile_read()
        s1 = cs.stats(reset=True)
        fl = FLOP_P2P * float(s1[0]) + FLOP_M2P * float(s1[1])
        sweep[str(th)] = {"interactions_per_s": float(s1[0] + s1[1]) / (m1 / 1e3),
                          "ms_per_step": m1,
                          "particle_steps_per_s": W["n"] * W["k"] / (m1 / 1e3),
                          "p2p_per_target": float(s1[0]) / max(int(s1[2]), 1),
                          "m2p_per_target": float(s1[1]) / max(int(s1[2]), 1),
                          "walk_frac_fp32_peak": fl / (wm / 1e3) / 1e12 / peak}
        cs.close()
    extra["theta_sweep"] = sweep

    # the Kelbg electron-ion law (Sec. 2.1 Eq. 3, lambda_ei = 0.05 in these units)
    # on the same workload: one block, FP32C
    ck = Context(c.n, c.q, c.m, leaf_cap=W["leaf_cap"], precision=UCP_FP32C, kelbg_lambda=0.05)
    ck.set_state(pos_d, vel_d, sp_d)
    ck.set_graphs(True)
    ck.profile(True)
    ck.step(W["dt_e"], W["k"], W["k"], W["theta"], W["eps"])
    torch.cuda.synchronize()
    mk, stk, wmk, wnk, _ = timed_steps(ck, 2, energy=False)
    extra["kelbg_fp32c"] = {
        "lambda_ei": 0.05, "ms_per_step": mk / 2,
        "interactions_per_s": float(stk[0] + stk[1]) / (mk / 1e3),
        "walk_ms_per_launch": wmk / max(wnk, 1),
        "note": "electron-ion direct pairs take the Kelbg form one source at a time"}
    ck.close()

    # ensemble of 64 independent clouds (sizes log-uniform 4096..65536, sigma_c =
    # (N_c/2048)^(1/3)) in one context: every stage one launch for all clouds
    from paper_0709_3331_gb300.inputs import batched_sizes, gaussian_cloud
    from paper_0709_3331_gb300.ucp import WALK_SHAPE_TABLE
    ns, _ = batched_sizes()
    cl = [gaussian_cloud(n, (n / 2048.0) ** (1.0 / 3.0), 4000 + i) for i, n in enumerate(ns)]
    bpos = torch.from_numpy(np.concatenate([x.pos for x in cl])).cuda()
    bvel = torch.from_numpy(np.concatenate([x.vel for x in cl])).cuda()
    bsp = torch.from_numpy(np.concatenate([x.species for x in cl])).cuda()
    ntot = int(sum(ns))
    cb = Context(ntot, c.q, c.m, leaf_cap=W["leaf_cap"], precision=UCP_FP32C, sizes=ns)
    cb.set_state(bpos, bvel, bsp)
    bshape, _ = cb.autotune(0.5, W["eps"])
    cb.step(W["dt_e"], W["k"], W["k"], 0.5, W["eps"])
    torch.cuda.synchronize()
    msb, stb, wmb, wnb, _ = timed_steps(cb, 2)
    extra["batched_64_clouds"] = {
        "n_total": ntot, "clouds": len(ns), "ms_per_step": msb / 2,
        "interactions_per_s": float(stb[0] + stb[1]) / (msb / 1e3),
        "particle_steps_per_s": ntot * W["k"] * 2 / (msb / 1e3),
        "walk_frac_fp32_peak": (FLOP_P2P * float(stb[0]) + FLOP_M2P * float(stb[1]))
        / (wmb / 1e3) / 1e12 / peak,
        "walk_shape": WALK_SHAPE_TABLE[bshape],
        "step": "one block of 10 electron substeps for all 64 clouds, theta 0.5, FP32C"}
    # the same ensemble for 500 electron substeps, each block a captured CUDA graph
    cb.set_graphs(True)
    cb.set_state(bpos, bvel, bsp)
    en0 = cb.energy_clouds(0.5, W["eps"])
    cb.step(W["dt_e"], W["k"], W["k"], 0.5, W["eps"])       # captures the block graph
    cb.stats(reset=True)
    torch.cuda.synchronize()
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    cb.step(W["dt_e"], W["k"], 490, 0.5, W["eps"])
    g1.record(stream)
    torch.cuda.synchronize()
    msg = g0.elapsed_time(g1)
    stg = cb.stats(reset=True)
    en1 = cb.energy_clouds(0.5, W["eps"])
    drift = np.abs(en1[:, 3] - en0[:, 3]) / (en0[:, 0] + en0[:, 1] + np.abs(en0[:, 2]))
    extra["batched_64_clouds"]["graphs_500_substeps"] = {
        "ms_per_block": msg / 49, "interactions_per_s": float(stg[0] + stg[1]) / (msg / 1e3),
        "particle_steps_per_s": ntot * 490 / (msg / 1e3),
        "energy_drift_max_over_clouds": float(drift.max()),
        "energy_drift_median": float(np.median(drift)),
        "note": "500 electron substeps: 1 block to capture the graph, 49 timed replays"}
    cb.close()

    # plain method in FP64: N = 131072, sigma 4, 1000 electron substeps (100 blocks)
    c1 = gaussian_cloud(131072, 4.0, 2)
    cp = Context(c1.n, c1.q, c1.m, leaf_cap=W["leaf_cap"], precision=UCP_FP64)
    cp.set_state(c1.pos, c1.vel, c1.species)
    e0 = cp.energy(0.5, W["eps"])
    # one block from the same state (compared with the oracle's block in the oracle leg)
    cp.step(W["dt_e"], W["k"], W["k"], 0.5, W["eps"])
    e10 = cp.energy(0.5, W["eps"])
    drift10 = abs(e10[3] - e0[3]) / (e0[0] + e0[1] + abs(e0[2]))
    cp.set_state(c1.pos, c1.vel, c1.species)
    e0 = cp.energy(0.5, W["eps"])
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    cp.step(W["dt_e"], W["k"], 1000, 0.5, W["eps"])
    t1.record(stream)
    torch.cuda.synchronize()
    mp = t0.elapsed_time(t1)
    e1 = cp.energy(0.5, W["eps"])
    # differentiation form: N = 262144 (sigma 6), FP32C forces with FP64 state,
    # gradient of the final electron kinetic energy w.r.t. the initial state
    # (200 electron substeps, checkpoint every 20), against the forward alone
    c4 = gaussian_cloud(262144, 6.0, 5)
    ca = Context(c4.n, c4.q, c4.m, leaf_cap=W["leaf_cap"], precision=UCP_FP32C)
    p4 = torch.from_numpy(c4.pos).cuda()
    v4 = torch.from_numpy(c4.vel).cuda()
    s4 = torch.from_numpy(c4.species).cuda()
    gx4 = torch.empty_like(p4)
    gv4 = torch.empty_like(v4)
    ca.set_state(p4, v4, s4)
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    ca.step(W["dt_e"], W["k"], 200, 0.5, W["eps"])
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - w0
    ca.set_state(p4, v4, s4)
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    L4, _, _ = ca.grad_ke_electrons(W["dt_e"], W["k"], 200, 0.5, W["eps"], 20, gx4, gv4)
    torch.cuda.synchronize()
    t_grad = time.perf_counter() - w0
    extra["adjoint_n262144"] = {
        "electron_steps": 200, "checkpoint_every": 20, "forward_s": t_fwd, "gradient_s": t_grad,
        "gradient_over_forward": t_grad / t_fwd, "loss": L4,
        "note": "gradient time includes the forward run, the checkpointed recomputation and "
                "201 FP32 adjoint walks"}
    ca.close()

    # the small workload (N = 2048, sigma 1, FP64): launch-bound, so each block of
    # 10 substeps is also run as a captured CUDA graph
    c0 = gaussian_cloud(2048, 1.0, 1)
    small = {}
    for graphs in (False, True):
        cs0 = Context(c0.n, c0.q, c0.m, leaf_cap=8, precision=UCP_FP64)
        cs0.set_state(c0.pos, c0.vel, c0.species)
        cs0.set_graphs(graphs)
        cs0.step(W["dt_e"], W["k"], 20, 0.5, W["eps"])
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        cs0.step(W["dt_e"], W["k"], 100, 0.5, W["eps"])
        t1.record(stream)
        torch.cuda.synchronize()
        ms_s = t0.elapsed_time(t1) / 10
        small["graphs" if graphs else "streams"] = {
            "ms_per_block": ms_s, "particle_steps_per_s": c0.n * W["k"] / (ms_s / 1e3)}
        if not graphs:   # walk time of the same run, from the library's own events
            cs0.profile(True)
            cs0.step(W["dt_e"], W["k"], 100, 0.5, W["eps"])
            torch.cuda.synchronize()
            wms, wn = cs0.profile_read()
            cs0.profile(False)
            small["streams"]["walk_ms_per_block"] = wms / 10
            small["streams"]["walk_launches_per_block"] = wn / 10
        cs0.close()
    extra["plain_fp64_n2048"] = small

    extra["plain_fp64_n131072"] = {
        "electron_steps": 1000, "ms": mp, "particle_steps_per_s": c1.n * 1000 / (mp / 1e3),
        "energy_drift": abs(e1[3] - e0[3]) / (e0[0] + e0[1] + abs(e0[2])),
        "drift_10_substeps_gpu": drift10}
    cp.close()
    # the same workload: drift over t = 0.5 against the electron step (FP32C walk,
    # captured blocks); close e-i encounters are resolved as dt_e falls
    dv = {}
    for dt in (1e-3, 5e-4, 2.5e-4, 1.25e-4):
        cd = Context(c1.n, c1.q, c1.m, leaf_cap=W["leaf_cap"], precision=UCP_FP32C)
        cd.set_state(c1.pos, c1.vel, c1.species)
        cd.set_graphs(True)
        d0 = cd.energy(0.5, W["eps"])
        nsub = int(round(0.5 / dt))
        cd.step(dt, W["k"], nsub, 0.5, W["eps"])
        d1 = cd.energy(0.5, W["eps"])
        dv[f"{dt:g}"] = {"substeps": nsub,
                         "energy_drift": abs(d1[3] - d0[3]) / (d0[0] + d0[1] + abs(d0[2]))}
        cd.close()
    extra["plain_n131072_drift_vs_dt"] = {
        "t": 0.5, "by_dt_e": dv,
        "note": "FP32C walk (forces within 1e-6 of FP64); drift = |E(t) - E(0)| / (KE + |PE|)"}
    return extra


def run_profile_case(args):
    """One named case through the C ABI, a fixed number of times, for a profiler
    to capture (no timing, no JSON line).  ``force``: tree build + one walk over
    every particle; ``step``: blocks of 10 electron substeps; ``grad``: the
    gradient over one block (checkpoint at its end)."""
    import torch

    from paper_0709_3331_gb300 import UCP_FP32C, UCP_FP64, Context
    from paper_0709_3331_gb300.inputs import WORKLOADS, gaussian_cloud

    w = dict(WORKLOADS[args.workload])
    if args.n:
        w["n"] = args.n
    c = gaussian_cloud(**w)
    dev = torch.device("cuda")
    prec = UCP_FP32C if args.precision == "fp32c" else UCP_FP64
    ctx = Context(c.n, c.q, c.m, leaf_cap=args.leaf_cap, precision=prec)
    ctx.set_state(torch.from_numpy(c.pos).to(dev), torch.from_numpy(c.vel).to(dev),
                  torch.from_numpy(c.species).to(dev))
    if prec == UCP_FP32C:
        ctx.set_walk_shape(args.shape)
    acc = torch.empty((c.n, 3), dtype=torch.float64, device=dev)
    phi = torch.empty(c.n, dtype=torch.float64, device=dev)
    for _ in range(args.repeat):
        if args.profile_case == "force":
            ctx.tree_force(args.theta, 0.01, acc, phi)
        elif args.profile_case == "grad":
            gx = torch.empty((c.n, 3), dtype=torch.float64, device=dev)
            gv = torch.empty_like(gx)
            ctx.grad_ke_electrons(1e-3, 10, 10, args.theta, 0.01, 10, gx, gv)
        else:
            ctx.step(1e-3, 10, 10, args.theta, 0.01)
    torch.cuda.synchronize()
    st = ctx.stats()
    print(f"n={c.n} walks={st[3]} p2p={st[0]} m2p={st[1]} boxes={st[4]} depth={st[5]}")
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--quick", action="store_true", help="skip the FP64 and theta-sweep lines")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer e2e leg")
    # a single untimed case for a profiler (see run_profile_case)
    ap.add_argument("--profile-case", choices=["force", "step", "grad"], default=None)
    ap.add_argument("--workload", default="precision_n524288")
    ap.add_argument("--n", type=int, default=0, help="profile case: override the particle count")
    ap.add_argument("--precision", default="fp32c", choices=["fp32c", "fp64"])
    ap.add_argument("--theta", type=float, default=0.5)
    ap.add_argument("--leaf-cap", type=int, default=None,
                    help="largest leaf population (default: the workload's)")
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--shape", type=int, default=0, help="profile case: FP32C walk launch shape")
    args = ap.parse_args()
    if args.leaf_cap is None:
        args.leaf_cap = WORKLOAD["leaf_cap"]
    WORKLOAD["leaf_cap"] = args.leaf_cap
    if args.profile_case:
        return run_profile_case(args)
    if args.warmup < 3 and args.impl == "gpu":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
