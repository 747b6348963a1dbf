#!/usr/bin/env python3
"""Benchmark of the fused FDLB time step (arXiv:1010.4124) on GB300.

Workload (default): the 4096 x 4096 Kelvin-Helmholtz shear layer in FP32
(D_v = D_rho = 16 cells, four seeded modes, dx = dy = 0.002, dt = tau = 1e-5,
periodic in x, outflow in y), the roofline configuration of the method.  One
"step" is one time step of the whole grid (one launch of the fused kernel).

Prints ONE JSON line (rank 0):
  value   Gcell-updates/s = nx * ny * steps / device time of the timed steps
          (inputs resident in HBM; 2 x 1.29 GB of f >> 129 MB L2, so every
          step streams from HBM without an explicit flush)
  e2e     the same metric through the C ABI with host buffers: klb_init_fields
          from pinned host fields, the steps, klb_moments back to pinned host
          memory, all inside the timed region
  roofline      the binding roofline of the step kernel: FP32 (or FP64)
                operations per node-update x rate, against the ALU peak
                (152 SMs x lanes x max clock); roofline_hbm beside it: 152
                (304) algorithmic bytes per node-update x rate against the
                measured copy bandwidth; traffic = ncu DRAM bytes per launch
  cpu_baseline  the FP64 oracle on the host cores, on a band of the workload
  clocks, gpu_launches, and the legs sweep (batched vs looped plain step),
  adjoint (checkpointed reverse sweep, 256^2; adjoint_4096: the FP32
  reverse step on the 4096^2 workload), schemes (the convection schemes of
  the paper's comparison) and paper_sweeps (its Kelvin-Helmholtz studies).

--impl reference times the FP64 CPU oracle (the baseline of this method: the
paper publishes no timings) on a bounded sample of the same workload.
N > 1 (torchrun): replicas only -- every rank runs its own copy of the
workload (the step does not need a collective); value sums over ranks and the
time is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NQ = 19  # velocities of the D2V19 set
BYTES_PER_NODE = {"fp32": 152, "fp64": 304}  # 19 reads + 19 writes per node-update
# FP32 lane operations of the FMA pipe per node-update (an fma counts as one):
# 30 WENO5 faces x 29, moments and state 74, collision with the conservative
# projection 223, flux differences 60 (the reciprocals, 4 per face and 2 per
# node, run on the MUFU unit and are not counted)
FP32_OPS_PER_NODE = 1227
# FP32 issue peak of the FMA pipes: 152 SMs x 128 lanes x 2070 MHz (max SM clock)
FP32_LANE_PEAK_T = 152 * 128 * 2.070e9 / 1e12
# FP64 path (the parity path, every operation rounded as the oracle rounds it):
# FP64-pipe instructions per node-update counted by ncu (DADD + DMUL + DFMA,
# the division sequences included; profiles/step_fp64_khi512_ncu.md), and the
# FP64 pipe peak: 152 SMs x 2 per clock x 2070 MHz
FP64_OPS_PER_NODE = 5214
FP64_PEAK_T = 152 * 2 * 2.070e9 / 1e12
STEP_KERNEL_SOURCES = ["paper_1010_4124_gb300/csrc/klb_step_f32.cuh", "paper_1010_4124_gb300/csrc/klb_step_f32.cu",
                       "paper_1010_4124_gb300/csrc/klb_device.cuh"]


def kernel_sha() -> str:
    h = hashlib.sha256()
    for f in STEP_KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def profiled_traffic(workload: str, precision: str, variant: int):
    """DRAM bytes per launch of the step kernel from the committed ncu summary,
    if it was taken on the current kernel source and tile shape."""
    path = os.path.join(ROOT, "profiles", f"step_{precision}_{workload}.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    if d.get("kernel_sha") != kernel_sha():
        return None
    t = d.get("traffic_bytes_per_launch")
    return t.get(str(variant)) if isinstance(t, dict) else None


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.tmp = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.tmp, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        self.tmp.flush()
        rows = []
        for line in open(self.tmp.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.tmp.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def workload_problem(name: str, steps: int):
    from paper_1010_4124_gb300 import inputs
    if name == "khi4096":
        pb = inputs.roofline_4096(steps)
    elif name == "khi2048":  # the same profile at 2048^2 (profiling case: 2 x 318 MB of f, > L2)
        pb = inputs.khi(2048, 2048, steps, Dv=16.0, Drho=16.0, modes=4, phase_seed=inputs.ROOFLINE_PHASE_SEED)
    elif name == "khi512":
        pb = inputs.khi(512, 512, steps)
    elif name in ("khi8192", "khi16384"):  # the same profile on larger grids (2 x 5.1 / 20.4 GB of f)
        n = int(name[3:])
        pb = inputs.khi(n, n, steps, Dv=16.0, Drho=16.0, modes=4, phase_seed=inputs.ROOFLINE_PHASE_SEED)
    else:
        raise SystemExit(f"unknown workload {name}")
    pb.sample_every = 0
    return pb


def max_over_ranks(x: float, ws: int, device: str = "cuda") -> float:
    """The largest value of x over the ranks (the job's time is its slowest
    replica's); x itself when the job has one rank."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(cells: int, steps: int, ws: int, seconds: float) -> float:
    """Whole-job Gcell-updates/s of ws replicas of one grid each (weak scaling):
    the units all ranks processed over the slowest rank's time."""
    return cells * steps * ws / seconds / 1e9


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def pick_variant(h, stream, torch, steps: int = 20):
    """Time both FP32 tile shapes on the workload itself and keep the faster
    (an untimed warm-up of the run; the state it leaves is re-initialised).
    The shapes are timed alternately, twice each, and compared by their best
    time, so that neither is judged on the GPU's first, colder steps."""
    best_ms = {}
    for v in (0, 1, 0, 1):
        h.variant = v
        h.step(3)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h.step(steps)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        best_ms[v] = min(ms, best_ms.get(v, ms))
    return min(best_ms, key=best_ms.get)


def run_ours(args):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1010_4124_gb300 import inputs, klb

    pb = workload_problem(args.workload, args.steps)
    prec = args.precision
    stream = torch.cuda.Stream()
    fields = [np.ascontiguousarray(a) for a in inputs.fields(pb)]
    h = klb.Klb.from_problem(pb, precision=prec, stream=stream.cuda_stream)
    h.init_fields(*fields)
    variant = max(args.variant, 0)
    if prec == "fp32" and args.variant < 0:
        variant = pick_variant(h, stream, torch)
    if prec == "fp32":
        h.variant = variant
    h.step(args.warmup)
    h.sync()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    # ---- device-resident timing: K steps bracketed by events on the launch stream
    n0 = h.launch_count
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0.record(stream)
        h.step(args.steps)
        e1.record(stream)
        e1.synchronize()
    torch.cuda.synchronize()
    barrier()
    launches = h.launch_count - n0
    ms = e0.elapsed_time(e1)
    clocks = clk.summary()
    ms = max_over_ranks(ms, ws)
    cells = pb.nx * pb.ny
    state_gb = NQ * pb.ny * pb.nx * (4 if prec == "fp32" else 8) / 1e9
    value = job_rate(cells, args.steps, ws, ms * 1e-3)
    per_step_ms = ms / args.steps
    achieved = BYTES_PER_NODE[prec] * cells / (per_step_ms * 1e-3) / 1e9  # GB/s
    peak, peak_kind = measured_peaks()

    kernel = "fdlb::step_f32_kernel" if prec == "fp32" else "fdlb::step_kernel<double>"
    traffic = profiled_traffic(args.workload, prec, variant if prec == "fp32" else 0)
    hbm_roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "peak_kind": peak_kind, "traffic": traffic,
                "algorithmic_bytes_per_node": BYTES_PER_NODE[prec], "kernel": kernel}
    if prec == "fp32":
        ops = FP32_OPS_PER_NODE * cells / (per_step_ms * 1e-3) / 1e12
        alu_roof = {"bound": "alu", "achieved": round(ops, 2), "peak": round(FP32_LANE_PEAK_T, 2),
                    "unit": "T FP32 lane-ops/s (fma = 1)", "frac": round(ops / FP32_LANE_PEAK_T, 4),
                    "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2070 MHz",
                    "traffic": traffic, "ops_per_node": FP32_OPS_PER_NODE, "kernel": kernel}
    else:
        ops = FP64_OPS_PER_NODE * cells / (per_step_ms * 1e-3) / 1e12
        alu_roof = {"bound": "alu", "achieved": round(ops, 4), "peak": round(FP64_PEAK_T, 4),
                    "unit": "T FP64 pipe instructions/s", "frac": round(ops / FP64_PEAK_T, 4),
                    "peak_kind": "derived: 152 SMs x 2 FP64 per clock x 2070 MHz",
                    "traffic": traffic, "ops_per_node": FP64_OPS_PER_NODE,
                    "ops_kind": "executed per node, counted by ncu", "kernel": kernel}

    # ---- end to end through the C ABI with host buffers (pinned)
    pin = [torch.from_numpy(a).pin_memory() for a in fields]
    outs = [torch.empty((pb.ny, pb.nx), dtype=torch.float64).pin_memory() for _ in range(4)]
    h.sync()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h.init_fields(*[p.numpy() for p in pin])
    h.step(args.steps)
    h.moments(tuple(o.numpy() for o in outs))  # synchronises
    t1 = time.perf_counter()
    e2e_s = t1 - t0
    e2e_s = max_over_ranks(e2e_s, ws)
    h.close()

    line = {
        "metric": "Gcell-updates/s (fused FDLB D2V19 WENO5 step)",
        "value": round(value, 4),
        "unit": "Gcell-updates/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(per_step_ms, 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if prec == "fp32" else "f64",
        "data": "synthetic (seeded KHI initial fields; f = f_eq of them)",
        "config": {"workload": f"KHI {pb.nx}x{pb.ny} {prec.upper()}, D_v=D_rho=16 cells, 4 seeded modes, "
                               f"periodic x / outflow y, dt=tau=1e-5, dx=dy=0.002",
                   "nx": pb.nx, "ny": pb.ny, "precision": prec, "diagnostics": "off in the timed steps",
                   "kernel_variant": variant if prec == "fp32" else 0,
                   "l2": f"inputs larger than L2 (2 x {state_gb:.2f} GB of f per step, L2 129 MB)",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "roofline": hbm_roof,
        "e2e": {"value": round(job_rate(cells, args.steps, ws, e2e_s), 4), "unit": "Gcell-updates/s",
                "h2d_bytes_per_step": round(4 * 8 * cells / args.steps, 1),
                "d2h_bytes_per_step": round(4 * 8 * cells / args.steps, 1)},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    # both steps are bound by their arithmetic units, not by HBM: the ALU
    # roofline is the binding one, the HBM fraction is reported beside it
    line["roofline"] = alu_roof
    line["roofline_hbm"] = hbm_roof
    if rank == 0 and not args.no_sweep:
        line["sweep"] = sweep_measure(args.sweep_steps, torch)
    if rank == 0 and not args.no_physics:
        line["paper_sweeps"] = physics_measure(torch)
    if rank == 0 and not args.no_schemes:
        line["schemes"] = schemes_measure(args.workload, 100, torch)
    if rank == 0 and not args.no_adjoint:
        line["adjoint"] = [adjoint_measure(p, args.adjoint_steps, torch) for p in ("fp32", "fp64")]
        if not args.no_adjoint_4096:
            line["adjoint_4096"] = adjoint_large(torch)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload, samples=40, rows=1024)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def sweep_measure(steps: int, torch):
    """The batched D_v x D_rho sweep (32 KHI instances on uneven grids drawn by
    seed, FP32, diagnostics every 10 steps): one persistent launch per step
    over all instances, replayed from a CUDA graph, tiles picked by the
    autotuner -- against looping the plain single-grid step (same tile shape)
    over the 32 instances one after another on the same GPU, and against the
    batch with the other tile shape."""
    import numpy as np
    from paper_1010_4124_gb300 import inputs, klb
    pbs = inputs.sweep_instances(steps)
    fields = [[np.ascontiguousarray(a) for a in inputs.fields(pb)] for pb in pbs]
    cells = sum(pb.nx * pb.ny for pb in pbs)
    stream = torch.cuda.Stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with klb.KlbBatch.from_problems(pbs, stream=stream.cuda_stream) as bt:
        for m, fl in zip(bt.members, fields):
            m.init_fields(*fl)
        variant = bt.autotune(steps=5)
        bt.step(70)  # warm-up: builds and replays the graph once
        bt.sync()
        n0 = bt.launch_count
        e0.record(stream)
        bt.step(steps)
        e1.record(stream)
        e1.synchronize()
        bt.sync()
        t_batch = e0.elapsed_time(e1) * 1e-3
        launches = bt.launch_count - n0
        tiles = bt.tiles
        # the other tile shape, timed the same way from the initial state:
        # evidence for the pick
        other = 1 - variant
        bt.variant = other
        for m, fl in zip(bt.members, fields):
            m.init_fields(*fl)
        bt.step(70)
        bt.sync()
        e0.record(stream)
        bt.step(steps)
        e1.record(stream)
        e1.synchronize()
        bt.sync()
        t_other = e0.elapsed_time(e1) * 1e-3
    # the plain step, looped over the instances, with the batch's tile shape
    hs = []
    for pb, fl in zip(pbs, fields):
        h = klb.Klb.from_problem(pb, precision="fp32", stream=stream.cuda_stream)
        h.variant = variant
        h.init_fields(*fl)
        h.step(80)  # warm-up: also captures the step graph the timed run replays
        hs.append(h)
    torch.cuda.synchronize()
    e0.record(stream)
    for h in hs:
        h.step(steps)
    e1.record(stream)
    e1.synchronize()
    t_loop = e0.elapsed_time(e1) * 1e-3
    for h in hs:
        h.sync()
        h.close()
    return {"instances": len(pbs), "cells": cells, "steps": steps, "kernel_variant": variant,
            "tiles_per_launch": tiles, "launches": launches,
            "batched_gcell_s": round(cells * steps / t_batch / 1e9, 4),
            "looped_plain_gcell_s": round(cells * steps / t_loop / 1e9, 4),
            "speedup_vs_looped_plain": round(t_loop / t_batch, 3),
            "other_tiles": {"kernel_variant": other, "batched_gcell_s": round(cells * steps / t_other / 1e9, 4)},
            "sizes": sorted({f"{pb.nx}x{pb.ny}" for pb in pbs})}


def adjoint_large(torch, steps: int = 20):
    """The FP32 adjoint on the 4096 x 4096 roofline workload (sampled every
    10 steps, a checkpoint every 10): forward plus reverse sweep of `steps`
    steps against the plain forward, and the reverse step's share of it,
    (adjoint - 2 forward) / steps (each reverse step also recomputes one
    forward step from its checkpoint)."""
    from paper_1010_4124_gb300 import inputs, klb
    pb = inputs.roofline_4096(steps).with_(sample_every=10)
    dev = [torch.as_tensor(a, device="cuda").contiguous() for a in inputs.fields(pb)]
    grads = tuple(torch.empty_like(dev[0]) for _ in range(4))
    with klb.KlbAdjoint.from_problem(pb, "fp32", checkpoint_every=10) as adj:
        adj.forward(*dev)
        adj.backward(1.0, 1.0, out=grads)  # warm
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        adj.forward(*dev)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        adj.backward(1.0, 1.0, out=grads)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
    t_fwd, t_all = t1 - t0, t2 - t0
    return {"workload": f"KHI 4096x4096 FP32, {steps} steps, sampled every 10, a checkpoint every 10",
            "adjoint_s": round(t_all, 4), "forward_with_checkpoints_s": round(t_fwd, 4),
            "reverse_step_ms": round((t_all - 2 * t_fwd) / steps * 1e3, 3),
            "adjoint_over_2x_forward": round(t_all / (2 * t_fwd), 3)}


def adjoint_measure(prec: str, steps: int, torch):
    """The adjoint run of the 256 x 256 KHI (sampled every 10 steps,
    objective KE + gamma): forward with a checkpoint every 45 steps plus the
    reverse sweep, against the same with every state stored (checkpoint
    every step: full-trajectory storage, no recomputation) and against two
    plain forward runs of the step."""
    from paper_1010_4124_gb300 import inputs, klb
    pb = inputs.khi(256, 256, steps, sample_every=10)
    dev = [torch.as_tensor(a, device="cuda").contiguous() for a in inputs.fields(pb)]
    grads = tuple(torch.empty_like(dev[0]) for _ in range(4))

    def run(ckpt):
        with klb.KlbAdjoint.from_problem(pb, prec, checkpoint_every=ckpt) as adj:
            adj.forward(*dev)
            adj.backward(1.0, 1.0, out=grads)  # warm (allocations, graphs, caches)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            adj.forward(*dev)
            adj.backward(1.0, 1.0, out=grads)
            torch.cuda.synchronize()
            return time.perf_counter() - t0

    t_ckpt = run(45)
    t_full = run(1)
    stream = torch.cuda.Stream()
    h = klb.Klb.from_problem(pb, precision=prec, stream=stream.cuda_stream)
    h.init_fields(*dev)
    if prec == "fp32":
        h.variant = pick_variant(h, stream, torch)
        h.init_fields(*dev)
    h.step(80)  # warm-up: also captures the step graph the timed run replays
    h.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    h.step(steps)
    e1.record(stream)
    e1.synchronize()
    t_fwd = e0.elapsed_time(e1) * 1e-3
    h.close()
    state_mb = NQ * (pb.ny + 6) * ((pb.nx + 7 + 31) // 32 * 32) * (4 if prec == "fp32" else 8) / 1e6
    # the same gradient (objective w.r.t. the four initial fields at every
    # node) by central differences: two plain forward runs per parameter
    n_params = 4 * pb.nx * pb.ny
    return {"workload": f"KHI 256x256 {prec.upper()}, {steps} steps, sampled every 10, objective KE + gamma",
            "precision": prec, "checkpoint_every": 45,
            "adjoint_s": round(t_ckpt, 4), "full_storage_s": round(t_full, 4), "plain_forward_s": round(t_fwd, 4),
            "adjoint_over_2x_forward": round(t_ckpt / (2 * t_fwd), 3),
            "speedup_vs_full_storage": round(t_full / t_ckpt, 3),
            "gradient_entries": n_params,
            "speedup_vs_looped_plain_central_fd": round(2 * n_params * t_fwd / t_ckpt, 1),
            "checkpoint_mb": round(((steps + 44) // 45) * state_mb, 1),
            "full_storage_mb": round(steps * state_mb, 1)}


def physics_measure(torch):
    """The paper's three Kelvin-Helmholtz sweeps (Sec. IV) on the batched
    engine (paper_1010_4124_gb300.sweeps): growth rates, the fitted laws of
    the paper's Figs. 7 and 9, and the batched throughput of each sweep."""
    from paper_1010_4124_gb300 import sweeps
    out = {"steps": 40000, "sample_every": 50, "paper": {"a": 2.70, "b": 0.07, "c": 5.28, "e": 0.62}}
    for name in ("velocity", "density", "hybrid"):
        pbs = sweeps.problems(name)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = sweeps.run(name)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        cells = sum(pb.nx * pb.ny for pb in pbs)
        rec = {"instances": len(pbs), "state": sweeps.SWEEPS[name][0], "seconds": round(dt, 3),
               "gcell_s": round(cells * 40000 / dt / 1e9, 3),
               "gamma": [[r["Dv"], r["Drho"], round(r["gamma"], 4)] for r in res]}
        if name == "velocity":
            a, b = sweeps.fit_velocity_law(res)
            rec["fit_a_b"] = [round(a, 4), round(b, 5)]
        if name == "density":
            c, e = sweeps.fit_density_law(res)
            rec["fit_c_e"] = [round(c, 4), round(e, 4)]
        out[name] = rec
    return out


SOD_P_STAR = 0.285975  # star pressure of the gamma = 2 Sod problem (exact Riemann solution)


def schemes_measure(workload: str, steps: int, torch):
    """The convection schemes of the paper's comparison (Sec. III.B, Fig. 2):
    FP32 step throughput of each on the bench workload, and the Sod tube
    (200 x 4, FP64, 5000 steps to t = 0.1) run with each: the shock width
    (10 %-90 % of the pressure jump, in cells) and the total variation of the
    density (0.875 for the exact, monotone profile)."""
    import numpy as np
    from paper_1010_4124_gb300 import inputs, klb
    names = ("weno5", "upwind1", "upwind2", "tvd")
    pb = workload_problem(workload, steps)
    fields = [np.ascontiguousarray(a) for a in inputs.fields(pb)]
    stream = torch.cuda.Stream()
    rate = {}
    for sch in names:
        with klb.Klb.from_problem(pb, precision="fp32", stream=stream.cuda_stream, scheme=sch) as h:
            h.init_fields(*fields)
            h.variant = pick_variant(h, stream, torch, steps=10)
            h.step(3)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h.step(steps)
            e1.record(stream)
            e1.synchronize()
            rate[sch] = round(pb.nx * pb.ny * steps / (e0.elapsed_time(e1) * 1e-3) / 1e9, 4)
    sod = inputs.sod(200, 4, 5000)
    sf = inputs.fields(sod)
    x = (np.arange(sod.nx) + 0.5) * sod.dx
    lo, hi = 0.1 + 0.1 * (SOD_P_STAR - 0.1), 0.1 + 0.9 * (SOD_P_STAR - 0.1)
    width, tv = {}, {}
    for sch in names:
        with klb.Klb.from_problem(sod, precision="fp64", scheme=sch) as h:
            h.init_fields(*sf)
            h.step(sod.steps)
            out = tuple(np.empty((sod.ny, sod.nx)) for _ in range(4))
            h.moments(out)
        r, p = out[0][0], out[0][0] * out[3][0]
        if not (np.isfinite(r).all() and np.isfinite(p).all()):
            width[sch], tv[sch] = None, None  # the run diverged
            continue
        sel = (x > 0.6) & (x < 0.8)
        xx, pp = x[sel], p[sel]

        def crossing(level):
            i = np.where((pp[:-1] >= level) & (pp[1:] < level))[0]
            if len(i) == 0:
                return None
            i = i[-1]
            return xx[i] + sod.dx * (pp[i] - level) / (pp[i] - pp[i + 1])

        a, b = crossing(lo), crossing(hi)
        width[sch] = round((a - b) / sod.dx, 3) if a is not None and b is not None else None
        tv[sch] = round(float(np.abs(np.diff(r)).sum()), 4)
    return {"fp32_workload": f"{pb.nx}x{pb.ny}", "fp32_steps": steps, "fp32_gcell_s": rate,
            "sod_fp64": {"workload": "Sod 200x4, dt = tau = 2e-5, 5000 steps (t = 0.1)",
                         "shock_width_cells": width, "tv_rho": tv, "tv_rho_exact": 0.875,
                         "null": "the run diverged (non-finite state)"}}


def _band(pb, rows: int):
    """A full-width band of `rows` rows (at most the workload's) centred on the
    shear layer of the workload."""
    from paper_1010_4124_gb300 import inputs
    rows = min(rows, pb.ny)
    band = pb.with_(ny=rows)
    full = inputs.fields(pb)
    j0 = pb.ny // 2 - rows // 2
    return band, [a[j0:j0 + rows].copy() for a in full]


def cpu_baseline(workload: str, samples: int = 3, rows: int = 256):
    """The FP64 oracle, as it stands, on a bounded sample of the workload: a
    full-width band of `rows` rows around the shear layer (outflow rows), a few steps."""
    import numpy as np
    from oracle import core
    pb = workload_problem(workload, 1)
    band, fl = _band(pb, rows)
    p = core.Params(nx=band.nx, ny=band.ny, dx=band.dx, dy=band.dy, dt=band.dt, tau=band.tau, v=band.v,
                    bc_x=band.bc_x, bc_y=band.bc_y)
    f = core.init_feq(p, *fl)
    core.step(p, f)  # warm-up (page-in, thread start)
    t0 = time.perf_counter()
    for _ in range(samples):
        f = core.step(p, f)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": round(band.nx * band.ny * samples / dt / 1e9, 6), "unit": "Gcell-updates/s",
            "cores": cores, "kind": "oracle",
            "sample": f"{samples} oracle steps (FP64, OpenMP over rows) on a {band.nx}x{band.ny} full-width band "
                      f"of the {pb.nx}x{pb.ny} workload around the shear layer"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import build as obuild
    obuild.build()
    import numpy as np
    from oracle import core
    pb = workload_problem(args.workload, 1)
    # the whole workload when the run stays within a few minutes of host time
    # (about a second per oracle step of 4096^2 on 16 cores), else a band of it
    rows = pb.ny if args.steps + args.warmup <= 100 else 64
    band, fl = _band(pb, rows)
    p = core.Params(nx=band.nx, ny=band.ny, dx=band.dx, dy=band.dy, dt=band.dt, tau=band.tau, v=band.v,
                    bc_x=band.bc_x, bc_y=band.bc_y)
    f = core.init_feq(p, *fl)
    for _ in range(args.warmup):
        f = core.step(p, f)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f = core.step(p, f)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    value = band.nx * band.ny * args.steps / dt / 1e9
    if band.ny == pb.ny:
        sample = f"each step = one oracle step (FP64, OpenMP over rows) of the whole {pb.nx}x{pb.ny} workload"
    else:
        sample = (f"each step = one oracle step (FP64, OpenMP over rows) on a {band.nx}x{band.ny} full-width band "
                  f"of the {pb.nx}x{pb.ny} workload around the shear layer")
    print(json.dumps({
        "impl": "reference", "metric": "Gcell-updates/s (fused FDLB D2V19 WENO5 step)", "value": round(value, 6),
        "unit": "Gcell-updates/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt / args.steps * 1e3, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"KHI {pb.nx}x{pb.ny} {args.precision.upper()}, D_v=D_rho=16 cells, 4 seeded modes, "
                               f"periodic x / outflow y, dt=tau=1e-5, dx=dy=0.002",
                   "nx": pb.nx, "ny": pb.ny, "precision": args.precision},
        "cpu_baseline": {"value": round(value, 6), "unit": "Gcell-updates/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 6), "unit": "Gcell-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="khi4096", choices=["khi4096", "khi2048", "khi512", "khi8192", "khi16384"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--variant", type=int, default=-1,
                    help="FP32 kernel tile shape (0: 32x16, 1: 32x8); -1 picks the faster by timing both")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--sweep-steps", type=int, default=2000)
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-schemes", action="store_true")
    ap.add_argument("--no-physics", action="store_true")
    ap.add_argument("--adjoint-steps", type=int, default=2000)
    ap.add_argument("--no-adjoint-4096", action="store_true", help="skip the FP32 adjoint on the 4096^2 workload")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
