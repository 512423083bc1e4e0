"""Throughput of the adaptive multiresolution finite-volume step on one GB300.

Default workload (N=1): 2D adaptive MR in single precision, 8 levels (8 -> 1024
cells per dimension), eps = 1e-3, global time stepping, CFL 0.5, seeded
four-quadrant Riemann data (rho in [0.5, 2], v in [-0.75, 0.75]^2,
p in [0.3, 1.5]), run from t = 0.  A step is one full pass of the method:
CFL reduction, ghost strips, two RK2 stages over every leaf of every level,
projection, flux correction, MR analysis, thresholding, tree update.

metric: leaf cell-updates per second (a leaf cell advanced one full step).
The state is a few tens of MB, smaller than L2, so L2 is flushed (a 512 MB
write) between timed steps, outside the timed events.

--impl reference times the CPU oracle (plain FP64 C) on the host cores, on the
same workload, each step a full oracle step.

Multi-GPU: the method has no exchange step in this build; N ranks run N
independent replicas ("scaling": "weak"), no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import mrfv_inputs as mi  # noqa: E402

WORKLOAD = "mr2d_fp32_L7"
WL = dict(dim=2, precision="fp32", levels=8, base_blocks=(1, 1, 1), adapt=True, eps=1e-3, cfl=0.5,
          t_end=0.25)
SEED = 0


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_solver(m, stream=None):
    s = m.Solver(dim=WL["dim"], precision=WL["precision"], levels=WL["levels"], base_blocks=WL["base_blocks"],
                 adapt=WL["adapt"], eps=WL["eps"], cfl=WL["cfl"], t_end=WL["t_end"], stream=stream)
    s.init_state(mi.IC_QUADRANTS, mi.quadrant_params(SEED))
    return s


def uniform_roofline(m, torch, hbm_peak, steps=6):
    """Stage kernel alone on a uniform 8192^2 single-precision grid (state 1 GB per
    buffer, far above L2): algorithmic bytes per launch / CUDA-event duration."""
    s = m.Solver(dim=2, precision="fp32", levels=1, base_blocks=(1024, 1024, 1), cfl=0.5)
    s.init_state(mi.IC_QUADRANTS, mi.quadrant_params(SEED))
    for _ in range(2):
        s.step(0.0, sync=False)
    s.profile_enable(True)
    for _ in range(steps):
        s.step(0.0, sync=False)
    p = s.profile_read()
    s.profile_enable(False)
    achieved = p["fv_bytes"] / (p["fv_ms"] * 1e-3) / 1e9
    out = {"workload": "uniform2d_fp32_8192", "bound": "hbm", "achieved": round(achieved, 1),
           "peak": hbm_peak, "unit": "GB/s", "frac": round(achieved / hbm_peak, 4),
           "launches": p["fv_launches"], "avg_launch_ms": round(p["fv_ms"] / max(1, p["fv_launches"]), 4),
           "cell_updates_per_s": 8192 * 8192 * steps / (p["fv_ms"] * 1e-3)}
    s.close()
    del s
    torch.cuda.empty_cache()
    return out


def oracle_sample(budget_s: float, max_steps: int = 50):
    """Oracle (FP64 C, one host thread) on the same workload from t = 0."""
    import oracle

    o = oracle.Oracle(2, WL["levels"], WL["base_blocks"])
    o.init(mi.IC_QUADRANTS, mi.quadrant_params(SEED))
    o.adapt(oracle.CRIT_MR, WL["eps"], precision=1)
    cells = 0
    steps = 0
    t0 = time.perf_counter()
    while steps < max_steps and time.perf_counter() - t0 < budget_s:
        leaves = sum(int(o.leaf_mask(l).sum()) for l in range(o.levels)) * 64
        o.step(o.dt(WL["cfl"]))
        o.adapt(oracle.CRIT_MR, WL["eps"], precision=1)
        cells += leaves
        steps += 1
    el = time.perf_counter() - t0
    return cells / el, steps, el


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    import oracle

    oracle.build()
    o = oracle.Oracle(2, WL["levels"], WL["base_blocks"])
    o.init(mi.IC_QUADRANTS, mi.quadrant_params(SEED))
    o.adapt(oracle.CRIT_MR, WL["eps"], precision=1)

    def one():
        leaves = sum(int(o.leaf_mask(l).sum()) for l in range(o.levels)) * 64
        o.step(o.dt(WL["cfl"]))
        o.adapt(oracle.CRIT_MR, WL["eps"], precision=1)
        return leaves

    for _ in range(args.warmup):
        one()
    cells = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        cells += one()
    el = time.perf_counter() - t0
    v = cells / el
    line = {"metric": "cell-updates/s", "value": v, "unit": "cell-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "levels": 8, "finest": 1024, "eps": WL["eps"],
                       "ic": "seeded four-quadrant Riemann (seed 0)"},
            "cpu_baseline": {"value": v, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} oracle steps after {args.warmup} warm-up steps"},
            "e2e": {"value": v, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_1603_05211_gb300 as m

    rank, world, local = dist_info()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    m.build()
    m.load()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    s = make_solver(m, stream)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        s.step(0.0, sync=False)
    s.synchronize()
    st0 = s.stats()
    s.profile_enable(True)   # reset the launch counter ...
    s.profile_enable(False)  # ... and keep the captured-graph replay for the timed steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)  # evict L2 between steps (outside the events)
        ev[k][0].record(stream)
        s.step(0.0, sync=False)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    launches = s.profile_read()["launches"]
    st1 = s.stats()
    cells = st1["cell_updates"] - st0["cell_updates"]
    # the same steps once more with every stage launch bracketed by CUDA events
    # (eager launches: events cannot be read per replay inside a graph)
    s.profile_enable(True)
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        s.step(0.0, sync=False)
    prof = s.profile_read()
    s.profile_enable(False)
    t_local = torch.tensor([ms], dtype=torch.float64, device=dev)
    c_all = torch.tensor([float(cells)], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t_local, op=dist.ReduceOp.MAX)
        dist.all_reduce(c_all, op=dist.ReduceOp.SUM)
    ms_max = float(t_local.item())
    value = float(c_all.item()) / (ms_max * 1e-3)
    hbm_peak, peak_kind = measured_peaks()

    result = None
    if rank == 0:
        fv_ach = prof["fv_bytes"] / (prof["fv_ms"] * 1e-3) / 1e9 if prof["fv_ms"] > 0 else 0.0
        roof = {"bound": "hbm", "achieved": round(fv_ach, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(fv_ach / hbm_peak, 4), "traffic": None,
                "kernel": "k_fv (fused reconstruct-flux-update stage)", "peak_kind": peak_kind,
                "timing": "CUDA events around each stage launch, same workload and step count, eager launches",
                "launches": prof["fv_launches"],
                "avg_launch_us": round(prof["fv_ms"] * 1e3 / max(1, prof["fv_launches"]), 2),
                "bytes_per_launch": prof["fv_bytes"] / max(1, prof["fv_launches"])}
        try:
            roof_u = uniform_roofline(m, torch, hbm_peak)
        except Exception as e:  # noqa: BLE001
            roof_u = {"error": str(e)}
        # end to end through the C interface: host initial state in, host state out
        e2e = run_e2e(m, torch, stream, args.steps)
        # CPU baseline: the oracle on a bounded sample of the same workload
        ob, osteps, osec = oracle_sample(budget_s=float(os.environ.get("MRFV_ORACLE_BUDGET", "15")))
        result = {
            "metric": "cell-updates/s", "value": value, "unit": "cell-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "levels": 8, "finest": 1024, "eps": WL["eps"], "cfl": WL["cfl"],
                       "ic": "seeded four-quadrant Riemann (seed 0)", "l2": "flushed between timed steps",
                       "leaves_per_step": cells / args.steps / 64, "parallelism": f"replicas x{world}"},
            "roofline": roof,
            "roofline_uniform": roof_u,
            "cpu_baseline": {"value": ob, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
                             "sample": f"{osteps} FP64 oracle steps of the same workload from t=0 ({osec:.1f} s)"},
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk,
        }
        print(json.dumps(result), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return result


def run_e2e(m, torch, stream, steps):
    """Same metric through the public C interface with host buffers: the finest-level
    initial state is copied in from host memory, `steps` steps run (each reading its
    dt back), and every level's state is copied out; wall-clock time."""
    import numpy as np

    s = make_solver(m, stream)
    L = WL["levels"] - 1
    ref = m.Solver(dim=2, precision="fp32", levels=WL["levels"], base_blocks=(1, 1, 1), adapt=False)
    ref.init_state(mi.IC_QUADRANTS, mi.quadrant_params(SEED + 1))
    host_in = ref.download_level(L)[0]
    full = [np.ones(s.blocks_shape(l), np.uint8) for l in range(WL["levels"])]
    ref.close()
    st0 = s.stats()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.set_tree(full)
    s.upload_level(L, host_in)
    s.restrict(0)
    s.adapt()
    for _ in range(steps):
        s.step(0.0, sync=True)
    out_bytes = 0
    for l in range(WL["levels"]):
        a, _ = s.download_level(l)
        out_bytes += a.nbytes
    el = time.perf_counter() - t0
    st1 = s.stats()
    s.close()
    cells = st1["cell_updates"] - st0["cell_updates"]
    return {"value": cells / el, "unit": "cell-updates/s", "h2d_bytes_per_step": host_in.nbytes / steps,
            "d2h_bytes_per_step": (out_bytes + 8 * steps) / steps}


def run_case(args):
    """Single uniform-grid case (the profiling workload): levels=1, n^d cells, CFL steps only."""
    import torch

    import paper_1603_05211_gb300 as m

    m.build()
    m.load()
    nb = args.n // 8
    prec = args.precision
    if args.dim == 2:
        s = m.Solver(dim=2, precision=prec, levels=1, base_blocks=(nb, nb, 1), cfl=0.5)
        s.init_state(mi.IC_QUADRANTS, mi.quadrant_params(SEED))
    else:
        s = m.Solver(dim=3, precision=prec, levels=1, base_blocks=(nb, nb, nb), lo=(-1, -1, -1), hi=(1, 1, 1), cfl=0.5)
        s.init_state(mi.IC_ELLIPSOID, mi.ellipsoid_params(SEED))
    for _ in range(args.warmup):
        s.step(0.0, sync=False)
    s.profile_enable(True)
    for _ in range(args.steps):
        s.step(0.0, sync=False)
    p = s.profile_read()
    hbm_peak, _ = measured_peaks()
    ach = p["fv_bytes"] / (p["fv_ms"] * 1e-3) / 1e9
    cells = args.n ** args.dim * args.steps
    print(json.dumps({"case": f"uniform{args.dim}d_{prec}_{args.n}", "fv_launches": p["fv_launches"],
                      "fv_avg_ms": p["fv_ms"] / max(1, p["fv_launches"]), "fv_GBps": ach,
                      "fv_frac_hbm": ach / hbm_peak, "cell_updates_per_s_fv_only": cells / (p["fv_ms"] * 1e-3)}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--case", default="adaptive", choices=["adaptive", "uniform"],
                    help="uniform: only the stage kernel on an n^d grid (profiling workload)")
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--dim", type=int, default=2)
    ap.add_argument("--precision", default="fp32")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.case == "uniform":
        run_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
