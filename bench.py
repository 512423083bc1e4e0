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

Multi-GPU: the single-GPU path has no exchange step; N ranks run N
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


def aggregate_ranks(ms: float, cells: float, world: int, dev) -> tuple:
    """Whole-job throughput of N replicas: the slowest rank's time (max over
    ranks) and the cell-updates of all ranks (sum), over the default process
    group when world > 1.  Returns (max ms, cell-updates/s)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(ms)], dtype=torch.float64, device=dev)
    c = torch.tensor([float(cells)], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
    ms_max = float(t.item())
    return ms_max, float(c.item()) / (ms_max * 1e-3)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def measured_bf16_tflops():
    """Burst bf16 tensor peak (a kernel timed alone), measured, else the fallback."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    return 1900.0, "fallback"


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


def uniform_roofline(m, torch, hbm_peak, steps=6, scheme="muscl_rk2"):
    """Stage kernel alone on a uniform 8192^2 single-precision grid (state 1 GB per
    buffer, far above L2): algorithmic bytes per launch / CUDA-event duration.
    MUSCL-Hancock: one stage per step, 2 nv words per cell."""
    s = m.Solver(dim=2, precision="fp32", levels=1, base_blocks=(1024, 1024, 1), cfl=0.4 if scheme == "hancock" else 0.5,
                 scheme=scheme)
    s.init_state(mi.IC_QUADRANTS, mi.quadrant_params(SEED))
    for _ in range(2):
        s.step(0.0, sync=False)
    s.profile_enable(True)
    for _ in range(steps):
        s.step(0.0, sync=False)
    p = s.profile_read()
    s.profile_enable(False)
    achieved = p["fv_bytes"] / (p["fv_ms"] * 1e-3) / 1e9
    out = {"workload": "uniform2d_fp32_8192", "scheme": scheme, "bound": "hbm", "achieved": round(achieved, 1),
           "peak": hbm_peak, "unit": "GB/s", "frac": round(achieved / hbm_peak, 4),
           "launches": p["fv_launches"], "avg_launch_ms": round(p["fv_ms"] / max(1, p["fv_launches"]), 4),
           "cell_updates_per_s": 8192 * 8192 * steps / (p["fv_ms"] * 1e-3),
           "kernel": stage_kernel_names(p.get("fv_kernels", 0))}
    s.close()
    del s
    torch.cuda.empty_cache()
    return out


# DRAM traffic of the stage kernel per launch on the default workload, from an ncu
# capture summarised under profiles/: a line
#   bench-traffic: kernel=<name> workload=<workload> source_sha256=<hash> bytes_per_launch=<N>
# The figure is reported only while the kernel's source still has that hash (the
# counters describe the kernel as it was built then); otherwise traffic is null.
KERNEL_SOURCES = {"k_fvt": ["paper_1603_05211_gb300/csrc/fvt.cu"],
                  "k_fv": ["paper_1603_05211_gb300/csrc/fv.cuh"],
                  "k_fvs": ["paper_1603_05211_gb300/csrc/fvh.cuh"],
                  "k_fvp": ["paper_1603_05211_gb300/csrc/fv.cuh"]}


def kernel_source_sha(kernel: str):
    import hashlib

    files = KERNEL_SOURCES.get(kernel)
    if not files:
        return None
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel_label: str, workload: str):
    """(bytes per launch, summary file) of the ncu capture of this kernel on this
    workload, or (None, reason) when there is none for the current source."""
    import glob
    import re

    kernel = kernel_label.split(" ")[0]
    sha = kernel_source_sha(kernel)
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        with open(path) as fh:
            for line in fh:
                mt = re.match(r"\s*bench-traffic: kernel=(\S+) workload=(\S+) source_sha256=(\S+) "
                              r"bytes_per_launch=([0-9.eE+]+)", line)
                if mt and mt.group(1) == kernel and mt.group(2) == workload:
                    if mt.group(3) != sha:
                        return None, f"{os.path.basename(path)}: kernel source changed since the capture"
                    return float(mt.group(4)), os.path.basename(path)
    return None, "no ncu capture of this kernel on this workload"


STAGE_KERNELS = ((1, "k_fv (pencil)"), (2, "k_fvs (staged)"), (4, "k_fv (pencil, two threads per line)"),
                 (8, "k_fvp (pencil on staged primitives)"), (16, "k_fvs (staged MUSCL-Hancock)"),
                 (32, "k_fvt (TMA-staged, packed x/y lines)"))


def stage_kernel_names(mask: int) -> str:
    """Names of the fused reconstruct-flux-update stage kernels a profile saw."""
    names = [n for bit, n in STAGE_KERNELS if mask & bit]
    return " + ".join(names) if names else "stage kernel"


def timed_steps(s, n: int, torch, stream, dt: float = 0.0) -> float:
    """GPU time (ms) of n asynchronous steps (dt <= 0: CFL steps), CUDA events on
    the solver's stream.  The first step (which captures the step graph on the
    host) runs untimed and counts as the mean of the others."""
    if n <= 1:
        s.step(dt, sync=True)
        return 0.0
    s.step(dt, sync=False)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(n - 1):
        s.step(dt, sync=False)
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) * n / (n - 1)


def count_steps_to_end(make, t_end: float) -> int:
    s = make()
    n = 0
    while True:
        dt = s.step(0.0, sync=True)
        n += 1
        if dt <= 0.0 or s.stats()["t"] >= t_end * (1 - 1e-12):
            break
    s.close()
    return n


def collect_snapshots(makes, nsnap, eps, t_end=0.0):
    """Up to nsnap (features at t, MR flags at t + dt) pairs from the runs the
    factories in `makes` build, in turn, each run to t_end (or until nsnap).
    Targets are 255 at positions whose parent block is absent at t (no logit can
    add them there), so snapshots of different trees train together."""
    import numpy as np

    feats, targets = [], []
    for make in makes:
        s = make()
        while len(feats) < nsnap:
            s.analyse(eps)
            f = s.proposer_features()
            parent = [np.zeros(int(np.prod(s.blocks_shape(0))), bool)]
            for l in range(1, s.levels):
                ex = s.get_tree(l - 1).astype(bool)
                up = ex
                for ax in range(ex.ndim):
                    up = np.repeat(up, 2, axis=ax)
                parent.append(up.ravel())
            parent = np.concatenate(parent)
            dt = s.step(0.0, sync=True)
            s.analyse(eps)
            t = np.concatenate([s.get_flags(l)[0].ravel() for l in range(s.levels)]).astype(np.uint8)
            t[~parent] = 255
            feats.append(f)
            targets.append(t)
            if dt <= 0.0 or (t_end > 0 and s.stats()["t"] >= t_end * (1 - 1e-12)):
                break
        s.close()
        if len(feats) >= nsnap:
            break
    return np.stack(feats), np.stack(targets)


def train_minibatch(m, make_full, feats, targets, steps, batch=32, lr=3e-3, seed=0):
    """Adam on random minibatches of the snapshots, on a solver of the same
    geometry with every block present (make_full), from small random weights.
    Returns (weights, record)."""
    import numpy as np

    tr = make_full()
    rng = np.random.default_rng(seed)
    tr.proposer_set_weights((rng.normal(0, 1, m.PROPOSER_NWEIGHTS) * 0.05).astype(np.float32))
    n = feats.shape[0]
    order = rng.permutation(n)
    t0 = time.perf_counter()
    losses = []
    for k in range(steps):
        idx = np.sort(order[np.arange(k * batch, (k + 1) * batch) % n])
        losses.append(tr.proposer_train(feats[idx], targets[idx], steps=1, lr=lr))
    sec = time.perf_counter() - t0
    w = tr.proposer_get_weights()
    tr.close()
    used = targets != 255
    return w, {"snapshots": int(n), "minibatch": batch, "adam_steps": steps,
               "loss_first": losses[0], "loss_last": float(np.mean(losses[-10:])), "seconds": sec,
               "positive_fraction": float((targets[used] == 1).mean())}


def train_proposer(m, make_snap, make_full, nsnap, steps, eps, batch=32):
    """Weights of the learned proposer trained on nsnap snapshots of the runs
    make_snap() builds."""
    feats, targets = collect_snapshots([make_snap] * 8, nsnap, eps)
    return train_minibatch(m, make_full, feats, targets, steps, batch=batch)


def matched_l1_2d(m, torch, stream, t_end=0.25, n=1024, eps=None, cache=None, proposer=False, snapshots=60,
                  train_steps=300, stage_kernel=1):
    """Adaptive MR (finest n^2, level 0 one block) vs the uniform n^2 solve, both
    to t_end, each L1(rho) measured against a uniform (2n)^2 solve restricted to
    n^2 (Section 3); GPU time of each (CUDA events, steps counted beforehand).
    `cache` (a dict) keeps the reference and the uniform run between calls."""
    import numpy as np

    P = mi.quadrant_params(SEED)
    eps = WL["eps"] if eps is None else eps
    levels = (n // 8).bit_length()  # level 0: one block of 8^2 cells
    cache = {} if cache is None else cache

    # Every run of the comparison takes the same stage kernel: the data develops
    # shear-layer instabilities that grow from rounding, so at 4096^2 and above two
    # correct single-precision kernels (which agree to 2e-7 relative L1 over 400
    # fixed steps at 2048^2) end at L1 values 25 % apart after 5800 steps.
    def uniform(k):
        s = m.Solver(dim=2, precision="fp32", levels=1, base_blocks=(k // 8, k // 8, 1), cfl=0.5, t_end=t_end,
                     stream=stream)
        s.init_state(mi.IC_QUADRANTS, P)
        s.set_launch_shape(stage_kernel=stage_kernel)
        return s

    def adaptive(lv=levels, prop=False, w=None):
        s = m.Solver(dim=2, precision="fp32", levels=lv, base_blocks=(1, 1, 1), adapt=True, eps=eps, cfl=0.5,
                     t_end=t_end, stream=stream, proposer=prop)
        s.init_state(mi.IC_QUADRANTS, P)
        s.set_launch_shape(stage_kernel=stage_kernel)
        if w is not None:
            s.proposer_set_weights(w)
        return s

    # reference (2n)^2, restricted to n^2
    if "ref" not in cache:
        r = uniform(2 * n)
        nref = 0
        while nref < 1000000:
            dt = r.step(0.0, sync=True)
            nref += 1
            if dt <= 0.0 or r.stats()["t"] >= t_end * (1 - 1e-12):
                break
        rho = r.download_level(0)[0][0]
        r.close()
        torch.cuda.empty_cache()
        cache["ref"], cache["nref"] = rho.reshape(n, 2, n, 2).mean(axis=(1, 3)), nref
    ref, nref = cache["ref"], cache["nref"]
    h2 = (1.0 / n) ** 2
    out = {"t_end": t_end, "finest": n, "levels": levels, "eps": eps,
           "stage_kernel": stage_kernel_names({1: 1, 2: 2, 3: 4, 4: 8, 5: 32}.get(stage_kernel, 0)),
           "reference": f"uniform {2 * n}^2 FP32 restricted to {n}^2", "reference_steps": nref}
    # uniform fine
    if "uniform" not in cache:
        nu = count_steps_to_end(lambda: uniform(n), t_end)
        u = uniform(n)
        ms_u = timed_steps(u, nu, torch, stream)
        l1_u = float(np.abs(u.download_level(0)[0][0] - ref).sum() * h2)
        u.close()
        cache["uniform"] = (nu, ms_u, l1_u)
    nu, ms_u, l1_u = cache["uniform"]
    # adaptive
    na = count_steps_to_end(adaptive, t_end)
    a = adaptive()
    st0 = a.stats()
    ms_a = timed_steps(a, na, torch, stream)
    st1 = a.stats()
    l1_a = float(np.abs(a.project_finest()[0] - ref).sum() * h2)
    a.close()
    leaves = (st1["cell_updates"] - st0["cell_updates"]) / max(1, na)
    out.update({
        "uniform_fine": {"steps": nu, "gpu_ms": ms_u, "l1_rho": l1_u},
        "adaptive": {"steps": na, "gpu_ms": ms_a, "l1_rho": l1_a, "mean_leaf_cells": leaves,
                     "mesh_compression": leaves / n ** 2},
        "accuracy_perturbation": abs(l1_u - l1_a) / l1_u,
        "matched": abs(l1_u - l1_a) / l1_u <= 0.05,
        "time_ratio_adaptive_over_uniform": ms_a / ms_u,
        "overhead_per_leaf": (ms_a / max(1.0, leaves * na)) / (ms_u / (n ** 2 * nu)) - 1.0,
    })
    if proposer:
        # the learned proposer, trained on snapshots of the 8-level workload (1024^2
        # finest, several seeds) on a full-tree solver of that geometry; the control:
        # the MR rule without safety zone (every logit negative)
        if "proposer_w" not in cache:
            wl_levels = WL["levels"]

            def snap_run(seed):
                def make():
                    s = m.Solver(dim=2, precision="fp32", levels=wl_levels, base_blocks=(1, 1, 1), adapt=True,
                                 eps=eps, cfl=0.5, t_end=t_end, stream=stream)
                    s.init_state(mi.IC_QUADRANTS, mi.quadrant_params(seed))
                    return s
                return make

            def full():
                s = m.Solver(dim=2, precision="fp32", levels=wl_levels, base_blocks=(1, 1, 1), cfl=0.5, stream=stream)
                s.init_state(mi.IC_QUADRANTS, mi.quadrant_params(SEED))
                return s

            feats, targets = collect_snapshots([snap_run(k) for k in range(10, 40)], snapshots, eps, t_end)
            cache["proposer_w"] = train_minibatch(m, full, feats, targets, train_steps)
            del feats, targets
        w, tr = cache["proposer_w"]
        out["proposer_training"] = dict(tr, levels=WL["levels"], source="2D MR workload, seeds 10..")
        control = np.zeros(m.PROPOSER_NWEIGHTS, np.float32)
        control[-1] = -1.0
        for name, wt in (("adaptive_control", control), ("adaptive_proposer", w)):
            make = lambda: adaptive(prop=True, w=wt)  # noqa: E731
            na = count_steps_to_end(make, t_end)
            a = make()
            st0 = a.stats()
            ms_p = timed_steps(a, na, torch, stream)
            st1 = a.stats()
            l1_p = float(np.abs(a.project_finest()[0] - ref).sum() * h2)
            a.close()
            lp = (st1["cell_updates"] - st0["cell_updates"]) / max(1, na)
            out[name] = {"steps": na, "gpu_ms": ms_p, "l1_rho": l1_p, "mean_leaf_cells": lp,
                         "mesh_compression": lp / n ** 2, "accuracy_perturbation": abs(l1_u - l1_p) / l1_u,
                         "matched": abs(l1_u - l1_p) / l1_u <= 0.05, "time_ratio_over_uniform": ms_p / ms_u}
    return out


def run_matched2d(args):
    """The matched-L1 comparison in 2D at a chosen finest resolution (--finest, a
    power of two): adaptive MR against the uniform solve at that resolution, L1
    against the uniform solve at twice it (Section 3)."""
    import torch

    import paper_1603_05211_gb300 as m

    m.build()
    m.load()
    stream = torch.cuda.current_stream()
    cache = {}
    for eps in [float(x) for x in args.eps_list.split(",")]:
        r = matched_l1_2d(m, torch, stream, n=args.finest, eps=eps, cache=cache, proposer=args.proposer2d,
                          stage_kernel=args.stage_kernel or 1,
                          snapshots=args.snapshots, train_steps=args.train_steps)
        print(json.dumps({"case": f"matched2d_fp32_{args.finest}", **r}), flush=True)


def blast3d(m, stream, levels, t_end, proposer=False, eps=1e-3):
    s = m.Solver(dim=3, precision="fp32", levels=levels, base_blocks=(2, 2, 2), lo=(-1, -1, -1), hi=(1, 1, 1),
                 adapt=levels > 1, eps=eps, cfl=0.5, t_end=t_end, stream=stream, proposer=proposer)
    s.init_state(mi.IC_ELLIPSOID, mi.ellipsoid_params(SEED))
    return s


def uniform3d(m, stream, n, t_end):
    s = m.Solver(dim=3, precision="fp32", levels=1, base_blocks=(n // 8,) * 3, lo=(-1, -1, -1), hi=(1, 1, 1),
                 cfl=0.5, t_end=t_end, stream=stream)
    s.init_state(mi.IC_ELLIPSOID, mi.ellipsoid_params(SEED))
    return s


def proposer_snapshots(m, stream, levels, t_end, nsnap, make=None, eps=None):
    """(features at t, MR flags at t + dt) pairs from the method's own run (the 3D
    blast, or the solver make() returns)."""
    import numpy as np

    eps = WL["eps"] if eps is None else eps
    s = make() if make is not None else blast3d(m, stream, levels, t_end)
    feats, targets = [], []
    for _ in range(nsnap):
        s.analyse(eps)
        f = s.proposer_features()
        s.step(0.0, sync=True)
        s.analyse(eps)
        feats.append(f)
        targets.append(np.concatenate([s.get_flags(l)[0].ravel() for l in range(s.levels)]))
    s.close()
    return np.stack(feats), np.stack(targets)


def proposer_miss_rate(m, stream, levels, t_end, w, nsteps):
    """Run the plain MR heuristic; at every step compare the proposer's positive
    blocks (plus the blocks the MR rule keeps without its safety zone) with the
    blocks found significant one step later.  miss = significant later but not
    proposed / significant later."""
    import numpy as np

    s = blast3d(m, stream, levels, t_end)
    s.proposer_set_weights(w)
    miss = tot = prop = 0
    for _ in range(nsteps):
        s.analyse(WL["eps"])
        z = s.proposer_infer()
        sig = np.concatenate([s.get_flags(l)[0].ravel() for l in range(s.levels)]).astype(bool)
        ex = np.concatenate([s.get_tree(l).ravel() for l in range(s.levels)]).astype(bool)
        keep = sig.copy()
        # children of significant blocks (refinement by one level) are kept too
        off = 0
        offs = []
        for l in range(s.levels):
            offs.append(off)
            off += int(np.prod(s.blocks_shape(l)))
        for l in range(s.levels - 1):
            sh = s.blocks_shape(l)
            sl = sig[offs[l]:offs[l] + int(np.prod(sh))].reshape(sh)
            ch = np.kron(sl, np.ones((2, 2, 2), bool))
            keep[offs[l + 1]:offs[l + 1] + ch.size] |= ch.ravel()
        proposed = (z > 0) | keep
        s.step(0.0, sync=True)
        s.analyse(WL["eps"])
        sig1 = np.concatenate([s.get_flags(l)[0].ravel() for l in range(s.levels)]).astype(bool)
        miss += int((sig1 & ~proposed).sum())
        tot += int(sig1.sum())
        prop += int(((z > 0) & ~ex).sum())
    s.close()
    return {"miss_rate": miss / max(1, tot), "significant_blocks": tot, "steps": nsteps,
            "proposed_new_blocks_per_step": prop / max(1, nsteps)}


def shock_stop_time(m, stream, levels, frac=0.8, max_steps=20000):
    """Stop rule of the 3D blast workload: the time at which the shock reaches frac
    of the domain half-width, taken as the outer face of the outermost block of
    the finest level that the MR analysis finds significant (run of the plain MR
    heuristic, CFL steps)."""
    import numpy as np

    s = blast3d(m, stream, levels, 0.0)
    nb = 2 << (levels - 1)  # finest blocks per side of [-1, 1]^3
    t = 0.0
    for _ in range(max_steps):
        s.step(0.0, sync=True)
        t = s.stats()["t"]
        f = s.get_flags(levels - 1)[0]
        idx = np.nonzero(f)
        if idx[0].size:
            r = max(float(np.max(np.maximum(np.abs(i / (nb / 2) - 1), np.abs((i + 1) / (nb / 2) - 1))))
                    for i in idx)
            if r >= frac:
                break
    s.close()
    return t


def run_to_end(s, t_end, torch, stream, max_steps=100000):
    """Steps to t_end (CFL steps clipped to end there) with CUDA events around each
    step: (steps, GPU ms).  The first step, which captures the step graph on the
    host, counts as the mean of the others."""
    ev = []
    n = 0
    while n < max_steps:
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        s.step(0.0, sync=False)
        b.record(stream)
        ev.append((a, b))
        n += 1
        torch.cuda.synchronize()
        if s.stats()["t"] >= t_end * (1 - 1e-12):
            break
    times = [x.elapsed_time(y) for x, y in ev]
    if len(times) > 1:
        times[0] = sum(times[1:]) / (len(times) - 1)
    return n, float(sum(times))


def matched_l1_3d(m, torch, stream, L, t_end=0.0, proposer=False, snapshots=60, train_steps=300):
    """3D ellipsoidal blast: adaptive MR (and, with `proposer`, the learned
    proposer) against the uniform solve on the finest grid, all to the stop rule
    of the workload (the shock at 0.8 of the half-width) unless t_end > 0,
    L1(rho) against a uniform solve at twice the finest resolution averaged onto
    it (Section 3); GPU time of each (CUDA events around each step)."""
    import numpy as np

    nfin = 16 << (L - 1)
    rule = "given" if t_end > 0 else "shock at 0.8 of the half-width"
    t_end = t_end if t_end > 0 else shock_stop_time(m, stream, L)
    h3 = (2.0 / nfin) ** 3
    out = {"case": f"blast3d_fp32_L{L - 1}", "finest": nfin, "t_end": t_end, "t_end_rule": rule, "eps": WL["eps"]}
    # reference: uniform at twice the finest resolution, density averaged onto the finest grid
    r = uniform3d(m, stream, 2 * nfin, t_end)
    nref = 0
    while r.stats()["t"] < t_end * (1 - 1e-12):
        r.step(0.0, sync=True)
        nref += 1
    ref = r.download_var(0, 0, 2)
    r.close()
    torch.cuda.empty_cache()
    out["reference"] = {"grid": 2 * nfin, "steps": nref}
    u = uniform3d(m, stream, nfin, t_end)
    nu, ms_u = run_to_end(u, t_end, torch, stream)
    l1_u = float(np.abs(u.download_var(0, 0, 1) - ref).sum() * h3)
    u.close()
    torch.cuda.empty_cache()
    out["uniform_fine"] = {"steps": nu, "gpu_ms": ms_u, "l1_rho": l1_u}
    runs = [("adaptive", False, None)]
    if proposer:
        # learned proposer: trained on snapshots of the 5-level blast workload (256^3
        # finest; ellipsoids of several seeds, each run to this stop time) on a
        # full-tree solver of that geometry; the control arm: the MR rule without
        # safety zone (every logit negative)
        def snap_run(seed):
            def make():
                s = m.Solver(dim=3, precision="fp32", levels=5, base_blocks=(2, 2, 2), lo=(-1, -1, -1),
                             hi=(1, 1, 1), adapt=True, eps=WL["eps"], cfl=0.5, t_end=t_end, stream=stream)
                s.init_state(mi.IC_ELLIPSOID, mi.ellipsoid_params(seed))
                return s
            return make

        def full():
            s = m.Solver(dim=3, precision="fp32", levels=5, base_blocks=(2, 2, 2), lo=(-1, -1, -1), hi=(1, 1, 1),
                         cfl=0.5, stream=stream)
            s.init_state(mi.IC_ELLIPSOID, mi.ellipsoid_params(SEED))
            return s

        feats, targets = collect_snapshots([snap_run(k) for k in range(10, 60)], snapshots, WL["eps"], t_end)
        w, tr = train_minibatch(m, full, feats, targets, train_steps)
        del feats, targets
        out["proposer_training"] = dict(tr, levels=5, source="3D blast workload, seeds 10..")
        control = np.zeros(m.PROPOSER_NWEIGHTS, np.float32)
        control[-1] = -1.0
        out["proposer_eval"] = proposer_miss_rate(m, stream, L, t_end, w, 40)
        out["control_eval"] = proposer_miss_rate(m, stream, L, t_end, control, 40)
        runs += [("adaptive_control", True, control), ("adaptive_proposer", True, w)]
    for name, prop, w in runs:
        a = blast3d(m, stream, L, t_end, proposer=prop)
        if prop:
            a.proposer_set_weights(w)
        st0 = a.stats()
        na, ms_a = run_to_end(a, t_end, torch, stream)
        st1 = a.stats()
        l1_a = float(np.abs(a.project_finest()[0] - ref).sum() * h3)
        a.close()
        torch.cuda.empty_cache()
        leaves = (st1["cell_updates"] - st0["cell_updates"]) / max(1, na)
        pert = abs(l1_u - l1_a) / l1_u
        out[name] = {"steps": na, "gpu_ms": ms_a, "l1_rho": l1_a, "mean_leaf_cells": leaves,
                     "mesh_compression": leaves / nfin ** 3, "accuracy_perturbation": pert,
                     "matched": pert <= 0.05, "time_ratio_over_uniform": ms_a / ms_u}
    return out


def run_matched3d(args):
    """--case matched3d: matched_l1_3d with the learned proposer."""
    import torch

    import paper_1603_05211_gb300 as m

    m.build()
    m.load()
    stream = torch.cuda.current_stream()
    out = matched_l1_3d(m, torch, stream, args.levels3d, t_end=args.t_end3d, proposer=True,
                        snapshots=args.snapshots, train_steps=args.train_steps)
    print(json.dumps(out), flush=True)


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


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:  # noqa: BLE001
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_omp_uniform(budget_s: float, n: int = 1024, max_steps: int = 200):
    """The oracle's OpenMP build (the same C source, its finite-volume loops over
    blocks on every host core) on a uniform n^2 FP64 grid of the seeded
    four-quadrant data: cell-updates/s, steps, seconds, threads."""
    import oracle

    o = oracle.Oracle(2, 1, (n // 8, n // 8, 1), openmp=True)
    o.init(mi.IC_QUADRANTS, mi.quadrant_params(SEED))
    o.step(o.dt(WL["cfl"]))  # warm-up (thread team, first touch)
    steps = 0
    t0 = time.perf_counter()
    while steps < max_steps and time.perf_counter() - t0 < budget_s:
        o.step(o.dt(WL["cfl"]))
        steps += 1
    el = time.perf_counter() - t0
    return n * n * steps / el, steps, el, oracle.threads(True)


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
    shape, tuned = {}, None
    if args.autotune:
        # the launch shape from the autotuner's cache, swept and cached first when absent
        from paper_1603_05211_gb300 import autotune

        tuned = autotune.tuned_shape(lambda: make_solver(m, stream), dict(WL, criterion="mr", scheme="muscl_rk2"),
                                     retune=args.autotune == "sweep", steps=20, warmup=5, passes=2)
        shape = tuned["shape"]
    s = make_solver(m, stream)
    if shape:
        s.set_launch_shape(**shape)
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
    prof_g = s.profile_read()
    launches = prof_g["launches"]
    st1 = s.stats()
    cells = st1["cell_updates"] - st0["cell_updates"]
    # the same steps once more with every stage launch bracketed by CUDA events
    # (eager launches: events cannot be read per replay inside a graph), in the
    # stage kernel the captured step graph uses
    graph_stage = {1: 1, 2: 2, 4: 3, 8: 4, 32: 5}.get(prof_g.get("graph_fv_kernels", 0), 0)
    if graph_stage:
        s.set_launch_shape(stage_kernel=graph_stage)
    s.profile_enable(True)
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        s.step(0.0, sync=False)
    prof = s.profile_read()
    s.profile_enable(False)
    if graph_stage:
        s.set_launch_shape(**dict(shape or {}, stage_kernel=(shape or {}).get("stage_kernel", 0)))
    ms_max, value = aggregate_ranks(ms, cells, world, dev)
    hbm_peak, peak_kind = measured_peaks()

    result = None
    if rank == 0:
        fv_ach = prof["fv_bytes"] / (prof["fv_ms"] * 1e-3) / 1e9 if prof["fv_ms"] > 0 else 0.0
        kname = stage_kernel_names(prof.get("fv_kernels", 0))
        traffic, traffic_src = profiled_traffic(kname, WORKLOAD)
        roof = {"bound": "hbm", "achieved": round(fv_ach, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(fv_ach / hbm_peak, 4), "traffic": traffic, "traffic_source": traffic_src,
                "kernel": kname, "peak_kind": peak_kind,
                "timing": "CUDA events around each stage launch, same workload and step count, eager launches",
                "launches": prof["fv_launches"],
                "avg_launch_us": round(prof["fv_ms"] * 1e3 / max(1, prof["fv_launches"]), 2),
                "bytes_per_launch": prof["fv_bytes"] / max(1, prof["fv_launches"])}
        try:
            roof_u = uniform_roofline(m, torch, hbm_peak)
        except Exception as e:  # noqa: BLE001
            roof_u = {"error": str(e)}
        try:
            roof_h = uniform_roofline(m, torch, hbm_peak, steps=4, scheme="hancock")
        except Exception as e:  # noqa: BLE001
            roof_h = {"error": str(e)}
        # end to end through the C interface: host initial state in, host state out
        e2e = run_e2e(m, torch, stream, args.steps)
        # adaptive against uniform-fine GPU time at matched L1 (Section 3): the default
        # workload (1024^2 finest), the same data at 4096^2 finest, and the 3D blast
        matched = {}
        try:
            matched["2d_1024"] = matched_l1_2d(m, torch, stream)
        except Exception as e:  # noqa: BLE001
            matched["2d_1024"] = {"error": str(e)}
        for sk in (1, 5):
            try:
                c4096 = {}
                matched[f"2d_4096_stage_kernel_{sk}"] = [
                    matched_l1_2d(m, torch, stream, n=4096, eps=e, cache=c4096, stage_kernel=sk) for e in (3e-4, 2e-4)]
                del c4096
            except Exception as e:  # noqa: BLE001
                matched[f"2d_4096_stage_kernel_{sk}"] = {"error": str(e)}
            torch.cuda.empty_cache()
        torch.cuda.empty_cache()
        try:
            matched["3d_blast_256"] = matched_l1_3d(m, torch, stream, 5)
        except Exception as e:  # noqa: BLE001
            matched["3d_blast_256"] = {"error": str(e)}
        torch.cuda.empty_cache()
        # CPU baseline: the oracle on a bounded sample of the same workload
        ob, osteps, osec = oracle_sample(budget_s=float(os.environ.get("MRFV_ORACLE_BUDGET", "15")))
        try:
            omp_v, omp_steps, omp_s, omp_threads = oracle_omp_uniform(
                budget_s=float(os.environ.get("MRFV_ORACLE_BUDGET", "15")) / 2)
            omp = {"value": omp_v, "unit": "cell-updates/s", "cores": omp_threads, "kind": "oracle (OpenMP build)",
                   "sample": f"{omp_steps} FP64 steps of the uniform 1024^2 grid of the same initial data "
                             f"({omp_s:.1f} s)"}
        except Exception as e:  # noqa: BLE001
            omp = {"error": str(e)}
        result = {
            "metric": "cell-updates/s", "value": value, "unit": "cell-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "levels": 8, "finest": 1024, "eps": WL["eps"], "cfl": WL["cfl"],
                       "ic": "seeded four-quadrant Riemann (seed 0)", "l2": "flushed between timed steps",
                       "leaves_per_step": cells / args.steps / 64, "parallelism": f"replicas x{world}",
                       "launch_shape": shape or "library defaults",
                       **({"autotune": {k: tuned[k] for k in ("ms_per_step", "default_ms_per_step", "cached")
                                        if k in tuned}} if tuned else {})},
            "roofline": roof,
            "roofline_uniform": roof_u, "roofline_hancock": roof_h,
            "cpu_baseline": {"value": ob, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
                             "sample": f"{osteps} FP64 oracle steps of the same workload from t=0 ({osec:.1f} s)",
                             "cpu_model": cpu_model(), "host_cores": os.cpu_count(),
                             "uniform_fv_all_cores": omp},
            "e2e": e2e,
            "matched_l1": matched,
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

    def pinned(shape):
        return torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()

    host_in = pinned((s.nv,) + s.cells_shape(L))
    ref.download_level(L, out=host_in)
    host_out = [pinned((s.nv,) + s.cells_shape(l)) for l in range(WL["levels"])]
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
        a, _ = s.download_level(l, out=host_out[l])
        out_bytes += a.nbytes
    el = time.perf_counter() - t0
    st1 = s.stats()
    s.close()
    cells = st1["cell_updates"] - st0["cell_updates"]
    return {"value": cells / el, "unit": "cell-updates/s", "h2d_bytes_per_step": host_in.nbytes / steps,
            "d2h_bytes_per_step": (out_bytes + 8 * steps) / steps}


def run_proposer(args):
    """The learned proposer's tensor-core convolution on the 3D blast hierarchy
    (levels3d levels, every block position of every level): CUDA-event time of the
    three tcgen05 layers per inference, algorithmic flops, fraction of the measured
    bf16 peak.  The GEMMs are 128 positions x 16 channels x K in {216, 432}: the
    kernel is bound by gathering its im2col rows, not by the tensor pipe."""
    import numpy as np
    import torch

    import paper_1603_05211_gb300 as m

    m.build()
    m.load()
    stream = torch.cuda.current_stream()
    L = args.levels3d
    s = blast3d(m, stream, L, 1.0, proposer=False)
    for _ in range(5):
        s.step(0.0, sync=False)
    s.analyse(WL["eps"])
    rng = np.random.default_rng(0)
    s.proposer_set_weights((rng.normal(0, 1, m.PROPOSER_NWEIGHTS) * 0.05).astype(np.float32))
    for _ in range(max(3, args.warmup)):
        s.proposer_infer()
    s.profile_enable(True)
    n = max(1, args.steps)
    for _ in range(n):
        s.proposer_infer()
    p = s.profile_read()
    s.profile_enable(False)
    peak, kind = measured_bf16_tflops()
    tf = p["prop_flops"] / (p["prop_ms"] * 1e-3) / 1e12
    npos = s.positions
    print(json.dumps({"case": f"proposer_conv_blast3d_L{L - 1}", "positions": npos, "inferences": n,
                      "conv_us_per_inference": 1000.0 * p["prop_ms"] / n,
                      "roofline": {"bound": "tensor", "achieved": round(tf, 3), "peak": peak, "unit": "TFLOP/s",
                                   "frac": round(tf / peak, 6), "peak_kind": kind,
                                   "kernel": "k_prop_conv_tc (tcgen05.mma kind::f16, 3 layers)"}}), flush=True)
    s.close()


def laxliu_solver(m, stream, n_cells, levels, scheme, adapt=False, lts=False, crit="mr", eps=0.0023, eps_w=0.05,
                  eps_r=0.0):
    """Lax-Liu #6 solver on [0,1]^2, single precision, Berger-Rigoutsos clustering"""
    return m.Solver(dim=2, precision="fp32", levels=levels, base_blocks=(n_cells // (8 << (levels - 1)),) * 2 + (1,),
                    adapt=adapt, lts=lts, criterion=crit, eps=eps, eps_w=eps_w, eta_tol=0.8, cfl=0.5,
                    stream=stream, scheme=scheme, clustering="br", eps_r=eps_r)


def laxliu_reference(m, torch, stream, nref, te):
    """density of the AMR scheme on a uniform nref^2 grid after 5120 nref/4096 steps
    to te (the reference of Tables 2-4), and the step count"""
    r = laxliu_solver(m, stream, nref, 1, "hancock")
    r.init_state(mi.IC_QUADRANTS, mi.laxliu6_params())
    nr_steps = 5120 * nref // 4096
    for _ in range(nr_steps):
        r.step(te / nr_steps, sync=False)
    rho_ref = r.download_level(0)[0][0]
    r.close()
    torch.cuda.empty_cache()
    return rho_ref, nr_steps


def run_richardson(args):
    """The Richardson estimate added to the AMR criterion (Section 2.2) on the
    paper's 2D benchmark: Lax-Liu configuration 6 to t_e = 0.25 with N_I fixed
    finest-level steps at scale level L, the AMR scheme, density-gradient flags
    eps_rho = 0.05 clustered by Berger-Rigoutsos, single precision.  Variants, with
    global and with level-dependent steps: gradient flags only, gradient flags and
    the estimate (eps_r = 1e-3), the estimate alone.  Reports L1(rho) against the
    4096^2 reference, accumulated leaves, GPU time of the timed run, and from a
    profiled eager run the estimate's time per launch, the blocks it estimates
    and its patch stage cell-updates per second."""
    import numpy as np
    import torch

    import paper_1603_05211_gb300 as m

    m.build()
    m.load()
    stream = torch.cuda.current_stream()
    P = mi.laxliu6_params()
    te = 0.25
    nref = args.laxliu_ref
    rho_ref, nr_steps = laxliu_reference(m, torch, stream, nref, te)
    # patch stage cell-updates per block of the AMR scheme in 2D (blocks away from
    # the walls): fine stages on 12^2 and 8^2 cells, the coarse stage on 4^2
    per_block = 144 + 64 + 16
    out = {"case": "richardson_laxliu6", "t_end": te, "scheme": "hancock",
           "reference": {"grid": nref, "steps": nr_steps}, "rows": []}
    for L in [int(x) for x in args.laxliu_levels.split(",")]:
        n = 1 << L
        NI = 160 << (L - 7)
        dt = te / NI
        levels = L - 2
        k = nref // n
        ref = rho_ref.reshape(n, k, n, k).mean(axis=(1, 3))
        row = {"L": L, "N": n, "N_I": NI}
        variants = []
        for lts in (False, True):
            t = "LT" if lts else ""
            variants += [(f"AMR{t}", lts, 0.05, 0.0), (f"AMR{t}+R", lts, 0.05, 1e-3), (f"R{t}", lts, 1e9, 1e-3)]
        for name, lts, eps_w, eps_r in variants:
            steps = NI >> (levels - 1) if lts else NI
            mult = (1 << (levels - 1)) if lts else 1

            def make():
                a = laxliu_solver(m, stream, n, levels, "hancock", adapt=True, lts=lts, crit="grad", eps_w=eps_w,
                                  eps_r=eps_r)
                a.init_state(mi.IC_QUADRANTS, P)
                return a

            a = make()
            Lf = 0
            for _ in range(steps):
                Lf += a.stats()["total_leaves"] * 64 * mult
                a.step(dt, sync=True)
            l1 = float(np.abs(a.project_finest()[0] - ref).sum() / (n * n))
            a.close()
            a = make()
            ms = timed_steps(a, steps, torch, stream, dt=dt)
            a.close()
            # profiled eager steps from halfway through the run
            a = make()
            for _ in range(steps // 2):
                a.step(dt, sync=False)
            a.profile_enable(True)
            nprof = max(1, min(20, steps - steps // 2))
            for _ in range(nprof):
                a.step(dt, sync=False)
            p = a.profile_read()
            a.close()
            torch.cuda.empty_cache()
            ent = {"eps_w": eps_w, "eps_r": eps_r, "l1_rho": l1, "leaves_1e6": Lf / 1e6,
                   "leaf_compression_pct": 100.0 * Lf / (NI * n * n), "gpu_ms": ms, "ms_per_step": ms / steps}
            if p["rich_launches"]:
                ent.update({"rich_launches_per_step": p["rich_launches"] / nprof,
                            "rich_ms_per_launch": p["rich_ms"] / p["rich_launches"],
                            "rich_blocks_per_launch": p["rich_blocks"] / p["rich_launches"],
                            "rich_us_per_block": 1e3 * p["rich_ms"] / max(1.0, p["rich_blocks"]),
                            "rich_patch_cell_updates_per_s": per_block * p["rich_blocks"] / (p["rich_ms"] * 1e-3),
                            "rich_pct_of_step": 100.0 * (p["rich_ms"] / nprof) / (ms / steps)})
            row[name] = ent
        out["rows"].append(row)
        print(json.dumps(row), flush=True)
    print(json.dumps(out), flush=True)


def run_richardson3d(args):
    """The Richardson estimate on the paper's 3D case (Section 4.2): the rotated
    ellipsoid on [-2,2]^3 with N_I = 16 * 2^(L-5) fixed steps to t_e = 0.28 at
    scale level L, the AMR scheme, density and pressure gradient flags
    (eps_rho = eps_p = 0.05) clustered by Berger-Rigoutsos, single precision,
    global and level-dependent steps, without and with the estimate
    (eps_r = 1e-3).  Reports accumulated leaves, GPU time per step and the
    estimate's time, blocks and patch stage cell-updates per second (3D AMR
    scheme: fine stages on 12^3 and 8^3 cells, the coarse stage on 4^3)."""
    import torch

    import paper_1603_05211_gb300 as m

    m.build()
    m.load()
    stream = torch.cuda.current_stream()
    P = mi.paper3d_params()
    te = 0.28
    per_block = 12 ** 3 + 8 ** 3 + 4 ** 3
    out = {"case": "richardson_paper3d", "t_end": te, "scheme": "hancock", "rows": []}
    for L in [int(x) for x in args.paper3d_levels.split(",")]:
        n = 1 << L
        NI = 16 << (L - 5)
        dt = te / NI
        levels = L - 2
        row = {"L": L, "N": n, "N_I": NI}
        for name, lts, eps_r in (("AMR", False, 0.0), ("AMR+R", False, 1e-3), ("AMRLT", True, 0.0),
                                 ("AMRLT+R", True, 1e-3)):
            steps = NI >> (levels - 1) if lts else NI
            mult = (1 << (levels - 1)) if lts else 1

            def make():
                a = m.Solver(dim=3, precision="fp32", levels=levels, base_blocks=(1, 1, 1), lo=(-2.0,) * 3,
                             hi=(2.0,) * 3, adapt=True, lts=lts, criterion="grad", eps_w=0.05, eps_p=0.05,
                             eta_tol=0.8, cfl=0.4, stream=stream, scheme="hancock", clustering="br", eps_r=eps_r)
                a.init_state(mi.IC_ROTATED_ELLIPSOID, P)
                return a

            a = make()
            Lf = 0
            for _ in range(steps):
                Lf += a.stats()["total_leaves"] * 512 * mult
                a.step(dt, sync=True)
            a.close()
            a = make()
            ms = timed_steps(a, steps, torch, stream, dt=dt)
            a.close()
            a = make()
            for _ in range(steps // 2):
                a.step(dt, sync=False)
            a.profile_enable(True)
            nprof = max(1, min(10, steps - steps // 2))
            for _ in range(nprof):
                a.step(dt, sync=False)
            p = a.profile_read()
            a.close()
            torch.cuda.empty_cache()
            ent = {"eps_r": eps_r, "leaves_1e6": Lf / 1e6, "leaf_compression_pct": 100.0 * Lf / (NI * n ** 3),
                   "gpu_ms": ms, "ms_per_step": ms / steps}
            if p["rich_launches"]:
                ent.update({"rich_launches_per_step": p["rich_launches"] / nprof,
                            "rich_ms_per_launch": p["rich_ms"] / p["rich_launches"],
                            "rich_blocks_per_launch": p["rich_blocks"] / p["rich_launches"],
                            "rich_us_per_block": 1e3 * p["rich_ms"] / max(1.0, p["rich_blocks"]),
                            "rich_patch_cell_updates_per_s": per_block * p["rich_blocks"] / (p["rich_ms"] * 1e-3),
                            "rich_pct_of_step": 100.0 * (p["rich_ms"] / nprof) / (ms / steps)})
            row[name] = ent
        out["rows"].append(row)
        print(json.dumps(row), flush=True)
    print(json.dumps(out), flush=True)


def run_adaptive3d(args):
    """A short adaptive MR run of the 3D blast (--levels3d levels, CFL steps):
    --warmup untimed steps, then --steps timed steps of the captured graph (the
    workload of the 3D launch list)."""
    import torch

    import paper_1603_05211_gb300 as m

    m.build()
    m.load()
    stream = torch.cuda.current_stream()
    s = blast3d(m, stream, args.levels3d, 0.0)
    for _ in range(max(1, args.warmup)):
        s.step(0.0, sync=False)
    st0 = s.stats()
    ms = timed_steps(s, args.steps, torch, stream)
    st1 = s.stats()
    cells = st1["cell_updates"] - st0["cell_updates"]
    print(json.dumps({"case": f"adaptive3d_fp32_L{args.levels3d - 1}", "steps": args.steps,
                      "ms_per_step": ms / max(1, args.steps), "leaf_cells_per_step": cells / max(1, args.steps),
                      "cell_updates_per_s": cells / (ms * 1e-3) if ms > 0 else None}), flush=True)


def run_adaptive2d(args):
    """The default workload's steps alone (no side measurements; the workload of the
    2D launch list and of the stage kernel's traffic capture): --warmup untimed
    steps, --steps steps of the captured graph timed with CUDA events (L2 flushed
    before each), then the same number of eager steps with every stage launch
    bracketed by CUDA events (the roofline pass of the default line)."""
    import torch

    import paper_1603_05211_gb300 as m

    m.build()
    m.load()
    stream = torch.cuda.current_stream()
    s = make_solver(m, stream)
    if args.stage_kernel:
        s.set_launch_shape(stage_kernel=args.stage_kernel)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    for _ in range(max(1, args.warmup)):
        s.step(0.0, sync=False)
    s.synchronize()
    st0 = s.stats()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        ev[k][0].record(stream)
        s.step(0.0, sync=False)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    cells = s.stats()["cell_updates"] - st0["cell_updates"]
    s.profile_enable(True)
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        s.step(0.0, sync=False)
    p = s.profile_read()
    hbm_peak, _ = measured_peaks()
    ach = p["fv_bytes"] / (p["fv_ms"] * 1e-3) / 1e9 if p["fv_ms"] > 0 else 0.0
    print(json.dumps({"case": WORKLOAD, "steps": args.steps, "ms_per_step": ms / max(1, args.steps),
                      "cell_updates_per_s": cells / (ms * 1e-3) if ms > 0 else None,
                      "stage_kernel": stage_kernel_names(p.get("fv_kernels", 0)),
                      "stage_avg_us": 1e3 * p["fv_ms"] / max(1, p["fv_launches"]),
                      "stage_bytes_per_launch": p["fv_bytes"] / max(1, p["fv_launches"]),
                      "stage_frac_hbm": ach / hbm_peak}), flush=True)


def run_autotune(args):
    """The launch-shape autotuner on one workload (a fresh sweep, printed with
    every candidate's time): --dim 2, the default adaptive 2D MR workload;
    --dim 3, the 3D blast with --levels3d levels."""
    import torch

    import paper_1603_05211_gb300 as m
    from paper_1603_05211_gb300 import autotune

    m.build()
    m.load()
    stream = torch.cuda.current_stream()
    if args.dim == 3:
        make = lambda: blast3d(m, stream, args.levels3d, 0.0)  # noqa: E731
        name = f"blast3d_fp32_L{args.levels3d - 1}"
    else:
        make = lambda: make_solver(m, stream)  # noqa: E731
        name = WORKLOAD
    r = autotune.tune(make, steps=20, warmup=5, passes=2)
    print(json.dumps({"case": "autotune", "workload": name, **r}), flush=True)


def run_laxliu(args):
    """The paper's 2D benchmark (Section 4.1, Tables 2-4): Lax-Liu configuration 6
    on [0,1]^2 to t_e = 0.25 with N_I = 160 * 2^(L-7) fixed steps at scale levels
    L = 7..10 (finest 2^L cells per side), single precision on the GPU.
    FV: uniform 2^L grid (MR scheme: van Albada / AUSM+ / RK2; AMR scheme:
    MUSCL-Hancock / Minmod / AUSMDV).  MR, MRLT: eps = 0.0023; AMR, AMRLT:
    density-gradient flags eps_rho = 0.05 clustered by Berger-Rigoutsos
    (eta 0.8), the AMR scheme.  Reference: the AMR scheme on a uniform 4096^2
    grid, 5120 steps, restricted by cell means.  Reports L1(rho), rates,
    perturbation, accumulated cells and leaves (with compression), GPU time and
    time compression against the FV run of the same scheme."""
    import numpy as np
    import torch

    import paper_1603_05211_gb300 as m

    m.build()
    m.load()
    stream = torch.cuda.current_stream()
    P = mi.laxliu6_params()
    te = 0.25
    Ls = [int(x) for x in args.laxliu_levels.split(",")]

    def solver(n_cells, levels, scheme, adapt=False, lts=False, crit="mr", eps=0.0023):
        return laxliu_solver(m, stream, n_cells, levels, scheme, adapt=adapt, lts=lts, crit=crit, eps=eps)

    nref = args.laxliu_ref
    rho_ref, nr_steps = laxliu_reference(m, torch, stream, nref, te)
    out = {"case": "laxliu6", "t_end": te, "reference": {"grid": nref, "steps": nr_steps, "scheme": "hancock"},
           "rows": []}

    def l1_at(rho, n):
        k = nref // n
        ref = rho_ref.reshape(n, k, n, k).mean(axis=(1, 3))
        return float(np.abs(rho - ref).sum() / (n * n))

    for L in Ls:
        n = 1 << L
        NI = 160 << (L - 7)
        dt = te / NI
        levels = L - 2  # blocks of 8 cells: level 0 has one block
        row = {"L": L, "N": n, "N_I": NI}
        for scheme, fvname in (("muscl_rk2", "FV_MR"), ("hancock", "FV_AMR")):
            u = solver(n, 1, scheme)
            u.init_state(mi.IC_QUADRANTS, P)
            ms = timed_steps(u, NI, torch, stream, dt=dt)
            row[fvname] = {"l1_rho": l1_at(u.download_level(0)[0][0], n), "gpu_ms": ms}
            u.close()
        variants = (("MR", "muscl_rk2", False, "mr", "FV_MR"), ("MRLT", "muscl_rk2", True, "mr", "FV_MR"),
                    ("AMR", "hancock", False, "grad", "FV_AMR"), ("AMRLT", "hancock", True, "grad", "FV_AMR"))
        for name, scheme, lts, crit, fvname in variants:
            steps = NI >> (levels - 1) if lts else NI
            # counting run: accumulated cells and leaves per finest step
            a = solver(n, levels, scheme, adapt=True, lts=lts, crit=crit)
            a.init_state(mi.IC_QUADRANTS, P)
            C = Lf = 0
            for _ in range(steps):
                st = a.stats()
                mult = (1 << (levels - 1)) if lts else 1
                C += st["total_blocks"] * 64 * mult
                Lf += st["total_leaves"] * 64 * mult
                a.step(dt, sync=True)
            l1 = l1_at(a.project_finest()[0], n)
            a.close()
            # timed run
            a = solver(n, levels, scheme, adapt=True, lts=lts, crit=crit)
            a.init_state(mi.IC_QUADRANTS, P)
            ms = timed_steps(a, steps, torch, stream, dt=dt)
            a.close()
            fv = row[fvname]
            row[name] = {"l1_rho": l1, "perturbation_pct": 100.0 * abs(l1 - fv["l1_rho"]) / fv["l1_rho"],
                         "cells_1e6": C / 1e6, "cell_compression_pct": 100.0 * C / (NI * n * n),
                         "leaves_1e6": Lf / 1e6, "leaf_compression_pct": 100.0 * Lf / (NI * n * n),
                         "gpu_ms": ms, "time_compression_pct": 100.0 * ms / fv["gpu_ms"]}
            torch.cuda.empty_cache()
        out["rows"].append(row)
        print(json.dumps(row), flush=True)
    for key in ("FV_MR", "FV_AMR", "MR", "MRLT", "AMR", "AMRLT"):
        e = [r_[key]["l1_rho"] for r_ in out["rows"]]
        out.setdefault("rates", {})[key] = [float(np.log2(e[i] / e[i + 1])) for i in range(len(e) - 1)]
    print(json.dumps(out), flush=True)


def run_epssweep(args):
    """The threshold study of Section 4.1: Lax-Liu configuration 6 at scale level
    L (default 10), MR and MRLT with eps in {0.0005, 0.0008, 0.0010, 0.0023,
    0.0025, 0.0028} (the paper's values, sorted), against the uniform FV-MR run
    and the 4096^2 AMR-scheme reference of --case laxliu: L1(rho), perturbation,
    accumulated cells and leaves, GPU time."""
    import numpy as np
    import torch

    import paper_1603_05211_gb300 as m

    m.build()
    m.load()
    stream = torch.cuda.current_stream()
    P = mi.laxliu6_params()
    te = 0.25
    L = args.eps_level
    n = 1 << L
    NI = 160 << (L - 7)
    dt = te / NI
    levels = L - 2
    nref = args.laxliu_ref

    def solver(n_cells, lv, adapt=False, lts=False, eps=0.0023, scheme="muscl_rk2"):
        return m.Solver(dim=2, precision="fp32", levels=lv, base_blocks=(n_cells // (8 << (lv - 1)),) * 2 + (1,),
                        adapt=adapt, lts=lts, criterion="mr", eps=eps, cfl=0.5, stream=stream, scheme=scheme)

    r = solver(nref, 1, scheme="hancock")
    r.init_state(mi.IC_QUADRANTS, P)
    nr_steps = 5120 * nref // 4096
    for _ in range(nr_steps):
        r.step(te / nr_steps, sync=False)
    rho_ref = r.download_level(0)[0][0]
    r.close()
    torch.cuda.empty_cache()
    k = nref // n
    ref = rho_ref.reshape(n, k, n, k).mean(axis=(1, 3))
    u = solver(n, 1)
    u.init_state(mi.IC_QUADRANTS, P)
    ms_fv = timed_steps(u, NI, torch, stream, dt=dt)
    l1_fv = float(np.abs(u.download_level(0)[0][0] - ref).sum() / (n * n))
    u.close()
    out = {"case": "epssweep_laxliu6", "L": L, "N_I": NI, "reference": {"grid": nref, "steps": nr_steps},
           "FV_MR": {"l1_rho": l1_fv, "gpu_ms": ms_fv}, "rows": []}
    for eps in (0.0005, 0.0008, 0.0010, 0.0023, 0.0025, 0.0028):
        row = {"eps": eps}
        for name, lts in (("MR", False), ("MRLT", True)):
            steps = NI >> (levels - 1) if lts else NI
            a = solver(n, levels, adapt=True, lts=lts, eps=eps)
            a.init_state(mi.IC_QUADRANTS, P)
            C = Lf = 0
            mult = (1 << (levels - 1)) if lts else 1
            for _ in range(steps):
                st = a.stats()
                C += st["total_blocks"] * 64 * mult
                Lf += st["total_leaves"] * 64 * mult
                a.step(dt, sync=True)
            l1 = float(np.abs(a.project_finest()[0] - ref).sum() / (n * n))
            a.close()
            a = solver(n, levels, adapt=True, lts=lts, eps=eps)
            a.init_state(mi.IC_QUADRANTS, P)
            ms = timed_steps(a, steps, torch, stream, dt=dt)
            a.close()
            row[name] = {"l1_rho": l1, "perturbation_pct": 100.0 * abs(l1 - l1_fv) / l1_fv,
                         "cell_compression_pct": 100.0 * C / (NI * n * n),
                         "leaf_compression_pct": 100.0 * Lf / (NI * n * n),
                         "gpu_ms": ms, "time_compression_pct": 100.0 * ms / ms_fv}
            torch.cuda.empty_cache()
        out["rows"].append(row)
        print(json.dumps(row), flush=True)
    print(json.dumps(out), flush=True)


def run_paper3d(args):
    """The paper's 3D benchmark (Section 4.2, Tables 6-8): the rotated ellipsoid on
    [-2,2]^3 to t_e = 0.28 with N_I = 16 * 2^(L-5) fixed steps at scale levels
    L = 5..8 (finest 2^L cells per side, level 0 one block of 8^3, the paper's
    8^3 base mesh), single precision on the GPU.  FV: uniform 2^L grid of each
    scheme.  MR, MRLT: eps = 0.013; AMR, AMRLT: density and pressure gradient
    flags (eps_rho = eps_p = 0.05) clustered by Berger-Rigoutsos (eta 0.8), the
    AMR scheme.  Reference: the AMR scheme on a uniform 1024^3 grid with CFL 0.4
    steps to t_e, cell means onto each level.  L1(rho) = sum |rho - rho_ref| h^3.
    Reports L1, rates, perturbation, accumulated cells and leaves (with
    compression), GPU time and time compression against the FV run of the same
    scheme."""
    import numpy as np
    import torch

    import paper_1603_05211_gb300 as m

    m.build()
    m.load()
    stream = torch.cuda.current_stream()
    P = mi.paper3d_params()
    te = 0.28
    Ls = [int(x) for x in args.paper3d_levels.split(",")]
    lo, hi = (-2.0, -2.0, -2.0), (2.0, 2.0, 2.0)

    def solver(n_cells, levels, scheme, adapt=False, lts=False, crit="mr", cfl=0.4, t_end=0.0):
        nb = n_cells // (8 << (levels - 1))
        return m.Solver(dim=3, precision="fp32", levels=levels, base_blocks=(nb, nb, nb), lo=lo, hi=hi,
                        adapt=adapt, lts=lts, criterion=crit, eps=0.013, eps_w=0.05, eps_p=0.05, eta_tol=0.8,
                        cfl=cfl, t_end=t_end, stream=stream, scheme=scheme, clustering="br")

    nref = args.paper3d_ref
    r = solver(nref, 1, "hancock", t_end=te)
    r.init_state(mi.IC_ROTATED_ELLIPSOID, P)
    nr_steps = 0
    t0 = time.perf_counter()
    while r.stats()["t"] < te * (1 - 1e-12) and nr_steps < 100000:
        r.step(0.0, sync=True)
        nr_steps += 1
    ref_s = time.perf_counter() - t0
    # cell means of the reference on each level: coarsened on the device to the
    # finest level asked for (a factor of at most 8), then on the host
    Lmax = max(Ls)
    base = r.download_var(0, 0, nref >> Lmax)
    refs = {}
    for L in Ls:
        k = 1 << (Lmax - L)
        n = 1 << L
        refs[L] = base.reshape(n, k, n, k, n, k).mean(axis=(1, 3, 5))
    r.close()
    torch.cuda.empty_cache()
    out = {"case": "paper3d_rotated_ellipsoid", "t_end": te,
           "reference": {"grid": nref, "steps": nr_steps, "cfl": 0.4, "scheme": "hancock", "wall_s": ref_s},
           "rows": []}

    def l1_at(rho, L):
        n = 1 << L
        return float(np.abs(rho - refs[L]).sum() * (4.0 / n) ** 3)

    for L in Ls:
        n = 1 << L
        NI = 16 << (L - 5)
        dt = te / NI
        levels = L - 2  # blocks of 8 cells: level 0 has one block
        row = {"L": L, "N": n, "N_I": NI}
        for scheme, fvname in (("muscl_rk2", "FV_MR"), ("hancock", "FV_AMR")):
            u = solver(n, 1, scheme)
            u.init_state(mi.IC_ROTATED_ELLIPSOID, P)
            ms = timed_steps(u, NI, torch, stream, dt=dt)
            row[fvname] = {"l1_rho": l1_at(u.download_var(0, 0, 1), L), "gpu_ms": ms}
            u.close()
        variants = (("MR", "muscl_rk2", False, "mr", "FV_MR"), ("MRLT", "muscl_rk2", True, "mr", "FV_MR"),
                    ("AMR", "hancock", False, "grad", "FV_AMR"), ("AMRLT", "hancock", True, "grad", "FV_AMR"))
        for name, scheme, lts, crit, fvname in variants:
            steps = NI >> (levels - 1) if lts else NI
            a = solver(n, levels, scheme, adapt=True, lts=lts, crit=crit)
            a.init_state(mi.IC_ROTATED_ELLIPSOID, P)
            C = Lf = 0
            mult = (1 << (levels - 1)) if lts else 1
            for _ in range(steps):
                st = a.stats()
                C += st["total_blocks"] * 512 * mult
                Lf += st["total_leaves"] * 512 * mult
                a.step(dt, sync=True)
            l1 = l1_at(a.project_finest()[0], L)
            a.close()
            a = solver(n, levels, scheme, adapt=True, lts=lts, crit=crit)
            a.init_state(mi.IC_ROTATED_ELLIPSOID, P)
            ms = timed_steps(a, steps, torch, stream, dt=dt)
            a.close()
            fv = row[fvname]
            row[name] = {"l1_rho": l1, "perturbation_pct": 100.0 * abs(l1 - fv["l1_rho"]) / fv["l1_rho"],
                         "cells_1e6": C / 1e6, "cell_compression_pct": 100.0 * C / (NI * n ** 3),
                         "leaves_1e6": Lf / 1e6, "leaf_compression_pct": 100.0 * Lf / (NI * n ** 3),
                         "gpu_ms": ms, "time_compression_pct": 100.0 * ms / fv["gpu_ms"]}
            torch.cuda.empty_cache()
        out["rows"].append(row)
        print(json.dumps(row), flush=True)
    for key in ("FV_MR", "FV_AMR", "MR", "MRLT", "AMR", "AMRLT"):
        e = [r_[key]["l1_rho"] for r_ in out["rows"]]
        out.setdefault("rates", {})[key] = [float(np.log2(e[i] / e[i + 1])) for i in range(len(e) - 1)]
    print(json.dumps(out), flush=True)


def run_case(args):
    """Single uniform-grid case (the profiling workload): levels=1, n^d cells, CFL steps only."""
    import torch

    import paper_1603_05211_gb300 as m

    m.build()
    m.load()
    nb = args.n // 8
    prec = args.precision
    cfl = 0.4 if args.scheme == "hancock" else 0.5
    if args.dim == 2:
        s = m.Solver(dim=2, precision=prec, levels=1, base_blocks=(nb, nb, 1), cfl=cfl, scheme=args.scheme)
        s.init_state(mi.IC_QUADRANTS, mi.quadrant_params(SEED))
    else:
        s = m.Solver(dim=3, precision=prec, levels=1, base_blocks=(nb, nb, nb), lo=(-1, -1, -1), hi=(1, 1, 1), cfl=cfl,
                     scheme=args.scheme)
        s.init_state(mi.IC_ELLIPSOID, mi.ellipsoid_params(SEED))
    if args.stage_kernel:
        s.set_launch_shape(stage_kernel=args.stage_kernel)
    for _ in range(args.warmup):
        s.step(0.0, sync=False)
    s.profile_enable(True)
    for _ in range(args.steps):
        s.step(0.0, sync=False)
    p = s.profile_read()
    hbm_peak, _ = measured_peaks()
    ach = p["fv_bytes"] / (p["fv_ms"] * 1e-3) / 1e9
    cells = args.n ** args.dim * args.steps
    print(json.dumps({"case": f"uniform{args.dim}d_{prec}_{args.n}", "scheme": args.scheme, "fv_launches": p["fv_launches"],
                      "fv_avg_ms": p["fv_ms"] / max(1, p["fv_launches"]), "fv_GBps": ach,
                      "fv_frac_hbm": ach / hbm_peak, "cell_updates_per_s_fv_only": cells / (p["fv_ms"] * 1e-3)}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--case", default="adaptive",
                    choices=["adaptive", "uniform", "matched3d", "proposer", "laxliu", "paper3d", "epssweep",
                             "richardson", "matched2d", "autotune", "adaptive3d", "adaptive2d"],
                    help="uniform: only the stage kernel on an n^d grid (profiling workload); "
                         "matched3d: 3D blast, adaptive (heuristic / learned proposer) vs uniform at matched L1")
    ap.add_argument("--levels3d", type=int, default=5)
    ap.add_argument("--t-end3d", dest="t_end3d", type=float, default=0.0,
                    help="end time of --case matched3d; 0: the workload's stop rule (shock at 0.8 of the half-width)")
    ap.add_argument("--snapshots", type=int, default=1000)
    ap.add_argument("--train-steps", dest="train_steps", type=int, default=300)
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--laxliu-levels", dest="laxliu_levels", default="7,8,9,10")
    ap.add_argument("--laxliu-ref", dest="laxliu_ref", type=int, default=4096, help="reference grid of --case laxliu")
    ap.add_argument("--paper3d-levels", dest="paper3d_levels", default="5,6,7,8")
    ap.add_argument("--eps-level", dest="eps_level", type=int, default=10, help="scale level L of --case epssweep")
    ap.add_argument("--paper3d-ref", dest="paper3d_ref", type=int, default=1024, help="reference grid of --case paper3d")
    ap.add_argument("--dim", type=int, default=2)
    ap.add_argument("--precision", default="fp32")
    ap.add_argument("--scheme", default="muscl_rk2", choices=["muscl_rk2", "hancock"],
                    help="finite-volume scheme of the uniform case")
    ap.add_argument("--finest", type=int, default=4096, help="finest resolution of --case matched2d")
    ap.add_argument("--eps-list", dest="eps_list", default="1e-3", help="MR thresholds of --case matched2d")
    ap.add_argument("--proposer2d", action="store_true", help="--case matched2d: also the learned proposer")
    ap.add_argument("--autotune", default="", choices=["", "cache", "sweep"],
                    help="default workload: take the launch shape from the autotuner (cache: the cached "
                         "choice, swept first when absent; sweep: sweep again)")
    ap.add_argument("--stage-kernel", dest="stage_kernel", type=int, default=0, choices=[0, 1, 2, 3, 4, 5],
                    help="uniform case: 0 by leaf count, 1 pencil kernel, 2 staged kernel, "
                         "3 split pencil kernel, 4 pencil kernel on staged primitives")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.case == "uniform":
        run_case(args)
    elif args.case == "matched3d":
        run_matched3d(args)
    elif args.case == "proposer":
        run_proposer(args)
    elif args.case == "adaptive2d":
        run_adaptive2d(args)
    elif args.case == "adaptive3d":
        run_adaptive3d(args)
    elif args.case == "autotune":
        run_autotune(args)
    elif args.case == "matched2d":
        run_matched2d(args)
    elif args.case == "richardson":
        if args.dim == 3:
            run_richardson3d(args)
        else:
            run_richardson(args)
    elif args.case == "laxliu":
        run_laxliu(args)
    elif args.case == "paper3d":
        run_paper3d(args)
    elif args.case == "epssweep":
        run_epssweep(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
