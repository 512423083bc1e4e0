"""Launch-shape autotuner: picks the CTA shapes of the persistent kernels and the
stage kernel for one workload by timing whole steps, and caches the choice in a
JSON file.

The shape is the four arguments of ``mrfv_set_launch_shape``: CTAs per SM of the
grid-stride kernels, of the one-block-per-CTA kernels and of the finite-volume
stage kernels, and the stage kernel of the MR scheme.  Every kernel loops over
its device-resident work list, so a shape changes the time of a step and never
its result.  The sweep is a coordinate descent: starting from the library's
defaults, each parameter in turn takes every value of its range while the others
stay at their best so far, for a few passes.  Each candidate runs on a fresh
solver from the caller's factory (same initial state), takes ``warmup`` untimed
steps (the first one captures the step graph) and is timed over ``steps`` steps
with CUDA events on the solver's stream.

The cache maps a workload key (device, SM count and the configuration that
decides the work lists) to the chosen shape and its time.  Its path is the
``path`` argument, else ``$MRFV_AUTOTUNE_CACHE``, else
``~/.cache/paper_1603_05211_gb300/launch_shapes.json``.
"""
from __future__ import annotations

import json
import os
import tempfile

# values tried per parameter; 0 means the library's default
SPACE = {
    "grid_ctas_per_sm": [0, 1, 2, 4, 8],
    "block_ctas_per_sm": [0, 2, 4, 8, 16],
    "fv_ctas_per_sm": [0, 1, 2, 4, 8],
    "stage_kernel": [0, 1, 2, 3, 4, 5],
}
DEFAULT_SHAPE = {k: 0 for k in SPACE}
# configuration fields that decide the work lists and the kernels a step runs
KEY_FIELDS = ("dim", "precision", "levels", "base_blocks", "bc", "adapt", "criterion", "lts", "scheme",
              "clustering", "proposer", "lts_remesh", "eps_r")


def cache_path(path: str | None = None) -> str:
    if path:
        return path
    env = os.environ.get("MRFV_AUTOTUNE_CACHE")
    if env:
        return env
    return os.path.join(os.path.expanduser("~"), ".cache", "paper_1603_05211_gb300", "launch_shapes.json")


def workload_key(config: dict, device: str, sm_count: int) -> str:
    """Stable key of a workload: the device and the configuration fields that
    decide the work (missing fields count as None)."""
    parts = {"device": device, "sms": int(sm_count)}
    for f in KEY_FIELDS:
        v = config.get(f)
        parts[f] = list(v) if isinstance(v, (tuple, list)) else v
    return json.dumps(parts, sort_keys=True)


def load_cache(path: str | None = None) -> dict:
    p = cache_path(path)
    try:
        with open(p) as fh:
            data = json.load(fh)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def lookup(key: str, path: str | None = None) -> dict | None:
    """The cached entry of a key ({"shape": ..., "ms_per_step": ...}) or None."""
    e = load_cache(path).get(key)
    if not isinstance(e, dict) or not isinstance(e.get("shape"), dict):
        return None
    if set(e["shape"]) != set(SPACE):
        return None
    return e


def store(key: str, entry: dict, path: str | None = None) -> str:
    """Merge one entry into the cache file (written atomically); returns the path."""
    p = cache_path(path)
    os.makedirs(os.path.dirname(os.path.abspath(p)), exist_ok=True)
    data = load_cache(p)
    data[key] = entry
    fd, tmp = tempfile.mkstemp(dir=os.path.dirname(os.path.abspath(p)), suffix=".tmp")
    with os.fdopen(fd, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, p)
    return p


def coordinate_descent(measure, space: dict | None = None, start: dict | None = None, passes: int = 2):
    """Minimise measure(shape) -> ms over the product of the value lists in
    `space`, one parameter at a time.  Returns (best shape, best ms, trials),
    trials = [(shape, ms)] in the order measured; a shape is measured once."""
    space = space or SPACE
    best = dict(start or DEFAULT_SHAPE)
    seen = {}

    def cost(shape):
        k = tuple(sorted(shape.items()))
        if k not in seen:
            seen[k] = float(measure(dict(shape)))
        return seen[k]

    best_ms = cost(best)
    trials_order = [dict(best)]
    for _ in range(max(1, passes)):
        changed = False
        for name, values in space.items():
            for v in values:
                if v == best[name]:
                    continue
                cand = dict(best)
                cand[name] = v
                k = tuple(sorted(cand.items()))
                fresh = k not in seen
                ms = cost(cand)
                if fresh:
                    trials_order.append(dict(cand))
                if ms < best_ms:
                    best, best_ms, changed = cand, ms, True
        if not changed:
            break
    trials = [(s, seen[tuple(sorted(s.items()))]) for s in trials_order]
    return best, best_ms, trials


def time_steps(solver, steps: int, warmup: int, dt: float = 0.0) -> float:
    """ms per step of `steps` asynchronous steps after `warmup` untimed ones
    (CUDA events on the solver's stream)."""
    import torch

    for _ in range(max(1, warmup)):
        solver.step(dt, sync=False)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    solver.synchronize()
    a.record(solver.stream)
    for _ in range(steps):
        solver.step(dt, sync=False)
    b.record(solver.stream)
    solver.synchronize()
    return a.elapsed_time(b) / steps


def tune(make, steps: int = 20, warmup: int = 5, passes: int = 2, space: dict | None = None, dt: float = 0.0):
    """Sweep the launch shapes of the workload that make() builds (a fresh,
    initialised Solver per call).  Returns {"shape", "ms_per_step",
    "default_ms_per_step", "trials"}."""

    def measure(shape):
        s = make()
        try:
            try:
                s.set_launch_shape(**shape)
            except Exception as e:  # a stage kernel this configuration does not have
                if getattr(e, "code", None) == -1:
                    return float("inf")
                raise
            return time_steps(s, steps, warmup, dt)
        finally:
            s.close()

    best, best_ms, trials = coordinate_descent(measure, space=space, passes=passes)
    default_ms = next(ms for sh, ms in trials if sh == DEFAULT_SHAPE)
    return {"shape": best, "ms_per_step": best_ms, "default_ms_per_step": default_ms,
            "trials": [{"shape": sh, "ms_per_step": ms} for sh, ms in trials]}


def tuned_shape(make, config: dict, path: str | None = None, retune: bool = False, **kw) -> dict:
    """The cached shape of this workload on the current device, tuning (and
    caching) it first when absent or when `retune`."""
    import torch

    dev = torch.cuda.current_device()
    props = torch.cuda.get_device_properties(dev)
    key = workload_key(config, props.name, props.multi_processor_count)
    if not retune:
        e = lookup(key, path)
        if e is not None:
            return dict(e, cached=True)
    r = tune(make, **kw)
    entry = {"shape": r["shape"], "ms_per_step": r["ms_per_step"], "default_ms_per_step": r["default_ms_per_step"],
             "candidates": len(r["trials"])}
    store(key, entry, path)
    return dict(entry, cached=False)
