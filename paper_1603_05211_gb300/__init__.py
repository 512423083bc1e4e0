"""GB300-native adaptive multiresolution finite volumes for the compressible Euler equations.

A thin ctypes binding of ``libmrfv.so`` (the C interface in ``include/mrfv.h``):
every step of the method runs in the library's CUDA kernels; this module only
marshals arguments.  PyTorch provides the device memory (the library's arena is
a ``torch.uint8`` CUDA tensor) and the CUDA stream.  There is no CPU path: if the
library is missing or no GPU is present, construction raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmrfv.so")

OK = 0
ERR_ARG, ERR_POOL_FULL, ERR_NONPHYSICAL, ERR_TIMEOUT, ERR_CUDA, ERR_STATE, ERR_TREE = -1, -2, -3, -4, -5, -6, -7
FP64, FP32 = 0, 1
BC_TRANSMISSIVE, BC_PERIODIC = 0, 1
CRIT_MR, CRIT_GRAD = 0, 1
SCHEME_MUSCL_RK2, SCHEME_HANCOCK = 0, 1
CLUSTER_ROWS, CLUSTER_BR = 0, 1
MAX_LEVELS = 12


class MRFVError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"mrfv error {code}: {msg}")
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("precision", ctypes.c_int), ("levels", ctypes.c_int),
        ("base_blocks", ctypes.c_int * 3),
        ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
        ("bc", ctypes.c_int), ("gamma", ctypes.c_double), ("cfl", ctypes.c_double),
        ("t_end", ctypes.c_double), ("adapt", ctypes.c_int), ("criterion", ctypes.c_int),
        ("eps", ctypes.c_double), ("eps_w", ctypes.c_double), ("eta_tol", ctypes.c_double),
        ("lts", ctypes.c_int), ("pool_blocks", ctypes.c_int64),
        ("stream", ctypes.c_void_p), ("device_arena", ctypes.c_void_p), ("arena_bytes", ctypes.c_size_t),
        ("use_graph", ctypes.c_int), ("proposer", ctypes.c_int), ("scheme", ctypes.c_int),
        ("clustering", ctypes.c_int), ("eps_p", ctypes.c_double), ("lts_remesh", ctypes.c_int),
        ("eps_r", ctypes.c_double), ("proposer_dense", ctypes.c_int),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("levels", ctypes.c_int),
        ("blocks", ctypes.c_int64 * MAX_LEVELS), ("leaves", ctypes.c_int64 * MAX_LEVELS),
        ("total_blocks", ctypes.c_int64), ("total_leaves", ctypes.c_int64), ("leaf_cells", ctypes.c_int64),
        ("pool_capacity", ctypes.c_int64), ("t", ctypes.c_double), ("last_dt", ctypes.c_double),
        ("steps", ctypes.c_int64), ("cell_updates", ctypes.c_int64),
    ]


class Profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("fv_launches", ctypes.c_int64),
                ("fv_ms", ctypes.c_double), ("fv_bytes", ctypes.c_double),
                ("prop_launches", ctypes.c_int64), ("prop_ms", ctypes.c_double), ("prop_flops", ctypes.c_double),
                ("fv_kernels", ctypes.c_int), ("graph_fv_kernels", ctypes.c_int),
                ("rich_launches", ctypes.c_int64), ("rich_ms", ctypes.c_double), ("rich_blocks", ctypes.c_double)]


# exported symbols of include/mrfv.h with their ctypes signatures
_P, _I, _D, _I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
_DP = ctypes.POINTER(ctypes.c_double)
_U8 = ctypes.POINTER(ctypes.c_uint8)
_I64P = ctypes.POINTER(ctypes.c_int64)
SIGNATURES = {
    "mrfv_config_default": (_I, [ctypes.POINTER(Config)]),
    "mrfv_arena_bytes": (ctypes.c_size_t, [ctypes.POINTER(Config)]),
    "mrfv_create": (_I, [ctypes.POINTER(Config), ctypes.POINTER(_P)]),
    "mrfv_destroy": (_I, [_P]),
    "mrfv_last_error": (ctypes.c_char_p, [_P]),
    "mrfv_init_state": (_I, [_P, _I, _DP, _I]),
    "mrfv_analyse": (_I, [_P, _D, _I64P]),
    "mrfv_adapt": (_I, [_P, _I, _I64P]),
    "mrfv_compute_dt": (_I, [_P, _DP]),
    "mrfv_fill_ghosts": (_I, [_P, _I, _I]),
    "mrfv_step": (_I, [_P, _D, _DP]),
    "mrfv_step_level": (_I, [_P, _I, _D]),
    "mrfv_restrict": (_I, [_P, _I]),
    "mrfv_conserved_totals": (_I, [_P, _DP, _I]),
    "mrfv_get_stats": (_I, [_P, ctypes.POINTER(Stats)]),
    "mrfv_download_level": (_I, [_P, _I, _DP, _I64, _U8]),
    "mrfv_download_var": (_I, [_P, _I, _I, _I, _DP, _I64]),
    "mrfv_upload_level": (_I, [_P, _I, _DP, _I64]),
    "mrfv_project_finest": (_I, [_P, _DP, _I64]),
    "mrfv_get_tree": (_I, [_P, _I, _U8, _I64]),
    "mrfv_set_tree": (_I, [_P, _U8, _I64]),
    "mrfv_get_flags": (_I, [_P, _I, _U8, _DP, _I64]),
    "mrfv_synchronize": (_I, [_P]),
    "mrfv_prolong": (_I, [_P, _I]),
    "mrfv_wait_selftest": (_I, [_P, _I64, _I]),
    "mrfv_profile_enable": (_I, [_P, _I]),
    "mrfv_profile_read": (_I, [_P, ctypes.POINTER(Profile)]),
    "mrfv_set_launch_shape": (_I, [_P, _I, _I, _I, _I]),
    "mrfv_cfl_dt_noalloc": (_I, [_I, _I, _P, _I64, _I64, _I64, _DP, _D, _D, _P, _P]),
    "mrfv_proposer_set_weights": (_I, [_P, ctypes.POINTER(ctypes.c_float), _I64]),
    "mrfv_proposer_get_weights": (_I, [_P, ctypes.POINTER(ctypes.c_float), _I64]),
    "mrfv_proposer_features": (_I, [_P, ctypes.POINTER(ctypes.c_float), _I64]),
    "mrfv_proposer_infer": (_I, [_P, ctypes.POINTER(ctypes.c_float), _I64]),
    "mrfv_proposer_train": (_I, [_P, ctypes.POINTER(ctypes.c_float), _U8, _I, _I, ctypes.c_float,
                                 ctypes.POINTER(ctypes.c_double)]),
    "mrfv_proposer_grad": (_I, [_P, ctypes.POINTER(ctypes.c_float), _U8, _I, ctypes.POINTER(ctypes.c_float), _I64,
                                ctypes.POINTER(ctypes.c_double)]),
    "mrfv_proposer_activations": (_I, [_P, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float), _I64]),
}
PROPOSER_NWEIGHTS = 8673

_lib = None


def build(force: bool = False) -> str:
    """Compile libmrfv.so for sm_103a (nvcc); see build.py."""
    return _build.build(force=force)


def load() -> ctypes.CDLL:
    """Load libmrfv.so; raises when it has not been built (there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_1603_05211_gb300.build() first")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(_DP)


def _u8(a):
    return a.ctypes.data_as(_U8)


class Solver:
    """One solver context (``mrfv_ctx``) on the current CUDA device.

    Keyword arguments mirror ``mrfv_config``.  ``precision`` is ``"fp64"`` or
    ``"fp32"``; ``criterion`` is ``"mr"`` or ``"grad"``.  The device arena is a
    PyTorch tensor owned by this object; work goes to ``stream`` (a
    ``torch.cuda.Stream``; default: the current stream).
    """

    def __init__(self, dim=2, precision="fp64", levels=1, base_blocks=(1, 1, 1), lo=(0.0, 0.0, 0.0),
                 hi=(1.0, 1.0, 1.0), bc=BC_TRANSMISSIVE, gamma=1.4, cfl=0.5, t_end=0.0, adapt=False,
                 criterion="mr", eps=1e-3, eps_w=0.05, eta_tol=0.8, lts=False, pool_blocks=0, stream=None,
                 use_graph=True, proposer=False, scheme="muscl_rk2", clustering="rows", eps_p=0.0,
                 lts_remesh=True, eps_r=0.0, proposer_dense=False):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("mrfv needs a CUDA GPU; there is no CPU path")
        lib = load()
        self.lib = lib
        cfg = Config()
        lib.mrfv_config_default(ctypes.byref(cfg))
        cfg.dim = dim
        cfg.precision = FP32 if str(precision).lower() in ("fp32", "float32", "1") else FP64
        cfg.levels = levels
        bb = (list(base_blocks) + [1, 1, 1])[:3]
        for d in range(3):
            cfg.base_blocks[d] = int(bb[d]) if d < dim else 1
            cfg.lo[d] = float((list(lo) + [0.0] * 3)[d])
            cfg.hi[d] = float((list(hi) + [1.0] * 3)[d])
        cfg.bc = bc
        cfg.gamma, cfg.cfl, cfg.t_end = gamma, cfl, t_end
        cfg.adapt = int(bool(adapt))
        cfg.criterion = CRIT_GRAD if str(criterion).lower() in ("grad", "1") else CRIT_MR
        cfg.eps, cfg.eps_w, cfg.eta_tol, cfg.eps_p = eps, eps_w, eta_tol, eps_p
        cfg.lts_remesh = int(bool(lts_remesh))
        cfg.eps_r = float(eps_r)
        cfg.lts = int(bool(lts))
        cfg.pool_blocks = int(pool_blocks)
        cfg.use_graph = int(bool(use_graph))
        cfg.proposer = int(bool(proposer))
        cfg.proposer_dense = int(bool(proposer_dense))
        cfg.scheme = SCHEME_HANCOCK if str(scheme).lower() in ("hancock", "1") else SCHEME_MUSCL_RK2
        cfg.clustering = CLUSTER_BR if str(clustering).lower() in ("br", "berger-rigoutsos", "1") else CLUSTER_ROWS
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        cfg.stream = self.stream.cuda_stream
        nbytes = lib.mrfv_arena_bytes(ctypes.byref(cfg))
        if nbytes == 0:
            raise MRFVError(ERR_ARG, "invalid configuration")
        self.arena = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        cfg.device_arena = self.arena.data_ptr()
        cfg.arena_bytes = nbytes
        h = ctypes.c_void_p()
        rc = lib.mrfv_create(ctypes.byref(cfg), ctypes.byref(h))
        if rc != OK:
            raise MRFVError(rc, lib.mrfv_last_error(None).decode())
        self._h = h
        self.cfg = cfg
        self.dim, self.nv, self.levels, self.L = dim, dim + 2, levels, levels - 1
        self.base_blocks = tuple(cfg.base_blocks[d] for d in range(3))

    # ------------------------------------------------------------------ helpers
    def _check(self, rc: int):
        if rc != OK:
            raise MRFVError(rc, self.lib.mrfv_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self.lib.mrfv_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def cells_shape(self, l: int):
        return tuple(reversed([self.base_blocks[d] * 8 << l for d in range(self.dim)]))

    def blocks_shape(self, l: int):
        return tuple(reversed([self.base_blocks[d] << l for d in range(self.dim)]))

    # ------------------------------------------------------------------ C ABI
    def init_state(self, kind: int, params) -> None:
        p = np.ascontiguousarray(params, dtype=np.float64)
        self._check(self.lib.mrfv_init_state(self._h, kind, _dp(p), len(p)))

    def analyse(self, eps: float) -> int:
        n = ctypes.c_int64(0)
        self._check(self.lib.mrfv_analyse(self._h, eps, ctypes.byref(n)))
        return n.value

    def adapt(self) -> int:
        n = ctypes.c_int64(0)
        self._check(self.lib.mrfv_adapt(self._h, 0, ctypes.byref(n)))
        return n.value

    def compute_dt(self) -> float:
        d = ctypes.c_double(0.0)
        self._check(self.lib.mrfv_compute_dt(self._h, ctypes.byref(d)))
        return d.value

    def fill_ghosts(self, level: int, buffer: int = 0) -> None:
        self._check(self.lib.mrfv_fill_ghosts(self._h, level, buffer))

    def step(self, dt: float = 0.0, sync: bool = True):
        """One step (dt <= 0: CFL step).  Returns the dt used when ``sync``."""
        if sync:
            d = ctypes.c_double(0.0)
            self._check(self.lib.mrfv_step(self._h, dt, ctypes.byref(d)))
            return d.value
        self._check(self.lib.mrfv_step(self._h, dt, None))
        return None

    def step_level(self, level: int, dt_finest: float) -> None:
        self._check(self.lib.mrfv_step_level(self._h, level, dt_finest))

    def restrict(self, fine_level: int = 0) -> None:
        self._check(self.lib.mrfv_restrict(self._h, fine_level))

    def prolong(self, coarse_level: int) -> None:
        """Overwrite every existing block of level coarse_level+1 by the
        third-order prediction from level coarse_level."""
        self._check(self.lib.mrfv_prolong(self._h, coarse_level))

    def totals(self) -> np.ndarray:
        out = np.zeros(5)
        self._check(self.lib.mrfv_conserved_totals(self._h, _dp(out), 5))
        return out[: self.nv]

    def stats(self) -> dict:
        s = Stats()
        self._check(self.lib.mrfv_get_stats(self._h, ctypes.byref(s)))
        return dict(levels=s.levels, blocks=list(s.blocks[: s.levels]), leaves=list(s.leaves[: s.levels]),
                    total_blocks=s.total_blocks, total_leaves=s.total_leaves, leaf_cells=s.leaf_cells,
                    pool_capacity=s.pool_capacity, t=s.t, last_dt=s.last_dt, steps=s.steps,
                    cell_updates=s.cell_updates)

    def download_level(self, level: int, out=None):
        """Dense level (nv, ...) with NaN where absent, and the block existence map.
        out: optional float64 C-contiguous array of that shape to fill (for
        example a view of pinned host memory)."""
        shape = (self.nv,) + self.cells_shape(level)
        if out is None:
            out = np.empty(shape, dtype=np.float64)
        elif out.shape != shape or out.dtype != np.float64 or not out.flags.c_contiguous:
            raise ValueError("download_level: out must be a C-contiguous float64 array of shape %s" % (shape,))
        ex = np.empty(self.blocks_shape(level), dtype=np.uint8)
        self._check(self.lib.mrfv_download_level(self._h, level, _dp(out), out.size, _u8(ex)))
        return out, ex

    def download_var(self, level: int, var: int = 0, coarsen: int = 1) -> np.ndarray:
        """One variable of a dense level, averaged over coarsen^d-cell cubes (NaN where absent)."""
        shape = tuple(n // coarsen for n in self.cells_shape(level))
        out = np.empty(shape, dtype=np.float64)
        self._check(self.lib.mrfv_download_var(self._h, level, var, coarsen, _dp(out), out.size))
        return out

    def upload_level(self, level: int, data) -> None:
        a = np.ascontiguousarray(data, dtype=np.float64)
        self._check(self.lib.mrfv_upload_level(self._h, level, _dp(a), a.size))

    def project_finest(self) -> np.ndarray:
        out = np.empty((self.nv,) + self.cells_shape(self.L), dtype=np.float64)
        self._check(self.lib.mrfv_project_finest(self._h, _dp(out), out.size))
        return out

    def get_tree(self, level: int) -> np.ndarray:
        ex = np.empty(self.blocks_shape(level), dtype=np.uint8)
        self._check(self.lib.mrfv_get_tree(self._h, level, _u8(ex), ex.size))
        return ex

    def set_tree(self, maps) -> None:
        a = np.ascontiguousarray(np.concatenate([np.asarray(m, dtype=np.uint8).ravel() for m in maps]))
        self._check(self.lib.mrfv_set_tree(self._h, _u8(a), a.size))

    def get_flags(self, level: int):
        f = np.empty(self.blocks_shape(level), dtype=np.uint8)
        m = np.empty(self.blocks_shape(level), dtype=np.float64)
        self._check(self.lib.mrfv_get_flags(self._h, level, _u8(f), _dp(m), f.size))
        return f, m

    def synchronize(self) -> None:
        self._check(self.lib.mrfv_synchronize(self._h))

    def wait_selftest(self, iterations: int, complete: bool) -> int:
        """Status of one bounded device wait on a phase that completes only when
        `complete` (OK, or ERR_TIMEOUT once `iterations` tries expired)."""
        return int(self.lib.mrfv_wait_selftest(self._h, int(iterations), int(bool(complete))))

    # ------------------------------------------------------------------ learned proposer
    @property
    def positions(self) -> int:
        """Block positions of every level (the proposer's grid)."""
        return sum(int(np.prod(self.blocks_shape(l))) for l in range(self.levels))

    def adapt_with(self, use_proposer: bool) -> int:
        n = ctypes.c_int64(0)
        self._check(self.lib.mrfv_adapt(self._h, int(bool(use_proposer)), ctypes.byref(n)))
        return n.value

    def proposer_set_weights(self, w) -> None:
        a = np.ascontiguousarray(w, dtype=np.float32)
        self._check(self.lib.mrfv_proposer_set_weights(self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), a.size))

    def proposer_get_weights(self) -> np.ndarray:
        a = np.empty(PROPOSER_NWEIGHTS, dtype=np.float32)
        self._check(self.lib.mrfv_proposer_get_weights(self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), a.size))
        return a

    def proposer_features(self) -> np.ndarray:
        a = np.empty((3, self.positions), dtype=np.float32)
        self._check(self.lib.mrfv_proposer_features(self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), a.size))
        return a

    def proposer_infer(self) -> np.ndarray:
        a = np.empty(self.positions, dtype=np.float32)
        self._check(self.lib.mrfv_proposer_infer(self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), a.size))
        return a

    def proposer_grad(self, feats, targets):
        """(loss, gradient) of the next training step, without the step."""
        f = np.ascontiguousarray(feats, dtype=np.float32)
        t = np.ascontiguousarray(targets, dtype=np.uint8)
        g = np.empty(PROPOSER_NWEIGHTS, np.float32)
        loss = ctypes.c_double(0.0)
        self._check(self.lib.mrfv_proposer_grad(self._h, f.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), _u8(t),
                                                f.shape[0], g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), g.size,
                                                ctypes.byref(loss)))
        return loss.value, g

    def proposer_activations(self):
        """BF16 inputs of layers 2 and 3 of the last inference, [positions][16] each."""
        n = self.positions
        h1 = np.empty((n, 16), np.float32)
        h2 = np.empty((n, 16), np.float32)
        self._check(self.lib.mrfv_proposer_activations(self._h, h1.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                                       h2.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), h1.size))
        return h1, h2

    def proposer_train(self, feats, targets, steps: int, lr: float) -> float:
        f = np.ascontiguousarray(feats, dtype=np.float32)
        t = np.ascontiguousarray(targets, dtype=np.uint8)
        ns = f.shape[0]
        loss = ctypes.c_double(0.0)
        self._check(self.lib.mrfv_proposer_train(self._h, f.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), _u8(t),
                                                 ns, steps, lr, ctypes.byref(loss)))
        return loss.value

    def profile_enable(self, enable: bool = True) -> None:
        self._check(self.lib.mrfv_profile_enable(self._h, int(bool(enable))))

    def set_launch_shape(self, grid_ctas_per_sm: int = 0, block_ctas_per_sm: int = 0, fv_ctas_per_sm: int = 0,
                         stage_kernel: int = 0) -> None:
        self._check(self.lib.mrfv_set_launch_shape(self._h, grid_ctas_per_sm, block_ctas_per_sm, fv_ctas_per_sm,
                                                   stage_kernel))

    def profile_read(self) -> dict:
        p = Profile()
        self._check(self.lib.mrfv_profile_read(self._h, ctypes.byref(p)))
        return dict(launches=p.launches, fv_launches=p.fv_launches, fv_ms=p.fv_ms, fv_bytes=p.fv_bytes,
                    prop_launches=p.prop_launches, prop_ms=p.prop_ms, prop_flops=p.prop_flops,
                    fv_kernels=p.fv_kernels, graph_fv_kernels=p.graph_fv_kernels,
                    rich_launches=p.rich_launches, rich_ms=p.rich_ms, rich_blocks=p.rich_blocks)
