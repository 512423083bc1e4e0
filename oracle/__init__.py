"""CPU oracle of the adaptive multiresolution finite-volume method (FP64, plain C).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use this package; the product path never does.
It shares no code with the CUDA path.  ``build()`` compiles ``liboracle.so`` next
to this file with ``-ffp-contract=off`` so every rounding happens where the C
source says it does.

The oracle's state is one dense array per level (``[v][cell]`` with
``cell = i + n0*(j + n1*k)``), NaN where no block exists, plus a dense byte map of
existing 8^d blocks per level.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mrfv_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
# the same source built with -fopenmp: the finite-volume loops over blocks run on
# every host core (identical results; the multi-core CPU baseline of the bench)
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")

BC_TRANSMISSIVE = 0
BC_PERIODIC = 1
CRIT_MR = 0
CRIT_GRAD = 1
SCHEME_MUSCL_RK2 = 0  # MUSCL / van Albada / AUSM+ / explicit midpoint RK2 (the MR scheme, Section 2)
SCHEME_HANCOCK = 1    # MUSCL-Hancock / Minmod / AUSMDV (the AMR scheme, Section 2)
CLUSTER_ROWS = 0      # gradient flags clustered in runs along the first direction
CLUSTER_BR = 1        # Berger-Rigoutsos clustering into boxes (Section 2.2)


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile liboracle.so (gcc, -O2, no floating-point contraction), or with
    openmp its OpenMP build liboracle_omp.so."""
    out = _LIB_OMP if openmp else _LIB
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off",
                               "-fno-fast-math", "-shared", "-fPIC"] + (["-fopenmp"] if openmp else [])
                              + [_SRC, "-o", tmp, "-lm"])
        os.replace(tmp, out)
    return out


_lib = None
_lib_omp = None


def _load(openmp: bool = False):
    global _lib, _lib_omp
    if (_lib_omp if openmp else _lib) is None:
        lib = ctypes.CDLL(build(openmp=openmp))
        P, I, D, L = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_long
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        u8 = ctypes.POINTER(ctypes.c_uint8)
        lp = ctypes.POINTER(ctypes.c_long)
        sig = {
            "orc_create": (P, [I, I, ip, dp, dp, D, I]),
            "orc_destroy": (None, [P]),
            "orc_init": (I, [P, I, dp, I]),
            "orc_level_cells": (L, [P, I]),
            "orc_level_blocks": (L, [P, I]),
            "orc_get_level": (None, [P, I, dp]),
            "orc_set_level": (None, [P, I, dp]),
            "orc_get_exist": (None, [P, I, u8]),
            "orc_set_exist": (None, [P, I, u8]),
            "orc_get_sig": (None, [P, I, u8, dp]),
            "orc_get_scale": (None, [P, dp]),
            "orc_restrict_all": (None, [P]),
            "orc_dt": (D, [P, D, I]),
            "orc_step": (None, [P, D, I]),
            "orc_analyse": (I, [P, D, I, lp]),
            "orc_adapt": (I, [P, I, D, D, D, I]),
            "orc_totals": (None, [P, dp]),
            "orc_project_finest": (None, [P, dp]),
            "orc_flux": (None, [P, I, dp, dp, dp]),
            "orc_physical_flux": (None, [P, I, dp, dp]),
            "orc_flux_ausmdv": (None, [P, I, dp, dp, dp]),
            "orc_set_scheme": (I, [P, I]),
            "orc_set_clustering": (I, [P, I]),
            "orc_set_eps_p": (I, [P, D]),
            "orc_set_eps_r": (I, [P, D]),
            "orc_rich_bad": (L, [P]),
            "orc_rich_tau": (L, [P, I, D, dp]),
            "orc_set_lts_remesh": (I, [P, I, I, D, D, D, I]),
            "orc_br_cluster": (None, [P, I, u8, D, u8]),
            "orc_predict": (D, [P, I, dp, I, I, I, I]),
            "orc_threads": (I, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        if openmp:
            _lib_omp = lib
        else:
            _lib = lib
    return _lib_omp if openmp else _lib


def threads(openmp: bool = False) -> int:
    """Threads of the finite-volume loops of the (OpenMP) oracle library."""
    return int(_load(openmp).orc_threads())


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _u8(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


class Oracle:
    """Dense per-level FP64 oracle.  ``levels`` counts levels 0..L; level l has
    ``base_blocks * 2^l`` blocks of 8 cells per dimension."""

    def __init__(self, dim: int, levels: int, base_blocks, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0),
                 gamma: float = 1.4, bc: int = BC_TRANSMISSIVE, scheme: int = SCHEME_MUSCL_RK2,
                 clustering: int = CLUSTER_ROWS, openmp: bool = False):
        lib = _load(openmp)
        nb = (ctypes.c_int * 3)(*[int(b) for b in (list(base_blocks) + [1, 1, 1])[:3]])
        lo3 = (ctypes.c_double * 3)(*[float(x) for x in (list(lo) + [0.0] * 3)[:3]])
        hi3 = (ctypes.c_double * 3)(*[float(x) for x in (list(hi) + [1.0] * 3)[:3]])
        self._h = lib.orc_create(dim, levels, nb, lo3, hi3, gamma, bc)
        if not self._h:
            raise ValueError("oracle: bad configuration")
        self.lib = lib
        if lib.orc_set_scheme(self._h, scheme) != 0:
            raise ValueError("oracle: bad scheme")
        self.scheme = scheme
        if lib.orc_set_clustering(self._h, clustering) != 0:
            raise ValueError("oracle: bad clustering")
        self.dim, self.levels, self.L, self.nv = dim, levels, levels - 1, dim + 2
        self.bc = bc
        self.base_blocks = tuple(int(b) for b in (list(base_blocks) + [1, 1, 1])[:3])
        self.lo = tuple(float(x) for x in (list(lo) + [0.0] * 3)[:3])
        self.hi = tuple(float(x) for x in (list(hi) + [1.0] * 3)[:3])

    def __del__(self):
        if getattr(self, "_h", None):
            self.lib.orc_destroy(self._h)
            self._h = None

    # geometry
    def cells_shape(self, l: int):
        n = [b * 8 << l for b in self.base_blocks[: self.dim]]
        return tuple(reversed(n))  # numpy order (k, j, i)

    def blocks_shape(self, l: int):
        n = [b << l for b in self.base_blocks[: self.dim]]
        return tuple(reversed(n))

    def dx(self, l: int):
        return [(self.hi[d] - self.lo[d]) / (self.base_blocks[d] * 8 << l) for d in range(self.dim)]

    # state
    def init(self, kind: int, params) -> None:
        p = np.ascontiguousarray(params, dtype=np.float64)
        self.lib.orc_init(self._h, kind, _dp(p), len(p))

    def get_level(self, l: int) -> np.ndarray:
        out = np.empty((self.nv,) + self.cells_shape(l), dtype=np.float64)
        self.lib.orc_get_level(self._h, l, _dp(out))
        return out

    def set_level(self, l: int, a: np.ndarray) -> None:
        a = np.ascontiguousarray(a, dtype=np.float64)
        assert a.size == self.nv * int(np.prod(self.cells_shape(l)))
        self.lib.orc_set_level(self._h, l, _dp(a))

    def get_exist(self, l: int) -> np.ndarray:
        out = np.empty(self.blocks_shape(l), dtype=np.uint8)
        self.lib.orc_get_exist(self._h, l, _u8(out))
        return out

    def set_exist(self, l: int, ex: np.ndarray) -> None:
        ex = np.ascontiguousarray(ex, dtype=np.uint8)
        self.lib.orc_set_exist(self._h, l, _u8(ex))

    def get_sig(self, l: int):
        s = np.empty(self.blocks_shape(l), dtype=np.uint8)
        m = np.empty(self.blocks_shape(l), dtype=np.float64)
        self.lib.orc_get_sig(self._h, l, _u8(s), _dp(m))
        return s, m

    def scale(self) -> np.ndarray:
        s = np.zeros(5)
        self.lib.orc_get_scale(self._h, _dp(s))
        return s[: self.nv]

    def leaf_mask(self, l: int) -> np.ndarray:
        ex = self.get_exist(l).astype(bool)
        if l == self.L:
            return ex
        ch = self.get_exist(l + 1).astype(bool)
        sl = tuple(slice(0, None, 2) for _ in range(self.dim))
        return ex & ~ch[sl]

    # method
    def restrict_all(self) -> None:
        self.lib.orc_restrict_all(self._h)

    def dt(self, cfl: float, lts: bool = False) -> float:
        return self.lib.orc_dt(self._h, cfl, int(lts))

    def step(self, dt: float, lts: bool = False) -> None:
        self.lib.orc_step(self._h, dt, int(lts))

    def analyse(self, eps: float, precision: int = 0) -> int:
        n = ctypes.c_long(0)
        self.lib.orc_analyse(self._h, eps, precision, ctypes.byref(n))
        return n.value

    def adapt(self, criterion: int = CRIT_MR, eps: float = 1e-3, eps_w: float = 0.05,
              eta_tol: float = 0.8, precision: int = 0, eps_p: float = 0.0, eps_r: float = 0.0) -> None:
        """eps_p > 0: the gradient criterion also tests pressure against eps_p;
        eps_r > 0: it also flags by the Richardson estimate of density."""
        if self.lib.orc_set_eps_p(self._h, eps_p) != 0 or self.lib.orc_set_eps_r(self._h, eps_r) != 0:
            raise ValueError("oracle: bad eps_p / eps_r")
        self.lib.orc_adapt(self._h, criterion, eps, eps_w, eta_tol, precision)

    def set_lts_remesh(self, on: bool = True, eps_w: float = 0.05, eta_tol: float = 0.8,
                       eps_p: float = 0.0, criterion: int = CRIT_GRAD, eps: float = 1e-3,
                       precision: int = 0, eps_r: float = 0.0) -> None:
        """Remesh the finer levels inside the level recursion (Fig. 2) when stepping
        with level-dependent steps, with the gradient (eps_w, eta_tol, eps_p, eps_r) or
        the MR criterion (eps, decided in single precision with precision 1)."""
        if self.lib.orc_set_eps_p(self._h, eps_p) != 0 or self.lib.orc_set_eps_r(self._h, eps_r) != 0 or \
                self.lib.orc_set_lts_remesh(self._h, int(bool(on)), criterion, eps, eps_w, eta_tol,
                                            precision) != 0:
            raise ValueError("oracle: bad remesh parameters")

    def rich_tau(self, l: int, dt: float):
        """Richardson estimate of density of level l with level step dt on the
        current state: (tau on the level's grid coarsened by 2, numpy order, and
        the number of non-finite estimates on coarse cells of existing blocks)."""
        shape = tuple(n // 2 for n in self.cells_shape(l))
        tau = np.empty(shape, dtype=np.float64)
        bad = self.lib.orc_rich_tau(self._h, l, dt, _dp(tau))
        return tau, int(bad)

    @property
    def rich_bad(self) -> int:
        """Richardson estimates on existing blocks that came out non-finite so far."""
        return int(self.lib.orc_rich_bad(self._h))

    def totals(self) -> np.ndarray:
        out = np.zeros(5)
        self.lib.orc_totals(self._h, _dp(out))
        return out[: self.nv]

    def project_finest(self) -> np.ndarray:
        out = np.empty((self.nv,) + self.cells_shape(self.L), dtype=np.float64)
        self.lib.orc_project_finest(self._h, _dp(out))
        return out

    def flux(self, nd: int, ql, qr) -> np.ndarray:
        a = np.zeros(5); b = np.zeros(5); F = np.zeros(5)
        a[: self.nv] = ql; b[: self.nv] = qr
        self.lib.orc_flux(self._h, nd, _dp(a), _dp(b), _dp(F))
        return F[: self.nv]

    def flux_ausmdv(self, nd: int, ql, qr) -> np.ndarray:
        a = np.zeros(5); b = np.zeros(5); F = np.zeros(5)
        a[: self.nv] = ql; b[: self.nv] = qr
        self.lib.orc_flux_ausmdv(self._h, nd, _dp(a), _dp(b), _dp(F))
        return F[: self.nv]

    def br_cluster(self, l: int, flags, eta: float) -> np.ndarray:
        """Berger-Rigoutsos boxes of a block flag map of level l (shape blocks_shape(l))."""
        fl = np.ascontiguousarray(flags, dtype=np.uint8)
        assert fl.shape == self.blocks_shape(l)
        out = np.zeros_like(fl)
        self.lib.orc_br_cluster(self._h, l, _u8(fl), eta, _u8(out))
        return out

    def physical_flux(self, nd: int, q) -> np.ndarray:
        a = np.zeros(5); F = np.zeros(5)
        a[: self.nv] = q
        self.lib.orc_physical_flux(self._h, nd, _dp(a), _dp(F))
        return F[: self.nv]

    def predict(self, lf: int, coarse: np.ndarray, v: int, i: int, j: int, k: int = 0) -> float:
        c = np.ascontiguousarray(coarse, dtype=np.float64)
        return self.lib.orc_predict(self._h, lf, _dp(c), v, i, j, k)
