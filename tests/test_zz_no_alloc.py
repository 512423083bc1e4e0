"""The allocation-free CFL entry point (mrfv_cfl_dt_noalloc) against mrfv_compute_dt.

For callers that cannot allocate device memory (stream capture, host frameworks
that own all device memory, latency-critical loops): the entry point takes the
state and the output from the caller and keeps its scratch in a static device
array.  This file runs last so that, if it fails, every other test has run.
It must pass alone in a fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest

import mrfv_inputs as mi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1603_05211_gb300 as m

    m.build()
    return m, torch


def _noalloc_dt(m, torch, s, level_state, precision, dx):
    """Call the C entry point on a device copy of the dense level."""
    dt = torch.empty(1, dtype=torch.float64, device="cuda")
    dev = torch.tensor(level_state, dtype=torch.float32 if precision == "fp32" else torch.float64, device="cuda")
    shape = level_state.shape[1:]  # (k, j, i) or (j, i)
    n = list(reversed(shape)) + [1] * (3 - len(shape))
    dxa = (ctypes.c_double * 3)(*(list(dx) + [1.0] * (3 - len(dx))))
    rc = m.load().mrfv_cfl_dt_noalloc(s.dim, m.FP32 if precision == "fp32" else m.FP64,
                                      ctypes.c_void_p(dev.data_ptr()), n[0], n[1], n[2],
                                      dxa, 1.4, 0.5, ctypes.cast(ctypes.c_void_p(dt.data_ptr()), ctypes.POINTER(ctypes.c_double)),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    torch.cuda.synchronize()
    return float(dt.item())


@pytest.mark.parametrize("dim,precision", [(2, "fp64"), (2, "fp32"), (3, "fp64"), (3, "fp32")])
def test_noalloc_dt_matches_compute_dt_twice(env, dim, precision):
    m, torch = env
    if dim == 2:
        s = m.Solver(dim=2, precision=precision, levels=1, base_blocks=(24, 16, 1), hi=(1.5, 1.0, 1.0))
        s.init_state(mi.IC_QUADRANTS, mi.quadrant_params(9))
        dx = [1.5 / 192, 1.0 / 128]
    else:
        s = m.Solver(dim=3, precision=precision, levels=1, base_blocks=(4, 4, 4), lo=(-1, -1, -1), hi=(1, 1, 1))
        s.init_state(mi.IC_ELLIPSOID, mi.ellipsoid_params(9))
        dx = [2.0 / 32] * 3
    tol = 0.0 if precision == "fp64" else 1e-6
    for _ in range(2):  # two calls in a row, on different states
        ref = s.compute_dt()
        got = _noalloc_dt(m, torch, s, s.download_level(0)[0], precision, dx)
        assert got == pytest.approx(ref, rel=tol, abs=0.0)
        s.step(0.0)


def test_noalloc_dt_rejects_oversize_and_flags_nonphysical(env):
    m, torch = env
    lib = m.load()
    big = (ctypes.c_double * 3)(1.0, 1.0, 1.0)
    dt = torch.empty(1, dtype=torch.float64, device="cuda")
    x = torch.ones(4, dtype=torch.float64, device="cuda")
    dtp = ctypes.cast(ctypes.c_void_p(dt.data_ptr()), ctypes.POINTER(ctypes.c_double))
    n = 1 << 15  # 2^30 cells > the stated maximum
    assert lib.mrfv_cfl_dt_noalloc(2, m.FP64, ctypes.c_void_p(x.data_ptr()), n, n, 1, big, 1.4, 0.5, dtp, None) == m.ERR_ARG
    state = np.zeros((4, 8, 8))
    state[0] = 1.0
    state[3] = -1.0  # negative energy: non-physical
    dev = torch.tensor(state, device="cuda")
    assert lib.mrfv_cfl_dt_noalloc(2, m.FP64, ctypes.c_void_p(dev.data_ptr()), 8, 8, 1, big, 1.4, 0.5, dtp, None) == 0
    torch.cuda.synchronize()
    assert dt.item() == -1.0
