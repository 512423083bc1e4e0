"""The C interface library builds, loads without a GPU and exports every symbol
that include/mrfv.h declares; host-only entry points behave as documented."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "mrfv.h")).read()
    return sorted(set(re.findall(r"\b(mrfv_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import paper_1603_05211_gb300 as m

    m.build()
    return m.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    import paper_1603_05211_gb300 as m

    assert sorted(m.SIGNATURES) == declared_symbols()


def test_config_default_and_arena_size(lib):
    import paper_1603_05211_gb300 as m

    cfg = m.Config()
    assert lib.mrfv_config_default(ctypes.byref(cfg)) == 0
    assert cfg.gamma == 1.4 and cfg.cfl == 0.5 and cfg.dim == 2
    n1 = lib.mrfv_arena_bytes(ctypes.byref(cfg))
    cfg.levels = 4
    n4 = lib.mrfv_arena_bytes(ctypes.byref(cfg))
    assert 0 < n1 < n4
    cfg.precision = m.FP32
    assert lib.mrfv_arena_bytes(ctypes.byref(cfg)) < n4
    cfg.dim = 5
    assert lib.mrfv_arena_bytes(ctypes.byref(cfg)) == 0


def test_create_without_gpu_fails_loudly(lib):
    import torch

    import paper_1603_05211_gb300 as m

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    cfg = m.Config()
    lib.mrfv_config_default(ctypes.byref(cfg))
    h = ctypes.c_void_p()
    rc = lib.mrfv_create(ctypes.byref(cfg), ctypes.byref(h))
    assert rc == m.ERR_CUDA
    assert b"no CUDA device" in lib.mrfv_last_error(None)
    with pytest.raises(RuntimeError):
        m.Solver()


def test_bad_config_is_rejected(lib):
    import paper_1603_05211_gb300 as m

    cfg = m.Config()
    lib.mrfv_config_default(ctypes.byref(cfg))
    cfg.levels = 0
    h = ctypes.c_void_p()
    assert lib.mrfv_create(ctypes.byref(cfg), ctypes.byref(h)) == m.ERR_ARG


def test_richardson_config_is_checked_and_sized(lib):
    """eps_r must be >= 0, only adds to the gradient criterion, and adds its mask
    and patch scratch to the arena only when on."""
    import paper_1603_05211_gb300 as m

    cfg = m.Config()
    lib.mrfv_config_default(ctypes.byref(cfg))
    cfg.levels = 3
    cfg.criterion = m.CRIT_GRAD
    off = lib.mrfv_arena_bytes(ctypes.byref(cfg))
    cfg.eps_r = 1e-3
    assert lib.mrfv_arena_bytes(ctypes.byref(cfg)) > off
    h = ctypes.c_void_p()
    for eps_r, crit in ((-1e-3, m.CRIT_GRAD), (float("nan"), m.CRIT_GRAD), (float("inf"), m.CRIT_GRAD),
                        (1e-3, m.CRIT_MR)):
        cfg.eps_r, cfg.criterion = eps_r, crit
        assert lib.mrfv_create(ctypes.byref(cfg), ctypes.byref(h)) == m.ERR_ARG
    cfg.levels = 1  # one level: nothing below the finest, no scratch
    cfg.criterion, cfg.eps_r = m.CRIT_GRAD, 1e-3
    n1 = lib.mrfv_arena_bytes(ctypes.byref(cfg))
    cfg.eps_r = 0.0
    assert lib.mrfv_arena_bytes(ctypes.byref(cfg)) == n1
