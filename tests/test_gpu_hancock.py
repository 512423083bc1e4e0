"""The MUSCL-Hancock / Minmod / AUSMDV scheme (the AMR scheme of Section 2) on
the GPU through the C interface, against the oracle element by element.

Bars as for the default scheme: FP64 per cell <= 1e-12 relative (same
expressions in the same order, so the runs are bit-exact in practice) with the
time steps and trees equal after every step; FP32 <= 2e-4 relative L1 density
and conserved totals within 1e-6 relative.
"""
import numpy as np
import pytest

import mrfv_inputs as mi
import oracle

pytestmark = pytest.mark.gpu

REL64 = 1e-12
CFL = 0.4


@pytest.fixture(scope="module")
def mrfv():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1603_05211_gb300 as m

    m.build()
    return m


def pair(m, dim, levels, base, lo=(0, 0, 0), hi=(1, 1, 1), bc=0, precision="fp64", adapt=False, criterion="mr",
         eps=1e-3, lts=False, ic=mi.IC_QUADRANTS, params=None):
    params = params if params is not None else mi.quadrant_params(0)
    s = m.Solver(dim=dim, precision=precision, levels=levels, base_blocks=base, lo=lo, hi=hi, bc=bc, adapt=adapt,
                 criterion=criterion, eps=eps, lts=lts, cfl=CFL, scheme="hancock")
    s.init_state(ic, params)
    o = oracle.Oracle(dim, levels, base, lo=lo, hi=hi, bc=bc, scheme=oracle.SCHEME_HANCOCK)
    o.init(ic, params)
    if adapt:
        o.adapt(oracle.CRIT_GRAD if criterion == "grad" else oracle.CRIT_MR, eps=eps,
                precision=1 if precision == "fp32" else 0)
    if adapt and lts:  # the solver's default: Remesh(l) inside the recursion (Fig. 2)
        o.set_lts_remesh(True, 0.05, 0.8, criterion=oracle.CRIT_GRAD if criterion == "grad" else oracle.CRIT_MR,
                         eps=eps, precision=1 if precision == "fp32" else 0)
    return s, o


def same_tree(s, o):
    for l in range(o.levels):
        assert np.array_equal(s.get_tree(l), o.get_exist(l)), f"tree differs on level {l}"


def levels_close(s, o, rel=REL64):
    for l in range(o.levels):
        g, _ = s.download_level(l)
        r = o.get_level(l)
        assert np.array_equal(np.isnan(g), np.isnan(r)), f"existence differs on level {l}"
        m = ~np.isnan(r)
        if m.any():
            err = np.abs(g[m] - r[m]).max()
            assert err <= rel * np.abs(r[m]).max(), f"level {l}: max abs err {err:.3e}"


def run(s, o, steps, lts=False, crit=None, eps=1e-3, tree=False):
    for _ in range(steps):
        dt_o = o.dt(CFL, lts)
        assert s.step(0.0) == dt_o
        o.step(dt_o, lts)
        if crit is not None:
            o.adapt(crit, eps=eps)
            if tree:
                same_tree(s, o)


@pytest.mark.parametrize("bc", [0, 1])
def test_hancock_uniform_ragged_fp64(mrfv, bc):
    s, o = pair(mrfv, 2, 1, (3, 5, 1), bc=bc, params=mi.quadrant_params(2))
    run(s, o, 40)
    levels_close(s, o)


def test_hancock_uniform_3d_fp64(mrfv):
    s, o = pair(mrfv, 3, 1, (2, 3, 2), lo=(-1, -1, -1), hi=(1, 1, 1), ic=mi.IC_ELLIPSOID,
                params=mi.ellipsoid_params(2))
    run(s, o, 8)
    levels_close(s, o)


@pytest.mark.parametrize("seed", [0, 1])
def test_hancock_adaptive_mr_fp64(mrfv, seed):
    s, o = pair(mrfv, 2, 5, (1, 1, 1), adapt=True, params=mi.quadrant_params(seed))
    same_tree(s, o)
    run(s, o, 25, crit=oracle.CRIT_MR, tree=True)
    levels_close(s, o)


def test_hancock_adaptive_periodic_conservation_fp64(mrfv):
    s, o = pair(mrfv, 2, 5, (1, 1, 1), bc=1, adapt=True, params=mi.quadrant_params(4))
    T0 = s.totals()
    run(s, o, 15, crit=oracle.CRIT_MR, tree=True)
    levels_close(s, o)
    assert np.all(np.abs(s.totals() - T0) <= 1e-12 * np.abs(T0).max())


def test_hancock_mrlt_fp64(mrfv):
    s, o = pair(mrfv, 2, 4, (2, 2, 1), adapt=True, lts=True, params=mi.quadrant_params(2))
    run(s, o, 3, lts=True, crit=oracle.CRIT_MR, tree=True)
    levels_close(s, o)


def test_hancock_amr_gradient_lts_fp64(mrfv):
    s, o = pair(mrfv, 2, 3, (4, 4, 1), adapt=True, criterion="grad", lts=True, params=mi.quadrant_params(3))
    same_tree(s, o)
    for _ in range(3):
        dt = o.dt(CFL, True)
        assert s.step(0.0) == dt
        o.step(dt, True)
        o.adapt(oracle.CRIT_GRAD)
        same_tree(s, o)
    levels_close(s, o)


def test_hancock_adaptive_3d_fp64(mrfv):
    s, o = pair(mrfv, 3, 3, (2, 2, 2), lo=(-1, -1, -1), hi=(1, 1, 1), adapt=True, ic=mi.IC_ELLIPSOID,
                params=mi.ellipsoid_params(1))
    same_tree(s, o)
    run(s, o, 4, crit=oracle.CRIT_MR, tree=True)
    levels_close(s, o)


def test_hancock_adaptive_3d_lts_fp64(mrfv):
    s, o = pair(mrfv, 3, 3, (2, 2, 2), lo=(-1, -1, -1), hi=(1, 1, 1), adapt=True, lts=True, ic=mi.IC_ELLIPSOID,
                params=mi.ellipsoid_params(3))
    run(s, o, 2, lts=True, crit=oracle.CRIT_MR, tree=True)
    levels_close(s, o)


def test_hancock_fp32_adaptive_l1_and_totals(mrfv):
    s, o = pair(mrfv, 2, 5, (1, 1, 1), bc=1, precision="fp32", adapt=True, params=mi.quadrant_params(6))
    T0 = o.totals()
    for _ in range(60):
        dt = o.dt(CFL)
        s.step(dt)
        o.step(dt)
        o.adapt(oracle.CRIT_MR, 1e-3, precision=1)
    o2 = oracle.Oracle(2, 5, (1, 1, 1), bc=1, scheme=oracle.SCHEME_HANCOCK)
    o2.init(mi.IC_QUADRANTS, mi.quadrant_params(6))
    for l in range(5):
        o2.set_exist(l, s.get_tree(l))
    for l in range(5):
        o2.set_level(l, s.download_level(l)[0])
    fg, fo = o2.project_finest()[0], o.project_finest()[0]
    assert np.abs(fg - fo).sum() / np.abs(fo).sum() <= 2e-4
    assert np.all(np.abs(s.totals() - o.totals()) <= 1e-6 * np.abs(T0).max())


def test_hancock_free_stream_bit_exact(mrfv):
    s = mrfv.Solver(dim=2, levels=4, base_blocks=(1, 1, 1), adapt=False, scheme="hancock")
    s.init_state(mi.IC_UNIFORM, [1.3, 0.4, -0.2, 0.0, 0.8])
    ex = [np.ones(s.blocks_shape(0), np.uint8), np.ones(s.blocks_shape(1), np.uint8)]
    for l in range(2, 4):
        m = np.zeros(s.blocks_shape(l), np.uint8)
        m[:2, :2] = 1  # a graded corner refinement: coarse-fine faces and halo corners
        ex.append(m)
    s.set_tree(ex)
    ref = [s.download_level(l)[0] for l in range(4)]
    for _ in range(5):
        s.step(0.002)
    for l in range(4):
        a = s.download_level(l)[0]
        m = ~np.isnan(a)
        assert np.array_equal(a[m], ref[l][m])
