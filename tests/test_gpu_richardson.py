"""The Richardson estimate added to the gradient criterion (Section 2.2) on the
GPU against the oracle, through the C ABI.

FP64: the trees (integer work) bit-exact after every step, the block flags
bit-exact, the per-block maxima of |tau| within 1e-12 of the largest, the state
within 1e-12.  FP32: the per-block maxima of the single-precision estimate
within 1 % on every block whose estimate is at least 5 % of the largest, and
flags that differ only where the oracle's estimate is within 2 % of eps_r.
Covered: both schemes, transmissive and periodic boundaries, global and
level-dependent steps (with the remesh inside the level recursion), 2D and 3D,
the degenerate thresholds and the estimate before the first step.
"""
import numpy as np
import pytest

import mrfv_inputs as mi
import oracle

pytestmark = pytest.mark.gpu

EPS_R = 5e-4


@pytest.fixture(scope="module")
def mrfv():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1603_05211_gb300 as m

    m.build()
    return m


def _pair(m, dim, levels, base, lts, scheme, bc=0, eps_w=0.05, eps_r=EPS_R, ic=mi.IC_QUADRANTS, params=None,
          lo=(0, 0, 0), hi=(1, 1, 1), precision="fp64", adapt=True, cfl=0.5):
    params = params if params is not None else mi.quadrant_params(4)
    s = m.Solver(dim=dim, levels=levels, base_blocks=base, adapt=adapt, criterion="grad", lts=lts, bc=bc, lo=lo,
                 hi=hi, eps_w=eps_w, eps_r=eps_r, scheme=scheme, precision=precision, cfl=cfl)
    s.init_state(ic, params)
    o = oracle.Oracle(dim, levels, base, bc=bc, lo=lo, hi=hi,
                      scheme=oracle.SCHEME_HANCOCK if scheme == "hancock" else oracle.SCHEME_MUSCL_RK2)
    o.init(ic, params)
    if adapt:
        o.adapt(oracle.CRIT_GRAD, eps_w=eps_w, eps_r=eps_r)
    if lts:
        o.set_lts_remesh(True, eps_w, 0.8, eps_r=eps_r)
    return s, o


def _same_tree(s, o):
    for l in range(o.levels):
        assert np.array_equal(s.get_tree(l), o.get_exist(l)), f"tree differs on level {l}"


def _same_flags(s, o):
    """flags bit-exact, per-block maxima of |tau| within 1e-12 of the largest"""
    top = max(float(o.get_sig(l)[1].max()) for l in range(o.L))
    for l in range(o.L):
        gf, gm = s.get_flags(l)
        of, om = o.get_sig(l)
        assert np.array_equal(gf, of), f"flags differ on level {l}"
        assert np.abs(gm - om).max() <= 1e-12 * top, (l, np.abs(gm - om).max(), top)
    return top


def _close(s, o):
    for l in range(o.levels):
        g, r = s.download_level(l)[0], o.get_level(l)
        assert np.array_equal(np.isnan(g), np.isnan(r))
        msk = ~np.isnan(r)
        if msk.any():
            assert np.abs(g[msk] - r[msk]).max() <= 1e-12 * np.abs(r[msk]).max()


def _run(s, o, steps, lts, eps_w, eps_r, cfl=0.5):
    tops = []
    for _ in range(steps):
        dt = o.dt(cfl, lts)
        assert s.step(0.0) == dt
        o.step(dt, lts)
        o.adapt(oracle.CRIT_GRAD, eps_w=eps_w, eps_r=eps_r)
        _same_tree(s, o)
        tops.append(_same_flags(s, o))
    assert o.rich_bad == 0
    return tops


@pytest.mark.parametrize("scheme", ["muscl_rk2", "hancock"])
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("lts", [False, True])
def test_richardson_2d_matches_oracle(mrfv, scheme, bc, lts):
    s, o = _pair(mrfv, 2, 4, (4, 4, 1), lts, scheme, bc=bc)
    _same_tree(s, o)
    tops = _run(s, o, 3, lts, 0.05, EPS_R)
    assert max(tops) > EPS_R  # the estimate decides some flags
    _close(s, o)


@pytest.mark.parametrize("scheme", ["muscl_rk2", "hancock"])
def test_richardson_alone_2d(mrfv, scheme):
    """gradient test off (eps_w huge): the tree grows from the estimate alone"""
    s, o = _pair(mrfv, 2, 3, (4, 4, 1), False, scheme, eps_w=1e9)
    _run(s, o, 3, False, 1e9, EPS_R)
    assert o.get_exist(1).any()
    _close(s, o)


def test_richardson_3d_sod_matches_oracle(mrfv):
    s, o = _pair(mrfv, 3, 3, (2, 2, 2), False, "muscl_rk2", ic=mi.IC_SHOCKTUBE, params=mi.sod_params(1, 0.4))
    _same_tree(s, o)
    _run(s, o, 2, False, 0.05, EPS_R)
    _close(s, o)


def test_richardson_3d_rotated_ellipsoid_hancock_lts(mrfv):
    """the 3D case of Section 4.2 at small size, level-dependent steps (remesh
    inside the recursion with the estimate)"""
    s, o = _pair(mrfv, 3, 3, (2, 2, 2), True, "hancock", ic=mi.IC_ROTATED_ELLIPSOID, params=mi.paper3d_params(),
                 lo=(-2, -2, -2), hi=(2, 2, 2), cfl=0.4)
    _same_tree(s, o)
    _run(s, o, 2, True, 0.05, EPS_R, cfl=0.4)
    _close(s, o)


def test_richardson_3d_periodic_alone(mrfv):
    s, o = _pair(mrfv, 3, 3, (2, 2, 2), False, "muscl_rk2", bc=1, eps_w=1e9, ic=mi.IC_ELLIPSOID,
                 params=[0.5, 0.5, 0.5, 0.3, 0.25, 0.2, 1.0, 1.0, 0.5, 0.5])
    _run(s, o, 2, False, 1e9, EPS_R)
    assert o.get_exist(2).any()
    _close(s, o)


@pytest.mark.parametrize("eps_r", [1e9, 1e-300])
def test_degenerate_thresholds(mrfv, eps_r):
    """eps_r huge: the gradient tree; eps_r tiny: every block with a nonzero
    estimate is flagged (the oracle decides the same)."""
    s, o = _pair(mrfv, 2, 3, (4, 4, 1), False, "muscl_rk2", eps_r=eps_r)
    _run(s, o, 2, False, 0.05, eps_r)
    if eps_r > 1.0:
        g = mrfv.Solver(dim=2, levels=3, base_blocks=(4, 4, 1), adapt=True, criterion="grad")
        g.init_state(mi.IC_QUADRANTS, mi.quadrant_params(4))
        g.step(0.0)
        g.step(0.0)
        for l in range(3):
            assert np.array_equal(g.get_tree(l), s.get_tree(l))


def test_no_estimate_before_the_first_step(mrfv):
    s, o = _pair(mrfv, 2, 3, (4, 4, 1), False, "muscl_rk2", eps_w=1e9, eps_r=1e-300)
    for l in range(3):
        gf, gm = s.get_flags(l)
        assert not gf.any() and not gm.any()
    _same_tree(s, o)


def test_richardson_fp32_estimates(mrfv):
    """single precision: the same tree on both sides (the solver adapts only when
    asked), one step, then one adaptation; estimates and flags compared"""
    s, o = _pair(mrfv, 2, 4, (4, 4, 1), False, "muscl_rk2", precision="fp32", adapt=False)
    o.adapt(oracle.CRIT_GRAD, eps_w=0.05, eps_r=EPS_R)
    s.set_tree([o.get_exist(l) for l in range(o.levels)])
    for l in range(o.levels):
        s.upload_level(l, o.get_level(l))
    dt = o.dt(0.5)
    s.step(dt)
    o.step(dt)
    s.adapt()
    o.adapt(oracle.CRIT_GRAD, eps_w=0.05, eps_r=EPS_R)
    top = max(float(o.get_sig(l)[1].max()) for l in range(o.L))
    assert top > EPS_R
    for l in range(o.L):
        gm, om = s.get_flags(l)[1], o.get_sig(l)[1]
        big = om >= 0.05 * top
        assert np.all(np.abs(gm[big] - om[big]) <= 1e-2 * om[big]), l
    # flags decided on opposite sides of eps_r only where the oracle's estimate is close to it
    for l in range(o.L):
        gm, om = s.get_flags(l)[1], o.get_sig(l)[1]
        differ = (gm > EPS_R) != (om > EPS_R)
        assert np.all(np.abs(om[differ] - EPS_R) <= 2e-2 * EPS_R), l
