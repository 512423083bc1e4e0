"""Pins of the oracle's Remesh(l) inside the level recursion (Fig. 2: AMR with
level-dependent steps regenerates the finer levels at the sub-steps of every
level, from gradient flags of data at one time).

Pinned by what must hold whatever the flags: conservation on a periodic domain,
the tree rules after every step, no effect when the flags cover everything (the
tree then never changes, so the run must equal the one without remeshing bit for
bit), and by the purpose of the rule: the run stays closer to the uniform solve
at the finest resolution than adapting once per coarse step does.
"""
import numpy as np
import pytest

import mrfv_inputs as mi
import oracle


def _amrlt(levels, base, seed, remesh, eps_w=0.05, scheme=oracle.SCHEME_MUSCL_RK2, dim=2, bc=oracle.BC_PERIODIC,
           steps=3, ic=mi.IC_QUADRANTS, params=None, lo=(0, 0, 0), hi=(1, 1, 1)):
    o = oracle.Oracle(dim, levels, base, bc=bc, clustering=oracle.CLUSTER_BR, scheme=scheme, lo=lo, hi=hi)
    o.init(ic, params if params is not None else mi.quadrant_params(seed))
    o.adapt(oracle.CRIT_GRAD, eps_w=eps_w, eta_tol=0.8)
    if remesh:
        o.set_lts_remesh(True, eps_w, 0.8)
    T0 = o.totals()
    dts = []
    for _ in range(steps):
        dt = o.dt(0.4, True)
        dts.append(dt)
        o.step(dt, True)
        _tree_rules(o)
        o.adapt(oracle.CRIT_GRAD, eps_w=eps_w, eta_tol=0.8)
    return o, T0, dts


def _tree_rules(o):
    for l in range(1, o.levels):
        ex, par = o.get_exist(l).astype(bool), o.get_exist(l - 1).astype(bool)
        idx = np.argwhere(ex)
        for p in idx:
            q = tuple(int(x) >> 1 for x in p)
            assert par[q], f"level {l}: block without parent"
            # complete sibling groups
            sl = tuple(slice(2 * x, 2 * x + 2) for x in q)
            assert ex[sl].all(), f"level {l}: incomplete sibling group"


@pytest.mark.parametrize("scheme", [oracle.SCHEME_MUSCL_RK2, oracle.SCHEME_HANCOCK])
def test_remesh_conserves_and_keeps_the_tree_rules(scheme):
    o, T0, _ = _amrlt(4, (2, 2, 1), 3, True, scheme=scheme)
    assert np.all(np.abs(o.totals() - T0) <= 1e-12 * np.abs(T0).max())


def test_remesh_conserves_3d():
    o, T0, _ = _amrlt(3, (2, 2, 2), 0, True, dim=3, steps=2, ic=mi.IC_ROTATED_ELLIPSOID,
                      params=mi.paper3d_params(), lo=(-2, -2, -2), hi=(2, 2, 2), scheme=oracle.SCHEME_HANCOCK)
    assert np.all(np.abs(o.totals() - T0) <= 1e-12 * np.abs(T0).max())


def test_remesh_changes_nothing_when_everything_is_flagged():
    """eps_w < 0 flags every cell: the tree is full and stays full, so remeshing
    must leave the run bit for bit as it is without it."""
    a, _, _ = _amrlt(3, (2, 2, 1), 1, False, eps_w=-1.0)
    b, _, _ = _amrlt(3, (2, 2, 1), 1, True, eps_w=-1.0)
    for l in range(3):
        assert np.array_equal(a.get_exist(l), b.get_exist(l))
        x, y = a.get_level(l), b.get_level(l)
        assert np.array_equal(np.isnan(x), np.isnan(y))
        m = ~np.isnan(x)
        assert np.array_equal(x[m], y[m])


@pytest.mark.parametrize("scheme", [oracle.SCHEME_MUSCL_RK2, oracle.SCHEME_HANCOCK])
def test_remesh_tracks_the_uniform_fine_solution_better(scheme):
    """Sod's shock tube with 5 levels: a coarse step spans 16 finest steps, long
    enough for the waves to leave the refined region laid at its start; with the
    finer levels regenerated at the sub-steps the run stays closer to the uniform
    solve on the finest grid (same finest steps)."""
    levels, base = 5, (2, 1, 1)
    runs = []
    for remesh in (False, True):
        o = oracle.Oracle(2, levels, base, clustering=oracle.CLUSTER_BR, scheme=scheme)
        o.init(mi.IC_SHOCKTUBE, mi.sod_params(0, 0.3))
        o.adapt(oracle.CRIT_GRAD, eps_w=0.05, eta_tol=0.8)
        if remesh:
            o.set_lts_remesh(True, 0.05, 0.8)
        dts = []
        for _ in range(3):
            dt = o.dt(0.4, True)
            dts.append(dt)
            o.step(dt, True)
            o.adapt(oracle.CRIT_GRAD, eps_w=0.05, eta_tol=0.8)
        runs.append((o, dts))
    u = oracle.Oracle(2, 1, (32, 16, 1), scheme=scheme)
    u.init(mi.IC_SHOCKTUBE, mi.sod_params(0, 0.3))
    for dt in runs[1][1]:
        for _ in range(1 << (levels - 1)):
            u.step(dt)
    ref = u.get_level(0)[0]
    ea = np.abs(runs[0][0].project_finest()[0] - ref).mean()
    eb = np.abs(runs[1][0].project_finest()[0] - ref).mean()
    assert eb < 0.8 * ea, (ea, eb)


# ---------------------------------------------------------------- MR criterion
def _mrlt(levels, base, seed, remesh, eps=1e-3, scheme=oracle.SCHEME_MUSCL_RK2, steps=3, bc=oracle.BC_PERIODIC):
    o = oracle.Oracle(2, levels, base, bc=bc, scheme=scheme)
    o.init(mi.IC_QUADRANTS, mi.quadrant_params(seed))
    o.adapt(oracle.CRIT_MR, eps=eps)
    if remesh:
        o.set_lts_remesh(True, criterion=oracle.CRIT_MR, eps=eps)
    T0 = o.totals()
    for _ in range(steps):
        o.step(o.dt(0.4, True), True)
        _tree_rules(o)
        o.adapt(oracle.CRIT_MR, eps=eps)
    return o, T0


@pytest.mark.parametrize("scheme", [oracle.SCHEME_MUSCL_RK2, oracle.SCHEME_HANCOCK])
def test_mr_remesh_conserves_and_keeps_the_tree_rules(scheme):
    o, T0 = _mrlt(4, (2, 2, 1), 2, True, scheme=scheme)
    assert np.all(np.abs(o.totals() - T0) <= 1e-12 * np.abs(T0).max())


def test_mr_remesh_changes_nothing_when_everything_is_significant():
    a, _ = _mrlt(3, (2, 2, 1), 1, False, eps=-1.0)
    b, _ = _mrlt(3, (2, 2, 1), 1, True, eps=-1.0)
    for l in range(3):
        assert np.array_equal(a.get_exist(l), b.get_exist(l))
        x, y = a.get_level(l), b.get_level(l)
        m = ~np.isnan(x)
        assert np.array_equal(np.isnan(x), np.isnan(y)) and np.array_equal(x[m], y[m])


def test_mr_remesh_tracks_the_uniform_fine_solution_better():
    levels = 5
    runs = []
    for remesh in (False, True):
        o = oracle.Oracle(2, levels, (2, 1, 1))
        o.init(mi.IC_SHOCKTUBE, mi.sod_params(0, 0.3))
        o.adapt(oracle.CRIT_MR, eps=1e-3)
        if remesh:
            o.set_lts_remesh(True, criterion=oracle.CRIT_MR, eps=1e-3)
        dts = []
        for _ in range(3):
            dt = o.dt(0.4, True)
            dts.append(dt)
            o.step(dt, True)
            o.adapt(oracle.CRIT_MR, eps=1e-3)
        runs.append((o, dts))
    u = oracle.Oracle(2, 1, (32, 16, 1))
    u.init(mi.IC_SHOCKTUBE, mi.sod_params(0, 0.3))
    for dt in runs[1][1]:
        for _ in range(1 << (levels - 1)):
            u.step(dt)
    ref = u.get_level(0)[0]
    ea = np.abs(runs[0][0].project_finest()[0] - ref).mean()
    eb = np.abs(runs[1][0].project_finest()[0] - ref).mean()
    assert eb < 0.5 * ea, (ea, eb)
