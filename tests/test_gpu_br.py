"""Berger-Rigoutsos clustering of gradient flags (Section 2.2) on the GPU
against the oracle: the trees (integer work) bit-exact after every step, the
FP64 state within 1e-12."""
import numpy as np
import pytest

import mrfv_inputs as mi
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mrfv():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1603_05211_gb300 as m

    m.build()
    return m


def _pair(m, levels, base, lts, seed, bc=0, dim=2, ic=mi.IC_QUADRANTS, params=None, lo=(0, 0, 0), hi=(1, 1, 1)):
    params = params if params is not None else mi.quadrant_params(seed)
    s = m.Solver(dim=dim, levels=levels, base_blocks=base, adapt=True, criterion="grad", lts=lts, bc=bc, lo=lo, hi=hi,
                 clustering="br")
    s.init_state(ic, params)
    o = oracle.Oracle(dim, levels, base, bc=bc, lo=lo, hi=hi, clustering=oracle.CLUSTER_BR)
    o.init(ic, params)
    o.adapt(oracle.CRIT_GRAD)
    if lts:
        o.set_lts_remesh(True, 0.05, 0.8)  # the solver's default (Fig. 2)
    return s, o


def _same(s, o):
    for l in range(o.levels):
        assert np.array_equal(s.get_tree(l), o.get_exist(l)), f"tree differs on level {l}"


def _close(s, o):
    for l in range(o.levels):
        g, r = s.download_level(l)[0], o.get_level(l)
        assert np.array_equal(np.isnan(g), np.isnan(r))
        m = ~np.isnan(r)
        if m.any():
            assert np.abs(g[m] - r[m]).max() <= 1e-12 * np.abs(r[m]).max()


@pytest.mark.parametrize("lts", [False, True])
@pytest.mark.parametrize("seed", [3, 7])
def test_br_amr_matches_oracle(mrfv, lts, seed):
    s, o = _pair(mrfv, 3, (8, 8, 1), lts, seed)
    _same(s, o)
    for l in range(2):
        assert np.array_equal(s.get_flags(l)[0], o.get_sig(l)[0])
    for _ in range(3):
        dt = o.dt(0.5, lts)
        assert s.step(0.0) == dt
        o.step(dt, lts)
        o.adapt(oracle.CRIT_GRAD)
        _same(s, o)
    _close(s, o)


def test_br_amr_base128_levels4_flags(mrfv):
    """The AMR workload's geometry (base 128^2, 4 levels): the clustered flags of
    every level after initialisation and after two steps."""
    s, o = _pair(mrfv, 4, (16, 16, 1), True, 0)
    _same(s, o)
    for _ in range(2):
        dt = o.dt(0.5, True)
        s.step(0.0)
        o.step(dt, True)
        o.adapt(oracle.CRIT_GRAD)
        _same(s, o)


def test_br_3d_matches_oracle(mrfv):
    s, o = _pair(mrfv, 3, (2, 2, 2), False, 0, dim=3, ic=mi.IC_SHOCKTUBE, params=mi.sod_params(1, 0.4))
    _same(s, o)
    for _ in range(2):
        dt = o.dt(0.5)
        assert s.step(0.0) == dt
        o.step(dt)
        o.adapt(oracle.CRIT_GRAD)
        _same(s, o)
    _close(s, o)


def _pair_p(m, dim, levels, base, lts, ic, params, clustering, scheme="muscl_rk2", lo=(0, 0, 0), hi=(1, 1, 1),
            cfl=0.5):
    """Gradient criterion on density and pressure (eps_w = eps_p = 0.05)."""
    s = m.Solver(dim=dim, levels=levels, base_blocks=base, adapt=True, criterion="grad", lts=lts, lo=lo, hi=hi,
                 clustering=clustering, eps_w=0.05, eps_p=0.05, scheme=scheme, cfl=cfl)
    s.init_state(ic, params)
    o = oracle.Oracle(dim, levels, base, lo=lo, hi=hi,
                      clustering=oracle.CLUSTER_BR if clustering == "br" else oracle.CLUSTER_ROWS,
                      scheme=oracle.SCHEME_HANCOCK if scheme == "hancock" else oracle.SCHEME_MUSCL_RK2)
    o.init(ic, params)
    o.adapt(oracle.CRIT_GRAD, eps_w=0.05, eps_p=0.05)
    if lts:
        o.set_lts_remesh(True, 0.05, 0.8, eps_p=0.05)
    return s, o


@pytest.mark.parametrize("clustering", ["rows", "br"])
def test_pressure_gradient_flags_2d(mrfv, clustering):
    s, o = _pair_p(mrfv, 2, 3, (4, 4, 1), False, mi.IC_QUADRANTS, mi.quadrant_params(5), clustering)
    _same(s, o)
    for _ in range(3):
        dt = o.dt(0.5)
        assert s.step(0.0) == dt
        o.step(dt)
        o.adapt(oracle.CRIT_GRAD, eps_w=0.05, eps_p=0.05)
        for l in range(2):
            assert np.array_equal(s.get_flags(l)[0], o.get_sig(l)[0])
        _same(s, o)
    _close(s, o)


def test_pressure_gradient_rotated_ellipsoid_3d_hancock_lts(mrfv):
    """The 3D case of Section 4.2 at small size: rotated ellipsoid on [-2,2]^3,
    AMR scheme, density and pressure flags clustered by Berger-Rigoutsos,
    level-dependent steps."""
    s, o = _pair_p(mrfv, 3, 3, (2, 2, 2), True, mi.IC_ROTATED_ELLIPSOID, mi.paper3d_params(), "br",
                   scheme="hancock", lo=(-2, -2, -2), hi=(2, 2, 2), cfl=0.4)
    _same(s, o)
    for _ in range(2):
        dt = o.dt(0.4, True)
        assert s.step(0.0) == dt
        o.step(dt, True)
        o.adapt(oracle.CRIT_GRAD, eps_w=0.05, eps_p=0.05)
        _same(s, o)
    _close(s, o)


@pytest.mark.parametrize("scheme", ["muscl_rk2", "hancock"])
def test_lts_remesh_inside_the_recursion_matches_oracle(mrfv, scheme):
    """Remesh(l) at the sub-steps (Fig. 2) on a moving shock whose waves leave
    the refined region within a coarse step: trees after every coarse step and the
    FP64 state against the oracle; the same run with the remesh switched off on
    both sides differs (the rule is exercised)."""
    def run(remesh):
        s = mrfv.Solver(dim=2, levels=5, base_blocks=(2, 1, 1), adapt=True, criterion="grad", lts=True,
                        clustering="br", scheme=scheme, cfl=0.4, lts_remesh=remesh)
        s.init_state(mi.IC_SHOCKTUBE, mi.sod_params(0, 0.3))
        o = oracle.Oracle(2, 5, (2, 1, 1), clustering=oracle.CLUSTER_BR,
                          scheme=oracle.SCHEME_HANCOCK if scheme == "hancock" else oracle.SCHEME_MUSCL_RK2)
        o.init(mi.IC_SHOCKTUBE, mi.sod_params(0, 0.3))
        o.adapt(oracle.CRIT_GRAD)
        o.set_lts_remesh(remesh, 0.05, 0.8)
        _same(s, o)
        for _ in range(3):
            dt = o.dt(0.4, True)
            assert s.step(0.0) == dt
            o.step(dt, True)
            o.adapt(oracle.CRIT_GRAD)
            _same(s, o)
        _close(s, o)
        return s
    a, b = run(True), run(False)
    assert any(not np.array_equal(a.download_level(l)[0], b.download_level(l)[0], equal_nan=True) for l in range(5))
