"""Long runs on the GPU against the oracle: the FP64 bar (every cell within 1e-12
relative, the time step and the tree bit-exact after every step) over 100 steps
for the 3D and AMR-side configurations, and the FP32 bar (2e-4 relative L1 of
the density projected to the finest level, conserved totals within 1e-6) over
25 steps of the 8-level 2D workload the bench times.

Schemes: the MR scheme of Section 2 (MUSCL / van Albada / AUSM+ / midpoint RK2)
and the AMR scheme (MUSCL-Hancock / Minmod / AUSMDV); criteria: MR thresholding
(Section 2.1) and gradient flags with Berger-Rigoutsos clustering (Section 2.2);
level-dependent steps follow Fig. 2.
"""
import numpy as np
import pytest

import mrfv_inputs as mi
import oracle

pytestmark = pytest.mark.gpu

REL64 = 1e-12


@pytest.fixture(scope="module")
def mrfv():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1603_05211_gb300 as m

    m.build()
    return m


def _pair(m, dim, levels, base, *, scheme="muscl_rk2", criterion="mr", clustering="rows", lts=False, ic, params,
          lo=(0, 0, 0), hi=(1, 1, 1), cfl=0.5, eps=1e-3, precision="fp64", t_end=0.0):
    s = m.Solver(dim=dim, precision=precision, levels=levels, base_blocks=base, lo=lo, hi=hi, adapt=True,
                 criterion=criterion, eps=eps, lts=lts, cfl=cfl, scheme=scheme, clustering=clustering, t_end=t_end)
    s.init_state(ic, params)
    o = oracle.Oracle(dim, levels, base, lo=lo, hi=hi,
                      scheme=oracle.SCHEME_HANCOCK if scheme == "hancock" else oracle.SCHEME_MUSCL_RK2,
                      clustering=oracle.CLUSTER_BR if clustering == "br" else oracle.CLUSTER_ROWS)
    o.init(ic, params)
    crit = oracle.CRIT_GRAD if criterion == "grad" else oracle.CRIT_MR
    p = 1 if precision == "fp32" else 0
    o.adapt(crit, eps=eps, precision=p)
    if lts:  # the solver's default: Remesh(l) inside the recursion (Fig. 2)
        o.set_lts_remesh(True, 0.05, 0.8, criterion=crit, eps=eps, precision=p)
    return s, o, crit


def _same_tree(s, o, k):
    for l in range(o.levels):
        assert np.array_equal(s.get_tree(l), o.get_exist(l)), f"step {k}: tree differs on level {l}"


def _close(s, o, k):
    for l in range(o.levels):
        g, _ = s.download_level(l)
        r = o.get_level(l)
        assert np.array_equal(np.isnan(g), np.isnan(r)), f"step {k}: existence differs on level {l}"
        msk = ~np.isnan(r)
        if msk.any():
            err = np.abs(g[msk] - r[msk]).max()
            assert err <= REL64 * np.abs(r[msk]).max(), f"step {k}, level {l}: max abs err {err:.3e}"


def _run_fp64(s, o, crit, steps, lts=False, cfl=0.5):
    _same_tree(s, o, 0)
    adaptive = 0  # steps after which the leaves lie on two levels or more
    for k in range(1, steps + 1):
        dt = o.dt(cfl, lts)
        assert s.step(0.0) == dt, f"step {k}: dt differs"
        o.step(dt, lts)
        o.adapt(crit, eps=1e-3)
        _same_tree(s, o, k)
        if k % 25 == 0:
            _close(s, o, k)
        adaptive += len([x for x in s.stats()["leaves"] if x]) >= 2
    assert adaptive >= steps // 4, f"the tree was adaptive after {adaptive} of {steps} steps only"


# A weak off-centre ellipsoidal blast (pressure ratio 2) on [-1, 1]^3, 4 levels (64^3 finest):
# the tree stays adaptive for most of the 100 steps (the workload's blast fills a
# 64^3 hierarchy at once) and the flow is fully three-dimensional.
BLAST_OFF_CENTRE = [-0.4, 0.3, 0.2, 0.12, 0.1, 0.15, 1.0, 2.0, 1.0, 1.0]


def test_adaptive_3d_mr_fp64_100_steps(mrfv):
    """3D blast, MR scheme and MR thresholding, 4 levels (64^3 finest)."""
    s, o, crit = _pair(mrfv, 3, 4, (1, 1, 1), lo=(-1, -1, -1), hi=(1, 1, 1), ic=mi.IC_ELLIPSOID,
                       params=BLAST_OFF_CENTRE)
    _run_fp64(s, o, crit, 100)


def test_hancock_adaptive_2d_fp64_100_steps(mrfv):
    """The AMR scheme under MR thresholding, 2D four-quadrant data, 5 levels."""
    s, o, crit = _pair(mrfv, 2, 5, (1, 1, 1), scheme="hancock", ic=mi.IC_QUADRANTS, params=mi.quadrant_params(0),
                       cfl=0.4)
    _run_fp64(s, o, crit, 100, cfl=0.4)


def test_hancock_adaptive_3d_fp64_100_steps(mrfv):
    """The AMR scheme under MR thresholding, the same 3D blast, 4 levels (64^3 finest)."""
    s, o, crit = _pair(mrfv, 3, 4, (1, 1, 1), scheme="hancock", lo=(-1, -1, -1), hi=(1, 1, 1), ic=mi.IC_ELLIPSOID,
                       params=BLAST_OFF_CENTRE, cfl=0.4)
    _run_fp64(s, o, crit, 100, cfl=0.4)


@pytest.mark.parametrize("scheme", ["muscl_rk2", "hancock"])
def test_amr_gradient_lts_fp64_100_coarse_steps(mrfv, scheme):
    """Gradient flags with level-dependent steps and Remesh(l) inside the
    recursion (Fig. 2), 3 levels on a 32^2 base: 100 coarse steps (400 finest)."""
    cfl = 0.4 if scheme == "hancock" else 0.5
    s, o, crit = _pair(mrfv, 2, 3, (4, 4, 1), scheme=scheme, criterion="grad", lts=True, ic=mi.IC_QUADRANTS,
                       params=mi.quadrant_params(3), cfl=cfl)
    _run_fp64(s, o, crit, 100, lts=True, cfl=cfl)


def test_br_3d_fp64_100_steps(mrfv):
    """Berger-Rigoutsos clustering of 3D gradient flags (Sod's tube along y), 3 levels."""
    s, o, crit = _pair(mrfv, 3, 3, (2, 2, 2), criterion="grad", clustering="br", ic=mi.IC_SHOCKTUBE,
                       params=mi.sod_params(1, 0.4))
    _run_fp64(s, o, crit, 100)


def test_mr2d_fp32_levels8_bench_workload_25_steps(mrfv):
    """The bench's workload (2D MR, FP32, 8 levels, 1024^2 finest, eps 1e-3) for 25
    steps with the oracle's time steps: the density of the leaves projected to the
    finest level within 2e-4 relative L1 of the FP64 oracle, totals within 1e-6."""
    P = mi.quadrant_params(0)
    s, o, crit = _pair(mrfv, 2, 8, (1, 1, 1), ic=mi.IC_QUADRANTS, params=P, precision="fp32", t_end=0.25)
    T0 = o.totals()
    for _ in range(25):
        dt = o.dt(0.5)
        s.step(dt)
        o.step(dt)
        o.adapt(crit, eps=1e-3, precision=1)
    gs = [s.download_level(l)[0] for l in range(8)]
    o2 = oracle.Oracle(2, 8, (1, 1, 1))
    o2.init(mi.IC_QUADRANTS, P)
    for l in range(8):
        o2.set_exist(l, s.get_tree(l))
    for l in range(8):
        o2.set_level(l, gs[l])
    fg = o2.project_finest()[0]
    fo = o.project_finest()[0]
    assert np.abs(fg - fo).sum() / np.abs(fo).sum() <= 2e-4
    assert np.all(np.abs(s.totals() - o.totals()) <= 1e-6 * np.abs(T0).max())
    assert s.stats()["total_leaves"] > 1000
