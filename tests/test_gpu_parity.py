"""GPU path (through the C interface) against the CPU oracle, element by element.

Bars: FP64 mode per cell <= 1e-12 relative (the kernels evaluate the same
expressions in the same order without contraction, so most cases are bit-exact);
thresholding flags bit-exact on identical input state; FP32 mode <= 2e-4 relative
L1 density error and conserved totals within 1e-6 relative.
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


def pair(m, dim, levels, base, lo=(0, 0, 0), hi=(1, 1, 1), bc=0, precision="fp64", adapt=False,
         criterion="mr", eps=1e-3, lts=False, ic=mi.IC_QUADRANTS, params=None, cfl=0.5):
    params = params if params is not None else mi.quadrant_params(0)
    s = m.Solver(dim=dim, precision=precision, levels=levels, base_blocks=base, lo=lo, hi=hi, bc=bc,
                 adapt=adapt, criterion=criterion, eps=eps, lts=lts, cfl=cfl)
    s.init_state(ic, params)
    o = oracle.Oracle(dim, levels, base, lo=lo, hi=hi, bc=bc)
    o.init(ic, params)
    if adapt:
        o.adapt(oracle.CRIT_GRAD if criterion == "grad" else oracle.CRIT_MR, eps=eps,
                precision=1 if precision == "fp32" else 0)
    if adapt and lts:  # the solver's default: Remesh(l) inside the recursion (Fig. 2)
        o.set_lts_remesh(True, 0.05, 0.8, criterion=oracle.CRIT_GRAD if criterion == "grad" else oracle.CRIT_MR,
                         eps=eps, precision=1 if precision == "fp32" else 0)
    return s, o


def assert_same_tree(s, o):
    for l in range(o.levels):
        assert np.array_equal(s.get_tree(l), o.get_exist(l)), f"tree differs on level {l}"


def assert_levels_close(s, o, rel=REL64):
    for l in range(o.levels):
        g, ex = s.download_level(l)
        r = o.get_level(l)
        assert np.array_equal(np.isnan(g), np.isnan(r)), f"existence differs on level {l}"
        m = ~np.isnan(r)
        if not m.any():
            continue
        scale = np.abs(r[m]).max()
        err = np.abs(g[m] - r[m]).max()
        assert err <= rel * scale, f"level {l}: max abs err {err:.3e} (scale {scale:.3e})"


def run_pair(s, o, steps, lts=False, adapt_crit=None, eps=1e-3, check_dt=True, precision=0):
    for _ in range(steps):
        dt_o = o.dt(0.5, lts)
        dt_g = s.step(0.0)
        if check_dt:
            assert dt_g == dt_o
        o.step(dt_o, lts)
        if adapt_crit is not None:
            o.adapt(adapt_crit, eps=eps, precision=precision)


# ----------------------------------------------------------------------------- uniform

def test_uniform_128_fp64_200_steps_then_analysis(mrfv):
    """128^2 four-quadrant Riemann data, CFL 0.5, 200 steps, then a 4-level MR analysis (eps 1e-3)."""
    s, o = pair(mrfv, 2, 4, (2, 2, 1), params=mi.quadrant_params(0))
    run_pair(s, o, 200)
    g, _ = s.download_level(3)
    r = o.get_level(3)
    assert np.abs(g - r).max() <= REL64 * np.abs(r).max()
    n_g = s.analyse(1e-3)
    n_o = o.analyse(1e-3)
    assert n_g == n_o
    for l in range(1, 4):
        fg, mg = s.get_flags(l)
        fo, mo = o.get_sig(l)
        assert np.array_equal(fg, fo)
        assert np.array_equal(mg, mo)


@pytest.mark.parametrize("bc", [0, 1])
def test_uniform_ragged_single_level(mrfv, bc):
    """Non-power-of-two block grid (3 x 5 blocks), both boundary rules."""
    s, o = pair(mrfv, 2, 1, (3, 5, 1), hi=(0.6, 1.0, 1.0), bc=bc, params=mi.quadrant_params(3))
    run_pair(s, o, 30)
    assert_levels_close(s, o)


def test_single_block_domain(mrfv):
    s, o = pair(mrfv, 2, 1, (1, 1, 1), params=mi.laxliu6_params())
    run_pair(s, o, 10)
    assert_levels_close(s, o)


def test_free_stream_bit_exact_gpu(mrfv):
    s, _ = pair(mrfv, 2, 5, (1, 1, 1), ic=mi.IC_UNIFORM, params=[1.3, 0.4, -0.2, 0.0, 0.8], adapt=True)
    ref = [s.download_level(l)[0] for l in range(5)]
    for _ in range(5):
        s.step(0.001)
    for l in range(5):
        g = s.download_level(l)[0]
        m = ~np.isnan(ref[l])
        assert np.array_equal(g[m], ref[l][m])


# ----------------------------------------------------------------------------- adaptive

@pytest.mark.parametrize("seed", [0, 1])
def test_adaptive_mr_fp64(mrfv, seed):
    s, o = pair(mrfv, 2, 5, (1, 1, 1), adapt=True, params=mi.quadrant_params(seed))
    assert_same_tree(s, o)
    for _ in range(25):
        run_pair(s, o, 1, adapt_crit=oracle.CRIT_MR)
        assert_same_tree(s, o)
    assert_levels_close(s, o)
    st = s.stats()
    assert len([x for x in st["leaves"] if x]) >= 2


@pytest.mark.parametrize("lts", [False, True])
def test_adaptive_mr_fp64_100_steps(mrfv, lts):
    """The FP64 bar over a long run: 100 (coarse) steps of adaptive MR on 4 levels,
    the tree bit-exact after every step, every cell within 1e-12 at the end,
    dt bit-exact every step."""
    s, o = pair(mrfv, 2, 4, (2, 2, 1), adapt=True, lts=lts, params=mi.quadrant_params(5))
    for k in range(100):
        run_pair(s, o, 1, lts=lts, adapt_crit=oracle.CRIT_MR)
        assert_same_tree(s, o)
        if k % 25 == 24:
            assert_levels_close(s, o)
    assert_levels_close(s, o)
    st = s.stats()
    assert len([x for x in st["leaves"] if x]) >= 2


def test_project_finest_matches_oracle(mrfv):
    s, o = pair(mrfv, 2, 5, (1, 1, 1), adapt=True, params=mi.quadrant_params(8))
    run_pair(s, o, 10, adapt_crit=oracle.CRIT_MR)
    assert_same_tree(s, o)
    g = s.project_finest()
    r = o.project_finest()
    assert np.abs(g - r).max() <= REL64 * np.abs(r).max()


def test_adaptive_mr_fp64_periodic_conservation(mrfv):
    s, o = pair(mrfv, 2, 5, (1, 1, 1), bc=1, adapt=True, params=mi.quadrant_params(5))
    T0 = s.totals()
    assert np.allclose(T0, o.totals(), rtol=1e-13)
    run_pair(s, o, 15, adapt_crit=oracle.CRIT_MR)
    assert_same_tree(s, o)
    assert_levels_close(s, o)
    T1 = s.totals()
    assert np.all(np.abs(T1 - T0) <= 1e-12 * np.abs(T0).max())


def test_mrlt_fp64(mrfv):
    s, o = pair(mrfv, 2, 4, (2, 2, 1), adapt=True, lts=True, params=mi.quadrant_params(2))
    for _ in range(3):
        run_pair(s, o, 1, lts=True, adapt_crit=oracle.CRIT_MR)
        assert_same_tree(s, o)
    assert_levels_close(s, o)


def test_amr_gradient_lts_fp64(mrfv):
    s, o = pair(mrfv, 2, 3, (4, 4, 1), adapt=True, criterion="grad", lts=True, params=mi.quadrant_params(3))
    assert_same_tree(s, o)
    for l in range(2):
        assert np.array_equal(s.get_flags(l)[0], o.get_sig(l)[0])
    for _ in range(3):
        run_pair(s, o, 1, lts=True, adapt_crit=oracle.CRIT_GRAD)
        assert_same_tree(s, o)
    assert_levels_close(s, o)


def test_adaptive_3d_fp64(mrfv):
    s, o = pair(mrfv, 3, 3, (2, 2, 2), lo=(-1, -1, -1), hi=(1, 1, 1), adapt=True, ic=mi.IC_ELLIPSOID,
                params=mi.ellipsoid_params(1))
    assert_same_tree(s, o)
    for _ in range(4):
        run_pair(s, o, 1, adapt_crit=oracle.CRIT_MR)
        assert_same_tree(s, o)
    assert_levels_close(s, o)


def test_flags_bit_exact_on_identical_fp32_state(mrfv):
    """Upload the GPU's single-precision state into the oracle and take the
    thresholding decision on both sides in single precision."""
    s = mrfv.Solver(dim=2, precision="fp32", levels=5, base_blocks=(1, 1, 1), adapt=True, eps=1e-3)
    s.init_state(mi.IC_QUADRANTS, mi.quadrant_params(4))
    for _ in range(10):
        s.step(0.0)
    o = oracle.Oracle(2, 5, (1, 1, 1))
    o.init(mi.IC_QUADRANTS, mi.quadrant_params(4))
    for l in range(5):
        o.set_exist(l, s.get_tree(l))
    for l in range(5):
        o.set_level(l, s.download_level(l)[0])
    n_g = s.analyse(1e-3)
    n_o = o.analyse(1e-3, precision=1)
    assert n_g == n_o
    for l in range(1, 5):
        assert np.array_equal(s.get_flags(l)[0], o.get_sig(l)[0])
        assert np.array_equal(s.get_flags(l)[1], o.get_sig(l)[1])


# ----------------------------------------------------------------------------- FP32

def test_fp32_adaptive_l1_and_totals(mrfv):
    s, o = pair(mrfv, 2, 5, (1, 1, 1), bc=1, precision="fp32", adapt=True, params=mi.quadrant_params(6))
    T0 = o.totals()
    for _ in range(100):
        dt = o.dt(0.5)
        s.step(dt)
        o.step(dt)
        o.adapt(oracle.CRIT_MR, 1e-3, precision=1)
    # compare on the finest level (trees may differ where a detail sits at eps)
    gs = [s.download_level(l)[0] for l in range(5)]
    o2 = oracle.Oracle(2, 5, (1, 1, 1), bc=1)
    o2.init(mi.IC_QUADRANTS, mi.quadrant_params(6))
    for l in range(5):
        o2.set_exist(l, s.get_tree(l))
    for l in range(5):
        o2.set_level(l, gs[l])
    fg = o2.project_finest()[0]
    fo = o.project_finest()[0]
    rel_l1 = np.abs(fg - fo).sum() / np.abs(fo).sum()
    assert rel_l1 <= 2e-4, rel_l1
    Tg = s.totals()
    assert np.all(np.abs(Tg - o.totals()) <= 1e-6 * np.abs(T0).max())


def test_fp32_uniform_l1(mrfv):
    s, o = pair(mrfv, 2, 1, (8, 8, 1), precision="fp32", params=mi.quadrant_params(7))
    for _ in range(100):
        dt = o.dt(0.5)
        s.step(dt)
        o.step(dt)
    g = s.download_level(0)[0][0]
    r = o.get_level(0)[0]
    assert np.abs(g - r).sum() / np.abs(r).sum() <= 2e-4


def test_cfl_dt_fp32_close(mrfv):
    s, o = pair(mrfv, 2, 1, (4, 4, 1), precision="fp32")
    assert s.compute_dt() == pytest.approx(o.dt(0.5), rel=1e-6)


# ----------------------------------------------------------------------------- full size

def test_mr2d_fp32_levels8_full_size_steps(mrfv):
    """The 8-level (1024^2 finest) adaptive FP32 workload for a few steps, as timed by the bench."""
    P = mi.quadrant_params(0)
    s = mrfv.Solver(dim=2, precision="fp32", levels=8, base_blocks=(1, 1, 1), adapt=True, eps=1e-3, t_end=0.25)
    s.init_state(mi.IC_QUADRANTS, P)
    o = oracle.Oracle(2, 8, (1, 1, 1))
    o.init(mi.IC_QUADRANTS, P)
    o.adapt(oracle.CRIT_MR, 1e-3, precision=1)
    for _ in range(3):
        dt = o.dt(0.5)
        s.step(dt)
        o.step(dt)
        o.adapt(oracle.CRIT_MR, 1e-3, precision=1)
    st = s.stats()
    assert st["total_leaves"] > 0
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


def test_errors_are_reported(mrfv):
    s = mrfv.Solver(dim=2, levels=2, base_blocks=(1, 1, 1))
    with pytest.raises(mrfv.MRFVError) as e:
        s.step(0.0)
    assert e.value.code == mrfv.ERR_STATE
    with pytest.raises(mrfv.MRFVError):
        s.init_state(99, [])
    s.init_state(mi.IC_QUADRANTS, mi.quadrant_params(0))
    bad = [np.ones(s.blocks_shape(0), np.uint8), np.zeros(s.blocks_shape(1), np.uint8)]
    bad[1][0, 0] = 1  # incomplete child set
    with pytest.raises(mrfv.MRFVError) as e:
        s.set_tree(bad)
    assert e.value.code == mrfv.ERR_ARG


def test_state_pool_and_nonphysical_errors(mrfv):
    # level-recursion step without the LTS start-state buffer
    s = mrfv.Solver(dim=2, levels=2, base_blocks=(1, 1, 1))
    s.init_state(mi.IC_QUADRANTS, mi.quadrant_params(0))
    with pytest.raises(mrfv.MRFVError) as e:
        s.step_level(0, 1e-4)
    assert e.value.code == mrfv.ERR_STATE
    # a pool smaller than the full tree cannot be initialised
    p = mrfv.Solver(dim=2, levels=3, base_blocks=(2, 2, 1), pool_blocks=4)
    with pytest.raises(mrfv.MRFVError) as e:
        p.init_state(mi.IC_QUADRANTS, mi.quadrant_params(0))
    assert e.value.code == mrfv.ERR_POOL_FULL
    # a cell with negative density is reported by the CFL reduction
    for prec in ("fp64", "fp32"):
        u = mrfv.Solver(dim=2, precision=prec, levels=1, base_blocks=(2, 2, 1))
        u.init_state(mi.IC_QUADRANTS, mi.quadrant_params(0))
        q, _ = u.download_level(0)
        q[0, 5, 7] = -1.0
        u.upload_level(0, q)
        with pytest.raises(mrfv.MRFVError) as e:
            u.step(0.0)
        assert e.value.code == mrfv.ERR_NONPHYSICAL


def _finest_rel_l1(s, o, make_oracle):
    """Relative L1 of the finest-level projection of the GPU state against the
    oracle's, with the GPU tree and data loaded into a fresh oracle."""
    o2 = make_oracle()
    for l in range(o.levels):
        o2.set_exist(l, s.get_tree(l))
    for l in range(o.levels):
        o2.set_level(l, s.download_level(l)[0])
    fg = o2.project_finest()[0]
    fo = o.project_finest()[0]
    return np.abs(fg - fo).sum() / np.abs(fo).sum()


def test_amr2d_fp32_base128_levels4_lts_full_size_steps(mrfv):
    """The gradient-flagged AMR workload (base 128^2, 4 levels, local time
    stepping) at full size, two coarse steps (16 finest sub-steps)."""
    P = mi.quadrant_params(0)
    kw = dict(dim=2, precision="fp32", levels=4, base_blocks=(16, 16, 1), adapt=True, criterion="grad", lts=True)
    s = mrfv.Solver(**kw)
    s.init_state(mi.IC_QUADRANTS, P)

    def make():
        o = oracle.Oracle(2, 4, (16, 16, 1))
        o.init(mi.IC_QUADRANTS, P)
        o.set_lts_remesh(True, 0.05, 0.8)
        return o

    o = make()
    o.adapt(oracle.CRIT_GRAD, precision=1)
    T0 = o.totals()
    for _ in range(2):
        dt = o.dt(0.5, True)
        s.step(dt)
        o.step(dt, True)
        o.adapt(oracle.CRIT_GRAD, precision=1)
    assert _finest_rel_l1(s, o, make) <= 2e-4
    assert np.all(np.abs(s.totals() - o.totals()) <= 1e-6 * np.abs(T0).max())


def test_blast3d_fp32_levels5_full_size_step(mrfv):
    """The 3D ellipsoidal blast (5 levels, 256^3 finest) at full size, one step."""
    P = mi.ellipsoid_params(0)
    lo, hi = (-1, -1, -1), (1, 1, 1)
    s = mrfv.Solver(dim=3, precision="fp32", levels=5, base_blocks=(2, 2, 2), lo=lo, hi=hi, adapt=True, eps=1e-3)
    s.init_state(mi.IC_ELLIPSOID, P)

    def make():
        o = oracle.Oracle(3, 5, (2, 2, 2), lo=lo, hi=hi)
        o.init(mi.IC_ELLIPSOID, P)
        return o

    o = make()
    o.adapt(oracle.CRIT_MR, 1e-3, precision=1)
    T0 = o.totals()
    dt = o.dt(0.5)
    s.step(dt)
    o.step(dt)
    o.adapt(oracle.CRIT_MR, 1e-3, precision=1)
    assert _finest_rel_l1(s, o, make) <= 2e-4
    assert np.all(np.abs(s.totals() - o.totals()) <= 1e-6 * np.abs(T0).max())


@pytest.mark.parametrize("kernel", [1, 2, 3, 4])
@pytest.mark.parametrize("case", ["uniform", "adaptive", "mrlt", "adaptive3d"])
def test_both_stage_kernels_match_oracle(mrfv, kernel, case):
    """The MR-scheme stage in the pencil kernel (1), the staged kernel (2), the
    pencil kernel with two threads per line (3) and the pencil kernel reading
    primitives staged in shared memory (4), each forced, against the oracle (the
    default picks one by leaf count)."""
    if case == "uniform":
        s, o = pair(mrfv, 2, 1, (3, 5, 1), params=mi.quadrant_params(5))
        steps, lts, crit = 30, False, None
    elif case == "adaptive":
        s, o = pair(mrfv, 2, 5, (1, 1, 1), adapt=True, params=mi.quadrant_params(1))
        steps, lts, crit = 15, False, oracle.CRIT_MR
    elif case == "mrlt":
        s, o = pair(mrfv, 2, 4, (2, 2, 1), adapt=True, lts=True, params=mi.quadrant_params(3))
        steps, lts, crit = 2, True, oracle.CRIT_MR
    else:
        s, o = pair(mrfv, 3, 3, (2, 2, 2), lo=(-1, -1, -1), hi=(1, 1, 1), adapt=True, ic=mi.IC_ELLIPSOID,
                    params=mi.ellipsoid_params(4))
        steps, lts, crit = 3, False, oracle.CRIT_MR
    s.set_launch_shape(stage_kernel=kernel)
    for _ in range(steps):
        run_pair(s, o, 1, lts=lts, adapt_crit=crit)
        assert_same_tree(s, o)
    assert_levels_close(s, o)


@pytest.mark.parametrize("case", ["uniform", "periodic", "adaptive", "adaptive_periodic", "mrlt"])
def test_tma_stage_kernel_fp32_matches_pencil_cell_by_cell(mrfv, case):
    """The TMA-staged stage kernel (5) against the pencil kernel (1) in single
    precision, every cell after two steps from the same state with the same time
    steps: same-level halos, ghost strips of coarse-fine faces, transmissive walls,
    periodic wrap and the flux registers (global and level-dependent steps) all
    enter.  The two kernels round differently (packed FP32x2 arithmetic and
    approximate reciprocals against the pencil kernel's expressions), so the bar is
    a few units of single-precision rounding of each variable's magnitude."""
    kw = dict(dim=2, precision="fp32")
    if case in ("uniform", "periodic"):
        kw.update(levels=1, base_blocks=(3, 5, 1), bc=1 if case == "periodic" else 0)
        P = mi.quadrant_params(5)
    else:
        kw.update(levels=5 if case != "mrlt" else 4, base_blocks=(1, 1, 1) if case != "mrlt" else (2, 2, 1),
                  adapt=True, eps=1e-3, lts=case == "mrlt", bc=1 if case == "adaptive_periodic" else 0)
        P = mi.quadrant_params(1)
    a = mrfv.Solver(**kw)
    b = mrfv.Solver(**kw)
    for s in (a, b):
        s.init_state(mi.IC_QUADRANTS, P)
    # a few steps of history on the pencil kernel so the halos and ghost strips are non-trivial
    for s in (a, b):
        s.set_launch_shape(stage_kernel=1)
        for _ in range(3):
            s.step(2e-4)
    a.set_launch_shape(stage_kernel=5)
    a.profile_enable(True)
    for _ in range(2):
        a.step(2e-4)
        b.step(2e-4)
    assert a.profile_read()["fv_kernels"] & 32, "the TMA-staged kernel did not run"
    for l in range(a.levels):
        assert np.array_equal(a.get_tree(l), b.get_tree(l))
        ga, _ = a.download_level(l)
        gb, _ = b.download_level(l)
        assert np.array_equal(np.isnan(ga), np.isnan(gb))
        m = ~np.isnan(gb[0])
        if not m.any():
            continue
        for v in range(4):
            scale = np.abs(gb[v][m]).max()
            err = np.abs(ga[v][m] - gb[v][m]).max()
            assert err <= 3e-6 * scale, (case, l, v, err, scale)


def test_tma_stage_kernel_fp32_mrlt_against_oracle(mrfv):
    """Level-dependent steps (flux registers accumulated over the fine sub-steps)
    on the TMA-staged kernel against the FP64 oracle: 2e-4 relative L1, totals 1e-6."""
    s, o = pair(mrfv, 2, 4, (2, 2, 1), precision="fp32", adapt=True, lts=True, params=mi.quadrant_params(3))
    s.set_launch_shape(stage_kernel=5)
    T0 = o.totals()
    for _ in range(6):
        dt = o.dt(0.5, True)
        s.step(dt)
        o.step(dt, True)
        o.adapt(oracle.CRIT_MR, 1e-3, precision=1)
    assert _finest_rel_l1(s, o, lambda: _fresh_oracle(2, 4, (2, 2, 1), mi.quadrant_params(3))) <= 2e-4
    assert np.all(np.abs(s.totals() - o.totals()) <= 1e-6 * np.abs(T0).max())


def _fresh_oracle(dim, levels, base, P):
    o = oracle.Oracle(dim, levels, base)
    o.init(mi.IC_QUADRANTS, P)
    return o


@pytest.mark.parametrize("dim", [2, 3])
def test_download_var_coarsened_means(mrfv, dim):
    """One variable averaged over coarsen^d cells equals the mean of the full download."""
    if dim == 2:
        s = mrfv.Solver(dim=2, levels=1, base_blocks=(3, 2, 1))
        s.init_state(mi.IC_QUADRANTS, mi.quadrant_params(1))
    else:
        s = mrfv.Solver(dim=3, levels=1, base_blocks=(2, 1, 2), lo=(-1, -1, -1), hi=(1, 1, 1))
        s.init_state(mi.IC_ELLIPSOID, mi.ellipsoid_params(1))
    s.step(0.0)
    full = s.download_level(0)[0]
    for var in range(dim + 2):
        assert np.array_equal(s.download_var(0, var, 1), full[var])
        for f in (2, 4):
            g = s.download_var(0, var, f)
            sh = full[var].shape
            blocks = full[var].reshape(*[x for n in sh for x in (n // f, f)])
            want = blocks.mean(axis=tuple(range(1, 2 * len(sh), 2)))
            assert np.allclose(g, want, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("lts", [False, True])
@pytest.mark.parametrize("eps", [1e9, -1.0])
def test_degenerate_thresholds(mrfv, eps, lts):
    """The two ends of the MR threshold: eps so large that nothing is significant
    (the tree collapses to level 0 and stays there) and eps < 0 (every block
    significant: the full tree), with global and level-dependent steps; trees and
    FP64 states against the oracle."""
    s, o = pair(mrfv, 2, 4, (2, 2, 1), adapt=True, lts=lts, eps=eps, params=mi.quadrant_params(4))
    assert_same_tree(s, o)
    for _ in range(3 if lts else 6):
        run_pair(s, o, 1, lts=lts, adapt_crit=oracle.CRIT_MR, eps=eps)
        assert_same_tree(s, o)
    if eps > 1:
        assert all(not s.get_tree(l).any() for l in range(1, 4))
    else:
        assert all(s.get_tree(l).all() for l in range(4))
    assert_levels_close(s, o)


def test_bounded_wait_expires_and_the_context_stays_usable(mrfv):
    """Failure detection without a GPU fault: a bounded mbarrier wait on a phase
    nothing completes returns ERR_TIMEOUT; the completed phase returns OK; the
    same context then steps normally."""
    s = mrfv.Solver(dim=2, levels=2, base_blocks=(2, 2, 1), adapt=True)
    s.init_state(mi.IC_QUADRANTS, mi.quadrant_params(1))
    assert s.wait_selftest(4096, True) == mrfv.OK
    assert s.wait_selftest(4096, False) == mrfv.ERR_TIMEOUT
    assert b"bounded device wait expired" in s.lib.mrfv_last_error(s._h)
    assert s.wait_selftest(4096, True) == mrfv.OK
    dt = s.step(0.0)
    assert dt > 0.0
    s.synchronize()


@pytest.mark.parametrize("dim", [2, 3])
def test_prolong_whole_level_matches_oracle_prediction(mrfv, dim):
    """mrfv_prolong overwrites a level by the third-order prediction of Section
    2.1; every cell against the oracle's prediction from the same coarse data
    (FP64, 1e-12)."""
    base = (2, 2, 1) if dim == 2 else (1, 1, 1)
    s = mrfv.Solver(dim=dim, levels=3, base_blocks=base, adapt=True, bc=1)
    ic = mi.IC_QUADRANTS if dim == 2 else mi.IC_ELLIPSOID
    params = mi.quadrant_params(3) if dim == 2 else [0.5, 0.5, 0.5, 0.3, 0.25, 0.2, 1.0, 1.0, 0.5, 0.5]
    s.init_state(ic, params)
    s.step(0.0)
    o = oracle.Oracle(dim, 3, base, bc=1)
    for lc in (0, 1):
        coarse = s.download_level(lc)[0]
        ex = s.get_tree(lc + 1).astype(bool)
        if not ex.any():
            continue
        s.prolong(lc)
        fine = s.download_level(lc + 1)[0]
        nv = dim + 2
        shape = fine.shape[1:]
        cflat = np.nan_to_num(coarse).reshape(nv, -1)
        checked = 0
        for idx in np.argwhere(~np.isnan(fine[0])):
            k, j, i = (0, *idx) if dim == 2 else tuple(idx)
            for v in range(nv):
                want = o.predict(lc + 1, cflat, v, int(i), int(j), int(k))
                got = fine[(v, *idx)]
                assert abs(got - want) <= 1e-12 * max(1.0, abs(want)), (lc, v, idx)
            checked += 1
            if checked >= 400:
                break
        assert checked > 0
