"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the physical
flux of Eq. 2.2, the exact Riemann solution (Toro), conservation on a periodic
domain, free-stream preservation, mirror symmetry, exactness of the third-order
prediction on quadratic cell averages (Section 2.1), exact MR reconstruction at
eps = 0, the tree rules of Section 2.1 (gradedness, complete child sets), and the
printed values of Table 1.
"""
import math
import os

import numpy as np
import pytest

import mrfv_inputs as mi
import oracle
import exact_riemann as er

HERE = os.path.dirname(os.path.abspath(__file__))


def _run(o, t_end, cfl=0.5, lts=False, adapt=None):
    t, n = 0.0, 0
    while t < t_end - 1e-14:
        dt = min(o.dt(cfl, lts), t_end - t)
        o.step(dt, lts)
        if adapt:
            adapt()
        t += dt
        n += 1
    return n


# --------------------------------------------------------------------------- fixtures of the paper

def test_laxliu6_matches_table1():
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "laxliu6_table1.txt"))
            if l.strip() and not l.startswith("#")]
    expect = []
    for _, rho, p, v1, v2 in rows:
        expect += [float(rho), float(v1), float(v2), float(p)]
    assert mi.laxliu6_params() == expect
    o = oracle.Oracle(2, 1, (2, 2, 1))
    o.init(mi.IC_QUADRANTS, expect)
    q = o.get_level(0)
    # cell (i, j): quadrant I is x >= 0.5, y >= 0.5
    for (j, i), quad in (((15, 15), 0), ((15, 0), 1), ((0, 0), 2), ((0, 15), 3)):
        rho, v1, v2, p = expect[4 * quad: 4 * quad + 4]
        assert q[0, j, i] == rho
        assert q[1, j, i] == pytest.approx(rho * v1, abs=0)
        assert q[2, j, i] == pytest.approx(rho * v2, abs=0)
        assert q[3, j, i] == pytest.approx(p / 0.4 + 0.5 * rho * (v1 * v1 + v2 * v2), rel=1e-15)


def test_exact_riemann_solver_matches_toro_table():
    vals = dict(l.split() for l in open(os.path.join(HERE, "golden", "sod_exact_t015.txt"))
                if l.strip() and not l.startswith("#"))
    ps, us = er.star_state((1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    assert ps == pytest.approx(float(vals["p_star"]), abs=1e-5)
    assert us == pytest.approx(float(vals["u_star"]), abs=1e-5)
    # densities just left / right of the contact
    rl = er.sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), us - 1e-9)[0]
    rr = er.sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), us + 1e-9)[0]
    assert rl == pytest.approx(float(vals["rho_star_left"]), abs=1e-5)
    assert rr == pytest.approx(float(vals["rho_star_right"]), abs=1e-5)


# --------------------------------------------------------------------------- flux

@pytest.mark.parametrize("dim", [2, 3])
def test_ausm_plus_consistency_with_physical_flux(dim):
    o = oracle.Oracle(dim, 1, (1, 1, 1))
    rng = np.random.default_rng(0)
    for _ in range(200):
        rho = rng.uniform(0.1, 3.0)
        v = rng.uniform(-3.0, 3.0, dim)  # sub- and supersonic
        p = rng.uniform(0.05, 3.0)
        q = np.r_[rho, rho * v, p / 0.4 + 0.5 * rho * v @ v]
        for nd in range(dim):
            F = o.flux(nd, q, q)
            f = o.physical_flux(nd, q)
            assert np.allclose(F, f, rtol=1e-13, atol=1e-13 * np.abs(f).max())


def test_ausm_plus_supersonic_is_upwind():
    o = oracle.Oracle(2, 1, (1, 1, 1))
    for sgn in (1.0, -1.0):
        ql = np.array([1.0, sgn * 3.0, 0.2, 1.0 / 0.4 + 0.5 * (9.0 + 0.04)])
        qr = np.array([0.5, sgn * 1.5, -0.1, 0.8 / 0.4 + 0.25 * (2.25 + 0.01)])
        F = o.flux(0, ql, qr)
        up = ql if sgn > 0 else qr
        assert np.allclose(F, o.physical_flux(0, up), rtol=1e-13)


def test_ausm_plus_mirror_symmetry():
    """Reflecting x -> -x swaps the states, negates v_n: mass and energy flux flip sign."""
    o = oracle.Oracle(2, 1, (1, 1, 1))
    rng = np.random.default_rng(1)
    for _ in range(100):
        a = np.r_[rng.uniform(0.2, 2), rng.uniform(-1, 1, 2), rng.uniform(0.2, 2)]
        b = np.r_[rng.uniform(0.2, 2), rng.uniform(-1, 1, 2), rng.uniform(0.2, 2)]
        cons = lambda w: np.r_[w[0], w[0] * w[1], w[0] * w[2], w[3] / 0.4 + 0.5 * w[0] * (w[1] ** 2 + w[2] ** 2)]
        mir = lambda w: np.r_[w[0], -w[1], w[2], w[3]]
        F = o.flux(0, cons(a), cons(b))
        G = o.flux(0, cons(mir(b)), cons(mir(a)))
        assert np.allclose(G, [-F[0], F[1], -F[2], -F[3]], rtol=1e-12, atol=1e-14)


# --------------------------------------------------------------------------- whole FV step

@pytest.mark.parametrize("axis,dim", [(0, 2), (1, 2), (2, 3)])
def test_sod_converges_to_exact_riemann_solution(axis, dim):
    left, right, t_end = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 0.15
    errs = []
    for N in (64, 128, 256):
        nb = [1, 1, 1]
        nb[axis] = N // 8
        hi = [8.0 / N] * 3
        hi[axis] = 1.0
        o = oracle.Oracle(dim, 1, nb, lo=(0, 0, 0), hi=hi)
        o.init(mi.IC_SHOCKTUBE, mi.sod_params(axis, 0.5))
        _run(o, t_end)
        rho = o.get_level(0)[0]
        line = np.moveaxis(rho, dim - 1 - axis, -1).reshape(-1, N)
        assert np.abs(line - line[0]).max() < 1e-12  # stays planar
        ex = er.cell_average_density(left, right, 0.5, t_end, np.linspace(0, 1, N + 1))
        errs.append(np.abs(line[0] - ex).mean())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 3e-3
    assert np.all(rates > 0.6) and np.all(rates < 1.4), (errs, rates)


def test_smooth_wave_second_order():
    errs = []
    for nb in (2, 4, 8):
        o = oracle.Oracle(2, 1, (nb, nb, 1), bc=oracle.BC_PERIODIC)
        o.init(mi.IC_WAVE, [0.2, 1.0, 1.0, 0.0, 1.0])
        t_end = 0.1
        _run(o, t_end, cfl=0.4)
        N = nb * 8
        x = (np.arange(N) + 0.5) / N
        X, Y = np.meshgrid(x, x)
        h = 1.0 / N
        # exact cell averages of the translated wave rho = 1 + 0.2 sin(2 pi (x + y - 2t))
        s = 2 * np.pi
        avg = 1 + 0.2 * (np.sin(s * (X + Y - 2 * t_end)) * (np.sin(s * h / 2) / (s * h / 2)) ** 2)
        errs.append(np.abs(o.get_level(0)[0] - avg).mean())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > 1.5, (errs, rates)


@pytest.mark.parametrize("dim", [2, 3])
def test_free_stream_is_bit_exact(dim):
    o = oracle.Oracle(dim, 3 if dim == 2 else 2, (1, 1, 1), bc=oracle.BC_TRANSMISSIVE)
    o.init(mi.IC_UNIFORM, [1.3, 0.4, -0.2, 0.3 if dim == 3 else 0.0, 0.8])
    # force a graded adaptive tree: keep only one corner refined
    ex = [o.get_exist(l) for l in range(o.levels)]
    for l in range(2, o.levels):
        m = np.zeros_like(ex[l])
        m[(slice(0, 4),) * dim] = 1
        o.set_exist(l, m)
    ref = [o.get_level(l) for l in range(o.levels)]
    for _ in range(4):
        o.step(0.002)
    for l in range(o.levels):
        a, b = o.get_level(l), ref[l]
        m = ~np.isnan(a)
        assert np.array_equal(a[m], b[m])


@pytest.mark.parametrize("lts", [False, True])
def test_adaptive_conservation_periodic(lts):
    o = oracle.Oracle(2, 6, (1, 1, 1), bc=oracle.BC_PERIODIC)
    o.init(mi.IC_QUADRANTS, mi.quadrant_params(1))
    o.adapt(oracle.CRIT_MR, 1e-3)
    T0 = o.totals()
    nleaf_levels = set()
    for _ in range(6 if not lts else 1):
        o.step(o.dt(0.5, lts), lts)
        o.adapt(oracle.CRIT_MR, 1e-3)
        nleaf_levels |= {l for l in range(o.levels) if o.leaf_mask(l).any()}
    assert len(nleaf_levels) >= 2  # a genuinely multi-level hierarchy
    T1 = o.totals()
    assert np.all(np.abs(T1 - T0) <= 1e-12 * np.abs(T0).max()), (T1 - T0)


def test_amr_gradient_lts_conservation_periodic():
    o = oracle.Oracle(2, 3, (4, 4, 1), bc=oracle.BC_PERIODIC)
    o.init(mi.IC_QUADRANTS, mi.quadrant_params(3))
    o.adapt(oracle.CRIT_GRAD, eps_w=0.05, eta_tol=0.8)
    T0 = o.totals()
    for _ in range(3):
        o.step(o.dt(0.5, True), True)
        o.adapt(oracle.CRIT_GRAD, eps_w=0.05, eta_tol=0.8)
    T1 = o.totals()
    assert np.all(np.abs(T1 - T0) <= 1e-12 * np.abs(T0).max())


def test_diagonal_symmetry_uniform_bit_exact():
    """Data symmetric under x <-> y with (v1, v2) <-> (v2, v1) stays symmetric."""
    P = [1.0, 0.3, 0.3, 1.0,   # I (u = v)
         2.0, 0.5, -0.2, 1.2,  # II
         0.8, -0.4, -0.4, 0.7,  # III (u = v)
         2.0, -0.2, 0.5, 1.2]  # IV = II mirrored
    o = oracle.Oracle(2, 1, (4, 4, 1))
    o.init(mi.IC_QUADRANTS, P)
    _run(o, 0.05)
    q = o.get_level(0)
    assert np.array_equal(q[0], q[0].T)
    assert np.array_equal(q[1], q[2].T)
    assert np.array_equal(q[3], q[3].T)


def test_diagonal_symmetry_adaptive():
    P = [1.0, 0.3, 0.3, 1.0, 2.0, 0.5, -0.2, 1.2, 0.8, -0.4, -0.4, 0.7, 2.0, -0.2, 0.5, 1.2]
    o = oracle.Oracle(2, 5, (1, 1, 1))
    o.init(mi.IC_QUADRANTS, P)
    o.adapt(oracle.CRIT_MR, 1e-3)
    _run(o, 0.03, adapt=lambda: o.adapt(oracle.CRIT_MR, 1e-3))
    for l in range(o.levels):
        ex = o.get_exist(l)
        assert np.array_equal(ex, ex.T)
    f = o.project_finest()
    assert np.abs(f[0] - f[0].T).max() < 1e-12
    assert np.abs(f[1] - f[2].T).max() < 1e-12


def test_ellipsoid_mirror_symmetry_3d():
    o = oracle.Oracle(3, 1, (2, 2, 2), lo=(-1, -1, -1), hi=(1, 1, 1))
    o.init(mi.IC_ELLIPSOID, mi.ellipsoid_params(5))
    for _ in range(3):
        o.step(o.dt(0.5))
    q = o.get_level(0)
    rho = q[0]
    for ax in range(3):
        assert np.abs(rho - np.flip(rho, ax)).max() < 1e-13
    # momentum normal to a mirror plane flips sign
    assert np.abs(q[1] + np.flip(q[1], 2)).max() < 1e-13


# --------------------------------------------------------------------------- multiresolution

def _avg_poly_1d(a, x0, x1):
    return (x1 ** (a + 1) - x0 ** (a + 1)) / ((a + 1) * (x1 - x0))


@pytest.mark.parametrize("dim", [2, 3])
def test_prediction_exact_on_quadratic_cell_averages(dim):
    o = oracle.Oracle(dim, 2, (1, 1, 1))
    rng = np.random.default_rng(7)
    coef = rng.normal(size=(3,) * dim)
    nc, nf = 8, 16

    def averages(n):
        e = np.linspace(0, 1, n + 1)
        A = [np.array([_avg_poly_1d(a, e[i], e[i + 1]) for i in range(n)]) for a in range(3)]
        out = np.zeros((n,) * dim)
        for idx in np.ndindex(*(3,) * dim):
            t = coef[idx]
            grids = np.meshgrid(*[A[idx[d]] for d in range(dim)], indexing="ij")
            term = np.ones_like(grids[0]) * t
            for g in grids:
                term = term * g
            out += term
        return out  # indexed [i, j, (k)]

    C = averages(nc)
    F = averages(nf)
    coarse = np.zeros((o.nv,) + (nc,) * dim)
    coarse[0] = np.transpose(C)  # oracle layout (k, j, i)
    for idx in np.ndindex(*(nf,) * dim):
        if min(idx) < 2 or max(idx) > nf - 3:
            continue  # the boundary rule is not polynomial
        I = list(idx) + [0] * (3 - dim)
        p = o.predict(1, coarse, 0, *I)
        assert p == pytest.approx(F[idx], abs=1e-13)


@pytest.mark.parametrize("dim", [2, 3])
def test_prediction_children_mean_equals_parent(dim):
    o = oracle.Oracle(dim, 2, (1, 1, 1), bc=oracle.BC_PERIODIC)
    rng = np.random.default_rng(3)
    coarse = rng.uniform(0.5, 2.0, (o.nv,) + (8,) * dim)
    for cidx in [(1, 2, 3), (0, 7, 4), (5, 5, 5)]:
        c = cidx[:dim]
        s = 0.0
        for off in np.ndindex(*(2,) * dim):
            I = [2 * c[d] + off[d] for d in range(dim)] + [0] * (3 - dim)
            s += o.predict(1, coarse, 0, *I)
        assert s / 2 ** dim == pytest.approx(coarse[(0,) + tuple(reversed(c))], rel=1e-14)


@pytest.mark.parametrize("dim,levels", [(2, 5), (3, 3)])
def test_mr_reconstruction_exact_at_eps_zero(dim, levels):
    kw = dict(lo=(-1, -1, -1), hi=(1, 1, 1)) if dim == 3 else {}
    o = oracle.Oracle(dim, levels, (1, 1, 1) if dim == 2 else (2, 2, 2), **kw)
    if dim == 2:
        o.init(mi.IC_QUADRANTS, mi.quadrant_params(4))
    else:
        o.init(mi.IC_ELLIPSOID, mi.ellipsoid_params(4))
    fine = o.get_level(o.L)
    o.adapt(oracle.CRIT_MR, 0.0)
    n_full = sum(int(np.prod(o.blocks_shape(l))) for l in range(o.levels))
    n_kept = sum(int(o.get_exist(l).sum()) for l in range(o.levels))
    assert n_kept < n_full  # constant regions were coarsened
    rec = o.project_finest()
    assert np.abs(rec - fine).max() < 1e-13


def _tree_invariants(o):
    dim = o.dim
    assert o.get_exist(0).all()
    for l in range(1, o.levels):
        ex = o.get_exist(l).astype(bool)
        par = o.get_exist(l - 1).astype(bool)
        # complete child sets and existing parents
        sh = ex.shape
        grp = ex.reshape([s for n in sh for s in (n // 2, 2)])
        grp = grp.transpose(list(range(0, 2 * dim, 2)) + list(range(1, 2 * dim, 2)))
        anyc = grp.reshape(grp.shape[:dim] + (-1,)).any(-1)
        allc = grp.reshape(grp.shape[:dim] + (-1,)).all(-1)
        assert np.array_equal(anyc, allc)
        assert np.all(par[anyc])
        # gradedness: every neighbour (in the domain) of a parent with children exists
        for idx in zip(*np.nonzero(anyc)):
            for off in np.ndindex(*(3,) * dim):
                nb = tuple(idx[d] + off[d] - 1 for d in range(dim))
                if all(0 <= nb[d] < par.shape[d] for d in range(dim)):
                    assert par[nb]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tree_rules_after_adapt(seed):
    o = oracle.Oracle(2, 6, (1, 1, 1))
    o.init(mi.IC_QUADRANTS, mi.quadrant_params(seed))
    o.adapt(oracle.CRIT_MR, 1e-3)
    _tree_invariants(o)
    for _ in range(3):
        old = [o.get_exist(l).astype(bool) for l in range(o.levels)]
        o.step(o.dt(0.5))
        o.adapt(oracle.CRIT_MR, 1e-3)
        _tree_invariants(o)
        for l in range(1, o.levels):
            sig, md = o.get_sig(l)
            assert not (sig.astype(bool) & ~old[l]).any()
            ex = o.get_exist(l).astype(bool)
            for idx in zip(*np.nonzero(sig)):
                assert md[idx] > 1e-3
                for off in np.ndindex(3, 3):  # safety zone
                    nb = (idx[0] + off[0] - 1, idx[1] + off[1] - 1)
                    if 0 <= nb[0] < ex.shape[0] and 0 <= nb[1] < ex.shape[1]:
                        assert ex[nb]
                if l < o.L:  # refined by one level
                    ch = o.get_exist(l + 1)
                    assert ch[2 * idx[0], 2 * idx[1]]


def test_full_tree_adaptive_step_equals_uniform():
    P = mi.quadrant_params(6)
    a = oracle.Oracle(2, 3, (1, 1, 1))
    a.init(mi.IC_QUADRANTS, P)
    a.adapt(oracle.CRIT_MR, -1.0)  # every block significant: full tree, leaves on the finest level
    b = oracle.Oracle(2, 1, (4, 4, 1))
    b.init(mi.IC_QUADRANTS, P)
    assert a.leaf_mask(2).all()
    for _ in range(5):
        dt = b.dt(0.5)
        assert a.dt(0.5) == dt
        a.step(dt)
        b.step(dt)
    assert np.array_equal(a.get_level(2), b.get_level(0))


def test_lts_full_tree_equals_global_fine_steps():
    P = mi.quadrant_params(8)
    a = oracle.Oracle(2, 3, (1, 1, 1))
    a.init(mi.IC_QUADRANTS, P)
    a.adapt(oracle.CRIT_MR, -1.0)
    b = oracle.Oracle(2, 1, (4, 4, 1))
    b.init(mi.IC_QUADRANTS, P)
    dt = b.dt(0.5)
    assert a.dt(0.5, True) == dt
    a.step(dt, True)  # one coarse step = 4 finest sub-steps
    for _ in range(4):
        b.step(dt)
    assert np.array_equal(a.get_level(2), b.get_level(0))


def test_gradient_flags_and_row_clustering_brute_force():
    o = oracle.Oracle(2, 2, (8, 8, 1), bc=oracle.BC_PERIODIC)
    o.init(mi.IC_QUADRANTS, mi.quadrant_params(11))
    rho = o.get_level(0)[0]  # level 0 fully exists: the scheme's array is the state
    eps, eta = 0.05, 0.8
    o.adapt(oracle.CRIT_GRAD, eps_w=eps, eta_tol=eta)
    sig, _ = o.get_sig(0)
    cell = np.zeros_like(rho, dtype=bool)
    for a, b in ((1, 0), (0, 1), (1, 1)):
        cell |= np.abs(np.roll(np.roll(rho, -b, 0), -a, 1) - rho) > eps
    dil = cell.copy()
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            dil |= np.roll(np.roll(cell, b, 0), a, 1)
    blk = dil.reshape(8, 8, 8, 8).any(axis=(1, 3))
    expect = np.zeros_like(blk)
    for j in range(8):
        x = 0
        while x < 8:
            if not blk[j, x]:
                x += 1
                continue
            best, cnt = x, 0
            for e in range(x, min(8, x + 8)):
                if blk[j, e]:
                    cnt += 1
                    if cnt >= eta * (e - x + 1):
                        best = e
            expect[j, x:best + 1] = True
            x = best + 1
    assert np.array_equal(sig.astype(bool), expect)
    assert blk.any() and not blk.all()
