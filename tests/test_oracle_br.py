"""Pins of the oracle's Berger-Rigoutsos clustering of gradient flags (Section 2.2,
the AMROC clustering; Berger and Rigoutsos 1991) on the block grid.

The expected boxes below are worked out by hand from the algorithm's rules
(shrink to the flags, accept at efficiency >= eta with sides <= 8 blocks, cut at
a signature hole, else at the strongest signature inflection, else bisect the
longest side), and chosen so that each rule decides the outcome of one case.
"""
import numpy as np
import pytest

import mrfv_inputs as mi
import oracle


def _o(nx, ny):
    return oracle.Oracle(2, 1, (nx, ny, 1))


def test_hole_separates_two_clusters():
    """Two 3x3 clusters (one block missing in the first) with an empty gap: the
    hole cut separates them; each 3x3 box is efficient (8/9 >= 0.8)."""
    f = np.zeros((16, 16), np.uint8)
    f[0:3, 0:3] = 1
    f[0:3, 8:11] = 1
    f[1, 1] = 0
    want = np.zeros_like(f)
    want[0:3, 0:3] = 1
    want[0:3, 8:11] = 1
    assert np.array_equal(_o(16, 16).br_cluster(0, f, 0.8), want)


def test_inflection_cut_beats_bisection():
    """Three full columns plus one row to the right: no hole, and the x signature
    [8,8,8,1,1,1,1,1] has its only second-difference sign change between columns
    2 and 3, so the cut gives two exact boxes.  Bisecting instead would accept
    columns 0..3 (25/32 >= 0.7) and cover 7 unflagged blocks."""
    f = np.zeros((8, 8), np.uint8)
    f[:, 0:3] = 1
    f[0, 3:8] = 1
    out = _o(8, 8).br_cluster(0, f, 0.7)
    assert np.array_equal(out, f)


def test_l_shape_inflection():
    f = np.zeros((8, 8), np.uint8)
    f[0:2, :] = 1
    f[:, 0:2] = 1
    assert np.array_equal(_o(8, 8).br_cluster(0, f, 0.9), f)


def test_diagonal_bisects_to_two_by_two_boxes():
    """A diagonal has no hole and flat signatures (no inflection): bisection down
    to 2x2 boxes, which reach efficiency 1/2."""
    f = np.eye(8, dtype=np.uint8)
    want = np.zeros_like(f)
    for k in range(4):
        want[2 * k:2 * k + 2, 2 * k:2 * k + 2] = 1
    assert np.array_equal(_o(8, 8).br_cluster(0, f, 0.5), want)


def test_efficient_but_long_box_is_split_to_the_side_limit():
    """A full row of 16 blocks is efficient but longer than 8 blocks: bisected;
    the union is the row itself."""
    f = np.zeros((4, 16), np.uint8)
    f[2, :] = 1
    assert np.array_equal(_o(16, 4).br_cluster(0, f, 0.9), f)


@pytest.mark.parametrize("seed", range(6))
def test_random_flags_are_covered_and_bounded(seed):
    rng = np.random.default_rng(seed)
    f = (rng.random((12, 20)) < 0.15).astype(np.uint8)
    f[3:7, 4:9] = 1
    eta = 0.7
    out = _o(20, 12).br_cluster(0, f, eta)
    assert np.all(out[f == 1] == 1)  # every flag is in a box
    ys, xs = np.nonzero(f)
    bb = np.zeros_like(f)
    bb[ys.min():ys.max() + 1, xs.min():xs.max() + 1] = 1
    assert np.all(out[bb == 0] == 0)  # no box leaves the flags' bounding box
    # accepted boxes are at least eta efficient, so the union is too
    assert f.sum() >= eta * out.sum() - 1e-9


def test_br_in_the_amr_cycle_conserves_and_grades():
    """Gradient flags clustered by Berger-Rigoutsos in the adaptation cycle with
    level-dependent steps: conservation on a periodic domain and the tree rules."""
    o = oracle.Oracle(2, 3, (4, 4, 1), bc=oracle.BC_PERIODIC, clustering=oracle.CLUSTER_BR)
    o.init(mi.IC_QUADRANTS, mi.quadrant_params(3))
    o.adapt(oracle.CRIT_GRAD, eps_w=0.05, eta_tol=0.8)
    T0 = o.totals()
    for _ in range(3):
        o.step(o.dt(0.5, True), True)
        o.adapt(oracle.CRIT_GRAD, eps_w=0.05, eta_tol=0.8)
    assert np.all(np.abs(o.totals() - T0) <= 1e-12 * np.abs(T0).max())
    for l in range(1, o.levels):
        ex, par = o.get_exist(l), o.get_exist(l - 1)
        ys, xs = np.nonzero(ex)
        assert np.all(par[ys // 2, xs // 2])  # every block has its parent
