"""Pins of the proposer oracle (CPU): the features of hand-built trees whose block
means have closed forms, the training gradient against finite differences of
the loss, and the Adam update against its closed form.

The proposer has no counterpart in the paper (it stands in for the safety zone
of Section 2.1's refinement rule); these pins fix what the oracle computes from
the definitions stated in include/mrfv.h, independently of the CUDA path.
"""
import numpy as np
import pytest

from oracle import proposer as P

GAMMA = 1.4


def _level(shape_cells, rho_fn, vel, p_fn):
    """Dense conserved state [nv][cells...] of a level from closed-form fields of
    the cell indices (k, j, i) (or (j, i) in 2D)."""
    idx = np.meshgrid(*[np.arange(n) for n in shape_cells], indexing="ij")
    rho = rho_fn(*idx)
    p = p_fn(*idx)
    dim = len(shape_cells)
    mom = [rho * vel[d] for d in range(dim)]
    E = p / (GAMMA - 1.0) + 0.5 * rho * sum(v * v for v in vel[:dim])
    return np.stack([rho] + mom + [E]).astype(np.float64)


def _absent(q, blocks_present, shape_blocks):
    """NaN every block of q not in blocks_present (tuples in the map's index order)."""
    q = q.copy()
    for b in np.ndindex(*shape_blocks):
        if b not in blocks_present:
            q[(slice(None),) + tuple(slice(8 * i, 8 * i + 8) for i in b)] = np.nan
    return q


def test_features_hand_built_2d_tree():
    """Three levels of a 2D tree.  Linear fields: a block (or quadrant) mean is the
    field at its centre, so every expected value below is worked out by hand."""
    eps = 1e-3
    vel = (0.3, -0.2)
    # level 0: rho = 1 + 0.01 i + 0.02 j, p = 0.7 + 0.001 i (cells (j, i))
    q0 = _level((8, 8), lambda j, i: 1 + 0.01 * i + 0.02 * j, vel, lambda j, i: 0.7 + 0.001 * i)
    # level 1: blocks (0,0) and (1,1) exist; rho = 2 + 0.005 i + 0.003 j, p = 0.5
    q1 = _level((16, 16), lambda j, i: 2 + 0.005 * i + 0.003 * j, vel, lambda j, i: 0.5 + 0 * i)
    q1 = _absent(q1, {(0, 0), (1, 1)}, (2, 2))
    # level 2: only block (1,1) exists (its parent (0,0) does); rho = 3, p = 0.4
    q2 = _level((32, 32), lambda j, i: 3 + 0 * i, vel, lambda j, i: 0.4 + 0 * i)
    q2 = _absent(q2, {(1, 1)}, (4, 4))
    ex = [np.ones((1, 1), np.uint8), np.array([[1, 0], [0, 1]], np.uint8), np.zeros((4, 4), np.uint8)]
    ex[2][1, 1] = 1
    md = [np.full((1, 1), 3 * eps), np.array([[20 * eps, 0], [0, 4 * eps]]), np.zeros((4, 4))]
    md[2][1, 1] = 0.0
    s_rho, s_E = 2.5, 5.0          # pressure scale (gamma - 1) s_E = 2
    f = P.features(2, GAMMA, eps, [q0, q1, q2], ex, md, [s_rho, 0.0, 0.0, s_E])
    shapes = P.level_shapes(2, 3, (1, 1))
    offs = np.cumsum([0] + [int(np.prod(s)) for s in shapes])

    def at(l, by, bx):
        return f[:, offs[l] + bx + shapes[l][2] * by]

    # level 0: centre (3.5, 3.5); detail 3 eps -> 3/8
    assert at(0, 0, 0) == pytest.approx([1.105 / 2.5, 0.7035 / 2, 0.375], rel=1e-12)
    # level 1 existing: clamp at 8 (20 eps -> 1), 4 eps -> 1/2
    assert at(1, 0, 0) == pytest.approx([2.028 / 2.5, 0.25, 1.0], rel=1e-12)
    assert at(1, 1, 1) == pytest.approx([2.092 / 2.5, 0.25, 0.5], rel=1e-12)
    # level 1 absent: the quadrant of the level-0 block that covers it, detail 0
    assert at(1, 0, 1) == pytest.approx([1.085 / 2.5, 0.7055 / 2, 0.0], rel=1e-12)   # x in [4,8), y in [0,4)
    assert at(1, 1, 0) == pytest.approx([1.125 / 2.5, 0.7015 / 2, 0.0], rel=1e-12)   # x in [0,4), y in [4,8)
    # level 2
    assert at(2, 1, 1) == pytest.approx([3 / 2.5, 0.2, 0.0], rel=1e-12)
    assert at(2, 0, 0) == pytest.approx([2.012 / 2.5, 0.25, 0.0], rel=1e-12)       # quadrant of level-1 (0,0)
    assert at(2, 3, 3) == pytest.approx([2.108 / 2.5, 0.25, 0.0], rel=1e-12)       # quadrant of level-1 (1,1)
    # no parent: all zero
    for by, bx in [(0, 2), (0, 3), (1, 2), (2, 0), (3, 1)]:
        assert np.all(at(2, by, bx) == 0.0)


def test_features_octant_3d():
    """3D: an absent child takes the octant of its parent that covers it."""
    eps = 1e-3
    vel = (0.1, 0.2, -0.3)
    q0 = _level((8, 8, 8), lambda k, j, i: 1 + 0.01 * i + 0.02 * j + 0.04 * k, vel,
                lambda k, j, i: 0.6 + 0.002 * k)
    q1 = _level((16, 16, 16), lambda k, j, i: 1.5 + 0 * i, vel, lambda k, j, i: 0.3 + 0 * i)
    present = {b for b in np.ndindex(2, 2, 2)} - {(1, 0, 1)}
    q1 = _absent(q1, present, (2, 2, 2))
    ex = [np.ones((1, 1, 1), np.uint8), np.ones((2, 2, 2), np.uint8)]
    ex[1][1, 0, 1] = 0
    md = [np.zeros((1, 1, 1)), np.full((2, 2, 2), 16 * eps)]
    f = P.features(3, GAMMA, eps, [q0, q1], ex, md, [2.0, 0, 0, 0, 1.0])   # s_p = 0.4
    n0 = 1
    # position (bz=1, by=0, bx=1) of level 1: octant x in [4,8), y in [0,4), z in [4,8)
    p = n0 + 1 + 2 * (0 + 2 * 1)
    assert f[:, p] == pytest.approx([(1 + 0.055 + 0.03 + 0.22) / 2.0, (0.6 + 0.011) / 0.4, 0.0], rel=1e-12)
    # an existing level-1 block: its own means, detail clamped
    assert f[:, n0] == pytest.approx([0.75, 0.75, 1.0], rel=1e-12)
    # level 0: centre (3.5, 3.5, 3.5)
    assert f[:, 0] == pytest.approx([(1 + 0.035 + 0.07 + 0.14) / 2.0, 0.607 / 0.4, 0.0], rel=1e-12)


def _random_case(dim, levels, base, seed):
    rng = np.random.default_rng(seed)
    w = rng.normal(0.0, 0.4, P.NWEIGHTS)
    shapes = P.level_shapes(dim, levels, base)
    n = sum(int(np.prod(s)) for s in shapes)
    feats = rng.uniform(-1.0, 1.0, (2, 3, n))
    targets = (rng.uniform(size=(2, n)) < 0.3).astype(np.uint8)
    ex = [rng.uniform(size=s) < 0.6 for s in shapes]
    use = P.parent_mask(shapes, ex)
    return w, shapes, feats, targets, use


@pytest.mark.parametrize("dim,levels,base", [(2, 3, (1, 2)), (3, 2, (2, 1, 2))])
def test_training_gradient_matches_finite_differences(dim, levels, base):
    w, shapes, feats, targets, use = _random_case(dim, levels, base, 3 + dim)
    assert use.sum() > 5
    inv = 1.0 / use.size
    L0, g = P.loss_and_grad(w, feats, targets, shapes, use, inv)
    rng = np.random.default_rng(11)
    # every bias, and weights of every layer (some taps leave a 2D grid: gradient 0)
    idx = list(range(16 * 81, 16 * 81 + 16)) + list(range(NW2 := 16 * 81 + 16 + 16 * 432, NW2 + 16)) + [P.NWEIGHTS - 1]
    idx += list(rng.choice(16 * 81, 40, replace=False)) + list(16 * 81 + 16 + rng.choice(16 * 432, 60, replace=False))
    idx += list(NW2 + 16 + rng.choice(432, 40, replace=False))
    h = 1e-6
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (P.loss_and_grad(wp, feats, targets, shapes, use, inv)[0]
              - P.loss_and_grad(wm, feats, targets, shapes, use, inv)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-9), i
    if dim == 2:
        # taps with dz != 0 read the zero padding of a one-cell-deep grid
        W1g = g[:16 * 81].reshape(16, 3, 27)
        assert np.all(W1g[:, :, :9] == 0) and np.all(W1g[:, :, 18:] == 0)


def test_training_loss_is_the_binary_cross_entropy():
    """Zero weights: every logit is the last bias b; the loss is then
    inv * (count of used positions) * the cross-entropy of sigmoid(b) against
    each target, summed by hand."""
    w = np.zeros(P.NWEIGHTS)
    w[-1] = 0.3
    shapes = P.level_shapes(2, 2, (1, 1))
    n = 1 + 4
    feats = np.zeros((1, 3, n))
    targets = np.array([[1, 1, 0, 1, 0]], np.uint8)
    use = np.array([False, True, True, True, False])
    L, g = P.loss_and_grad(w, feats, targets, shapes, use, 0.5)
    s = 1.0 / (1.0 + np.exp(-0.3))
    assert L == pytest.approx(0.5 * (2 * -np.log(s) + -np.log(1 - s)), rel=1e-14)
    # dL/db3 = inv * sum over used positions of (sigmoid(b) - y)
    assert g[-1] == pytest.approx(0.5 * ((s - 1) * 2 + s), rel=1e-14)
    # a target of 255 leaves its position out of the loss
    t2 = targets.copy()
    t2[0, 2] = 255
    L2, g2 = P.loss_and_grad(w, feats, t2, shapes, use, 0.5)
    assert L2 == pytest.approx(0.5 * (2 * -np.log(s)), rel=1e-14)
    assert g2[-1] == pytest.approx(0.5 * ((s - 1) * 2), rel=1e-14)


def test_adam_closed_form():
    """Step 1 with zero moments moves each weight by lr g / (|g| + eps); step 2
    from the hand-computed moments."""
    w = np.array([1.0, -2.0, 0.5, 0.0])
    g1 = np.array([0.2, -3.0, 0.0, 1e-3])
    m = np.zeros(4)
    v = np.zeros(4)
    w1, m1, v1 = P.adam(w, g1, m, v, 1, 0.01)
    assert w1 == pytest.approx(w - 0.01 * g1 / (np.abs(g1) + 1e-8), rel=1e-13, abs=1e-15)
    g2 = np.array([0.1, 1.0, -0.5, 1e-3])
    w2, m2, v2 = P.adam(w1, g2, m1, v1, 2, 0.01)
    mm = 0.9 * 0.1 * g1 + 0.1 * g2
    vv = 0.999 * 0.001 * g1 ** 2 + 0.001 * g2 ** 2
    assert m2 == pytest.approx(mm, rel=1e-14) and v2 == pytest.approx(vv, rel=1e-14)
    assert w2 == pytest.approx(w1 - 0.01 * (mm / 0.19) / (np.sqrt(vv / (1 - 0.999 ** 2)) + 1e-8), rel=1e-13)


@pytest.mark.parametrize("dim,levels,base", [(2, 3, (1, 2)), (3, 2, (2, 1, 2))])
def test_bf16_training_gradient_reduces_to_the_pinned_one(dim, levels, base):
    """With its rounding taken out, the bfloat16 training gradient is the gradient
    pinned by finite differences above; with it, it stays close (the rounding
    points move each operand by at most 2^-8 relative)."""
    w, shapes, feats, targets, use = _random_case(dim, levels, base, 7 + dim)
    inv = 1.0 / use.size
    L, g = P.loss_and_grad(w, feats, targets, shapes, use, inv)
    Li, gi = P.loss_and_grad_bf16(w, feats, targets, shapes, use, inv, rnd=lambda a: np.asarray(a, np.float64))
    assert Li == pytest.approx(L, rel=1e-12)
    assert np.allclose(gi, g, rtol=1e-10, atol=1e-14)
    Lb, gb = P.loss_and_grad_bf16(w, feats, targets, shapes, use, inv)
    assert Lb == pytest.approx(L, rel=0.05)
    assert np.abs(gb - g).max() <= 0.1 * np.abs(g).max()
    assert not np.array_equal(gb, g)
