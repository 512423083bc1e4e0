"""Learned refinement proposer: oracle pins (CPU) and tensor-core inference,
features and training on the GPU against the oracle."""
import numpy as np
import pytest

import mrfv_inputs as mi
from oracle import proposer as P


def random_weights(seed: int, scale: float = 0.3) -> np.ndarray:
    rng = np.random.default_rng(seed)
    w = rng.normal(0.0, 1.0, P.NWEIGHTS).astype(np.float32)
    (W1, B1), (W2, B2), (W3, B3) = P.unpack(w)
    W1 *= scale / np.sqrt(81); W2 *= scale * 2 / np.sqrt(432); W3 *= scale * 2 / np.sqrt(432)
    return w


# ----------------------------------------------------------------------------- oracle pins

def test_bf16_rounding_known_values():
    x = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -9, 1 + 2 ** -7, -2.5, 0.0, 3.0e38], dtype=np.float32)
    r = P.bf16_round(x)
    assert r[0] == 1.0
    assert r[1] == 1.0                  # tie -> even
    assert r[2] == np.float32(1 + 2 ** -7)  # above the tie -> up
    assert r[3] == np.float32(1 + 2 ** -7)
    assert r[4] == -2.5 and r[5] == 0.0
    assert np.isfinite(r[6])


def test_conv_level_matches_brute_force():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 3, 4, 5))
    W = rng.normal(size=(3, 2, 27))
    b = rng.normal(size=3)
    y = P.conv_level(x, W, b)
    for co in range(3):
        for z in range(3):
            for yy in range(4):
                for xx in range(5):
                    s = b[co]
                    for ci in range(2):
                        for t in range(27):
                            dz, dy, dx = t // 9 - 1, (t // 3) % 3 - 1, t % 3 - 1
                            zz, y2, x2 = z + dz, yy + dy, xx + dx
                            if 0 <= zz < 3 and 0 <= y2 < 4 and 0 <= x2 < 5:
                                s += W[co, ci, t] * x[ci, zz, y2, x2]
                    assert y[co, z, yy, xx] == pytest.approx(s, abs=1e-12)


def test_forward_bias_only_is_constant_and_levels_independent():
    w = np.zeros(P.NWEIGHTS, np.float32)
    (W1, B1), (W2, B2), (W3, B3) = P.unpack(w)
    B3[0] = 0.75
    shapes = P.level_shapes(2, 3, (2, 2))
    n = sum(int(np.prod(s)) for s in shapes)
    z = P.forward(w, np.random.default_rng(0).normal(size=(3, n)), shapes)
    assert np.all(z == 0.75)


# ----------------------------------------------------------------------------- GPU

@pytest.fixture(scope="module")
def mrfv():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1603_05211_gb300 as m

    m.build()
    return m


def _oracle_features(s, dim, eps):
    levels = [s.download_level(l)[0] for l in range(s.levels)]
    ex = [s.get_tree(l) for l in range(s.levels)]
    md = [s.get_flags(l)[1] for l in range(s.levels)]
    # the analysis scales: recompute the level-0 maxima (same definition as the library)
    q0 = levels[0]
    rho = np.abs(q0[0]).max()
    E = np.abs(q0[dim + 1]).max()
    return P.features(dim, 1.4, eps, levels, ex, md, [rho] + [0.0] * dim + [E])


def _bf16_tie_distance(v: np.ndarray) -> np.ndarray:
    """Distance of each value to the nearest rounding midpoint of the bfloat16 grid."""
    a = np.abs(v).astype(np.float32)
    lo = (a.view(np.uint32) & np.uint32(0xFFFF0000)).view(np.float32).astype(np.float64)
    ulp = np.ldexp(1.0, np.frexp(np.maximum(lo, 1e-30))[1] - 8)
    return np.abs(np.abs(v) - (lo + 0.5 * ulp))


def _check_bf16_layer(h_gpu, pre, bound):
    """h_gpu: the kernel's bfloat16 ReLU outputs; pre: the oracle's exact
    pre-activations of the same inputs; bound: the FP32-accumulation error bound
    per output.  Exact equality with bf16(relu(pre)) except where pre lies
    within the bound of a rounding midpoint (or of 0), where the two
    neighbouring bfloat16 values are both correct.  Returns (outputs within the
    bound of a tie, outputs)."""
    ref = P.bf16_round(np.maximum(pre, 0.0).astype(np.float32)).astype(np.float64)
    near = (_bf16_tie_distance(pre) <= bound) | (np.abs(pre) <= bound)
    exact = ~near
    assert np.array_equal(h_gpu[exact], ref[exact]), np.abs(h_gpu[exact] - ref[exact]).max()
    ulp = np.ldexp(1.0, np.frexp(np.maximum(np.abs(pre[near]) + bound[near], 1e-30))[1] - 7)
    assert np.all(np.abs(h_gpu[near] - ref[near]) <= ulp)
    return int(near.sum()), near.size


@pytest.mark.gpu
@pytest.mark.parametrize("dim", [2, 3])
def test_proposer_features_and_tensor_core_inference_match_oracle(mrfv, dim):
    """Features within FP32 rounding of the oracle's block means; each tensor-core
    layer fed its own input checked against the oracle's exact convolution:
    BF16 outputs identical except at rounding ties within the FP32 accumulation
    error, logits within that error."""
    if dim == 2:
        s = mrfv.Solver(dim=2, precision="fp32", levels=5, base_blocks=(2, 2, 1), adapt=True, eps=1e-3)
        s.init_state(mi.IC_QUADRANTS, mi.quadrant_params(3))
        shapes = P.level_shapes(2, 5, (2, 2))
    else:
        s = mrfv.Solver(dim=3, precision="fp32", levels=3, base_blocks=(2, 2, 2), lo=(-1, -1, -1), hi=(1, 1, 1),
                        adapt=True, eps=1e-3)
        s.init_state(mi.IC_ELLIPSOID, mi.ellipsoid_params(3))
        shapes = P.level_shapes(3, 3, (2, 2, 2))
    for _ in range(3):
        s.step(0.0)
    s.analyse(1e-3)
    fg = s.proposer_features()
    fo = _oracle_features(s, dim, 1e-3)
    assert np.allclose(fg, fo, rtol=2e-5, atol=2e-6)
    w = random_weights(5)
    s.proposer_set_weights(w)
    zg = s.proposer_infer()
    h1g, h2g = s.proposer_activations()
    (W1, B1), (W2, B2), (W3, B3) = P.unpack(w)
    W1, W2, W3 = [P.bf16_round(W).astype(np.float64) for W in (W1, W2, W3)]
    # FP32 accumulation of K products: error below K * 2^-22 * sum |w| |x| (a factor 4 over
    # the sequential-summation bound, the tensor core's adder order being unspecified)
    off = 0
    near = total = 0
    for sh in shapes:
        n = int(np.prod(sh))
        x = P.bf16_round(fg[:, off:off + n]).astype(np.float64).reshape((3,) + sh)
        a1 = P.conv_level(x, W1, B1)
        b1 = 224 * 2.0 ** -22 * P.conv_level(np.abs(x), np.abs(W1), np.abs(B1))
        k, m = _check_bf16_layer(h1g[off:off + n].T.reshape((16,) + sh), a1, b1)
        near, total = near + k, total + m
        h1 = h1g[off:off + n].T.reshape((16,) + sh).astype(np.float64)
        a2 = P.conv_level(h1, W2, B2)
        b2 = 432 * 2.0 ** -22 * P.conv_level(np.abs(h1), np.abs(W2), np.abs(B2))
        k, m = _check_bf16_layer(h2g[off:off + n].T.reshape((16,) + sh), a2, b2)
        near, total = near + k, total + m
        h2 = h2g[off:off + n].T.reshape((16,) + sh).astype(np.float64)
        z = P.conv_level(h2, W3, B3)[0].reshape(-1)
        bz = (432 * 2.0 ** -22 * P.conv_level(np.abs(h2), np.abs(W3), np.abs(B3)))[0].reshape(-1)
        assert np.all(np.abs(zg[off:off + n] - z) <= bz + 1e-30), np.abs(zg[off:off + n] - z).max()
        off += n
    assert near < 0.3 * total, (near, total)   # the bound leaves most outputs decided exactly
    # end to end, the decisions agree wherever the oracle's own BF16 chain is clear of 0
    zo = P.forward(w, fg, shapes)
    clear = np.abs(zo) > 2e-3 * np.abs(zo).max()
    assert np.array_equal(zg[clear] > 0, zo[clear] > 0)


def _snapshots(mrfv, kw, nsnap, seed=2):
    s = mrfv.Solver(**kw)
    s.init_state(mi.IC_QUADRANTS, mi.quadrant_params(seed))
    feats, targets = [], []
    for _ in range(nsnap):
        s.analyse(1e-3)
        f = s.proposer_features()
        s.step(0.0)
        s.analyse(1e-3)
        feats.append(f)
        targets.append(np.concatenate([s.get_flags(l)[0].ravel() for l in range(s.levels)]))
    return s, np.stack(feats), np.stack(targets)


@pytest.mark.gpu
@pytest.mark.parametrize("dim", [2, 3])
def test_proposer_training_gradient_and_adam_match_oracle(mrfv, dim):
    """The training kernels (the tensor-core forward pass, the BCE gradient, the
    mirrored-tap tensor-core convolutions for the gradients of the layer inputs
    with the ReLU masks, the weight gradients from the BF16 rows) against the
    oracle's bfloat16 backward pass, layer by layer; then three Adam steps against
    the oracle's Adam on the same gradients.  The two sides round the same values
    to bfloat16; they differ where FP32 accumulation in a different order crosses a
    rounding tie, so each layer's gradient must agree within 0.5 % of its largest
    entry (a wrong tap, sign or mask changes entries by their own size)."""
    if dim == 2:
        kw = dict(dim=2, precision="fp32", levels=5, base_blocks=(2, 2, 1), adapt=True, eps=1e-3, bc=1)
    else:
        kw = dict(dim=3, precision="fp32", levels=3, base_blocks=(2, 2, 2), lo=(-1, -1, -1), hi=(1, 1, 1),
                  adapt=True, eps=1e-3)
    if dim == 2:
        s, feats, targets = _snapshots(mrfv, kw, 3)
    else:
        s = mrfv.Solver(**kw)
        s.init_state(mi.IC_ELLIPSOID, mi.ellipsoid_params(3))
        fl, tl = [], []
        for _ in range(2):
            s.analyse(1e-3)
            fl.append(s.proposer_features())
            s.step(0.0)
            s.analyse(1e-3)
            tl.append(np.concatenate([s.get_flags(l)[0].ravel() for l in range(s.levels)]))
        feats, targets = np.stack(fl), np.stack(tl)
    shapes = P.level_shapes(dim, s.levels, s.base_blocks[:dim])
    # leave a tenth of the positions out of the loss (target 255)
    targets = targets.copy()
    targets[np.random.default_rng(5).uniform(size=targets.shape) < 0.1] = 255
    w = random_weights(7)
    s.proposer_set_weights(w)
    ex = [s.get_tree(l) for l in range(s.levels)]
    use = P.parent_mask(shapes, ex)
    n0 = int(np.prod(shapes[0]))
    inv = 1.0 / (feats.shape[0] * (use.size - n0))
    lg, gg = s.proposer_grad(feats, targets)
    lo, go = P.loss_and_grad_bf16(w.astype(np.float64), feats, targets, shapes, use, inv)
    assert lg == pytest.approx(lo, rel=1e-4)
    o = 0
    for name, size in (("W1", 16 * 81), ("B1", 16), ("W2", 16 * 432), ("B2", 16), ("W3", 432), ("B3", 1)):
        a, b = gg[o:o + size], go[o:o + size]
        assert np.abs(a - b).max() <= 5e-3 * np.abs(b).max() + 1e-12, (name, np.abs(a - b).max(), np.abs(b).max())
        o += size
    # Adam: each step applies the gradient the grad entry point reports for the current weights
    m = np.zeros(P.NWEIGHTS)
    v = np.zeros(P.NWEIGHTS)
    wc = s.proposer_get_weights().astype(np.float64)
    lr = 1e-2
    for t in range(1, 4):
        _, g = s.proposer_grad(feats, targets)
        we, m, v = P.adam(wc, g.astype(np.float64), m, v, t, lr)
        s.proposer_train(feats, targets, steps=1, lr=lr)
        wc = s.proposer_get_weights().astype(np.float64)
        assert np.all(np.abs(wc - we) <= 2e-6 * lr + 1e-6 * np.abs(we)), np.abs(wc - we).max()


@pytest.mark.gpu
@pytest.mark.parametrize("dim", [2, 3])
def test_restricted_inference_adds_the_blocks_dense_inference_adds(mrfv, dim):
    """In the adaptation the convolutions cover only the tiles whose logits can add
    a block; the trees and states must equal those of dense inference over every
    position, and the net must add blocks the rule without safety zone (all
    logits negative) does not."""
    if dim == 2:
        kw = dict(dim=2, precision="fp32", levels=8, base_blocks=(1, 1, 1), adapt=True, eps=1e-3)
        ic, params = mi.IC_QUADRANTS, mi.quadrant_params(4)
    else:
        kw = dict(dim=3, precision="fp32", levels=4, base_blocks=(1, 1, 1), lo=(-1, -1, -1), hi=(1, 1, 1),
                  adapt=True, eps=1e-3)
        ic, params = mi.IC_ELLIPSOID, [-0.4, 0.3, 0.2, 0.12, 0.1, 0.15, 1.0, 2.0, 1.0, 1.0]
    w = random_weights(11)
    w[-1] = 0.4                      # output bias: the net proposes blocks
    control = np.zeros(len(w), np.float32)
    control[-1] = -1.0               # every logit negative: the MR rule without safety zone
    runs = {}
    for name, dense, weights in (("restricted", False, w), ("dense", True, w), ("control", False, control)):
        s = mrfv.Solver(proposer=True, proposer_dense=dense, **kw)
        s.init_state(ic, params)
        s.proposer_set_weights(weights)
        # one stage kernel for every run: the automatic choice follows the leaf count,
        # which the profiled (eager) run reads every step and a captured graph keeps
        # from its capture, and single-precision kernels differ in the last bit
        s.set_launch_shape(stage_kernel=1)
        if name == "restricted":
            s.profile_enable(True)
        for _ in range(4):
            s.step(0.0)
        runs[name] = s
    a, b, c = runs["restricted"], runs["dense"], runs["control"]
    for l in range(a.levels):
        assert np.array_equal(a.get_tree(l), b.get_tree(l)), l
        ga, gb = a.download_level(l)[0], b.download_level(l)[0]
        assert np.array_equal(np.isnan(ga), np.isnan(gb))
        m = ~np.isnan(ga)
        assert np.array_equal(ga[m], gb[m])
    assert sum(int(a.get_tree(l).sum()) for l in range(a.levels)) > sum(int(c.get_tree(l).sum())
                                                                          for l in range(c.levels))
    # the flagged tiles' positions at most (every tile: all positions rounded up to whole tiles)
    p = a.profile_read()
    tiles = (a.positions + 127) // 128
    whole = 2.0 * tiles * 128 * (16 * 81 + 16 * 432 + 432) * p["prop_launches"] / 3
    assert 0 < p["prop_flops"] <= whole


@pytest.mark.gpu
def test_proposer_training_and_deployment(mrfv):
    """Snapshots from the method itself (features at t, MR flags at t + dt), a few
    Adam steps on the GPU, then adaptation with the proposer: the loss falls and
    the run stays conservative and graded."""
    kw = dict(dim=2, precision="fp32", levels=5, base_blocks=(2, 2, 1), adapt=True, eps=1e-3, bc=1)
    s = mrfv.Solver(**kw)
    s.init_state(mi.IC_QUADRANTS, mi.quadrant_params(2))
    feats, targets = [], []
    for _ in range(6):
        s.analyse(1e-3)
        f = s.proposer_features()
        s.step(0.0)
        s.analyse(1e-3)
        t = np.concatenate([s.get_flags(l)[0].ravel() for l in range(s.levels)])
        feats.append(f)
        targets.append(t)
    s.proposer_set_weights(random_weights(7))
    l0 = s.proposer_train(np.stack(feats), np.stack(targets), steps=1, lr=1e-3)
    l1 = s.proposer_train(np.stack(feats), np.stack(targets), steps=40, lr=1e-2)
    assert l1 < l0
    w = s.proposer_get_weights()
    assert np.all(np.isfinite(w))
    # deploy
    p = mrfv.Solver(proposer=True, **kw)
    p.init_state(mi.IC_QUADRANTS, mi.quadrant_params(2))
    p.proposer_set_weights(w)
    T0 = p.totals()
    for _ in range(5):
        p.step(0.0)
    T1 = p.totals()
    assert np.all(np.abs(T1 - T0) <= 1e-5 * np.abs(T0).max())
    st = p.stats()
    assert st["total_leaves"] > 0
