"""The launch-shape autotuner on the GPU: a restricted sweep on a small adaptive
workload returns a shape of its space, caches it, and reuses the cache; a shape
changes the time of a step, never its result (trees bit-exact, FP64 state within
1e-12 of the default shape's)."""
import numpy as np
import pytest

import mrfv_inputs as mi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mrfv():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1603_05211_gb300 as m

    m.build()
    return m


def _make(m, precision="fp64"):
    def make():
        s = m.Solver(dim=2, precision=precision, levels=4, base_blocks=(2, 2, 1), adapt=True)
        s.init_state(mi.IC_QUADRANTS, mi.quadrant_params(2))
        return s
    return make


def test_restricted_sweep_and_cache(mrfv, tmp_path):
    from paper_1603_05211_gb300 import autotune as at

    space = {"grid_ctas_per_sm": [0, 2], "block_ctas_per_sm": [0, 8], "fv_ctas_per_sm": [0, 2],
             "stage_kernel": [0, 2]}
    r = at.tune(_make(mrfv, "fp32"), steps=4, warmup=2, passes=1, space=space)
    assert r["ms_per_step"] > 0 and r["ms_per_step"] <= r["default_ms_per_step"]
    for k, v in r["shape"].items():
        assert v in space[k]
    assert 1 < len(r["trials"]) <= 1 + sum(len(v) - 1 for v in space.values())
    p = str(tmp_path / "shapes.json")
    cfg = dict(dim=2, precision="fp32", levels=4, base_blocks=(2, 2, 1), adapt=True)
    t1 = at.tuned_shape(_make(mrfv, "fp32"), cfg, path=p, steps=3, warmup=2, passes=1, space=space)
    assert not t1["cached"]
    t2 = at.tuned_shape(_make(mrfv, "fp32"), cfg, path=p)
    assert t2["cached"] and t2["shape"] == t1["shape"]


@pytest.mark.parametrize("shape", [dict(grid_ctas_per_sm=1, block_ctas_per_sm=16, fv_ctas_per_sm=1, stage_kernel=2),
                                   dict(grid_ctas_per_sm=8, block_ctas_per_sm=2, fv_ctas_per_sm=8, stage_kernel=3)])
def test_a_shape_never_changes_the_result(mrfv, shape):
    a, b = _make(mrfv)(), _make(mrfv)()
    b.set_launch_shape(**shape)
    for _ in range(6):
        assert a.step(0.0) == b.step(0.0)
    for l in range(4):
        assert np.array_equal(a.get_tree(l), b.get_tree(l))
        x, y = a.download_level(l)[0], b.download_level(l)[0]
        m = ~np.isnan(x)
        assert np.array_equal(m, ~np.isnan(y))
        if m.any():
            assert np.abs(x[m] - y[m]).max() <= 1e-12 * np.abs(x[m]).max()
