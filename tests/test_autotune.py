"""The launch-shape autotuner's host logic: workload keys, the JSON cache and the
coordinate-descent sweep (on synthetic cost functions; the GPU sweep itself is in
tests/test_gpu_autotune.py)."""
import itertools
import json

import pytest

from paper_1603_05211_gb300 import autotune as at


def test_workload_key_is_stable_and_sensitive():
    base = dict(dim=2, precision="fp32", levels=8, base_blocks=(1, 1, 1), adapt=True, criterion="mr")
    k0 = at.workload_key(base, "GB300", 152)
    assert k0 == at.workload_key(dict(base, base_blocks=[1, 1, 1]), "GB300", 152)
    assert k0 == at.workload_key(dict(base, eps=5e-3, t_end=1.0), "GB300", 152)  # not in the key
    for change in (dict(dim=3), dict(levels=7), dict(precision="fp64"), dict(lts=True), dict(scheme="hancock")):
        assert at.workload_key(dict(base, **change), "GB300", 152) != k0
    assert at.workload_key(base, "GB300", 148) != k0
    assert json.loads(k0)["device"] == "GB300"


def test_cache_round_trip_merge_and_corruption(tmp_path):
    p = str(tmp_path / "sub" / "shapes.json")
    assert at.lookup("k1", p) is None
    e1 = {"shape": dict(at.DEFAULT_SHAPE, grid_ctas_per_sm=4), "ms_per_step": 0.15}
    e2 = {"shape": dict(at.DEFAULT_SHAPE, stage_kernel=2), "ms_per_step": 0.2}
    at.store("k1", e1, p)
    at.store("k2", e2, p)
    assert at.lookup("k1", p) == e1 and at.lookup("k2", p) == e2
    at.store("k1", e2, p)  # replace one, keep the other
    assert at.lookup("k1", p) == e2 and at.lookup("k2", p) == e2
    with open(p, "w") as fh:
        fh.write("{not json")
    assert at.lookup("k1", p) is None and at.load_cache(p) == {}
    with open(p, "w") as fh:
        json.dump({"k3": {"shape": {"grid_ctas_per_sm": 1}}}, fh)  # incomplete shape
    assert at.lookup("k3", p) is None


def test_cache_path_from_environment(monkeypatch, tmp_path):
    monkeypatch.setenv("MRFV_AUTOTUNE_CACHE", str(tmp_path / "x.json"))
    assert at.cache_path() == str(tmp_path / "x.json")
    assert at.cache_path(str(tmp_path / "y.json")) == str(tmp_path / "y.json")
    monkeypatch.delenv("MRFV_AUTOTUNE_CACHE")
    assert at.cache_path().endswith("launch_shapes.json")


def _all_shapes(space):
    names = list(space)
    for vals in itertools.product(*(space[n] for n in names)):
        yield dict(zip(names, vals))


def test_descent_finds_the_minimum_of_a_separable_cost():
    target = {"grid_ctas_per_sm": 4, "block_ctas_per_sm": 2, "fv_ctas_per_sm": 8, "stage_kernel": 3}
    calls = []

    def cost(shape):
        calls.append(shape)
        return 1.0 + sum((at.SPACE[k].index(shape[k]) - at.SPACE[k].index(target[k])) ** 2 for k in shape)

    best, ms, trials = at.coordinate_descent(cost)
    assert best == target and ms == 1.0
    assert trials[0][0] == at.DEFAULT_SHAPE  # starts from the library's defaults
    keys = [tuple(sorted(c.items())) for c in calls]
    assert len(keys) == len(set(keys))  # each shape measured once
    assert len(calls) < sum(1 for _ in _all_shapes(at.SPACE)) // 10  # far fewer than the full grid


def test_descent_never_returns_worse_than_the_defaults():
    # a non-separable cost with an interaction term: the result is a local minimum along every
    # axis and no worse than the defaults
    def cost(s):
        a, b = at.SPACE["grid_ctas_per_sm"].index(s["grid_ctas_per_sm"]), at.SPACE["fv_ctas_per_sm"].index(
            s["fv_ctas_per_sm"])
        return 5.0 + (a - 2) ** 2 + (b - 3) ** 2 - 1.5 * (a * b == 6) + 0.1 * s["stage_kernel"]

    best, ms, trials = at.coordinate_descent(cost, passes=3)
    assert ms <= cost(at.DEFAULT_SHAPE)
    for name, values in at.SPACE.items():
        for v in values:
            assert cost(dict(best, **{name: v})) >= ms
    assert ms == min(t[1] for t in trials)


def test_descent_respects_a_restricted_space():
    space = {"grid_ctas_per_sm": [0, 2], "block_ctas_per_sm": [0], "fv_ctas_per_sm": [0, 4], "stage_kernel": [0]}
    best, ms, trials = at.coordinate_descent(lambda s: 10 - s["grid_ctas_per_sm"] - s["fv_ctas_per_sm"], space=space)
    assert best == {"grid_ctas_per_sm": 2, "block_ctas_per_sm": 0, "fv_ctas_per_sm": 4, "stage_kernel": 0}
    assert ms == 4
    for sh, _ in trials:
        for k, v in sh.items():
            assert v in space[k]


def test_tuned_shape_uses_the_cache_without_measuring(monkeypatch, tmp_path):
    torch = pytest.importorskip("torch")
    p = str(tmp_path / "c.json")

    class Props:
        name, multi_processor_count = "FakeGPU", 7

    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda d: Props())
    cfg = dict(dim=2, levels=3)
    key = at.workload_key(cfg, "FakeGPU", 7)
    at.store(key, {"shape": dict(at.DEFAULT_SHAPE, block_ctas_per_sm=8), "ms_per_step": 1.0}, p)

    def make():
        raise AssertionError("a cached workload is not measured")

    r = at.tuned_shape(make, cfg, path=p)
    assert r["cached"] and r["shape"]["block_ctas_per_sm"] == 8
