"""The schedule autotuner: coordinate descent, counter checks, cache."""
from __future__ import annotations

import pytest

from paper_1705_09358_gb300 import autotune


def test_descent_finds_the_grid_minimum():
    space = {"a": [1, 2, 3, 4], "b": [10, 20, 30]}
    cost = lambda p: (p["a"] - 3) ** 2 + (p["b"] - 10) ** 2 / 100.0
    point, best, table = autotune.coordinate_descent(lambda p: (cost(p), (1, 2, 3, 4)), space, rounds=3)
    assert point == {"a": 3, "b": 10} and best == cost(point)
    assert len(table) <= len(space["a"]) * len(space["b"])


def test_a_schedule_that_changes_counters_is_an_error():
    space = {"a": [1, 2]}
    with pytest.raises(ValueError):
        autotune.coordinate_descent(lambda p: (1.0, (p["a"], 0, 0, 0)), space)


def test_cache_roundtrip_and_keys(tmp_path):
    path = str(tmp_path / "tune.json")
    assert autotune.lookup("x", path) == {}
    autotune.save({"x": {"opts": {"frames_per_warp": 64}, "seconds": 0.1}}, path)
    assert autotune.lookup("x", path) == {"frames_per_warp": 64}
    assert autotune.workload_key(2, 2000, 24, 3) == "kernel2:n2048:k32:algo3"
    assert autotune.workload_key(1, 100000, 128, 0) == "kernel1:n131072:k128:algo0"


@pytest.mark.gpu
def test_tuning_a_gpu_workload_keeps_the_counters(tmp_path):
    from gen import configs
    from gpu_common import engine
    w = configs.cl10k()
    E = engine()
    tid = E.load_target(w.targets[0])
    pids = [E.load_pattern(p) for p in w.patterns]
    small = {"frames_per_warp": [16, 64], "steal_granularity": [2, 8], "donate_every_us": [500, 2000]}
    out = autotune.tune_batch(E, [tid] * len(pids), pids, algo=3, reps=1, path=str(tmp_path / "t.json"),
                              space=small)
    assert set(out["opts"]) <= set(small) and out["seconds"] <= out["default_seconds"]
    assert autotune.lookup(out["key"], str(tmp_path / "t.json")) == out["opts"]
    assert out["key"] == autotune.batch_key(3, 10_000, 64, len(pids))


def test_batch_keys_and_the_package_cache(tmp_path):
    assert autotune.batch_key(0, 500, 64, 200_000, labelled=True) == "algo0:n512:k64:pairs262144:und:elab"
    assert autotune.batch_key(3, 2000, 24, 5) == "algo3:n2048:k32:pairs16:und:plain"
    # a user cache entry wins over the shipped one; a missing user entry falls back to it
    shipped = autotune.load(autotune.PACKAGE_CACHE)
    for key, ent in shipped.items():
        assert set(ent["opts"]) <= autotune.SCHEDULE_KEYS, key
        assert autotune.lookup(key, str(tmp_path / "none.json"), package=True) == ent["opts"]
    user = str(tmp_path / "user.json")
    autotune.save({"algo0:n2:k2:pairs1:und:plain": {"opts": {"split_depth": 2}}}, user)
    assert autotune.lookup("algo0:n2:k2:pairs1:und:plain", user, package=True) == {"split_depth": 2}
    assert autotune.lookup("algo9:none", user, package=True) == {}


@pytest.mark.gpu
def test_count_batch_applies_the_tuned_schedule_without_changing_counters(tmp_path):
    import numpy as np
    from gen import configs
    from gpu_common import engine
    w = configs.cl10k()
    E = engine()
    tid = E.load_target(w.targets[0])
    pids = [E.load_pattern(p) for p in w.patterns]
    key = E.batch_key([tid] * len(pids), pids, 3)
    old = E.autotune_cache
    E.autotune_cache = str(tmp_path / "user.json")
    E._tuned.clear()
    try:
        autotune.save({key: {"opts": {"split_depth": 2, "frames_per_warp": 4}}}, E.autotune_cache)
        assert E.tuned_schedule([tid] * len(pids), pids, 3) == {"split_depth": 2, "frames_per_warp": 4}
        rc, tuned = E.count_batch([tid] * len(pids), pids, algo=3)
        rc, plain = E.count_batch([tid] * len(pids), pids, algo=3, tuned=False)
        assert int(tuned["split_depth"][0]) == 2
        for k in ("matches", "states", "nodes", "hash"):
            assert np.array_equal(tuned[k], plain[k]), k
    finally:
        E.autotune_cache = old
        E._tuned.clear()
