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
    assert set(out["opts"]) == set(small)
    assert autotune.lookup(out["key"], str(tmp_path / "t.json")) == out["opts"]
