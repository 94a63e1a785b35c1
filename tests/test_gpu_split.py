"""The breadth-first split under a frontier budget (sge_opts.frontier_kib).

Unsharded runs split in one pass per level: a frame's candidates are tested
and counted once, and its children are appended at reserved offsets.  A level
whose children do not fit the frontier is abandoned after it was counted: its
frames go to the search as counted ranges (or, on a pattern's last position,
as empty ranges), so the search must count from the next level on.  Whatever
level that happens at -- the roots, a middle level, a level where some pairs
are on their last position -- the counters stay those of the oracle."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from brute import plant, random_graph
from gen import configs
from gpu_common import counters, engine, golden, golden_counters

pytestmark = pytest.mark.gpu

BUDGET = -4
KIBS = (1, 2, 3, 5, 8, 21, 55, 144, 377, 987, 2584, 6765, 17711, 46368, 121393)


def _unload(E, tids=(), pids=()):
    from paper_1705_09358_gb300 import sge_unload_pattern, sge_unload_target
    for p in pids:
        sge_unload_pattern(E.h, p)
    for t in tids:
        sge_unload_target(E.h, t)


@pytest.mark.parametrize("algo", [0, 3])
def test_cl10k_batch_under_small_frontiers(algo):
    """The 10 deep patterns (32..64 vertices) batched: with the default frontier
    the split runs to the bottom; small frontiers stop it at every depth."""
    w = configs.cl10k()
    g = golden("cl10k")
    E = engine()
    tid = E.load_target(w.targets[0])
    pids = [E.load_pattern(p) for p in w.patterns]
    want = [golden_counters(ent["algos"][str(algo)]) for ent in g["patterns"]]
    try:
        rc, rows = E.count_batch([tid] * len(pids), pids, algo=algo, kernel=1)
        assert [counters(r) for r in rows] == want
        full_depth = int(rows[0]["split_depth"])
        depths = set()
        for kib in KIBS:
            rc, rows = E.count_batch([tid] * len(pids), pids, algo=algo, kernel=1, frontier_kib=kib)
            assert [counters(r) for r in rows] == want, kib
            depths.add(int(rows[0]["split_depth"]))
        assert min(depths) < full_depth and len(depths) >= 3, (depths, full_depth)
    finally:
        _unload(E, [tid], pids)


@pytest.mark.parametrize("directed", [False, True])
def test_mixed_pattern_sizes_under_small_frontiers(directed):
    """Pairs of 2..7 pattern vertices in one batch, so the abandoned level holds
    frames on their pattern's last position beside frames with children."""
    E = engine()
    rng = np.random.default_rng(1705 + directed)
    pairs = []
    for _ in range(32):
        n = int(rng.integers(6, 17))
        t = random_graph(rng, n, float(rng.uniform(0.3, 0.9)), int(rng.integers(1, 3)), 1, directed)
        p = plant(rng, t, int(rng.integers(2, min(n, 7) + 1)), float(rng.uniform(0.4, 1.0)))
        pairs.append((t, p))
    tids = [E.load_target(t) for t, _ in pairs]
    pids = [E.load_pattern(p) for _, p in pairs]
    try:
        for algo in (0, 3):
            want = [counters(oracle.run(t, p, algo)) for t, p in pairs]
            for kib in (1, 2, 3, 4, 6, 9):
                for kernel in ((1,) if directed else (1, 2)):   # (the bitset kernel is undirected only)
                    rc, rows = E.count_batch(tids, pids, algo=algo, kernel=kernel, frontier_kib=kib,
                                             split_depth=6)
                    assert [counters(r) for r in rows] == want, (algo, kib, kernel)
    finally:
        _unload(E, tids, pids)


def test_bitset_kernel_under_small_frontiers():
    w = configs.er2000()
    g = golden("er2000")
    E = engine()
    tid = E.load_target(w.targets[0])
    pids = [E.load_pattern(p) for p in w.patterns]
    want = [golden_counters(ent["algos"]["3"]) for ent in g["patterns"]]
    try:
        for kib in (1, 4, 16, 64):
            rc, rows = E.count_batch([tid] * len(pids), pids, algo=3, kernel=2, frontier_kib=kib)
            assert [counters(r) for r in rows] == want, kib
    finally:
        _unload(E, [tid], pids)


def test_sharded_split_under_small_frontiers():
    """Sharded runs keep the ordered two-pass split; a level that does not fit is
    not written at all, and the shards still sum to the whole."""
    w = configs.cl10k()
    g = golden("cl10k")
    E = engine()
    tid = E.load_target(w.targets[0])
    pids = [E.load_pattern(p) for p in w.patterns[:4]]
    want = np.array([golden_counters(ent["algos"]["3"]) for ent in g["patterns"][:4]], dtype=np.uint64)
    try:
        for kib in (2, 21):
            tot = np.zeros_like(want)
            for s in range(3):
                rc, rows = E.count_batch([tid] * len(pids), pids, algo=3, kernel=1, frontier_kib=kib,
                                         shard_index=s, shard_count=3)
                tot += np.array([counters(r) for r in rows], dtype=np.uint64)
            assert np.array_equal(tot, want), kib
    finally:
        _unload(E, [tid], pids)


def test_counted_frames_survive_a_checkpoint():
    """A state budget stops the search while it still holds frames of an abandoned
    split level; the checkpoint carries them and the resumed run finishes exactly."""
    w = configs.cl10k()
    g = golden("cl10k")
    E = engine()
    tid = E.load_target(w.targets[0])
    pids = [E.load_pattern(p) for p in w.patterns]
    want = [golden_counters(ent["algos"]["3"]) for ent in g["patterns"]]
    try:
        budget = max(1, sorted(x[1] for x in want)[len(want) // 2] // 2)
        for kib in (1, 8):
            rc, rows, blob = E.count_batch_ckpt([tid] * len(pids), pids, algo=3, kernel=1, frontier_kib=kib,
                                                state_budget=budget)
            calls = 0
            while blob is not None:
                rc, rows, blob = E.resume(blob, kernel=1, state_budget=budget)
                calls += 1
                assert calls <= 400
            assert [counters(r) for r in rows] == want, kib
    finally:
        _unload(E, [tid], pids)


def test_negative_frontier_is_an_argument_error():
    import paper_1705_09358_gb300 as sge
    from brute import complete
    E = engine()
    tid, pid = E.load_target(complete(5)), E.load_pattern(complete(3))
    try:
        assert E.count(tid, pid, check=False, frontier_kib=-1)["rc"] == sge.SGE_ERR_ARG
    finally:
        _unload(E, [tid], [pid])
