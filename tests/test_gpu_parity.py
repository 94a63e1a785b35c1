"""Parity of the CUDA path with the CPU oracle, through the C ABI.

Everything here compares exact integers: matches, states, nodes and the
64-bit match hash (and for enumeration the full sorted match list).  The
oracle runs live on the same seeded inputs, or its stored results are read
from tests/golden (written by tests/golden/make_expected.py, which calls
only the oracle).
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from brute import random_graph, plant, plant_connected, complete, cycle, star, path, edges_graph
from gen import configs
from gen.graphs import Graph
from gpu_common import engine, counters, golden, golden_counters, table_digest

pytestmark = pytest.mark.gpu

ALGOS = [0, 1, 2, 3]


def _case(seed, directed=False, n_lo=3, n_hi=9, kmax=6):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(n_lo, n_hi))
    k = int(rng.integers(1, min(n, kmax) + 1))
    t = random_graph(rng, n, float(rng.uniform(0.2, 0.9)), int(rng.integers(1, 4)), int(rng.integers(1, 3)), directed)
    if rng.random() < 0.7:
        p = plant(rng, t, k, float(rng.uniform(0.3, 1.0)))
    else:
        p = random_graph(rng, k, float(rng.uniform(0.0, 0.8)), int(rng.integers(1, 3)), int(rng.integers(1, 3)), directed)
        if t.elabel is None:
            p.elabel = None
    return t, p


ORACLE_BUDGET = 50_000_000   # a case larger than this is a test-construction error


def _check_pair(E, t, p, algos=ALGOS, kernels=(0, 1), want_list=False, **opts):
    tid = E.load_target(t)
    pid = E.load_pattern(p)
    try:
        for algo in algos:
            want = oracle.run(t, p, algo, want_matches=want_list, state_budget=ORACLE_BUDGET)
            assert not want["budget_exceeded"], "test instance too large for the oracle"
            for kern in kernels:
                if want_list:
                    got = E.enumerate(tid, pid, algo=algo, kernel=kern, **opts)
                    assert np.array_equal(got["match_list"].reshape(-1, p.n) if p.n else got["match_list"],
                                          want["match_list"]), (algo, kern)
                else:
                    got = E.count(tid, pid, algo=algo, kernel=kern, **opts)
                assert counters(got) == counters(want), (algo, kern, counters(got), counters(want))
    finally:
        from paper_1705_09358_gb300 import sge_unload_target, sge_unload_pattern
        sge_unload_target(E.h, tid)
        sge_unload_pattern(E.h, pid)


# ---------------------------------------------------------------- tiny cases
@pytest.mark.parametrize("seed", range(40))
def test_tiny_undirected(seed):
    t, p = _case(seed * 7)
    _check_pair(engine(), t, p, want_list=(seed % 4 == 0))


@pytest.mark.parametrize("seed", range(20))
def test_tiny_directed(seed):
    t, p = _case(seed * 7 + 1000, directed=True)
    _check_pair(engine(), t, p, kernels=(0,))


def test_closed_forms():
    E = engine()
    for t, p in [(complete(9), complete(5)), (cycle(12), cycle(12)), (star(9), star(4)), (cycle(11), path(6))]:
        _check_pair(E, t, p)


def test_edge_cases():
    E = engine()
    empty = Graph(0, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32))
    _check_pair(E, complete(5), empty)
    _check_pair(E, complete(5), complete(6))
    p = complete(3)
    p.vlabel[:] = 9                       # label absent from the target
    _check_pair(E, complete(6), p)
    iso = Graph(4, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(4, np.int32))
    _check_pair(E, cycle(9), iso)         # every position unparented


# ------------------------------------------------- several tiles, ragged tail
@pytest.mark.parametrize("seed", range(12))
def test_medium_dense(seed):
    """Targets of 150-700 vertices (3-11 bitset words, ragged), dense planted patterns."""
    rng = np.random.default_rng(40000 + seed)
    n = int(rng.integers(150, 700))
    t = random_graph(rng, n, float(rng.uniform(0.03, 0.12)), int(rng.integers(2, 5)), 1)
    from gen.patterns import dense_walk_pattern
    from gen.rng import Stream
    p = dense_walk_pattern(t, int(rng.integers(5, 11)), Stream(int(rng.integers(1 << 40))))
    _check_pair(engine(), t, p)


@pytest.mark.parametrize("seed", range(8))
def test_medium_labelled_edges(seed):
    rng = np.random.default_rng(50000 + seed)
    n = int(rng.integers(60, 200))
    t = random_graph(rng, n, 0.08, 3, 3)
    p = plant_connected(rng, t, int(rng.integers(4, 8)))
    _check_pair(engine(), t, p, kernels=(0, 1))


@pytest.mark.parametrize("seed", range(6))
def test_medium_directed(seed):
    rng = np.random.default_rng(60000 + seed)
    n = int(rng.integers(40, 120))
    t = random_graph(rng, n, 0.08, 2, 2, directed=True)
    p = plant_connected(rng, t, int(rng.integers(3, 7)))
    _check_pair(engine(), t, p, kernels=(0,))


@pytest.mark.parametrize("seed", range(6))
def test_medium_directed_labelled_match_lists(seed):
    """Full sorted match lists on directed targets with edge labels (several bitset words, ragged
    tails), every variant."""
    rng = np.random.default_rng(61000 + seed)
    n = int(rng.integers(100, 330))
    t = random_graph(rng, n, 0.04, 2, 3, directed=True)
    p = plant_connected(rng, t, int(rng.integers(3, 7)))
    _check_pair(engine(), t, p, kernels=(0,), want_list=True)


@pytest.mark.parametrize("seed", range(6))
def test_medium_match_lists_both_kernels(seed):
    """Full sorted match lists on undirected vertex-labelled targets (several bitset words,
    ragged tails), the CSR and the bitset kernel, every variant."""
    rng = np.random.default_rng(62000 + seed)
    n = int(rng.integers(100, 330))
    t = random_graph(rng, n, 0.05, 3, 1)
    p = plant_connected(rng, t, int(rng.integers(3, 7)))
    _check_pair(engine(), t, p, kernels=(1, 2), want_list=True)


# ------------------------------------------------------------- workload 1
def test_er1000_full_match_list():
    w = configs.er1000()
    t, p = w.targets[0], w.patterns[0]
    g = golden("er1000")
    assert t.sha256() == g["target_sha256"] and p.sha256() == g["pattern_sha256"]
    E = engine()
    tid, pid = E.load_target(t), E.load_pattern(p)
    want = oracle.run(t, p, 0, want_matches=True)["match_list"]
    for algo in ALGOS:
        for kern in (1, 2):
            got = E.enumerate(tid, pid, algo=algo, kernel=kern)
            assert counters(got) == golden_counters(g["algos"][str(algo)]), (algo, kern)
            assert np.array_equal(got["match_list"], want), (algo, kern)


# ------------------------------------------------------------- workload 3
def test_cl10k_all_patterns():
    w = configs.cl10k()
    g = golden("cl10k")
    assert w.targets[0].sha256() == g["target_sha256"]
    E = engine()
    tid = E.load_target(w.targets[0])
    for ent, p in zip(g["patterns"], w.patterns):
        assert p.sha256() == ent["pattern_sha256"]
        pid = E.load_pattern(p)
        for algo in ALGOS:
            got = E.count(tid, pid, algo=algo)
            assert counters(got) == golden_counters(ent["algos"][str(algo)]), (ent["slot"], algo)


# --------------------------------------------- schedule independence
SCHEDULES = [dict(split_depth=1), dict(split_depth=3), dict(frames_per_warp=1), dict(frames_per_warp=64),
             dict(steal_granularity=1), dict(steal_granularity=64), dict(no_donation=1), dict(blocks_per_sm=1),
             dict(blocks_per_sm=2, frames_per_warp=2)]


def test_schedule_invariance_csr():
    """Counters are fixed by the search tree: every split depth, frame count,
    donation granularity and grid size must give the same four numbers."""
    w = configs.cl10k()
    E = engine()
    tid = E.load_target(w.targets[0])
    pid = E.load_pattern(w.patterns[4])
    base = counters(E.count(tid, pid, algo=3))
    for opts in SCHEDULES:
        assert counters(E.count(tid, pid, algo=3, **opts)) == base, opts


def test_schedule_invariance_bitset():
    w = configs.er2000()
    g = golden("er2000")["patterns"][1]
    E = engine()
    tid = E.load_target(w.targets[0])
    pid = E.load_pattern(w.patterns[1])
    want = golden_counters(g["algos"]["3"])
    for opts in SCHEDULES + [dict(kernel=1), dict(kernel=2)]:
        assert counters(E.count(tid, pid, algo=3, **opts)) == want, opts


def test_shards_sum_to_whole():
    w = configs.er1000()
    E = engine()
    tid, pid = E.load_target(w.targets[0]), E.load_pattern(w.patterns[0])
    for algo in (0, 3):
        whole = counters(E.count(tid, pid, algo=algo))
        for depth in (1, 2, 3):
            for count in (2, 3):
                parts = [counters(E.count(tid, pid, algo=algo, split_depth=depth, shard_index=s, shard_count=count))
                         for s in range(count)]
                tot = tuple(sum(x[i] for x in parts) % (1 << 64) for i in range(4))
                assert tot == whole, (algo, depth, count)
                want = [oracle.run(w.targets[0], w.patterns[0], algo, shard=(depth, s, count)) for s in range(count)]
                assert [counters(x) for x in want] == parts


# ------------------------------------------------------------ stop paths
def test_budget_and_timeout_return_status():
    import paper_1705_09358_gb300 as sge
    E = engine()
    t, p = complete(40), complete(8)
    tid, pid = E.load_target(t), E.load_pattern(p)
    r = E.count(tid, pid, check=False, state_budget=100000)
    assert r["rc"] == sge.SGE_ERR_BUDGET and r["states"] >= 100000
    r = E.count(tid, pid, check=False, time_limit_ms=50)
    assert r["rc"] == sge.SGE_ERR_TIMEOUT
    # the context stays usable
    small = E.load_pattern(complete(3))
    assert E.count(tid, small)["matches"] == 40 * 39 * 38
