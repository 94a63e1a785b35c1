"""Inputs at the edges of what the library takes (Section 2.1's problem at its extremes):
the largest pattern (128 vertices) against closed forms and the oracle on both kernels, one
vertex more refused, empty and edgeless targets, and one batched call mixing patterns larger
than their target, empty patterns and ordinary pairs.  Counters are exact: matches, states,
nodes and the match hash."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_1705_09358_gb300 as sge
from brute import complete, cycle, edges_graph, path, random_graph, plant_connected
from gen.graphs import Graph
from gpu_common import counters, engine

pytestmark = pytest.mark.gpu

ALGOS = (0, 1, 2, 3)


def _empty(n: int, labels=None, directed: bool = False) -> Graph:
    vl = np.zeros(n, np.int32) if labels is None else np.asarray(labels, np.int32)
    return Graph(n, np.zeros(0, np.int32), np.zeros(0, np.int32), vl, None, directed)


def _unload(E, tids, pids):
    for p in pids:
        sge.sge_unload_pattern(E.h, p)
    for t in tids:
        sge.sge_unload_target(E.h, t)


def _check(E, t, p, matches=None, kernels=(0, 1, 2)):
    tid, pid = E.load_target(t), E.load_pattern(p)
    try:
        for algo in ALGOS:
            want = oracle.run(t, p, algo)
            if matches is not None:
                assert want["matches"] == matches, (algo, want["matches"], matches)
            for kern in kernels:
                got = E.count(tid, pid, algo=algo, kernel=kern)
                assert counters(got) == counters(want), (algo, kern, counters(got), counters(want))
    finally:
        _unload(E, [tid], [pid])


def test_largest_pattern_closed_forms():
    """128-vertex patterns: a path in a 200-cycle (a start vertex and a direction: 400), the
    128-cycle in itself (its 256 automorphisms), a path in a path two vertices longer (three
    placements, two directions: 6)."""
    E = engine()
    for t, p, m in [(cycle(200), path(128), 400), (cycle(128), cycle(128), 256), (path(130), path(128), 6)]:
        assert p.n == 128
        _check(E, t, p, matches=m)


def _cycle_directed(n: int) -> Graph:
    return edges_graph(n, [(i, (i + 1) % n) for i in range(n)], directed=True)


def _path_directed(n: int) -> Graph:
    return edges_graph(n, [(i, i + 1) for i in range(n - 1)], directed=True)


def test_largest_pattern_match_lists():
    """Full sorted match lists of a 128-vertex pattern (the match sink at its widest rows): the
    path in the 200-cycle (400 matches) on both kernels, and the directed path in the directed
    200-cycle (one direction: 200 matches)."""
    E = engine()
    for t, p, m, kernels in [(cycle(200), path(128), 400, (1, 2)),
                             (_cycle_directed(200), _path_directed(128), 200, (1,))]:
        tid, pid = E.load_target(t), E.load_pattern(p)
        try:
            for algo in (0, 3):
                want = oracle.run(t, p, algo, want_matches=True)
                assert want["matches"] == m and want["match_list"].shape == (m, 128)
                for kern in kernels:
                    got = E.enumerate(tid, pid, algo=algo, kernel=kern)
                    assert np.array_equal(got["match_list"].reshape(-1, 128), want["match_list"]), (algo, kern)
                    assert counters(got) == counters(want), (algo, kern)
        finally:
            _unload(E, [tid], [pid])


def test_pattern_of_129_vertices_is_refused():
    E = engine()
    with pytest.raises(sge.SgeError) as err:
        E.load_pattern(path(129))
    assert err.value.code == sge.SGE_ERR_ARG


def test_empty_and_edgeless_targets():
    """No target vertices at all, and vertices without edges: an edgeless 3-vertex pattern with
    labels (0, 0, 1) in six isolated vertices, three of each label, has 3 x 2 x 3 = 18 matches;
    any pattern edge has none."""
    E = engine()
    edgeless = _empty(6, [0, 0, 0, 1, 1, 1])
    _check(E, _empty(0), _empty(0), kernels=(0, 1))
    _check(E, _empty(0), complete(3), matches=0, kernels=(0, 1))
    _check(E, edgeless, _empty(3, [0, 0, 1]), matches=18)
    _check(E, edgeless, path(2), matches=0)


@pytest.mark.parametrize("directed", [False, True])
def test_batch_mixing_oversized_empty_and_ordinary_pairs(directed):
    """One batched call whose pairs include patterns with more vertices than their target, the
    empty pattern and ordinary connected patterns on random labelled targets, every variant:
    each row equals the oracle's counters for its own pair."""
    E = engine()
    rng = np.random.default_rng(4242 + directed)
    targets = [random_graph(rng, int(rng.integers(20, 120)), 0.08, 3, 2, directed) for _ in range(6)]
    patterns = [plant_connected(rng, targets[i % 6], int(rng.integers(3, 7))) for i in range(8)]
    if directed:
        patterns += [_cycle_directed(30), _path_directed(128), _empty(0, directed=True),
                     edges_graph(2, [(0, 1)], labels=[7, 7], directed=True)]
    else:
        patterns += [complete(30), path(128), _empty(0), edges_graph(2, [(0, 1)], labels=[7, 7])]
    tids = [E.load_target(t) for t in targets]
    pids = [E.load_pattern(p) for p in patterns]
    pairs = [(i, j) for i in range(len(targets)) for j in range(len(patterns))]
    try:
        for algo in ALGOS:
            want = [counters(oracle.run(targets[i], patterns[j], algo)) for i, j in pairs]
            rc, rows = E.count_batch([tids[i] for i, _ in pairs], [pids[j] for _, j in pairs], algo=algo)
            assert [counters(r) for r in rows] == want, algo
    finally:
        _unload(E, tids, pids)


@pytest.mark.parametrize("directed", [False, True])
def test_serving_at_the_limits(directed):
    """Served queries of every kind at once, on two targets (160 and 40 vertices): ordinary
    patterns, a 128-vertex pattern (larger than the small target), the empty pattern and an
    edgeless one, all four variants: each result equals the oracle's counters for its pair."""
    E = engine()
    rng = np.random.default_rng(777 + directed)
    targets = [random_graph(rng, 160, 0.05, 3, 2, directed), random_graph(rng, 40, 0.1, 3, 2, directed)]
    pats = [plant_connected(rng, targets[i % 2], int(rng.integers(3, 8))) for i in range(12)]
    if directed:
        pats += [_path_directed(128), _empty(0, directed=True), _empty(3, [0, 1, 2], True)]
    else:
        pats += [path(128), _empty(0), _empty(3, [0, 1, 2])]
    tids = [E.load_target(t) for t in targets]
    pids = [E.load_pattern(p) for p in pats]
    try:
        subs = []
        for rep in range(3):
            for i in range(len(targets)):
                for j, pid in enumerate(pids):
                    algo = (i + j + rep) % 4
                    subs.append((i, j, algo, E.serve_submit(tids[i], pid, algo=algo)))
        E.serve_drain()
        for i, j, algo, tk in subs:
            r = E.serve_poll(tk)
            assert r is not None and r["status"] == 0, (i, j, algo, r and r["status"])
            assert counters(r) == counters(oracle.run(targets[i], pats[j], algo)), (i, j, algo)
    finally:
        _unload(E, tids, pids)
