"""Target ingest on the device: the CSR built from the caller's edge list
(rows sorted, repeats merged) must give the oracle's results for every
shape of row the ingest kernels treat differently -- rows of at most 32
arcs (sorted across one warp), longer rows (ranked in shared memory) and
rows beyond the shared-memory limit (ranked in global memory) -- and bad
edge lists must be refused."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from brute import edges_graph, path, star, complete
from gen.graphs import Graph
from gpu_common import engine, counters

pytestmark = pytest.mark.gpu


def _count_both(t, p, algos=(0, 3)):
    E = engine()
    tid = E.load_target(t)
    pid = E.load_pattern(p)
    try:
        for algo in algos:
            want = oracle.run(t, p, algo, state_budget=50_000_000)
            assert not want["budget_exceeded"]
            for kern in (0, 1):
                got = E.count(tid, pid, algo=algo, kernel=kern)
                assert counters(got) == counters(want), (algo, kern)
    finally:
        from paper_1705_09358_gb300 import sge_unload_target, sge_unload_pattern
        sge_unload_target(E.h, tid)
        sge_unload_pattern(E.h, pid)


def _shuffled_with_repeats(g: Graph, rng, repeat_frac=0.5, flip=True) -> Graph:
    """The same graph given with edges in random order, some repeated and some reversed."""
    m = g.m
    extra = rng.choice(m, size=int(m * repeat_frac), replace=True) if m else np.zeros(0, np.int64)
    idx = np.concatenate([np.arange(m), extra])
    rng.shuffle(idx)
    src, dst = g.src[idx].copy(), g.dst[idx].copy()
    if flip and not g.directed:
        sw = rng.random(len(idx)) < 0.5
        src[sw], dst[sw] = dst[sw], src[sw]
    el = None if g.elabel is None else g.elabel[idx].copy()
    return Graph(g.n, src.astype(np.int32), dst.astype(np.int32), g.vlabel.copy(), el, g.directed)


@pytest.mark.parametrize("seed", range(6))
def test_repeated_and_reordered_edges(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(40, 90))
    # random graph with rows of mixed lengths, edge labels on half the cases
    p_edge = float(rng.uniform(0.05, 0.6))
    iu = np.triu_indices(n, 1)
    keep = rng.random(len(iu[0])) < p_edge
    src, dst = iu[0][keep].astype(np.int32), iu[1][keep].astype(np.int32)
    el = rng.integers(0, 3, size=len(src)).astype(np.int32) if seed % 2 else None
    t = Graph(n, src, dst, rng.integers(0, 2, size=n).astype(np.int32), el)
    t2 = _shuffled_with_repeats(t, rng)
    k = 3
    p = edges_graph(k, [(0, 1), (1, 2)], labels=[int(t.vlabel[0])] * k,
                    elabels=None if el is None else [0, 1])
    _count_both(t2, p)


@pytest.mark.parametrize("extra", [0, 6000])
def test_long_rows_in_shared_and_global_memory(extra):
    # hubs of degree 40 (shared-memory ranking), 5000 and 9000 (beyond the shared-memory
    # limit of 4096 keys), edges given in random order with repeats; a repeat left unmerged
    # (a row sorted wrongly) would change `states`.  With `extra` isolated vertices the
    # target passes the adjacency-bitset limit and the hubs get bitset rows instead.
    rng = np.random.default_rng(7)
    n = 1 + 40 + 1 + 5000 + 1 + 9000 + extra
    edges = []
    base = 0
    for deg in (40, 5000, 9000):
        hub = base
        edges += [(hub, hub + 1 + i) for i in range(deg)]
        edges += [(hub + 1 + i, hub + 2 + i) for i in range(0, deg - 1, 3)]   # some short rows too
        base += deg + 1
    src = np.array([a for a, b in edges], np.int32)
    dst = np.array([b for a, b in edges], np.int32)
    t = Graph(n, src, dst, np.zeros(n, np.int32))
    t2 = _shuffled_with_repeats(t, rng, repeat_frac=0.3)
    _count_both(t2, path(2), algos=(0, 3))    # every arc once per direction: 2 m


def test_directed_rows():
    rng = np.random.default_rng(3)
    n = 60
    a = rng.integers(0, n, 700)
    b = rng.integers(0, n, 700)
    keep = a != b
    t = Graph(n, a[keep].astype(np.int32), b[keep].astype(np.int32), rng.integers(0, 2, n).astype(np.int32),
              None, True)
    # repeated arcs merge; (a, b) and (b, a) stay distinct arcs
    t2 = _shuffled_with_repeats(t, rng, flip=False)
    p = edges_graph(3, [(0, 1), (1, 2)], labels=[0, 0, 0], directed=True)
    _count_both(t2, p, algos=(0, 1))


def test_bad_edge_lists_are_refused():
    from paper_1705_09358_gb300 import SgeError
    E = engine()
    z = np.zeros(4, np.int32)
    cases = [
        ([0, 1], [1, 1], None),            # self-loop
        ([0, 1], [1, 4], None),            # endpoint out of range
        ([0, 1], [-1, 2], None),           # negative endpoint
        ([0, 1, 1], [1, 2, 0], [1, 2, 3]),  # edge {0,1} twice with labels 1 and 3
    ]
    for s, d, el in cases:
        g = Graph(4, np.array(s, np.int32), np.array(d, np.int32), z.copy(),
                  None if el is None else np.array(el, np.int32))
        with pytest.raises(SgeError):
            E.load_target(g)
    # the same edge twice with the same label is merged, not refused
    g = Graph(4, np.array([0, 1, 1], np.int32), np.array([1, 0, 2], np.int32), z.copy(),
              np.array([5, 5, 1], np.int32))
    tid = E.load_target(g)
    from paper_1705_09358_gb300 import sge_unload_target
    sge_unload_target(E.h, tid)


def test_empty_and_edgeless_targets():
    _count_both(Graph(5, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(5, np.int32)),
                Graph(2, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(2, np.int32)))
    _count_both(complete(7), star(3))


def test_unloaded_blocks_are_reused_without_stale_data():
    # Unloaded graphs leave their device blocks in the context for later loads.  Load,
    # count and unload targets and patterns of changing sizes in turn, so that each load
    # takes blocks still holding an earlier graph's rows, adjacency bits and labels; every
    # count must still be the oracle's.
    rng = np.random.default_rng(11)
    for n, p_edge in [(300, 0.2), (260, 0.25), (150, 0.3), (300, 0.15), (290, 0.2)]:
        iu = np.triu_indices(n, 1)
        keep = rng.random(len(iu[0])) < p_edge
        t = Graph(n, iu[0][keep].astype(np.int32), iu[1][keep].astype(np.int32),
                  rng.integers(0, 2, size=n).astype(np.int32))
        k = int(rng.integers(3, 5))   # cycles of 3 or 4: a few million states for the oracle
        p = edges_graph(k, [(i, i + 1) for i in range(k - 1)] + [(0, k - 1)],
                        labels=[int(x) for x in rng.integers(0, 2, size=k)])
        _count_both(t, p)
