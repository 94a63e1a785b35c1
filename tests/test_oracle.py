"""Pins of the CPU oracle against things other than itself.

* brute force over all injections (the problem definition, Section 2.1);
* closed-form counts (complete graphs, cycles, stars, paths, isolated
  vertices) and automorphism-group orders of named graphs;
* the paper's worked forward-checking example (Section 4.2);
* the arc-consistency / forward-checking fixpoint recomputed under another
  schedule, with the soundness of every removal checked against the matches;
* per-depth node and state counts recomputed by brute force over prefixes
  of the ordering;
* hand-derived orderings for each tie-break of GreatestConstraintFirst.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np
import pytest

import oracle
from brute import (brute_force, list_hash, random_graph, plant, edges_graph, complete, cycle, path,
                   star, petersen, cube, arcs)
from gen.graphs import Graph

HERE = os.path.dirname(os.path.abspath(__file__))
ALGOS = [0, 1, 2, 3]


def _perm(n, k):
    return math.factorial(n) // math.factorial(n - k)


# ------------------------------------------------------------ brute force
def _random_case(seed: int, directed: bool = False):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 9))
    k = int(rng.integers(1, min(n, 6) + 1))
    t = random_graph(rng, n, float(rng.uniform(0.2, 0.9)), int(rng.integers(1, 4)),
                     int(rng.integers(1, 3)), directed)
    if rng.random() < 0.7:
        p = plant(rng, t, k, float(rng.uniform(0.3, 1.0)))
    else:
        p = random_graph(rng, k, float(rng.uniform(0.0, 0.8)), int(rng.integers(1, 3)),
                         int(rng.integers(1, 3)), directed)
        if t.elabel is None:
            p.elabel = None
    return t, p


@pytest.mark.parametrize("seed", range(80))
@pytest.mark.parametrize("directed", [False, True])
def test_brute_force_all_variants(seed, directed):
    t, p = _random_case(seed * 7 + (1000 if directed else 0), directed)
    want = brute_force(t, p)
    for algo in ALGOS:
        r = oracle.run(t, p, algo, want_matches=True)
        assert r["matches"] == want.shape[0], (algo, r["matches"], want.shape[0])
        assert np.array_equal(r["match_list"], want), algo
        assert r["hash"] == list_hash(want), algo


# ----------------------------------------------------------- closed forms
@pytest.mark.parametrize("n,k", [(5, 3), (6, 4), (7, 7), (9, 5), (12, 3)])
def test_complete_in_complete(n, k):
    r = oracle.run(complete(n), complete(k), 0)
    assert r["matches"] == _perm(n, k)


@pytest.mark.parametrize("k", [3, 4, 7, 12, 128])
def test_cycle_in_itself(k):
    for algo in ALGOS:
        assert oracle.run(cycle(k), cycle(k), algo)["matches"] == 2 * k


@pytest.mark.parametrize("n,k", [(5, 2), (6, 3), (8, 5), (9, 9), (4, 1)])
def test_star_in_star(n, k):
    want = _perm(n, k) if k >= 2 else 2 * n
    for algo in ALGOS:
        assert oracle.run(star(n), star(k), algo)["matches"] == want


@pytest.mark.parametrize("n,k", [(5, 2), (6, 4), (9, 9), (11, 6), (200, 128)])
def test_path_in_cycle(n, k):
    for algo in ALGOS:
        assert oracle.run(cycle(n), path(k), algo)["matches"] == 2 * n


@pytest.mark.parametrize("n,k", [(5, 2), (10, 4), (7, 7), (130, 128)])
def test_path_in_path(n, k):
    # a placement of the k-path on the n-path (n - k + 1) times two directions
    for algo in ALGOS:
        assert oracle.run(path(n), path(k), algo)["matches"] == 2 * (n - k + 1)


@pytest.mark.parametrize("n,k", [(6, 2), (9, 4), (7, 7), (200, 128)])
def test_directed_path_in_directed_cycle(n, k):
    # one direction only: a start vertex each
    c = edges_graph(n, [(i, (i + 1) % n) for i in range(n)], directed=True)
    pk = edges_graph(k, [(i, i + 1) for i in range(k - 1)], directed=True)
    for algo in ALGOS:
        assert oracle.run(c, pk, algo)["matches"] == n


@pytest.mark.parametrize("tl,pl", [([0, 0, 0, 1, 1, 1], [0, 0, 1]), ([0, 1, 2, 2, 2], [2, 2, 1]), ([0, 0], [1])])
def test_labelled_isolated_vertices(tl, pl):
    # edgeless graphs: each label's pattern vertices go injectively to that label's target vertices
    t = Graph(len(tl), np.zeros(0, np.int32), np.zeros(0, np.int32), np.array(tl, np.int32))
    p = Graph(len(pl), np.zeros(0, np.int32), np.zeros(0, np.int32), np.array(pl, np.int32))
    want = 1
    for lab in set(pl):
        a, b = tl.count(lab), pl.count(lab)
        want *= _perm(a, b) if b <= a else 0
    for algo in ALGOS:
        assert oracle.run(t, p, algo)["matches"] == want


@pytest.mark.parametrize("n,k", [(6, 3), (7, 2), (5, 5)])
def test_isolated_vertices(n, k):
    iso = Graph(k, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(k, np.int32))
    for t in (complete(n), cycle(n)):
        for algo in ALGOS:
            assert oracle.run(t, iso, algo)["matches"] == _perm(n, k)


@pytest.mark.parametrize("g,aut", [(petersen(), 120), (cube(), 48), (cycle(9), 18), (complete(6), 720)])
def test_automorphism_orders(g, aut):
    for algo in ALGOS:
        assert oracle.run(g, g, algo)["matches"] == aut


@pytest.mark.parametrize("seed", range(20))
def test_count_divisible_by_automorphisms(seed):
    rng = np.random.default_rng(5000 + seed)
    t = random_graph(rng, 14, 0.35, 2, 1)
    p = plant(rng, t, 5, 1.0)
    p.vlabel[:] = 0
    t.vlabel[:] = 0
    aut = oracle.run(p, p, 0)["matches"]
    cnt = oracle.run(t, p, 0)["matches"]
    assert aut >= 1 and cnt % aut == 0


# ------------------------------------------------- forward checking (paper)
def test_forward_checking_paper_example():
    with open(os.path.join(HERE, "golden", "fc_example.json")) as f:
        ex = json.load(f)
    nt = ex["n_targets"]
    dom = np.zeros((len(ex["initial"]), nt), dtype=np.uint8)
    for v, vals in enumerate(ex["initial"]):
        dom[v, vals] = 1
    out = oracle.forward_check(dom)
    got = [sorted(np.nonzero(row)[0].tolist()) for row in out]
    assert got == ex["result"]


# --------------------------------------------------- domains under AC / FC
def _supported(t: Graph, p: Graph, D, v, x, ta, pa) -> bool:
    for (a, b), lab in pa.items():
        if a == v:   # pattern arc v -> b needs a target arc x -> y, y in D(b)
            if not any(ta.get((x, y)) == lab and D[b][y] for y in range(t.n)):
                return False
        if p.directed and b == v:  # pattern arc a -> v needs a target arc y -> x
            if not any(ta.get((y, x)) == lab and D[a][y] for y in range(t.n)):
                return False
    return True


def _jacobi_domains(t: Graph, p: Graph, algo: int):
    """Greatest AC (and FC) fixpoint, removing everything unsupported at once."""
    ta, pa = arcs(t), arcs(p)
    tdeg_o = np.zeros(t.n, int); tdeg_i = np.zeros(t.n, int)
    pdeg_o = np.zeros(p.n, int); pdeg_i = np.zeros(p.n, int)
    for (a, b) in ta:
        tdeg_o[a] += 1; tdeg_i[b] += 1
    for (a, b) in pa:
        pdeg_o[a] += 1; pdeg_i[b] += 1
    D = [[int(t.vlabel[x] == p.vlabel[v] and tdeg_o[x] >= pdeg_o[v] and tdeg_i[x] >= pdeg_i[v])
          for x in range(t.n)] for v in range(p.n)]
    while True:
        rem = [(v, x) for v in range(p.n) for x in range(t.n)
               if D[v][x] and not _supported(t, p, D, v, x, ta, pa)]
        if algo == 3:
            for u in range(p.n):
                if sum(D[u]) == 1:
                    x = D[u].index(1)
                    rem += [(v, x) for v in range(p.n) if v != u and D[v][x]]
        if not rem:
            return np.array(D, dtype=np.uint8)
        for v, x in rem:
            D[v][x] = 0
        if any(sum(row) == 0 for row in D):
            return np.array(D, dtype=np.uint8)


@pytest.mark.parametrize("seed", range(40))
def test_domains_fixpoint_and_soundness(seed):
    t, p = _random_case(3000 + seed, directed=bool(seed % 4 == 3))
    matches = brute_force(t, p)
    for algo in (1, 3):
        got = oracle.domains(t, p, algo)
        want = _jacobi_domains(t, p, algo)
        if (got.sum(axis=1) > 0).all() and (want.sum(axis=1) > 0).all():
            assert np.array_equal(got, want), algo
        else:
            assert matches.shape[0] == 0
        for row in matches:           # no value used by a match is ever removed
            for v, x in enumerate(row):
                assert got[v, x] == 1


# ----------------------------------------------- per-depth counts by brute force
def _prefix_counts(t: Graph, p: Graph, algo: int, mu, par, dom):
    """(nodes per position, states per position) from prefix injections."""
    import itertools
    ta, pa = arcs(t), arcs(p)
    k, n = p.n, t.n
    out_deg = np.zeros(n, int); in_deg = np.zeros(n, int)
    for (a, b) in ta:
        out_deg[a] += 1; in_deg[b] += 1
    pout = np.zeros(k, int); pin = np.zeros(k, int)
    for (a, b) in pa:
        pout[a] += 1; pin[b] += 1
    out_rows = {x: [y for (a, y) in ta if a == x] for x in range(n)}
    in_rows = {x: [a for (a, y) in ta if y == x] for x in range(n)}

    def ok_prefix(g):
        d = len(g)
        for j in range(d):
            u, x = int(mu[j]), g[j]
            if t.vlabel[x] != p.vlabel[u] or out_deg[x] < pout[u] or in_deg[x] < pin[u]:
                return False
            if dom is not None and not dom[u][x]:
                return False
        for a in range(d):
            for b in range(d):
                lab = pa.get((int(mu[a]), int(mu[b])))
                if lab is not None and ta.get((g[a], g[b])) != lab:
                    return False
        return True

    def cand_count(g, i):
        if par[i] < 0:
            return n if dom is None else int(dom[int(mu[i])].sum())
        a = g[par[i]]
        if (int(mu[par[i]]), int(mu[i])) in pa or not t.directed:
            return len(out_rows[a])
        return len(in_rows[a])

    nodes, states = [], []
    prev = [()]
    for d in range(k):
        states.append(sum(cand_count(g, d) for g in prev))
        cur = [g for g in itertools.permutations(range(n), d + 1) if ok_prefix(g)]
        nodes.append(len(cur))
        prev = cur
    return nodes, states


@pytest.mark.parametrize("seed", range(30))
def test_level_counts_by_prefix_brute_force(seed):
    t, p = _random_case(7000 + seed, directed=bool(seed % 3 == 2))
    if p.n > 5:
        pytest.skip("prefix brute force kept to k <= 5")
    for algo in ALGOS:
        r = oracle.run(t, p, algo, want_levels=True)
        dom = None
        if algo != 0:
            dom = oracle.domains(t, p, algo)
            if (dom.sum(axis=1) == 0).any():
                assert r["states"] == 0 and r["nodes"] == 0 and r["matches"] == 0
                continue
        nodes, states = _prefix_counts(t, p, algo, r["order"], r["parent"], dom)
        assert list(r["level_nodes"]) == nodes, algo
        assert list(r["level_states"]) == states, algo
        assert r["nodes"] == sum(nodes) and r["states"] == sum(states)


# ------------------------------------------------------ ordering tie-breaks
def test_ordering_wn_decides():
    # Vertex 0 has the highest degree.  Then 1, 2, 3, 5 each have one
    # neighbour in mu; only 1 and 5 reach mu through a vertex outside it
    # (w_n = 1), and 1 wins the degree tie with 5 by lower id; 2 and 3 have
    # the higher degree but w_n = 0.  5 then has two neighbours in mu.
    g = edges_graph(10, [(0, 1), (0, 2), (0, 3), (0, 5), (1, 5), (2, 6), (2, 7), (3, 8), (3, 9)])
    mu, par = oracle.order(g, 0)
    assert mu.tolist() == [0, 1, 5, 2, 3, 6, 7, 8, 9, 4]
    assert par.tolist() == [-1, 0, 0, 0, 0, 3, 3, 4, 4, -1]


def test_ordering_degree_decides():
    # 1, 2, 3 all have (w_m, w_n) = (1, 1) after mu = [0]; 2 has the highest
    # degree.  Next 1 has two neighbours in mu, then 3 does.
    g = edges_graph(9, [(0, 1), (0, 2), (1, 2), (0, 3), (1, 3), (2, 4), (2, 5), (0, 6), (0, 7), (0, 8)])
    mu, par = oracle.order(g, 0)
    assert mu.tolist() == [0, 2, 1, 3, 4, 5, 6, 7, 8]
    assert par.tolist() == [-1, 0, 0, 0, 1, 1, 0, 0, 0]


def test_ordering_domain_size_tie_break():
    # Leaves 1, 2, 3 of a star tie on w_m, w_n and degree; SI takes the
    # smaller domain first, plain RI-DS the lower id (Section 4.1).
    g = star(3)
    sizes = np.array([5, 9, 4, 7], dtype=np.int64)
    assert oracle.order(g, 2, sizes)[0].tolist() == [0, 2, 3, 1]
    assert oracle.order(g, 1, sizes)[0].tolist() == [0, 1, 2, 3]
    # first vertex: all degrees equal on a 4-cycle; SI takes the smallest domain
    sizes = np.array([5, 3, 3, 9], dtype=np.int64)
    assert oracle.order(cycle(4), 2, sizes)[0][0] == 1
    assert oracle.order(cycle(4), 1, sizes)[0][0] == 0


def test_ordering_singletons_first():
    sizes = np.array([3, 1, 5, 1], dtype=np.int64)
    mu, par = oracle.order(path(4), 1, sizes)
    assert mu.tolist() == [1, 3, 2, 0]
    assert par.tolist() == [-1, -1, 0, 0]


# ------------------------------------------------------------ invariants
def test_cross_variant_er1000():
    from gen import configs
    w = configs.er1000()
    res = [oracle.run(w.targets[0], w.patterns[0], a) for a in ALGOS]
    assert len({(r["matches"], r["hash"]) for r in res}) == 1
    assert res[0]["matches"] >= 1


@pytest.mark.parametrize("seed", range(10))
def test_shards_sum_to_whole(seed):
    rng = np.random.default_rng(9000 + seed)
    t = random_graph(rng, 30, 0.25, 2, 1)
    p = plant(rng, t, 5, 0.8)
    for algo in (0, 3):
        whole = oracle.run(t, p, algo)
        for depth in (1, 2, 3):
            for count in (2, 3):
                parts = [oracle.run(t, p, algo, shard=(depth, s, count)) for s in range(count)]
                for key in ("matches", "states", "nodes"):
                    assert sum(q[key] for q in parts) == whole[key], (key, depth, count)
                assert sum(q["hash"] for q in parts) % (1 << 64) == whole["hash"]


def test_edge_cases():
    t = complete(5)
    empty = Graph(0, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32))
    r = oracle.run(t, empty, 0)
    assert (r["matches"], r["states"], r["nodes"]) == (0, 0, 0)
    r = oracle.run(t, complete(6), 0)
    assert (r["matches"], r["states"], r["nodes"]) == (0, 0, 0)
    # a label absent from the target: no match, but the root candidates are still considered
    p = complete(2)
    p.vlabel[:] = 7
    r = oracle.run(t, p, 0)
    assert r["matches"] == 0 and r["states"] == 5 and r["nodes"] == 0
    # RI-DS sees the empty domain first and searches nothing
    r = oracle.run(t, p, 1)
    assert (r["matches"], r["states"], r["nodes"]) == (0, 0, 0)
    with pytest.raises(ValueError):
        oracle.run(edges_graph(3, [(0, 0)]), complete(2), 0)
    with pytest.raises(ValueError):
        oracle.run(edges_graph(3, [(0, 1), (1, 0)], elabels=[1, 2]), complete(2), 0)
    # a repeated edge with the same label is one edge
    a = oracle.run(edges_graph(3, [(0, 1), (1, 2), (1, 0)]), complete(2), 0)
    b = oracle.run(edges_graph(3, [(0, 1), (1, 2)]), complete(2), 0)
    assert a["matches"] == b["matches"] == 4 and a["states"] == b["states"]


def test_budget_stops_search():
    r = oracle.run(complete(9), complete(6), 0, state_budget=100)
    assert r["budget_exceeded"]
