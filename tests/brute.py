"""Brute force straight from the problem definition (Section 2.1, Eqs. 1-3).

Used only to pin the oracle on tiny inputs: every injection V_p -> V_t is
tried, and one is kept when every pattern edge maps onto a target edge with
the same edge label and every pattern vertex onto a target vertex with the
same label (non-induced: target edges between images of non-adjacent
pattern vertices are allowed).
"""
from __future__ import annotations

import itertools

import numpy as np

from gen.graphs import Graph

_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_MASK = (1 << 64) - 1


def arcs(g: Graph) -> dict:
    """(a, b) -> label for every arc; undirected edges give both arcs."""
    out = {}
    for e in range(g.m):
        a, b = int(g.src[e]), int(g.dst[e])
        lab = 0 if g.elabel is None else int(g.elabel[e])
        out[(a, b)] = lab
        if not g.directed:
            out[(b, a)] = lab
    return out


def brute_force(target: Graph, pattern: Graph) -> np.ndarray:
    """Sorted (lexicographic) array of all matches, row = image of vertex 0..k-1."""
    k, n = pattern.n, target.n
    if k == 0 or k > n:
        return np.zeros((0, k), dtype=np.int32)
    ta, pa = arcs(target), arcs(pattern)
    tl = [int(x) for x in target.vlabel]
    pl = [int(x) for x in pattern.vlabel]
    rows = []
    for f in itertools.permutations(range(n), k):
        if any(tl[f[u]] != pl[u] for u in range(k)):
            continue
        if all(ta.get((f[a], f[b])) == lab for (a, b), lab in pa.items()):
            rows.append(f)
    arr = np.array(rows, dtype=np.int32).reshape(-1, k)
    if arr.shape[0]:
        arr = arr[np.lexsort(arr.T[::-1])]
    return arr


def fmix64(z: int) -> int:
    z &= _MASK
    z = ((z ^ (z >> 30)) * _M1) & _MASK
    z = ((z ^ (z >> 27)) * _M2) & _MASK
    return z ^ (z >> 31)


def match_hash(f) -> int:
    s = 0
    for u, v in enumerate(f):
        s = (s + fmix64(((u << 32) | int(v)) + 0x9E3779B97F4A7C15)) & _MASK
    return fmix64(s)


def list_hash(rows) -> int:
    return sum(match_hash(r) for r in rows) & _MASK


def random_graph(rng: np.random.Generator, n: int, p: float, nlab: int, nelab: int,
                 directed: bool = False) -> Graph:
    src, dst = [], []
    for a in range(n):
        for b in range(n):
            if a == b or (not directed and b <= a):
                continue
            if rng.random() < p:
                src.append(a)
                dst.append(b)
    el = None
    if nelab > 1:
        el = rng.integers(0, nelab, len(src)).astype(np.int32)
    return Graph(n, np.array(src, dtype=np.int32), np.array(dst, dtype=np.int32),
                 rng.integers(0, nlab, n).astype(np.int32), el, directed)


def plant(rng: np.random.Generator, target: Graph, k: int, keep: float) -> Graph:
    """A pattern on k random target vertices keeping a random subset of the
    induced edges (so at least one match exists)."""
    verts = [int(x) for x in rng.permutation(target.n)[:k]]
    pos = {v: i for i, v in enumerate(verts)}
    src, dst, lab = [], [], []
    for e in range(target.m):
        a, b = int(target.src[e]), int(target.dst[e])
        if a in pos and b in pos and rng.random() < keep:
            src.append(pos[a])
            dst.append(pos[b])
            lab.append(0 if target.elabel is None else int(target.elabel[e]))
    el = None if target.elabel is None else np.array(lab, dtype=np.int32)
    return Graph(k, np.array(src, dtype=np.int32), np.array(dst, dtype=np.int32),
                 np.array([int(target.vlabel[v]) for v in verts], dtype=np.int32), el, target.directed)


def plant_connected(rng: np.random.Generator, target: Graph, k: int) -> Graph:
    """A pattern induced on k target vertices that are connected in the
    target's undirected view (grown from a random vertex), so the search is
    driven by adjacency rather than by whole-vertex-set candidate lists."""
    nb = {v: set() for v in range(target.n)}
    for a, b in zip(target.src.tolist(), target.dst.tolist()):
        nb[a].add(b)
        nb[b].add(a)
    for _ in range(100):
        start = int(rng.integers(target.n))
        verts, frontier = [start], sorted(nb[start])
        while len(verts) < k and frontier:
            x = frontier[int(rng.integers(len(frontier)))]
            verts.append(x)
            frontier = sorted(set(frontier).union(nb[x]).difference(verts))
        if len(verts) == k:
            break
    pos = {v: i for i, v in enumerate(verts)}
    src, dst, lab = [], [], []
    for e in range(target.m):
        a, b = int(target.src[e]), int(target.dst[e])
        if a in pos and b in pos:
            src.append(pos[a])
            dst.append(pos[b])
            lab.append(0 if target.elabel is None else int(target.elabel[e]))
    el = None if target.elabel is None else np.array(lab, dtype=np.int32)
    return Graph(len(verts), np.array(src, dtype=np.int32), np.array(dst, dtype=np.int32),
                 np.array([int(target.vlabel[v]) for v in verts], dtype=np.int32), el, target.directed)


def edges_graph(n: int, edges, labels=None, elabels=None, directed: bool = False) -> Graph:
    src = np.array([a for a, _ in edges], dtype=np.int32)
    dst = np.array([b for _, b in edges], dtype=np.int32)
    vl = np.zeros(n, dtype=np.int32) if labels is None else np.array(labels, dtype=np.int32)
    el = None if elabels is None else np.array(elabels, dtype=np.int32)
    return Graph(n, src, dst, vl, el, directed)


def complete(n: int) -> Graph:
    return edges_graph(n, [(a, b) for a in range(n) for b in range(a + 1, n)])


def cycle(n: int) -> Graph:
    return edges_graph(n, [(i, (i + 1) % n) for i in range(n)])


def path(n: int) -> Graph:
    return edges_graph(n, [(i, i + 1) for i in range(n - 1)])


def star(leaves: int) -> Graph:
    return edges_graph(leaves + 1, [(0, i) for i in range(1, leaves + 1)])


def petersen() -> Graph:
    outer = [(i, (i + 1) % 5) for i in range(5)]
    spokes = [(i, i + 5) for i in range(5)]
    inner = [(5 + i, 5 + (i + 2) % 5) for i in range(5)]
    return edges_graph(10, outer + spokes + inner)


def cube() -> Graph:
    return edges_graph(8, [(a, a ^ (1 << b)) for a in range(8) for b in range(3) if a < a ^ (1 << b)])
