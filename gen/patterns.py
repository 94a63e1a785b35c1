"""Pattern graphs sampled from a target, so that at least one match exists.

Two samplers:

* `random_walk_pattern` -- a plain random walk until k distinct vertices are
  visited; the pattern is the subgraph induced on them (every target edge
  among them is kept, with its labels).  On sparse targets this gives
  near-tree patterns, as in the molecule collection.
* `dense_walk_pattern` -- a connected vertex set grown one vertex at a time,
  drawing the next vertex from the boundary with probability proportional to
  (edges into the set)^beta.  This yields the "dense" pattern class of the
  interaction-network collections; plain walks there produce patterns with
  astronomically many embeddings.

Pattern vertex i is the i-th sampled target vertex, so the identity of the
sample order is one embedding.  This module holds no part of the enumeration
method.
"""
from __future__ import annotations

import numpy as np

from .graphs import Graph, neighbour_lists
from .rng import Stream


class _Adj:
    def __init__(self, g: Graph):
        self.indptr, self.nbr, self.eidx = neighbour_lists(g)

    def row(self, v: int):
        return self.nbr[self.indptr[v]:self.indptr[v + 1]]


def induced_pattern(g: Graph, verts: list[int]) -> Graph:
    """Subgraph of undirected `g` induced on `verts`, vertex i = verts[i]."""
    pos = {v: i for i, v in enumerate(verts)}
    sel_src, sel_dst, sel_lab = [], [], []
    for e in range(g.m):
        a, b = int(g.src[e]), int(g.dst[e])
        if a in pos and b in pos:
            sel_src.append(pos[a])
            sel_dst.append(pos[b])
            if g.elabel is not None:
                sel_lab.append(int(g.elabel[e]))
    vl = np.array([int(g.vlabel[v]) for v in verts], dtype=np.int32)
    el = np.array(sel_lab, dtype=np.int32) if g.elabel is not None else None
    return Graph(len(verts), np.array(sel_src, dtype=np.int32), np.array(sel_dst, dtype=np.int32),
                 vl, el, False, {"sampled_from": list(map(int, verts))})


def _induced_fast(g: Graph, adj: _Adj, verts: list[int]) -> Graph:
    pos = {v: i for i, v in enumerate(verts)}
    src, dst, lab = [], [], []
    for i, v in enumerate(verts):
        lo, hi = adj.indptr[v], adj.indptr[v + 1]
        for t in range(lo, hi):
            w = int(adj.nbr[t])
            j = pos.get(w)
            if j is not None and i < j:
                src.append(i)
                dst.append(j)
                if g.elabel is not None:
                    lab.append(int(g.elabel[adj.eidx[t]]))
    vl = np.array([int(g.vlabel[v]) for v in verts], dtype=np.int32)
    el = np.array(lab, dtype=np.int32) if g.elabel is not None else None
    return Graph(len(verts), np.array(src, dtype=np.int32), np.array(dst, dtype=np.int32),
                 vl, el, False, {"sampled_from": list(map(int, verts))})


def random_walk_pattern(g: Graph, k: int, stream: Stream, adj: _Adj | None = None,
                        max_restarts: int = 1000) -> Graph:
    adj = adj or _Adj(g)
    deg = np.diff(adj.indptr)
    starts = np.nonzero(deg > 0)[0]
    if k == 1:
        return _induced_fast(g, adj, [int(starts[stream.one_below(starts.shape[0])])])
    for _ in range(max_restarts):
        cur = int(starts[stream.one_below(starts.shape[0])])
        seen = [cur]
        seen_set = {cur}
        steps = 0
        while len(seen) < k and steps < 200 * k:
            row = adj.row(cur)
            cur = int(row[stream.one_below(row.shape[0])])
            if cur not in seen_set:
                seen_set.add(cur)
                seen.append(cur)
            steps += 1
        if len(seen) == k:
            return _induced_fast(g, adj, seen)
    raise RuntimeError("random walk could not reach k distinct vertices")


def dense_walk_pattern(g: Graph, k: int, stream: Stream, beta: int = 4, adj: _Adj | None = None,
                       max_restarts: int = 1000) -> Graph:
    adj = adj or _Adj(g)
    deg = np.diff(adj.indptr)
    starts = np.nonzero(deg > 0)[0]
    conn = np.zeros(g.n, dtype=np.int64)      # edges from each boundary vertex into the set
    in_set = np.zeros(g.n, dtype=bool)
    for _ in range(max_restarts):
        first = int(starts[stream.one_below(starts.shape[0])])
        chosen = [first]
        in_set[first] = True
        keys = np.zeros(0, dtype=np.int64)    # boundary vertices, ascending

        def add_boundary(x, keys):
            row = adj.row(x)
            row = row[~in_set[row]]
            fresh = row[conn[row] == 0]
            conn[row] += 1                    # rows hold no repeated neighbour
            # both ascending and disjoint (a fresh vertex is not yet on the boundary)
            return np.insert(keys, np.searchsorted(keys, fresh), fresh) if fresh.shape[0] else keys

        keys = add_boundary(first, keys)
        while len(chosen) < k and keys.shape[0]:
            cum = np.cumsum(conn[keys] ** beta)
            total = int(cum[-1])
            r = int(stream.u64(1)[0]) % total
            i = int(np.searchsorted(cum, r, side="right"))
            pick = int(keys[i])
            chosen.append(pick)
            in_set[pick] = True
            keys = np.delete(keys, i)
            conn[pick] = 0
            keys = add_boundary(pick, keys)
        conn[keys] = 0
        in_set[np.array(chosen, dtype=np.int64)] = False
        if len(chosen) == k:
            return _induced_fast(g, adj, chosen)
    raise RuntimeError("dense walk could not reach k vertices")
