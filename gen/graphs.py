"""Seeded synthetic graphs shaped like the paper's biochemical collections.

The paper evaluates on PDBSv1 (sparse molecule graphs, mean degree 3.06, 5-8
labels), PPIS32 and GRAEMLIN32 (dense interaction networks, mean degrees 27.4
and 55.4, 32 labels) -- Section 5, "Data collections" and its table of graph
collections.  Those collections are not available here; the generators below
produce graphs of the same shape (size, degree distribution, label skew) from a
seed.  This module holds no part of the enumeration method: it only builds
edge lists and labels.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import hashlib

import numpy as np

from .rng import Stream, quantise_cdf


@dataclass
class Graph:
    """A labelled graph as an edge list.

    Undirected graphs list each edge once; `src[i]`, `dst[i]` and
    `elabel[i]` describe edge i.  Vertex ids are 0..n-1.
    """

    n: int
    src: np.ndarray
    dst: np.ndarray
    vlabel: np.ndarray
    elabel: np.ndarray | None = None
    directed: bool = False
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.src.shape[0])

    def sha256(self) -> str:
        h = hashlib.sha256()
        h.update(np.int64(self.n).tobytes())
        h.update(np.int8(1 if self.directed else 0).tobytes())
        for a in (self.src, self.dst, self.vlabel):
            h.update(np.ascontiguousarray(a, dtype=np.int32).tobytes())
        if self.elabel is not None:
            h.update(np.ascontiguousarray(self.elabel, dtype=np.int32).tobytes())
        return h.hexdigest()


def neighbour_lists(g: Graph):
    """(indptr, nbr, edge_index) adjacency of an undirected edge list, rows sorted."""
    u = np.concatenate([g.src, g.dst]).astype(np.int64)
    v = np.concatenate([g.dst, g.src]).astype(np.int64)
    e = np.concatenate([np.arange(g.m), np.arange(g.m)]).astype(np.int64)
    order = np.lexsort((v, u))
    u, v, e = u[order], v[order], e[order]
    indptr = np.zeros(g.n + 1, dtype=np.int64)
    np.add.at(indptr, u + 1, 1)
    indptr = np.cumsum(indptr)
    return indptr, v, e


def _dedup_undirected(a: np.ndarray, b: np.ndarray, n: int):
    """Drop self-loops and repeated pairs, keeping first occurrence order."""
    lo = np.minimum(a, b).astype(np.int64)
    hi = np.maximum(a, b).astype(np.int64)
    keep = lo != hi
    lo, hi = lo[keep], hi[keep]
    key = lo * n + hi
    _, first = np.unique(key, return_index=True)
    first.sort()
    return lo[first], hi[first]


def erdos_renyi(n: int, p: float, stream: Stream) -> tuple[np.ndarray, np.ndarray]:
    """G(n, p): every pair i < j kept independently with probability p."""
    iu, ju = np.triu_indices(n, k=1)
    thr = np.uint64(int(p * float(1 << 32)))
    keep = stream.u32(iu.shape[0]).astype(np.uint64) < thr
    return iu[keep].astype(np.int32), ju[keep].astype(np.int32)


def power_law_weights(n: int, gamma: float, mean_degree: float) -> np.ndarray:
    """Expected degrees w_i proportional to (i + 1)^(-1/(gamma-1)), mean `mean_degree`.

    The largest weights are capped at sqrt(n * mean_degree) (the structural
    cut-off of a Chung-Lu graph) and the mean is restored after capping.
    Returned as integers on a 2**16 scale so that later steps are exact.
    """
    alpha = 1.0 / (gamma - 1.0)
    w = np.power(np.arange(1, n + 1, dtype=np.float64), -alpha)
    cap = np.sqrt(n * mean_degree)
    for _ in range(50):
        w = w * (mean_degree * n / w.sum())
        w = np.minimum(w, cap)
    w = w * (mean_degree * n / w.sum())
    return np.floor(w * 65536.0 + 0.5).astype(np.int64)


def chung_lu(n: int, gamma: float, mean_degree: float, stream: Stream):
    """Chung-Lu-type power-law graph by weighted endpoint sampling.

    Each edge picks both endpoints independently with probability
    proportional to the expected-degree weight; self-loops and repeats are
    dropped, and sampling continues until n * mean_degree / 2 distinct edges
    exist.  This is the edge-sampling form of the Chung-Lu model (the
    expected degree of a vertex is proportional to its weight).
    """
    w = power_law_weights(n, gamma, mean_degree)
    thr = quantise_cdf(w.astype(np.float64))
    target = int(round(n * mean_degree / 2.0))
    have_lo = np.zeros(0, dtype=np.int64)
    have_hi = np.zeros(0, dtype=np.int64)
    batch = target
    while have_lo.shape[0] < target:
        a = stream.choice_thresholds(thr, batch)
        b = stream.choice_thresholds(thr, batch)
        lo, hi = _dedup_undirected(np.concatenate([have_lo, a]), np.concatenate([have_hi, b]), n)
        have_lo, have_hi = lo, hi
        batch = max(1024, (target - have_lo.shape[0]) * 2)
    return have_lo[:target].astype(np.int32), have_hi[:target].astype(np.int32)


def molecule_tree(n: int, stream: Stream, max_degree: int = 4, closure_frac: float = 0.1):
    """Near-tree molecule-shaped graph.

    A random tree in which vertex i attaches to a uniformly drawn earlier
    vertex of degree below `max_degree`, plus ceil(closure_frac * n) ring
    closures between vertices at tree distance 4 or 5 that keep every
    degree at most `max_degree`.
    """
    deg = np.zeros(n, dtype=np.int64)
    adj: list[list[int]] = [[] for _ in range(n)]
    src, dst = [], []
    for i in range(1, n):
        open_ = np.nonzero(deg[:i] < max_degree)[0]
        j = int(open_[stream.one_below(open_.shape[0])])
        src.append(j)
        dst.append(i)
        deg[i] += 1
        deg[j] += 1
        adj[i].append(j)
        adj[j].append(i)
    want = int(np.ceil(closure_frac * n))
    made = 0
    tries = 0
    edges = set(zip(src, dst))
    while made < want and tries < 50 * want:
        tries += 1
        a = stream.one_below(n)
        if deg[a] >= max_degree:
            continue
        # tree distances from a up to 5, breadth first
        dist = {a: 0}
        frontier = [a]
        for d in range(1, 6):
            nxt = []
            for x in frontier:
                for y in adj[x]:
                    if y not in dist:
                        dist[y] = d
                        nxt.append(y)
            frontier = nxt
        far = sorted(v for v, d in dist.items() if d in (4, 5) and deg[v] < max_degree)
        if not far:
            continue
        b = far[stream.one_below(len(far))]
        key = (min(a, b), max(a, b))
        if key in edges:
            continue
        edges.add(key)
        src.append(key[0])
        dst.append(key[1])
        deg[a] += 1
        deg[b] += 1
        made += 1
    return np.array(src, dtype=np.int32), np.array(dst, dtype=np.int32)


def uniform_labels(n: int, count: int, stream: Stream) -> np.ndarray:
    return stream.below(count, n).astype(np.int32)


def zipf_labels(n: int, count: int, s: float, stream: Stream) -> np.ndarray:
    """Label r (0-based) drawn with probability proportional to (r + 1)^(-s)."""
    w = np.power(np.arange(1, count + 1, dtype=np.float64), -s)
    return stream.choice_thresholds(quantise_cdf(w), n).astype(np.int32)


def categorical_labels(n: int, probs, stream: Stream, offset: int = 0) -> np.ndarray:
    return (stream.choice_thresholds(quantise_cdf(probs), n) + offset).astype(np.int32)


def molecule_label_probs() -> list[float]:
    """12 vertex labels: 0.60, 0.15, 0.15, and 0.10 spread geometrically over 9."""
    tail = np.power(0.5, np.arange(9, dtype=np.float64))
    tail = 0.10 * tail / tail.sum()
    return [0.60, 0.15, 0.15] + [float(x) for x in tail]
