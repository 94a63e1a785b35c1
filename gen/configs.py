"""The five synthetic workloads, each fixed by a master seed.

1. ``er1000``: plain RI, one query.  Target G(1000, p) with mean degree 8,
   vertex labels uniform over 8 values, no edge labels; one 8-vertex pattern
   from a random walk on the target.
2. ``er2000``: RI-DS on a dense target.  G(2000, 0.05) (about 100k edges),
   4 uniform labels; 5 dense-walk patterns of 16, 18, 20, 22 and 24 vertices.
3. ``cl10k``: interaction-network shape.  Chung-Lu power-law target, 10,000
   vertices, exponent 2.3, mean degree 20, 32 labels Zipf(1.2); 10 dense-walk
   patterns of 32, 48 and 64 vertices with at least 100 edges.
4. ``mol200``: batched molecule shape.  200 near-tree targets of 20-500
   vertices (max degree 4, about 1.1 edges per vertex), 12 skewed vertex
   labels, edge labels in {1, 2, 3}; 1000 random-walk patterns of 4-64
   vertices; all 200,000 (pattern, target) pairs.
5. ``cl100k``: serving.  Chung-Lu target, 100,000 vertices, exponent 2.2,
   mean degree 16, 64 labels Zipf(1.1); a Poisson stream of queries of 8-128
   vertices (log-uniform sizes) sampled from the target.

Patterns of workloads 2, 3 and 5 are drawn from candidate seeds; a pattern
whose exhaustive search is too large for the time limit is skipped in favour
of the next candidate (the paper counts instances over its 180 s limit as
unsolved, Section 5).  The accepted candidate index of each slot is read
from ``admitted.json`` beside this file; a slot missing there uses
candidate 0.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import json
import os

import numpy as np

from .graphs import (Graph, chung_lu, erdos_renyi, molecule_tree, uniform_labels, zipf_labels,
                     categorical_labels, molecule_label_probs)
from .patterns import _Adj, dense_walk_pattern, random_walk_pattern
from .rng import Stream, sub_seed, quantise_cdf

MASTER = 20170526
ALGO_RI, ALGO_RIDS, ALGO_RIDS_SI, ALGO_RIDS_SI_FC = 0, 1, 2, 3

_HERE = os.path.dirname(os.path.abspath(__file__))
ADMITTED_PATH = os.path.join(_HERE, "admitted.json")


def load_admitted() -> dict:
    if os.path.exists(ADMITTED_PATH):
        with open(ADMITTED_PATH) as f:
            return json.load(f)
    return {}


@dataclass
class Workload:
    name: str
    targets: list
    patterns: list
    pairs: np.ndarray          # (P, 2) int32: (target index, pattern index)
    algo: int
    meta: dict = field(default_factory=dict)


def master_seed(index: int) -> int:
    return MASTER + index


def log_uniform_sizes(lo: int, hi: int, count: int, stream: Stream) -> np.ndarray:
    """Integer sizes in [lo, hi], P(k) proportional to ln(k + 1) - ln(k)."""
    ks = np.arange(lo, hi + 1)
    w = np.log(ks + 1.0) - np.log(ks.astype(np.float64))
    return ks[stream.choice_thresholds(quantise_cdf(w), count)]


# ---------------------------------------------------------------- workload 1
def er1000_target() -> Graph:
    m = master_seed(1)
    s, d = erdos_renyi(1000, 8.0 / 999.0, Stream(sub_seed(m, 0)))
    lab = uniform_labels(1000, 8, Stream(sub_seed(m, 1)))
    return Graph(1000, s, d, lab, None, False, {"name": "er1000"})


def er1000(admitted: dict | None = None) -> Workload:
    t = er1000_target()
    p = random_walk_pattern(t, 8, Stream(sub_seed(master_seed(1), 100)))
    return Workload("er1000", [t], [p], np.array([[0, 0]], dtype=np.int32), ALGO_RI,
                    {"output": "sorted match list"})


# ---------------------------------------------------------------- workload 2
ER2000_SIZES = [16, 18, 20, 22, 24]


def er2000_target() -> Graph:
    m = master_seed(2)
    s, d = erdos_renyi(2000, 0.05, Stream(sub_seed(m, 0)))
    lab = uniform_labels(2000, 4, Stream(sub_seed(m, 1)))
    return Graph(2000, s, d, lab, None, False, {"name": "er2000"})


def er2000_candidate(t: Graph, slot: int, cand: int, adj=None) -> Graph:
    seed = sub_seed(sub_seed(master_seed(2), 100 + slot), cand)
    return dense_walk_pattern(t, ER2000_SIZES[slot], Stream(seed), beta=4, adj=adj)


def er2000(admitted: dict | None = None) -> Workload:
    adm = (admitted if admitted is not None else load_admitted()).get("er2000", {})
    t = er2000_target()
    adj = _Adj(t)
    pats = [er2000_candidate(t, i, int(adm.get(str(i), 0)), adj) for i in range(len(ER2000_SIZES))]
    pairs = np.array([[0, i] for i in range(len(pats))], dtype=np.int32)
    return Workload("er2000", [t], pats, pairs, ALGO_RIDS_SI_FC, {})


# ---------------------------------------------------------------- workload 3
CL10K_SIZES = [32, 32, 32, 48, 48, 48, 64, 64, 64, 64]


def cl10k_target() -> Graph:
    m = master_seed(3)
    s, d = chung_lu(10000, 2.3, 20.0, Stream(sub_seed(m, 0)))
    lab = zipf_labels(10000, 32, 1.2, Stream(sub_seed(m, 1)))
    return Graph(10000, s, d, lab, None, False, {"name": "cl10k"})


def cl10k_candidate(t: Graph, slot: int, cand: int, adj=None) -> Graph:
    # a candidate with fewer than 100 edges is replaced by the next sub-seed
    j = 0
    while True:
        seed = sub_seed(sub_seed(master_seed(3), 100 + slot), 1000 * cand + j)
        p = dense_walk_pattern(t, CL10K_SIZES[slot], Stream(seed), beta=4, adj=adj)
        if p.m >= 100 or j >= 999:
            return p
        j += 1


def cl10k(admitted: dict | None = None) -> Workload:
    adm = (admitted if admitted is not None else load_admitted()).get("cl10k", {})
    t = cl10k_target()
    adj = _Adj(t)
    pats = [cl10k_candidate(t, i, int(adm.get(str(i), 0)), adj) for i in range(len(CL10K_SIZES))]
    pairs = np.array([[0, i] for i in range(len(pats))], dtype=np.int32)
    return Workload("cl10k", [t], pats, pairs, ALGO_RIDS_SI_FC, {"also": ALGO_RI})


# ---------------------------------------------------------------- workload 4
def mol_targets(count: int = 200) -> list:
    m = master_seed(4)
    sizes = 20 + Stream(sub_seed(m, 0)).below(481, count)
    out = []
    probs = molecule_label_probs()
    for i in range(count):
        base = sub_seed(sub_seed(m, 1), i)
        n = int(sizes[i])
        s, d = molecule_tree(n, Stream(sub_seed(base, 0)))
        lab = categorical_labels(n, probs, Stream(sub_seed(base, 1)))
        el = categorical_labels(s.shape[0], [0.80, 0.15, 0.05], Stream(sub_seed(base, 2)), offset=1)
        out.append(Graph(n, s, d, lab, el, False, {"name": f"mol{i}"}))
    return out


def mol_patterns(targets: list, count: int = 1000) -> list:
    m = master_seed(4)
    ks = log_uniform_sizes(4, 64, count, Stream(sub_seed(m, 2)))
    pick = Stream(sub_seed(m, 3))
    adjs: dict[int, _Adj] = {}
    out = []
    for i in range(count):
        k = int(ks[i])
        ok = [j for j, t in enumerate(targets) if t.n >= k]
        ti = ok[pick.one_below(len(ok))]
        if ti not in adjs:
            adjs[ti] = _Adj(targets[ti])
        p = random_walk_pattern(targets[ti], k, Stream(sub_seed(sub_seed(m, 4), i)), adj=adjs[ti])
        p.meta["source_target"] = ti
        out.append(p)
    return out


def mol200(n_targets: int = 200, n_patterns: int = 1000) -> Workload:
    ts = mol_targets(n_targets)
    ps = mol_patterns(ts, n_patterns)
    ti, pi = np.meshgrid(np.arange(len(ts)), np.arange(len(ps)), indexing="ij")
    pairs = np.stack([ti.ravel(), pi.ravel()], axis=1).astype(np.int32)
    return Workload("mol200", ts, ps, pairs, ALGO_RI, {})


# ---------------------------------------------------------------- workload 5
def cl100k_target() -> Graph:
    m = master_seed(5)
    s, d = chung_lu(100000, 2.2, 16.0, Stream(sub_seed(m, 0)))
    lab = zipf_labels(100000, 64, 1.1, Stream(sub_seed(m, 1)))
    return Graph(100000, s, d, lab, None, False, {"name": "cl100k"})


def cl100k_sizes(count: int = 5000) -> np.ndarray:
    return log_uniform_sizes(8, 128, count, Stream(sub_seed(master_seed(5), 2)))


def cl100k_candidate(t: Graph, slot: int, k: int, cand: int, adj=None) -> Graph:
    seed = sub_seed(sub_seed(master_seed(5), 100 + slot), cand)
    return dense_walk_pattern(t, k, Stream(seed), beta=4, adj=adj)


def cl100k_arrivals(count: int, rate_per_s: float) -> np.ndarray:
    """Poisson arrival times (seconds) at `rate_per_s`."""
    u = Stream(sub_seed(master_seed(5), 3)).uniform(count)
    gaps = -np.log1p(-u) / rate_per_s
    return np.cumsum(gaps)


def cl100k(count: int = 5000, admitted: dict | None = None, target: Graph | None = None) -> Workload:
    adm = (admitted if admitted is not None else load_admitted()).get("cl100k", {})
    t = target if target is not None else cl100k_target()
    adj = _Adj(t)
    ks = cl100k_sizes(5000)[:count]
    pats = [cl100k_candidate(t, i, int(ks[i]), int(adm.get(str(i), 0)), adj) for i in range(count)]
    pairs = np.array([[0, i] for i in range(count)], dtype=np.int32)
    return Workload("cl100k", [t], pats, pairs, ALGO_RI, {})


BUILDERS = {"er1000": er1000, "er2000": er2000, "cl10k": cl10k, "mol200": mol200, "cl100k": cl100k}
