"""Parity of the bitset search kernel when a bitset row spans several words per lane.

The bitset kernel keeps ceil(n_t / 64) 64-bit words per row, word q in lane
q mod 32, so a target of more than 2048 vertices puts two or four words in
every lane (NWL = 2 or 4; up to 8192 vertices).  These cases compare that
path with the oracle (Section 2.1, Eqs. 1-3 for the result; the RI and RI-DS
searches for the states and nodes) on unlabelled-edge undirected ER targets
of 2049, 3000, 6000 and 8192 vertices: ragged last words (2049: one lane of
the second word; 3000: fifteen lanes; 6000: thirty lanes of the third word),
the full four words (8192), the used-vertex bitset spread over several
registers, and levels whose survivors overflow the shared-memory list and go
to the per-warp global slab.  A batch that pairs a 300-vertex target with a
6000-vertex one runs both at the larger word count.

Targets: G(n, p) with vertex labels drawn from a skewed mix (label 0 with
probability 1/2, labels 1..15 sharing the rest), so a common label lets one
level keep more than 64 survivors while the rare labels keep the match
counts small.  Patterns: dense walks (gen.patterns).  Every value compared
is an exact integer.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from gen.graphs import Graph, categorical_labels, erdos_renyi, neighbour_lists
from gen.patterns import dense_walk_pattern
from gen.rng import Stream
from gpu_common import counters, engine

ORACLE_BUDGET = 60_000_000
LIST_CAP = 64          # shared-memory survivor list of the bitset kernel for patterns of <= 32 vertices

# (n, p, [(k, candidate seed)]): chosen so that every variant stays within the oracle budget
CASES = {
    2049: (0.1, [(10, 0), (12, 0), (16, 2)]),
    3000: (0.08, [(12, 0), (12, 2), (16, 1)]),
    6000: (0.05, [(14, 2), (16, 0)]),
    8192: (0.04, [(16, 0), (16, 1)]),
}
SPILLING = {(6000, 16, 0), (8192, 16, 0)}   # an expansion keeps > LIST_CAP survivors (checked below)

_targets = {}


def skewed_er(n: int, p: float) -> Graph:
    if n not in _targets:
        s = Stream(7100 + n)
        a, b = erdos_renyi(n, p, s)
        _targets[n] = Graph(n, a, b, categorical_labels(n, [0.5] + [0.5 / 15] * 15, s))
    return _targets[n]


def pattern(t: Graph, k: int, cand: int) -> Graph:
    return dense_walk_pattern(t, k, Stream(t.n * 31 + k * 7 + cand))


def words_per_lane(n: int) -> int:
    dw = (n + 63) // 64
    w = 1
    while w < (dw + 31) // 32:
        w *= 2
    return w


def most_survivors_at_position_1(t: Graph, p: Graph) -> int:
    """Largest survivor count of an expansion of RI position 1 (candidates: the
    row of M(mu_0) filtered by mu_1's label and degree) over every root choice.
    With the split stopped at depth 1 the search kernel performs exactly these
    expansions."""
    ip, nb, _ = neighbour_lists(t)
    deg = np.diff(ip)
    pdeg = np.diff(neighbour_lists(p)[0])
    mu, _ = oracle.order(p, 0)
    ok0 = (t.vlabel == p.vlabel[mu[0]]) & (deg >= pdeg[mu[0]])
    ok1 = (t.vlabel == p.vlabel[mu[1]]) & (deg >= pdeg[mu[1]])
    return max(int(ok1[nb[ip[v]:ip[v + 1]]].sum()) for v in np.nonzero(ok0)[0])


def _unload(E, tid=None, pids=()):
    from paper_1705_09358_gb300 import sge_unload_pattern, sge_unload_target
    for pid in pids:
        sge_unload_pattern(E.h, pid)
    if tid is not None:
        sge_unload_target(E.h, tid)


def test_multiword_cases_are_admissible():
    """Host-side check of the case construction: two or four words per lane, every
    variant within the oracle budget, and the spilling cases really overflow the
    shared-memory survivor list."""
    for n, (p_edge, pats) in CASES.items():
        t = skewed_er(n, p_edge)
        assert words_per_lane(n) in (2, 4)
        ot = oracle.Target(t)
        for k, cand in pats:
            p = pattern(t, k, cand)
            for algo in range(4):
                assert not oracle.run(ot, p, algo, state_budget=ORACLE_BUDGET)["budget_exceeded"], (n, k, cand)
            spill = most_survivors_at_position_1(t, p)
            assert (spill > LIST_CAP) == ((n, k, cand) in SPILLING), (n, k, cand, spill)


@pytest.mark.gpu
@pytest.mark.parametrize("n", sorted(CASES))
def test_multiword_bitset_matches_oracle(n):
    p_edge, pats = CASES[n]
    t = skewed_er(n, p_edge)
    assert words_per_lane(n) in (2, 4)
    E = engine()
    tid = E.load_target(t)
    ot = oracle.Target(t)
    pids = []
    try:
        for k, cand in pats:
            p = pattern(t, k, cand)
            pid = E.load_pattern(p)
            pids.append(pid)
            for algo in range(4):
                want = oracle.run(ot, p, algo, state_budget=ORACLE_BUDGET)
                assert not want["budget_exceeded"], "test instance too large for the oracle"
                for kern in (0, 2, 1):
                    for sched in ({}, {"split_depth": 1}, {"split_depth": 2, "steal_granularity": 1}):
                        got = E.count(tid, pid, algo=algo, kernel=kern, **sched)
                        if kern != 1:
                            assert got["kernel"] == 2, "the bitset kernel should take this target"
                        assert counters(got) == counters(want), (n, k, cand, algo, kern, sched)
    finally:
        _unload(E, tid, pids)


@pytest.mark.gpu
def test_multiword_enumeration_lists():
    """Full sorted match lists through the bitset kernel at two and four words per lane."""
    E = engine()
    for n, k, cand in ((3000, 12, 0), (6000, 14, 2)):
        t = skewed_er(n, CASES[n][0])
        p = pattern(t, k, cand)
        tid, pid = E.load_target(t), E.load_pattern(p)
        try:
            want = oracle.run(t, p, 3, want_matches=True, state_budget=ORACLE_BUDGET)
            for algo in (0, 3):
                got = E.enumerate(tid, pid, algo=algo, kernel=2)
                assert got["kernel"] == 2
                assert np.array_equal(got["match_list"], want["match_list"]), (n, algo)
        finally:
            _unload(E, tid, [pid])


@pytest.mark.gpu
def test_mixed_batch_small_and_large_targets():
    """One batch holding a 300-vertex and a 6000-vertex target: both searched at
    four words per lane; every pair equals its own oracle run."""
    E = engine()
    small = skewed_er(300, 0.08)
    big = skewed_er(6000, CASES[6000][0])
    ps = [pattern(small, 8, 0), pattern(small, 10, 1), pattern(big, 16, 0), pattern(big, 14, 2)]
    ts_ = {0: small, 1: big}
    pairs = [(0, 0), (1, 2), (0, 1), (1, 3), (0, 3), (0, 2)]
    tids = {0: E.load_target(small), 1: E.load_target(big)}
    pids = [E.load_pattern(p) for p in ps]
    try:
        for algo in (0, 3):
            want = [counters(oracle.run(ts_[a], ps[b], algo, state_budget=ORACLE_BUDGET)) for a, b in pairs]
            for sched in ({}, {"split_depth": 1}):
                rc, rows = E.count_batch([tids[a] for a, _ in pairs], [pids[b] for _, b in pairs], algo=algo,
                                         **sched)
                assert set(int(x) for x in rows["kernel"]) == {2}
                got = [counters(r) for r in rows]
                assert got == want, (algo, sched)
    finally:
        _unload(E, None, pids)
        _unload(E, tids[0])
        _unload(E, tids[1])
