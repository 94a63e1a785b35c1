"""RI-DS domains (Section 4: initialisation, arc consistency, forward checking of
singletons) reached by the two device schedules: sweeps over the whole device
under a host loop, and each pair's whole fixpoint inside one block.  Both must
give the oracle's counters (the search then runs on the same domains, so any
difference in a domain shows up in states, nodes or matches)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from brute import plant, plant_connected, random_graph
from gen import configs
from gpu_common import counters, engine, golden, golden_counters, workload

pytestmark = pytest.mark.gpu

SWEEPS, BLOCKS = 1, 2


def _unload(E, tids=(), pids=()):
    from paper_1705_09358_gb300 import sge_unload_pattern, sge_unload_target
    for p in pids:
        sge_unload_pattern(E.h, p)
    for t in tids:
        sge_unload_target(E.h, t)


@pytest.mark.parametrize("directed", [False, True])
def test_block_fixpoint_on_tiny_random_cases(directed):
    """Random labelled (and directed) tiny pairs batched together, every RI-DS variant."""
    E = engine()
    rng = np.random.default_rng(91 + directed)
    pairs = []
    for _ in range(24):
        n = int(rng.integers(4, 12))
        t = random_graph(rng, n, float(rng.uniform(0.2, 0.8)), int(rng.integers(1, 4)), int(rng.integers(1, 3)),
                         directed)
        p = plant(rng, t, int(rng.integers(2, min(n, 6) + 1)), float(rng.uniform(0.3, 1.0)))
        pairs.append((t, p))
    tids = [E.load_target(t) for t, _ in pairs]
    pids = [E.load_pattern(p) for _, p in pairs]
    try:
        for algo in (1, 2, 3):
            want = [counters(oracle.run(t, p, algo)) for t, p in pairs]
            for mode in (SWEEPS, BLOCKS):
                rc, rows = E.count_batch(tids, pids, algo=algo, domain_fixpoint=mode)
                assert [counters(r) for r in rows] == want, (algo, mode)
    finally:
        _unload(E, tids, pids)


@pytest.mark.parametrize("directed", [False, True])
def test_block_fixpoint_on_many_small_random_cases(directed):
    """A batch of 1,000 pairs: enough that the fixpoint runs in blocks of four warps, as many as
    are resident, each taking pairs from the counter; 100 random labelled pairs (one to four
    domain words per pattern vertex), each repeated ten times across the batch, every RI-DS
    variant, against the oracle and the sweep schedule."""
    E = engine()
    rng = np.random.default_rng(191 + directed)
    pairs = []
    for i in range(100):
        if i % 2 == 0:   # one domain word per pattern vertex
            n = int(rng.integers(4, 16))
            t = random_graph(rng, n, float(rng.uniform(0.2, 0.8)), int(rng.integers(1, 4)),
                             int(rng.integers(1, 3)), directed)
            p = plant(rng, t, int(rng.integers(2, min(n, 6) + 1)), float(rng.uniform(0.3, 1.0)))
        else:            # two to four words: sparse targets, connected patterns
            n = int(rng.integers(65, 257))
            t = random_graph(rng, n, float(rng.uniform(0.02, 0.05)), int(rng.integers(2, 5)),
                             int(rng.integers(1, 3)), directed)
            p = plant_connected(rng, t, int(rng.integers(3, 9)))
        pairs.append((t, p))
    tids = [E.load_target(t) for t, _ in pairs]
    pids = [E.load_pattern(p) for _, p in pairs]
    order = np.tile(np.arange(len(pairs)), 10)
    rng.shuffle(order)
    T = np.array(tids, np.int32)[order]
    P = np.array(pids, np.int32)[order]
    try:
        for algo in (1, 2, 3):
            want = [counters(oracle.run(t, p, algo)) for t, p in pairs]
            rc, blocks = E.count_batch(T, P, algo=algo, domain_fixpoint=BLOCKS)
            assert [counters(r) for r in blocks] == [want[i] for i in order], algo
            rc, sweeps = E.count_batch(T, P, algo=algo, domain_fixpoint=SWEEPS)
            assert [counters(r) for r in sweeps] == [want[i] for i in order], algo
    finally:
        _unload(E, tids, pids)


def test_block_fixpoint_cl10k_and_er2000():
    E = engine()
    for name in ("cl10k", "er2000"):
        w = configs.BUILDERS[name]()
        g = golden(name)
        tid = E.load_target(w.targets[0])
        pids = [E.load_pattern(p) for p in w.patterns]
        try:
            for algo in (1, 2, 3):
                want = [golden_counters(ent["algos"][str(algo)]) for ent in g["patterns"]]
                for mode in (SWEEPS, BLOCKS):
                    rc, rows = E.count_batch([tid] * len(pids), pids, algo=algo, domain_fixpoint=mode)
                    assert [counters(r) for r in rows] == want, (name, algo, mode)
        finally:
            _unload(E, [tid], pids)


def test_block_fixpoint_on_the_100k_vertex_target():
    """Large domains (k x 100,000 bits) worked through by one block per query: the first
    16 queries against the live oracle, the first 400 against the sweep schedule."""
    t = workload("cl100k_target")
    w = workload("cl100k")
    E = engine()
    tid = E.load_target(t)
    pids = [E.load_pattern(p) for p in w.patterns[:400]]
    ot = oracle.Target(t)
    for algo in (1, 3):
        rc, blocks = E.count_batch([tid] * len(pids), pids, algo=algo, domain_fixpoint=BLOCKS)
        rc, sweeps = E.count_batch([tid] * len(pids), pids, algo=algo, domain_fixpoint=SWEEPS)
        assert [counters(r) for r in blocks] == [counters(r) for r in sweeps], algo
        for i in range(16):
            assert counters(blocks[i]) == counters(oracle.run(ot, w.patterns[i], algo)), (algo, i)


def test_unknown_domain_mode_is_an_argument_error():
    import paper_1705_09358_gb300 as sge
    from brute import complete
    E = engine()
    tid, pid = E.load_target(complete(5)), E.load_pattern(complete(3))
    r = E.count(tid, pid, check=False, algo=1, domain_fixpoint=7)
    assert r["rc"] == sge.SGE_ERR_ARG
