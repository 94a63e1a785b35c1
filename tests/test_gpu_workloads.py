"""Full-size parity on the five synthetic workloads, in the launch
configurations the bench uses, against the oracle's stored results
(tests/golden/expected_*.json, written by tests/golden/make_expected.py)."""
from __future__ import annotations

import threading
import time

import numpy as np
import pytest

from brute import complete
from gen import configs
from gpu_common import engine, counters, golden, golden_counters, table_digest, workload

pytestmark = pytest.mark.gpu


def test_er2000_single_and_batched():
    w = configs.er2000()
    g = golden("er2000")
    assert w.targets[0].sha256() == g["target_sha256"]
    E = engine()
    tid = E.load_target(w.targets[0])
    pids = [E.load_pattern(p) for p in w.patterns]
    for ent, p in zip(g["patterns"], w.patterns):
        assert p.sha256() == ent["pattern_sha256"]
    # the bench's configuration: all five pairs in one batched call, RI-DS-SI-FC
    rc, rows = E.count_batch([tid] * 5, pids, algo=3)
    for ent, row in zip(g["patterns"], rows):
        assert counters(row) == golden_counters(ent["algos"]["3"]), ent["slot"]
    # every variant, both kernel families, one pattern at a time
    for ent, pid in zip(g["patterns"], pids):
        for algo in range(4):
            want = ent["algos"][str(algo)]
            if want is None:
                continue
            for kern in (1, 2):
                got = E.count(tid, pid, algo=algo, kernel=kern)
                assert counters(got) == golden_counters(want), (ent["slot"], algo, kern)


@pytest.mark.parametrize("algo", [0, 3])
def test_mol200_all_pairs_batched(algo):
    ts = workload("mol_targets")
    ps = workload("mol_patterns")
    g = golden("mol200")
    E = engine()
    tids = [E.load_target(t) for t in ts]
    pids = [E.load_pattern(p) for p in ps]
    T = np.repeat(np.array(tids, np.int32), len(pids))
    P = np.tile(np.array(pids, np.int32), len(tids))
    rc, rows = E.count_batch(T, P, algo=algo)
    table = np.stack([rows["matches"], rows["states"], rows["nodes"], rows["hash"]], axis=1).astype(np.uint64)
    want = g["algos"][str(algo)]
    sample = np.array(want["sample_every_997"], dtype=np.uint64)
    assert np.array_equal(table[::997], sample)
    assert int(table[:, 1].sum()) == want["totals"]["states"]
    assert table_digest(table) == want["per_pair_sha256"]


def test_cl100k_queries_batched_and_alone():
    g = golden("cl100k")
    t = workload("cl100k_target")
    assert t.sha256() == g["target_sha256"]
    w = workload("cl100k")
    E = engine()
    tid = E.load_target(t)
    pids = [E.load_pattern(p) for p in w.patterns[:200]]
    rc, rows = E.count_batch([tid] * len(pids), pids, algo=0)
    want = np.array(g["first_200"], dtype=np.uint64)
    got = np.stack([rows["matches"], rows["states"], rows["nodes"], rows["hash"]], axis=1).astype(np.uint64)
    assert np.array_equal(got, want)
    for i in range(0, 200, 20):
        assert counters(E.count(tid, pids[i], algo=0)) == tuple(int(x) for x in want[i]), i


def test_cl100k_all_5000_digest():
    g = golden("cl100k")
    t = workload("cl100k_target")
    w = workload("cl100k")
    E = engine()
    tid = E.load_target(t)
    pids = [E.load_pattern(p) for p in w.patterns]
    rc, rows = E.count_batch([tid] * len(pids), pids, algo=0)
    table = np.stack([rows["matches"], rows["states"], rows["nodes"], rows["hash"]], axis=1).astype(np.uint64)
    assert int(table[:, 1].sum()) == g["totals"]["states"]
    assert table_digest(table) == g["per_query_sha256"]


def test_serving_results_same_alone_and_in_mix():
    """Queries submitted while others run are admitted, batched and overlapped;
    every result equals the query's result run alone (and the oracle's)."""
    g = golden("cl100k")
    t = workload("cl100k_target")
    w = workload("cl100k")
    E = engine()
    tid = E.load_target(t)
    pids = [E.load_pattern(p) for p in w.patterns[:200]]
    tickets = []
    for i, pid in enumerate(pids):
        tickets.append(E.serve_submit(tid, pid, algo=0))
        if i % 16 == 15:
            time.sleep(0.001)
    E.serve_drain()
    want = np.array(g["first_200"], dtype=np.uint64)
    for i, tk in enumerate(tickets):
        r = E.serve_poll(tk)
        assert r is not None and r["status"] == 0
        assert counters(r) == tuple(int(x) for x in want[i]), i
    for i in range(0, 200, 25):
        assert counters(E.count(tid, pids[i], algo=0)) == tuple(int(x) for x in want[i])


def test_serving_concurrent_groups_of_different_sizes():
    """Several scheduler threads launch groups of different pattern sizes at the
    same time (their kernels need different amounts of shared memory); every
    query must succeed with its own result, round after round."""
    g = golden("cl100k")
    t = workload("cl100k_target")
    w = workload("cl100k")
    E = engine()
    tid = E.load_target(t)
    pids = [E.load_pattern(p) for p in w.patterns[:200]]
    want = np.array(g["first_200"], dtype=np.uint64)
    order = np.random.default_rng(5).permutation(len(pids))
    for rnd in range(4):
        tickets = []
        for j, i in enumerate(order):
            tickets.append((int(i), E.serve_submit(tid, pids[int(i)], algo=0)))
            if j % 50 == 49:
                time.sleep(0.0005 * rnd)
        E.serve_drain()
        for i, tk in tickets:
            r = E.serve_poll(tk)
            assert r is not None and r["status"] == 0, (rnd, i, r and r["status"])
            assert counters(r) == tuple(int(x) for x in want[i]), (rnd, i)


def test_cancel_from_another_thread():
    import paper_1705_09358_gb300 as sge
    E = engine()
    tid, pid = E.load_target(complete(48)), E.load_pattern(complete(9))
    out = {}

    def run():
        out["r"] = E.count(tid, pid, check=False)

    th = threading.Thread(target=run)
    th.start()
    time.sleep(1.0)
    E.cancel()
    th.join(timeout=120)
    assert not th.is_alive()
    assert out["r"]["rc"] == sge.SGE_ERR_CANCELLED
    assert E.count(tid, E.load_pattern(complete(2)))["matches"] == 48 * 47


def test_cl100k_rids_variants_sample():
    """RI-DS (all three variants) on the 100k-vertex serving target: domains of
    k x 100,000 bits per query, checked against the live oracle."""
    import oracle
    t = workload("cl100k_target")
    w = workload("cl100k")
    E = engine()
    tid = E.load_target(t)
    pats = w.patterns[:40]
    pids = [E.load_pattern(p) for p in pats]
    ot = oracle.Target(t)
    for algo in (1, 2, 3):
        rc, rows = E.count_batch([tid] * len(pids), pids, algo=algo)
        for i, p in enumerate(pats):
            want = oracle.run(ot, p, algo)
            assert counters(rows[i]) == counters(want), (algo, i)


def test_domain_word_sweeps_match_candidate_sweeps():
    """Arc consistency runs over candidate lists, or over 64-target words when the lists
    would be too large; both must reach the same fixpoint.  The word sweeps are forced
    (SGE_DOMAIN_WORDS=1, read once per process) in a child process on cl10k."""
    import json
    import os
    import subprocess
    import sys
    g = golden("cl10k")
    code = (
        "import json, sys\n"
        "sys.path.insert(0, 'tests'); sys.path.insert(0, '.')\n"
        "from gen import configs\n"
        "import paper_1705_09358_gb300 as sge\n"
        "w = configs.cl10k()\n"
        "with sge.Context(0) as E:\n"
        "    tid = E.load_target(w.targets[0])\n"
        "    pids = [E.load_pattern(p) for p in w.patterns]\n"
        "    rc, rows = E.count_batch([tid] * len(pids), pids, algo=3)\n"
        "    print(json.dumps([[int(r[k]) for k in ('matches', 'states', 'nodes', 'hash')] for r in rows]))\n"
    )
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, SGE_DOMAIN_WORDS="1")
    out = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    got = json.loads(out.stdout.strip().splitlines()[-1])
    want = [list(golden_counters(ent["algos"]["3"])) for ent in g["patterns"]]
    assert got == want
