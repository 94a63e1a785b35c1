"""Checkpoint and resume: a batched search stopped by a time limit or a state
budget, then resumed (possibly with another kernel family, another schedule
or in shards) until nothing is left, gives exactly the counters of one
uninterrupted run, which the golden files hold from the oracle."""
from __future__ import annotations

import ctypes as C
import struct

import numpy as np
import pytest

from gen import configs
from gpu_common import engine, counters, golden, golden_counters, workload
from paper_1705_09358_gb300 import SgeError, load_library, sge_ckpt_info, sge_result

pytestmark = pytest.mark.gpu

TIMEOUT, BUDGET = -5, -4


def _er2000():
    w = configs.er2000()
    g = golden("er2000")
    E = engine()
    tid = E.load_target(w.targets[0])
    pids = [E.load_pattern(p) for p in w.patterns]
    return E, tid, pids, g


def _drain(E, blob, max_calls=400, **opts):
    """Resume until the search finishes; returns (final rows, resume calls)."""
    rows, calls = None, 0
    while blob is not None:
        rc, rows, blob = E.resume(blob, **opts)
        assert rc in (0, TIMEOUT, BUDGET), rc
        assert (blob is None) == (rc == 0)
        calls += 1
        assert calls <= max_calls, "resume made no progress"
    return rows, calls


def _table(rows):
    return [counters(r) for r in rows]


def test_er2000_time_limit_resume_bitset():
    E, tid, pids, g = _er2000()
    want = [golden_counters(ent["algos"]["3"]) for ent in g["patterns"]]
    # the batched search kernel runs ~9 ms, so a 1 ms limit stops it
    rc, rows, blob = E.count_batch_ckpt([tid] * 5, pids, algo=3, time_limit_ms=1)
    assert rc == TIMEOUT and blob is not None
    npairs, nframes = sge_ckpt_info(blob)
    assert npairs == 5 and nframes > 0
    partial = _table(rows)
    assert all(p[1] <= w[1] and p[2] <= w[2] for p, w in zip(partial, want))
    rows, calls = _drain(E, blob, time_limit_ms=2)
    assert calls >= 2
    assert _table(rows) == want


def test_er2000_checkpoint_resumed_by_other_kernel_and_schedule():
    # frames are ranges of candidate lists, so either kernel family continues them
    E, tid, pids, g = _er2000()
    want = [golden_counters(ent["algos"]["3"]) for ent in g["patterns"]]
    rc, rows, blob = E.count_batch_ckpt([tid] * 5, pids, algo=3, kernel=2, time_limit_ms=1)
    assert rc == TIMEOUT and blob is not None
    rows, calls = _drain(E, blob, kernel=1, steal_granularity=1, frames_per_warp=8)
    assert calls == 1
    assert _table(rows) == want
    rc, rows, blob = E.count_batch_ckpt([tid] * 5, pids, algo=3, kernel=1, time_limit_ms=1)
    if blob is not None:
        rows, _ = _drain(E, blob, kernel=2)
    assert _table(rows) == want


@pytest.mark.parametrize("algo", [0, 1])
def test_er2000_state_budget_resume_csr(algo):
    E, tid, pids, g = _er2000()
    want = [golden_counters(ent["algos"][str(algo)]) for ent in g["patterns"]]
    budget = max(w[1] for w in want) // 6
    rc, rows, blob = E.count_batch_ckpt([tid] * 5, pids, algo=algo, kernel=1, state_budget=budget)
    assert rc == BUDGET and blob is not None
    rows, calls = _drain(E, blob, kernel=1, state_budget=budget)
    assert calls >= 1
    assert _table(rows) == want


def test_er2000_sharded_checkpoints():
    E, tid, pids, g = _er2000()
    want = np.array([golden_counters(ent["algos"]["3"]) for ent in g["patterns"]], dtype=np.uint64)
    total = np.zeros_like(want)
    for shard in range(2):
        rc, rows, blob = E.count_batch_ckpt([tid] * 5, pids, algo=3, shard_index=shard, shard_count=2,
                                            time_limit_ms=1)
        if blob is not None:
            rows, _ = _drain(E, blob, time_limit_ms=3)
        total += np.array(_table(rows), dtype=np.uint64)   # uint64 wraps like the hash
    assert np.array_equal(total, want)


def test_cl100k_budget_resume():
    g = golden("cl100k")
    w = workload("cl100k")
    E = engine()
    tid = E.load_target(workload("cl100k_target"))
    pids = [E.load_pattern(p) for p in w.patterns[:60]]
    want = [tuple(int(x) for x in row) for row in g["first_200"][:60]]
    budget = max(1, sorted(r[1] for r in want)[len(want) // 2] // 2)
    rc, rows, blob = E.count_batch_ckpt([tid] * len(pids), pids, algo=0, state_budget=budget)
    assert rc in (0, BUDGET)
    if blob is not None:
        rows, calls = _drain(E, blob)
        assert calls == 1
    assert _table(rows) == want


@pytest.mark.parametrize("algo", [0, 3])
def test_directed_labelled_budget_resume(algo):
    """A directed, edge-labelled batch (the CSR kernel's in/out rows and direction-aware back-edge
    checks) cut by a state budget below the persistent kernel (split depth 1) and resumed to the
    end: every pair's counters equal the oracle's."""
    import oracle
    from brute import plant_connected, random_graph
    rng = np.random.default_rng(880)
    t = random_graph(rng, 300, 0.05, 2, 2, directed=True)
    pats = [plant_connected(rng, t, int(rng.integers(4, 8))) for _ in range(24)]
    E = engine()
    tid = E.load_target(t)
    pids = [E.load_pattern(p) for p in pats]
    want = [counters(oracle.run(t, p, algo)) for p in pats]
    budget = max(w[1] for w in want) // 5
    rc, rows, blob = E.count_batch_ckpt([tid] * len(pids), pids, algo=algo, split_depth=1, state_budget=budget)
    assert rc == BUDGET and blob is not None
    rows, calls = _drain(E, blob, state_budget=budget)
    assert calls >= 1
    assert _table(rows) == want


def test_finished_search_leaves_no_checkpoint():
    E, tid, pids, g = _er2000()
    rc, rows, blob = E.count_batch_ckpt([tid] * 5, pids, algo=3)
    assert rc == 0 and blob is None
    assert _table(rows) == [golden_counters(ent["algos"]["3"]) for ent in g["patterns"]]


def test_malformed_checkpoints_are_rejected():
    E, tid, pids, g = _er2000()
    rc, rows, blob = E.count_batch_ckpt([tid] * 5, pids, algo=3, time_limit_ms=1)
    assert blob is not None
    ARG = -1
    # an unknown target id
    bad = bytearray(blob)
    struct.pack_into("<i", bad, 32, 2 ** 30)
    assert E.resume(bytes(bad), check=False)[0] == ARG
    # a frame image outside the target: the first frame's first image (if it has one)
    npairs = struct.unpack_from("<q", blob, 16)[0]
    at = 32 + 48 * npairs
    kmax, np_g, nf = struct.unpack_from("<iiq", blob, at)
    at += 16 + 4 * (np_g + (np_g & 1))
    stride = 4 + kmax
    for f in range(nf):
        depth = struct.unpack_from("<i", blob, at + 4 * (f * stride + 1))[0] & 0xFFFF
        if depth > 0:
            bad = bytearray(blob)
            struct.pack_into("<i", bad, at + 4 * (f * stride + 4), 10 ** 9)
            assert E.resume(bytes(bad), check=False)[0] == ARG
            break
    # truncated, and trailing bytes: the binding's size check and the library's own
    with pytest.raises(SgeError):
        E.resume(blob[:-4])
    for bad in (blob[:-4], blob + b"\0\0\0\0"):
        out = (sge_result * 5)()
        ptr, nbytes = C.c_void_p(), C.c_int64(0)
        rc = load_library().sge_resume(E.h, bad, len(bad), None, C.cast(out, C.c_void_p), C.byref(ptr),
                                       C.byref(nbytes))
        assert rc == ARG and not ptr.value
    # the intact blob still resumes to the full counts
    rows, _ = _drain(E, blob)
    assert _table(rows) == [golden_counters(ent["algos"]["3"]) for ent in g["patterns"]]
