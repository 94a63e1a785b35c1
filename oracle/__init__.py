"""CPU oracle -- TEST INFRASTRUCTURE ONLY.

A plain single-threaded C statement of RI / RI-DS / RI-DS-SI / RI-DS-SI-FC
(arXiv 1705.09358, Section "RI" and Section 4), used to check the CUDA path
and as the timed CPU baseline.  Only the tests, the smoke check and the
bench's CPU-baseline leg may import this package; the library never does.

This module only marshals arguments into the C code in ``sge_oracle.c``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sge_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libsge_oracle.so")
_lock = threading.Lock()
_lib = None

ALGO_RI, ALGO_RIDS, ALGO_RIDS_SI, ALGO_RIDS_SI_FC = 0, 1, 2, 3
OR_BUDGET = 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no target-specific flags)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
            P = C.c_void_p
            lib.oracle_run.restype = C.c_int
            lib.oracle_run.argtypes = [C.c_int, C.c_int64, P, P, P, P, C.c_int,
                                       C.c_int, C.c_int64, P, P, P, P,
                                       C.c_int, C.c_int64, P, P, P, P, P, C.c_int64, P, P, P,
                                       C.c_int, C.c_int, C.c_int]
            lib.oracle_target_new.restype = C.c_void_p
            lib.oracle_target_new.argtypes = [C.c_int, C.c_int64, P, P, P, P, C.c_int, P]
            lib.oracle_target_free.restype = None
            lib.oracle_target_free.argtypes = [C.c_void_p]
            lib.oracle_run_t.restype = C.c_int
            lib.oracle_run_t.argtypes = [C.c_void_p, C.c_int, C.c_int64, P, P, P, P,
                                         C.c_int, C.c_int64, P, P, P, P, P, C.c_int64, P, P, P,
                                         C.c_int, C.c_int, C.c_int]
            lib.oracle_domains.restype = C.c_int
            lib.oracle_domains.argtypes = [C.c_int, C.c_int64, P, P, P, P, C.c_int,
                                           C.c_int, C.c_int64, P, P, P, P, C.c_int, P]
            lib.oracle_fc.restype = C.c_int
            lib.oracle_fc.argtypes = [C.c_int, C.c_int, P]
            lib.oracle_order.restype = C.c_int
            lib.oracle_order.argtypes = [C.c_int, C.c_int64, P, P, C.c_int, C.c_int, P, P, P]
            lib.oracle_match_hash.restype = C.c_uint64
            lib.oracle_match_hash.argtypes = [C.c_int, i32p]
            _lib = lib
    return _lib


def _i32(a):
    if a is None:
        return None
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _graph_args(g):
    src, dst, vl, el = _i32(g.src), _i32(g.dst), _i32(g.vlabel), _i32(g.elabel)
    keep = (src, dst, vl, el)
    return keep, [int(g.n), int(src.shape[0]), _ptr(src), _ptr(dst), _ptr(vl), _ptr(el)]


class Target:
    """A target graph built once inside the oracle for many runs."""

    def __init__(self, g):
        lib = _load()
        self.n = int(g.n)
        self.directed = bool(g.directed)
        keep, a = _graph_args(g)
        rc = np.zeros(1, dtype=np.int32)
        self._h = lib.oracle_target_new(*a, int(self.directed), _ptr(rc))
        if not self._h:
            raise ValueError(f"oracle_target_new rejected its input (code {int(rc[0])})")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.oracle_target_free(h)
            self._h = None


def run(target, pattern, algo: int = ALGO_RI, state_budget: int = 0, want_matches: bool = False,
        match_cap: int = 1 << 22, want_levels: bool = False, shard=None) -> dict:
    """Run one (target, pattern) instance.

    `target` is a graph or a prebuilt `Target`.  Returns a dict with
    matches, states, nodes, hash, order (mu), parent (position of P(mu_i) or
    -1), domain sizes (RI-DS), the sorted match list when `want_matches`,
    per-position node / state counts when `want_levels`, and
    `budget_exceeded`.  `shard=(depth, index, count)` restricts the search to
    one shard of the frontier at `depth`.
    """
    lib = _load()
    tgt = target if isinstance(target, Target) else Target(target)
    if tgt.directed != bool(pattern.directed):
        raise ValueError("target and pattern must both be directed or both undirected")
    pk, pa = _graph_args(pattern)
    k = int(pattern.n)
    counters = np.zeros(4, dtype=np.uint64)
    mu = np.full(max(k, 1), -1, dtype=np.int32)
    par = np.full(max(k, 1), -1, dtype=np.int32)
    dsz = np.zeros(max(k, 1), dtype=np.int64)
    mout = np.zeros(max(1, match_cap * max(k, 1)), dtype=np.int32) if want_matches else None
    mlen = np.zeros(1, dtype=np.int64)
    lvn = np.zeros(max(k, 1), dtype=np.uint64) if want_levels else None
    lvs = np.zeros(max(k, 1), dtype=np.uint64) if want_levels else None
    sd, si, sc = shard if shard is not None else (0, 0, 1)
    rc = lib.oracle_run_t(tgt._h, *pa[:6],
                          int(algo), int(state_budget), _ptr(counters), _ptr(mu), _ptr(par), _ptr(dsz),
                          _ptr(mout), int(match_cap if want_matches else 0), _ptr(mlen),
                          _ptr(lvn), _ptr(lvs), int(sd), int(si), int(sc))
    del pk
    if rc < 0:
        raise ValueError(f"oracle_run rejected its input (code {rc})")
    out = {
        "matches": int(counters[0]), "states": int(counters[1]), "nodes": int(counters[2]),
        "hash": int(counters[3]), "order": mu[:k].copy(), "parent": par[:k].copy(),
        "domain_sizes": dsz[:k].copy(), "budget_exceeded": rc == OR_BUDGET,
    }
    if want_matches:
        n = int(mlen[0])
        if n > match_cap:
            raise ValueError("match list larger than match_cap")
        rows = mout[: n * k].reshape(n, k) if k > 0 else np.zeros((0, 0), np.int32)
        if n > 0:
            rows = rows[np.lexsort(rows.T[::-1])]
        out["match_list"] = rows.copy()
    if want_levels:
        out["level_nodes"] = lvn[:k].astype(np.int64)
        out["level_states"] = lvs[:k].astype(np.int64)
    return out


def domains(target, pattern, algo: int) -> np.ndarray:
    """Final domains as a (k, n_t) 0/1 array (RI: the label/degree filter only)."""
    lib = _load()
    tk, ta = _graph_args(target)
    pk, pa = _graph_args(pattern)
    dom = np.zeros((pattern.n, target.n), dtype=np.uint8)
    rc = lib.oracle_domains(*ta[:6], int(bool(target.directed)), *pa[:6], int(algo), _ptr(dom))
    if rc < 0:
        raise ValueError(f"oracle_domains rejected its input (code {rc})")
    return dom


def forward_check(dom: np.ndarray) -> np.ndarray:
    """Forward checking of singleton domains alone, on a (k, n_t) 0/1 array."""
    lib = _load()
    d = np.ascontiguousarray(dom, dtype=np.uint8).copy()
    rc = lib.oracle_fc(int(d.shape[0]), int(d.shape[1]), _ptr(d))
    if rc < 0:
        raise ValueError("oracle_fc failed")
    return d


def order(pattern, algo: int = ALGO_RI, domain_sizes=None):
    """(mu, parent positions) of the GreatestConstraintFirst ordering."""
    lib = _load()
    src, dst = _i32(pattern.src), _i32(pattern.dst)
    k = int(pattern.n)
    mu = np.zeros(max(k, 1), dtype=np.int32)
    par = np.zeros(max(k, 1), dtype=np.int32)
    ds = None if domain_sizes is None else np.ascontiguousarray(domain_sizes, dtype=np.int64)
    rc = lib.oracle_order(k, int(src.shape[0]), _ptr(src), _ptr(dst), int(bool(pattern.directed)),
                          int(algo), _ptr(ds), _ptr(mu), _ptr(par))
    if rc < 0:
        raise ValueError(f"oracle_order rejected its input (code {rc})")
    return mu[:k].copy(), par[:k].copy()


def match_hash(f) -> int:
    """h(f) of one match given in pattern-vertex order."""
    f = np.ascontiguousarray(f, dtype=np.int32)
    return int(_load().oracle_match_hash(int(f.shape[0]), f))
