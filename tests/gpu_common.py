"""Helpers of the GPU tests: a shared engine context and oracle comparisons."""
from __future__ import annotations

import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden")
KEYS = ("matches", "states", "nodes", "hash")

_ctx = None


def engine():
    """One Context for the whole test session (built on first use)."""
    global _ctx
    if _ctx is None:
        from paper_1705_09358_gb300 import build, Context
        build.build()
        _ctx = Context(0)
    return _ctx


_cache = {}


def workload(name: str, **kw):
    """Generated workloads, built once per test session."""
    from gen import configs
    key = (name, tuple(sorted(kw.items())))
    if key not in _cache:
        if name == "cl100k_target":
            _cache[key] = configs.cl100k_target()
        elif name == "cl100k":
            _cache[key] = configs.cl100k(count=5000, target=workload("cl100k_target"))
        elif name == "mol_targets":
            _cache[key] = configs.mol_targets(200)
        elif name == "mol_patterns":
            _cache[key] = configs.mol_patterns(workload("mol_targets"), 1000)
        else:
            _cache[key] = configs.BUILDERS[name](**kw)
    return _cache[key]


def counters(d) -> tuple:
    return tuple(int(d[k]) for k in KEYS)


def golden(name: str) -> dict:
    with open(os.path.join(GOLDEN, f"expected_{name}.json")) as f:
        return json.load(f)


def golden_counters(g) -> tuple:
    return (int(g["matches"]), int(g["states"]), int(g["nodes"]), int(g["hash"]))


def table_digest(table) -> str:
    import hashlib
    return hashlib.sha256(np.ascontiguousarray(table, dtype=np.uint64).tobytes()).hexdigest()
