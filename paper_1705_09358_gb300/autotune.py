"""Schedule autotuner: picks split target, steal granularity and donation cadence.

The search tree is fixed by the method, so every schedule gives the same four
counters; only the time changes.  The tuner times the engine (through the C
ABI) on a caller's workload over a small grid of schedule points by
coordinate descent, keeps the fastest point whose counters equal the
baseline's (a point that changes them is reported as an error, never
chosen), and records it in a JSON cache keyed by the workload class:
(kernel family, n_t bucket, k bucket, variant).
"""
from __future__ import annotations

import json
import math
import os
import time

SPACE = {
    "frames_per_warp": [4, 8, 16, 32, 64],
    "steal_granularity": [1, 2, 4, 8, 16, 32],
    "donate_every_us": [20, 50, 100, 200, 500],
}
DEFAULT_PATH = os.path.join(os.path.expanduser("~"), ".cache", "sge_autotune.json")


def workload_key(kernel: int, n_t: int, k_max: int, algo: int) -> str:
    """Class of a workload: kernel family, n_t and k rounded to powers of two, variant."""
    nb = 1 << max(0, math.ceil(math.log2(max(1, n_t))))
    kb = 1 << max(0, math.ceil(math.log2(max(1, k_max))))
    return f"kernel{kernel}:n{nb}:k{kb}:algo{algo}"


def coordinate_descent(measure, space=SPACE, start=None, rounds: int = 2):
    """Minimise measure(point) over the grid, one coordinate at a time.

    `measure` returns (seconds, counters); points whose counters differ from
    the first measured point's raise ValueError.  Returns (best point, best
    seconds, table of every measured point)."""
    point = dict(start or {name: values[len(values) // 2] for name, values in space.items()})
    table = {}
    ref = None

    def run(p):
        nonlocal ref
        key = tuple(sorted(p.items()))
        if key not in table:
            secs, counters = measure(dict(p))
            if ref is None:
                ref = counters
            elif counters != ref:
                raise ValueError(f"schedule {p} changed the counters: {counters} != {ref}")
            table[key] = secs
        return table[key]

    best = run(point)
    for _ in range(rounds):
        moved = False
        for name, values in space.items():
            for v in values:
                cand = dict(point, **{name: v})
                t = run(cand)
                if t < best:
                    best, point, moved = t, cand, True
        if not moved:
            break
    return point, best, [{**dict(k), "seconds": v} for k, v in table.items()]


def load(path: str = DEFAULT_PATH) -> dict:
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


def save(cache: dict, path: str = DEFAULT_PATH) -> None:
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def lookup(key: str, path: str = DEFAULT_PATH) -> dict:
    """Tuned options for a workload class ({} if not tuned yet)."""
    return dict(load(path).get(key, {}).get("opts", {}))


def tune_batch(ctx, target_ids, pattern_ids, algo: int = 0, reps: int = 2, path: str | None = DEFAULT_PATH,
               space=SPACE, key: str | None = None) -> dict:
    """Tune the schedule of one batched workload on `ctx` (a Context).

    Each point runs the batch `reps` times after one warm-up call and scores
    the median search-kernel time (CUDA events inside the engine).  Returns
    {"key", "opts", "seconds", "table"} and stores it in the cache at `path`
    (None: do not store)."""
    import numpy as np

    def measure(p):
        ctx.count_batch(target_ids, pattern_ids, algo=algo, **p)
        times = []
        for _ in range(reps):
            rc, rows = ctx.count_batch(target_ids, pattern_ids, algo=algo, **p)
            times.append(float(np.max(rows["search_kernel_ms"])) / 1000.0)
        counters = tuple(int(np.sum(rows[k], dtype=np.uint64)) for k in ("matches", "states", "nodes", "hash"))
        return sorted(times)[len(times) // 2], counters

    t0 = time.perf_counter()
    point, best, table = coordinate_descent(measure, space)
    if key is None:
        rc, rows = ctx.count_batch(target_ids[:1], pattern_ids[:1], algo=algo)
        key = f"kernel{int(rows['kernel'][0])}:algo{algo}:pairs{len(target_ids)}"
    out = {"key": key, "opts": point, "seconds": best, "table": table,
           "tuning_seconds": time.perf_counter() - t0}
    if path:
        cache = load(path)
        cache[key] = {"opts": point, "seconds": best}
        save(cache, path)
    return out
