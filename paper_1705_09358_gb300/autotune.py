"""Schedule autotuner: picks split depth, frames per warp, steal granularity and donation cadence.

The search tree is fixed by the method, so every schedule gives the same four
counters; only the time changes.  The tuner times the engine (through the C
ABI) on a caller's workload over a small grid of schedule points by
coordinate descent, keeps the fastest point whose counters equal the
baseline's (a point that changes them is reported as an error, never
chosen), and records it in a JSON cache keyed by the workload class
(`batch_key`: variant, largest target and pattern rounded to powers of two,
batch size rounded to a power of four, edge labels, direction).

`Context.count_batch` looks the class of every call up (the user cache at
DEFAULT_PATH first, then the cache shipped with the package, written by
tuning on a GB300) and runs with the tuned schedule unless the caller sets
a schedule option itself.  The paper's counterpart is the task-group size
of its work-stealing runtime (Section 3), chosen there by a sweep.
"""
from __future__ import annotations

import json
import math
import os
import time

SPACE = {
    "split_depth": [0, 1, 2, 3, 4, 6],     # 0: the library's own split policy
    "frames_per_warp": [4, 8, 16, 32, 64],
    "steal_granularity": [1, 2, 4, 8, 16, 32],
    "donate_every_us": [20, 50, 100, 200, 500],
}
# options that make up a schedule: a call that sets any of them is not given a tuned one
SCHEDULE_KEYS = frozenset(SPACE) | {"donate_every_iters", "blocks_per_sm", "no_donation"}
DEFAULT_PATH = os.path.join(os.path.expanduser("~"), ".cache", "sge_autotune.json")
PACKAGE_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "autotune_cache.json")


def workload_key(kernel: int, n_t: int, k_max: int, algo: int) -> str:
    """Class of a workload: kernel family, n_t and k rounded to powers of two, variant."""
    nb = 1 << max(0, math.ceil(math.log2(max(1, n_t))))
    kb = 1 << max(0, math.ceil(math.log2(max(1, k_max))))
    return f"kernel{kernel}:n{nb}:k{kb}:algo{algo}"


def _pow_bucket(x: int, base: int) -> int:
    b = 1
    while b < x:
        b *= base
    return b


def batch_key(algo: int, n_max: int, k_max: int, npairs: int, labelled: bool = False,
              directed: bool = False) -> str:
    """Class of a batched call: variant, largest target and pattern (powers of two), number of
    pairs (power of four), edge labels, direction."""
    return (f"algo{algo}:n{_pow_bucket(max(1, n_max), 2)}:k{_pow_bucket(max(1, k_max), 2)}:"
            f"pairs{_pow_bucket(max(1, npairs), 4)}:{'dir' if directed else 'und'}:{'elab' if labelled else 'plain'}")


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


def lookup(key: str, path: str = DEFAULT_PATH, package: bool = False) -> dict:
    """Tuned options for a workload class ({} if not tuned yet): from the cache at `path`,
    else (with `package`) from the cache shipped with the package."""
    hit = load(path).get(key) if path else None
    if hit is None and package:
        hit = load(PACKAGE_CACHE).get(key)
    return dict((hit or {}).get("opts", {}))


MIN_GAIN = 0.03   # a tuned point must beat the library defaults by this fraction to be kept


def tune_batch(ctx, target_ids, pattern_ids, algo: int = 0, reps: int = 5, path: str | None = DEFAULT_PATH,
               space=SPACE, key: str | None = None, rounds: int = 2) -> dict:
    """Tune the schedule of one batched workload on `ctx` (a Context).

    Each point runs the batch `reps` times after one warm-up call and scores
    the median time of the whole call (host clock around it, device synchronised:
    domains, split and search, which is what a caller waits for).  The best point
    is then timed again against the defaults and kept only if it is at least
    MIN_GAIN faster (else the defaults stand: most apparent gains of a few percent
    are run-to-run noise).  Returns {"key", "opts", "seconds", "default_seconds",
    "table"} and stores the point in the cache at `path` (None: do not store)
    under the call's workload class."""
    import numpy as np

    def measure(p):
        opts = {k: v for k, v in p.items() if v != 0}
        ctx.count_batch(target_ids, pattern_ids, algo=algo, tuned=False, **opts)
        times = []
        for _ in range(reps):
            ctx.synchronize()
            t0 = time.perf_counter()
            rc, rows = ctx.count_batch(target_ids, pattern_ids, algo=algo, tuned=False, **opts)
            ctx.synchronize()
            times.append(time.perf_counter() - t0)
        counters = tuple(int(np.sum(rows[k], dtype=np.uint64)) for k in ("matches", "states", "nodes", "hash"))
        return sorted(times)[len(times) // 2], counters

    t0 = time.perf_counter()
    start = {name: (0 if name == "split_depth" else values[len(values) // 2]) for name, values in space.items()}
    defaults = {name: 0 for name in space}
    default_s, ref = measure(defaults)

    def checked(p):
        secs, counters = measure(p)
        if counters != ref:
            raise ValueError(f"schedule {p} changed the counters: {counters} != {ref}")
        return secs, counters

    point, best, table = coordinate_descent(checked, space, start=start, rounds=rounds)
    # confirm against the defaults, interleaved, before keeping a point
    if point != defaults:
        a, b = [], []
        for _ in range(3):
            a.append(measure(point)[0])
            b.append(measure(defaults)[0])
        best, default_s = sorted(a)[1], sorted(b)[1]
    if best > default_s * (1.0 - MIN_GAIN):
        point, best = defaults, default_s
    if key is None:
        key = ctx.batch_key(target_ids, pattern_ids, algo)
    out = {"key": key, "opts": {k: v for k, v in point.items() if v != 0}, "seconds": best,
           "default_seconds": default_s, "table": table, "tuning_seconds": time.perf_counter() - t0}
    if path:
        cache = load(path)
        cache[key] = {"opts": out["opts"], "seconds": best, "default_seconds": default_s}
        save(cache, path)
    return out
