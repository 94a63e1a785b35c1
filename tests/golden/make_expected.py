"""Admit workload patterns and record the oracle's expected results.

Run:  python tests/golden/make_expected.py [er1000 er2000 cl10k mol200 cl100k]

Calls only the CPU oracle (``oracle/``) and the seeded generators (``gen/``).
It writes

* ``gen/admitted.json`` -- for workloads whose patterns are drawn from
  candidate seeds, the index of the accepted candidate of every slot.  A
  candidate is accepted when its exhaustive search fits the state window of
  its workload (the paper likewise sets aside instances that exceed its time
  limit, Section 5);
* ``tests/golden/expected_<workload>.json`` -- the oracle's counters
  (matches, states, nodes, hash) per instance and algorithm, totals, and for
  the batched workloads a SHA-256 digest of the per-pair counter table.

Nothing here reads or runs the CUDA path.
"""
from __future__ import annotations

import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from gen import configs  # noqa: E402
from gen.patterns import _Adj  # noqa: E402

ER2000_WINDOW = (100_000_000, 2_000_000_000)   # RI-DS-SI-FC states per pattern
CL10K_BUDGET = 1_000_000_000
CL100K_BUDGET = 10_000_000                      # RI states per query
MOL_ALGOS = (0, 3)


def _counters(r) -> dict:
    return {"matches": r["matches"], "states": r["states"], "nodes": r["nodes"], "hash": str(r["hash"])}


def digest(table: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(table, dtype=np.uint64).tobytes()).hexdigest()


def _write(name: str, obj: dict):
    with open(os.path.join(HERE, f"expected_{name}.json"), "w") as f:
        json.dump(obj, f, indent=1)
        f.write("\n")


def _update_admitted(name: str, slots: dict):
    adm = configs.load_admitted()
    adm[name] = {str(k): int(v) for k, v in sorted(slots.items())}
    with open(configs.ADMITTED_PATH, "w") as f:
        json.dump(adm, f, indent=1, sort_keys=True)
        f.write("\n")


# ------------------------------------------------------------------ er1000
def do_er1000():
    w = configs.er1000()
    t, p = w.targets[0], w.patterns[0]
    out = {"target_sha256": t.sha256(), "pattern_sha256": p.sha256(), "algos": {}}
    for a in range(4):
        r = oracle.run(t, p, a, want_matches=True)
        rows = r["match_list"]
        out["algos"][str(a)] = _counters(r)
        out["match_list_sha256"] = hashlib.sha256(np.ascontiguousarray(rows, np.int32).tobytes()).hexdigest()
        out["match_list_len"] = int(rows.shape[0])
    _write("er1000", out)


# ------------------------------------------------------------------ er2000
_G = {}


def _er2000_init():
    t = configs.er2000_target()
    _G["t"] = t
    _G["adj"] = _Adj(t)
    _G["ot"] = oracle.Target(t)


def _er2000_try(args):
    slot, cand, algo, budget = args
    p = configs.er2000_candidate(_G["t"], slot, cand, _G["adj"])
    t0 = time.time()
    r = oracle.run(_G["ot"], p, algo, state_budget=budget)
    return slot, cand, algo, r, time.time() - t0, p.sha256()


def do_er2000(pool_size):
    lo, hi = ER2000_WINDOW
    ctx = mp.get_context("spawn")
    accepted = {}
    tried = {s: [] for s in range(len(configs.ER2000_SIZES))}
    with ctx.Pool(pool_size, initializer=_er2000_init) as pool:
        batch = 0
        while len(accepted) < len(configs.ER2000_SIZES):
            todo = [(s, batch * 8 + j, 3, hi) for s in range(len(configs.ER2000_SIZES)) if s not in accepted
                    for j in range(8)]
            for slot, cand, algo, r, dt, sha in pool.imap_unordered(_er2000_try, todo):
                tried[slot].append((cand, r, dt, sha))
                print(f"er2000 slot {slot} cand {cand}: states {r['states']} over={r['budget_exceeded']} {dt:.1f}s",
                      flush=True)
            for s in tried:
                if s in accepted:
                    continue
                for cand, r, dt, sha in sorted(tried[s], key=lambda x: x[0]):
                    if not r["budget_exceeded"] and lo <= r["states"] <= hi:
                        accepted[s] = (cand, r, dt, sha)
                        break
            batch += 1
        _update_admitted("er2000", {s: accepted[s][0] for s in accepted})
        # the other RI-DS variants (and plain RI when it fits the window's top)
        extra = [(s, accepted[s][0], a, 4 * hi) for s in accepted for a in (0, 1, 2)]
        more = {}
        for slot, cand, algo, r, dt, sha in pool.imap_unordered(_er2000_try, extra):
            more[(slot, algo)] = (r, dt)
            print(f"er2000 slot {slot} algo {algo}: states {r['states']} over={r['budget_exceeded']} {dt:.1f}s",
                  flush=True)
    t = configs.er2000_target()
    out = {"target_sha256": t.sha256(), "window": list(ER2000_WINDOW), "patterns": []}
    for s in sorted(accepted):
        cand, r, dt, sha = accepted[s]
        ent = {"slot": s, "k": configs.ER2000_SIZES[s], "candidate": cand, "pattern_sha256": sha,
               "oracle_seconds": {"3": round(dt, 2)}, "algos": {"3": _counters(r)},
               "order": r["order"].tolist(), "domain_sizes": r["domain_sizes"].tolist()}
        for a in (0, 1, 2):
            ra, dta = more[(s, a)]
            ent["algos"][str(a)] = None if ra["budget_exceeded"] else _counters(ra)
            ent["oracle_seconds"][str(a)] = round(dta, 2)
        out["patterns"].append(ent)
    _write("er2000", out)


# ------------------------------------------------------------------- cl10k
def _cl10k_init():
    t = configs.cl10k_target()
    _G["t"] = t
    _G["adj"] = _Adj(t)
    _G["ot"] = oracle.Target(t)


def _cl10k_try(args):
    slot, cand = args
    p = configs.cl10k_candidate(_G["t"], slot, cand, _G["adj"])
    res = {}
    for a in range(4):
        res[a] = oracle.run(_G["ot"], p, a, state_budget=CL10K_BUDGET)
    return slot, cand, res, p.sha256(), p.m


def do_cl10k(pool_size):
    ctx = mp.get_context("spawn")
    accepted = {}
    with ctx.Pool(pool_size, initializer=_cl10k_init) as pool:
        cand = 0
        while len(accepted) < len(configs.CL10K_SIZES):
            todo = [(s, cand) for s in range(len(configs.CL10K_SIZES)) if s not in accepted]
            for slot, c, res, sha, m in pool.imap_unordered(_cl10k_try, todo):
                if not any(r["budget_exceeded"] for r in res.values()):
                    accepted[slot] = (c, res, sha, m)
            cand += 1
    _update_admitted("cl10k", {s: accepted[s][0] for s in accepted})
    t = configs.cl10k_target()
    out = {"target_sha256": t.sha256(), "patterns": []}
    for s in sorted(accepted):
        c, res, sha, m = accepted[s]
        out["patterns"].append({"slot": s, "k": configs.CL10K_SIZES[s], "edges": m, "candidate": c,
                                "pattern_sha256": sha,
                                "algos": {str(a): _counters(r) for a, r in res.items()}})
    _write("cl10k", out)


# ------------------------------------------------------------------ mol200
def _mol_init():
    ts = configs.mol_targets(200)
    _G["ts"] = ts
    _G["ps"] = configs.mol_patterns(ts, 1000)


def _mol_target(ti):
    ot = oracle.Target(_G["ts"][ti])
    rows = {a: np.zeros((len(_G["ps"]), 4), dtype=np.uint64) for a in MOL_ALGOS}
    for pi, p in enumerate(_G["ps"]):
        for a in MOL_ALGOS:
            r = oracle.run(ot, p, a)
            rows[a][pi] = [r["matches"], r["states"], r["nodes"], r["hash"]]
    return ti, rows


def do_mol200(pool_size):
    ctx = mp.get_context("spawn")
    tables = {a: np.zeros((200 * 1000, 4), dtype=np.uint64) for a in MOL_ALGOS}
    t0 = time.time()
    with ctx.Pool(pool_size, initializer=_mol_init) as pool:
        for ti, rows in pool.imap_unordered(_mol_target, range(200), chunksize=2):
            for a in MOL_ALGOS:
                tables[a][ti * 1000:(ti + 1) * 1000] = rows[a]
    secs = time.time() - t0
    ts = configs.mol_targets(200)
    ps = configs.mol_patterns(ts, 1000)
    h = hashlib.sha256()
    for g in ts + ps:
        h.update(g.sha256().encode())
    out = {"inputs_sha256": h.hexdigest(), "pairs": 200 * 1000, "pair_order": "target-major: pair = t * 1000 + p",
           "oracle_seconds_all_algos": round(secs, 1), "algos": {}}
    for a in MOL_ALGOS:
        tab = tables[a]
        out["algos"][str(a)] = {
            "totals": {"matches": int(tab[:, 0].sum()), "states": int(tab[:, 1].sum()),
                       "nodes": int(tab[:, 2].sum()), "hash": str(int(tab[:, 3].sum(dtype=np.uint64)))},
            "per_pair_sha256": digest(tab),
            "sample_every_997": [[int(x) for x in tab[i]] for i in range(0, tab.shape[0], 997)],
        }
    _write("mol200", out)


# ------------------------------------------------------------------ cl100k
def _cl100k_init():
    t = configs.cl100k_target()
    _G["t"] = t
    _G["adj"] = _Adj(t)
    _G["ot"] = oracle.Target(t)
    _G["ks"] = configs.cl100k_sizes(5000)


def _cl100k_slot(slot):
    k = int(_G["ks"][slot])
    for cand in range(200):
        p = configs.cl100k_candidate(_G["t"], slot, k, cand, _G["adj"])
        r = oracle.run(_G["ot"], p, 0, state_budget=CL100K_BUDGET)
        if not r["budget_exceeded"]:
            return slot, cand, r, p.m
    raise RuntimeError(f"no admissible candidate for slot {slot}")


def do_cl100k(pool_size, count=5000):
    ctx = mp.get_context("spawn")
    res = {}
    t0 = time.time()
    with ctx.Pool(pool_size, initializer=_cl100k_init) as pool:
        for slot, cand, r, m in pool.imap_unordered(_cl100k_slot, range(count), chunksize=4):
            res[slot] = (cand, r, m)
            if len(res) % 250 == 0:
                print(f"cl100k {len(res)}/{count} {time.time() - t0:.0f}s", flush=True)
    _update_admitted("cl100k", {s: res[s][0] for s in res})
    tab = np.zeros((count, 4), dtype=np.uint64)
    for s in range(count):
        r = res[s][1]
        tab[s] = [r["matches"], r["states"], r["nodes"], r["hash"]]
    t = configs.cl100k_target()
    out = {"target_sha256": t.sha256(), "queries": count, "algo": 0, "budget_states": CL100K_BUDGET,
           "rejected_candidates": int(sum(res[s][0] for s in res)),
           "totals": {"matches": int(tab[:, 0].sum()), "states": int(tab[:, 1].sum()),
                      "nodes": int(tab[:, 2].sum()), "hash": str(int(tab[:, 3].sum(dtype=np.uint64)))},
           "per_query_sha256": digest(tab),
           "first_200": [[int(x) for x in tab[i]] for i in range(min(200, count))]}
    _write("cl100k", out)


if __name__ == "__main__":
    which = sys.argv[1:] or ["er1000", "er2000", "cl10k", "mol200", "cl100k"]
    procs = int(os.environ.get("SGE_ORACLE_PROCS", max(1, (os.cpu_count() or 2))))
    for w in which:
        t0 = time.time()
        if w == "er1000":
            do_er1000()
        elif w == "er2000":
            do_er2000(procs)
        elif w == "cl10k":
            do_cl10k(procs)
        elif w == "mol200":
            do_mol200(procs)
        elif w == "cl100k":
            do_cl100k(procs)
        print(f"{w} done in {time.time() - t0:.0f}s", flush=True)
