#!/usr/bin/env python
"""Throughput benchmark: search states/sec (and matches/sec) on one GB300.

Default workload (the dense RI-DS configuration): target G(2000, 0.05) with
4 uniform vertex labels, five dense-walk patterns of 16, 18, 20, 22 and 24
vertices, RI-DS-SI-FC.  One step = one batched launch sequence over the five
(target, pattern) pairs through the C ABI: domains (init, arc consistency,
forward checking), ordering, breadth-first split and the persistent search.
Inputs are resident in device memory before timing; L2 is flushed (256 MB
write) between timed steps.  The line also carries the end-to-end number
(host buffers in, results out, through the public API), the roofline of the
persistent search kernel, the CPU oracle on a bounded sample, and the
batched-vs-per-query speedup on a sample of the molecule workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With N > 1 (torchrun, one rank per GPU) every rank runs its own replica of
the workload (weak scaling); ranks exchange only the timing maximum.
"""
from __future__ import annotations

import argparse
import datetime
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "search states/sec and matches/sec on 1 GB300; batched vs per-query speedup"
UNIT = "states/s"
WORKLOAD = ("er2000: ER G(2000, p=0.05) target, 4 uniform vertex labels, 5 dense-walk patterns "
            "(16, 18, 20, 22, 24 vertices), RI-DS-SI-FC, all five pairs per step in one batched launch sequence")
ALGO = 3


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples of the SM clock, its maximum and the throttle reasons, kept
    for the timed region only: each sample carries nvidia-smi's timestamp, compared
    with the host clock at the region's start and end (same host, local time)."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None
        self.t0 = self.t1 = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            # let the sampler write its first line before the timed region starts (2 s at most)
            limit = time.time() + 2.0
            while time.time() < limit and self.proc.poll() is None and os.path.getsize(self.path) == 0:
                time.sleep(0.02)
        except Exception:
            self.proc = None
        return self

    def start(self):
        self.t0 = datetime.datetime.now()

    def stop(self):
        self.t1 = datetime.datetime.now()

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self) -> dict:
        rows = []   # (time or None, sm MHz, max MHz, active reasons)
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [x.strip() for x in line.split(",")]
                    if len(parts) < 8:
                        continue
                    try:
                        sm, mx = float(parts[1]), float(parts[2])
                    except ValueError:
                        continue
                    try:
                        ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f")
                    except ValueError:
                        ts = None
                    act = {nm for nm, v in zip(self.REASONS, parts[4:8]) if v.lower() == "active"}
                    rows.append((ts, sm, mx, act))
            os.unlink(self.path)
        except Exception:
            pass
        window = "whole run"
        if self.t0 is not None and self.t1 is not None:
            pad = datetime.timedelta(milliseconds=50)
            inside = [r for r in rows if r[0] is not None and self.t0 - pad <= r[0] <= self.t1 + pad]
            if inside:
                rows, window = inside, "timed region"
        sm = [r[1] for r in rows]
        reasons = set().union(*[r[3] for r in rows]) if rows else set()
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(r[2] for r in rows) if rows else None,
                "samples": len(rows), "window": window, "reasons": sorted(reasons)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    return world, rank, local


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    import torch
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()


# ----------------------------------------------------------- CPU oracle leg
def oracle_sample(workload, budget_per_pattern: int) -> dict:
    """The oracle as it stands, one thread, on every pattern with a state budget."""
    import oracle
    t = workload.targets[0]
    ot = oracle.Target(t)
    states = matches = 0
    t0 = time.perf_counter()
    for p in workload.patterns:
        r = oracle.run(ot, p, ALGO, state_budget=budget_per_pattern)
        states += r["states"]
        matches += r["matches"]
    dt = time.perf_counter() - t0
    return {"states": states, "matches": matches, "seconds": dt}


def run_reference(args, world, rank):
    from gen import configs
    if rank != 0:
        return
    w = configs.er2000()
    budget = 10_000_000
    for _ in range(args.warmup):
        oracle_sample(w, budget)
    tot_s = tot_t = tot_m = 0.0
    for _ in range(args.steps):
        r = oracle_sample(w, budget)
        tot_s += r["states"]
        tot_m += r["matches"]
        tot_t += r["seconds"]
    value = tot_s / tot_t
    sample = f"each step: the oracle on all 5 patterns, each stopped after {budget} states (bounded sample)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": {"workload": WORKLOAD},
            "matches_per_sec": tot_m / tot_t,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "search_kernel_traffic.txt")
# the sources whose change invalidates the recorded per-launch counts: the kernels and the host
# code that sets the search schedule (split depth, frames, donation cadence)
COUNTED_SOURCES = [os.path.join(ROOT, "paper_1705_09358_gb300", "csrc", f)
                   for f in ("sge_kernels.cu", "sge_internal.h", "sge_host.cpp")]


def sources_sha256() -> str:
    import hashlib
    h = hashlib.sha256()
    for path in COUNTED_SOURCES:
        with open(path, "rb") as f:
            h.update(hashlib.sha256(f.read()).digest())
    return h.hexdigest()


def _measured_record() -> dict:
    """Per search-kernel launch, from the last ncu capture of this workload: DRAM bytes
    (read + write) and warp instructions executed; empty when the kernel or schedule
    sources have changed since that capture."""
    try:
        rec = dict(line.strip().split("=", 1) for line in open(TRAFFIC_FILE)
                   if "=" in line and not line.startswith("#"))
        src = sources_sha256()
    except OSError:
        return {}
    if rec.get("sources_sha256") != src:
        return {}
    return rec


WARP_SCHEDULERS_PER_SM = 4   # each issues at most one warp instruction per cycle


def search_roofline(kernel_s: float, alg_bytes: float, nodes: float, sm_mhz, sms: int) -> dict:
    """Roofline of the persistent bitset search kernel (one launch per step).

    The kernel's data (adjacency bitset, domains, frames) is L2-resident, so
    DRAM moves a few MB per launch while the algorithmic bytes are ~14 GB; the
    binding resource is instruction issue.  achieved = warp instructions of one
    launch (ncu count of the current sources) / the live CUDA-event time of one
    launch; peak = SMs x 4 schedulers x 1 warp instruction per cycle x the
    median SM clock sampled in the timed region.  The bytes-based figures stay
    beside it as secondary fields."""
    hbm, hbm_kind = _peaks()
    rec = _measured_record()
    traffic = int(rec["dram_bytes_per_launch"]) if "dram_bytes_per_launch" in rec else None
    inst = int(rec["warp_instructions_per_launch"]) if "warp_instructions_per_launch" in rec else None
    mhz = float(sm_mhz) if sm_mhz else 2070.0
    peak = sms * WARP_SCHEDULERS_PER_SM * mhz * 1e6
    alg_gbs = alg_bytes / kernel_s / 1e9
    out = {"bound": "alu", "limiter": "warp-instruction issue (data L2-resident)",
           "achieved": inst / kernel_s if inst else None, "peak": peak, "unit": "warp instructions/s",
           "frac": inst / kernel_s / peak if inst else None, "traffic": traffic,
           "kernel": "k_search_bits<1> (persistent bitset search)", "kernel_ms_per_launch": kernel_s * 1e3,
           "instructions_per_launch": inst, "instructions_per_search_node": inst / nodes if inst and nodes else None,
           "peak_kind": f"{sms} SMs x {WARP_SCHEDULERS_PER_SM} schedulers x 1 warp instruction/cycle x "
                        f"{mhz:.0f} MHz (median SM clock in the timed region)",
           "frac_at_max_clock": inst / kernel_s / (sms * WARP_SCHEDULERS_PER_SM * 2070e6) if inst else None,
           "alg_bytes_per_launch": alg_bytes, "alg_bytes_gbs": alg_gbs, "alg_bytes_frac_of_hbm": alg_gbs / hbm,
           "dram_gbs": traffic / kernel_s / 1e9 if traffic else None,
           "dram_frac_of_hbm": traffic / kernel_s / 1e9 / hbm if traffic else None,
           "hbm_peak_gbs": hbm, "hbm_peak_kind": f"of {hbm_kind} HBM copy"}
    return out


def run_ours(args, world, rank, local):
    import torch
    import paper_1705_09358_gb300 as sge
    from gen import configs
    sge.build.build()
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    w = configs.er2000()
    t = w.targets[0]
    E = sge.Context(local, stream=stream)
    tid = E.load_target(t)
    pids = [E.load_pattern(p) for p in w.patterns]
    tids = [tid] * len(pids)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{local}")

    def step():
        rc, rows = E.count_batch(tids, pids, algo=ALGO)
        return rows

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    barrier(world)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    states = matches = alg_bytes = launches = nodes = 0
    kernel_ms = 0.0
    kernel_launches = 0
    with Clocks(local) as clk:
        clk.start()
        with torch.cuda.stream(stream):
            for i in range(args.steps):
                flush.zero_()                       # evict L2 between timed steps
                ev[i][0].record(stream)
                rows = step()
                ev[i][1].record(stream)
                states += int(rows["states"].sum())
                matches += int(rows["matches"].sum())
                alg_bytes += int(rows["alg_bytes"].sum())
                nodes += int(rows["nodes"].sum())
                launches += int(rows["launches"][0])
                kernel_ms += float(rows["search_kernel_ms"][0])
                kernel_launches += 1
        barrier(world)
        clk.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = sum(step_ms) / 1000.0
    total_s = max_over_ranks(total_s, world)
    value = world * states / total_s
    clocks = clk.summary()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    roofline = search_roofline(kernel_ms / kernel_launches / 1000.0, alg_bytes / kernel_launches,
                               nodes / kernel_launches, clocks.get("sm_mhz"), sms)

    # ------------------------------------------------------ end to end
    def pinned(a):
        """The array staged in pinned host memory (the step's inputs are copied from there)."""
        if a is None:
            return None
        buf = torch.empty(a.shape, dtype=torch.int32, pin_memory=True)
        buf.numpy()[...] = a
        return buf.numpy()

    tp = (pinned(t.src), pinned(t.dst), pinned(t.vlabel), pinned(t.elabel))
    srcs = [(p.n, pinned(p.src), pinned(p.dst), pinned(p.vlabel), pinned(p.elabel)) for p in w.patterns]
    h2d = 4 * (t.src.size + t.dst.size + t.vlabel.size) + sum(4 * (s.size + d.size + v.size) for _, s, d, v, _ in srcs)
    d2h = len(w.patterns) * 128
    e2e_steps = max(3, args.steps // 2)
    e2e_states = 0
    barrier(world)
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for _ in range(e2e_steps):
            flush.zero_()
            tt = sge.sge_load_target(E.h, t.n, tp[0], tp[1], tp[2], tp[3], False)
            pp = [sge.sge_load_pattern(E.h, n, s, d, v, e, False) for n, s, d, v, e in srcs]
            rc, rows = E.count_batch([tt] * len(pp), pp, algo=ALGO)
            e2e_states += int(rows["states"].sum())
            for x in pp:
                sge.sge_unload_pattern(E.h, x)
            sge.sge_unload_target(E.h, tt)
    barrier(world)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    e2e = {"value": world * e2e_states / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(d2h),
           "note": "sge_load_target (device ingest) + 5 x sge_load_pattern from pinned host arrays, "
                   "sge_count_batch, results to host, unload"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * total_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "l2": "flushed between timed steps (256 MB write)",
                       "parallelism": f"replicas x{world}"},
            "matches_per_sec": world * matches / total_s,
            "states_per_step": states // args.steps, "matches_per_step": matches // args.steps,
            "gpu_launches": launches, "roofline": roofline, "e2e": e2e}
    if rank == 0 and world == 1 and not args.no_extras:
        line["batched_vs_per_query"] = batched_vs_per_query(E, args)
        line["serving"] = serving_latency(E)
        smp = oracle_sample(w, 200_000_000)
        line["cpu_baseline"] = {"value": smp["states"] / smp["seconds"], "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": "the oracle (one thread) on all 5 patterns, each stopped after 2e8 states; "
                                          f"{smp['states']} states in {smp['seconds']:.1f} s"}
    line["clocks"] = clocks
    E.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def batched_vs_per_query(E, args) -> dict:
    """Molecule workload: all 200,000 (target, pattern) pairs in one batched
    call vs one call per pair (per-pair rate from an evenly spaced sample)."""
    import torch
    from gen import configs
    ts = configs.mol_targets(200)
    ps = configs.mol_patterns(ts, 1000)
    tids = [E.load_target(t) for t in ts]
    pids = [E.load_pattern(p) for p in ps]
    T = np.repeat(np.array(tids, np.int32), len(pids))
    P = np.tile(np.array(pids, np.int32), len(tids))
    E.count_batch(T[:4096], P[:4096])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc, rows = E.count_batch(T, P)
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0
    sb = int(rows["states"].sum())
    idx = np.arange(0, len(T), 100)
    t0 = time.perf_counter()
    s1 = 0
    for i in idx:
        s1 += E.count(int(T[i]), int(P[i]))["states"]
    torch.cuda.synchronize()
    t1 = time.perf_counter() - t0
    b_rate, q_rate = sb / tb, s1 / t1
    return {"workload": "mol200: 200 molecule-shaped targets x 1000 patterns, RI, all 200,000 pairs",
            "pairs_batched": int(len(T)), "batched_seconds": tb, "batched_states_per_s": b_rate,
            "pairs_per_query_sample": int(len(idx)), "per_query_ms_per_pair": 1000.0 * t1 / len(idx),
            "per_query_states_per_s": q_rate, "speedup": b_rate / q_rate}


def serving_latency(E, n_queries: int = 1000) -> dict:
    """Serving on the 100k-vertex power-law target: queries arrive as a
    Poisson stream and are admitted by the engine's continuous-batching
    scheduler; latency is submit-to-completion.  The offered load is 0.8 x
    the serving path's own saturation throughput (every query submitted at
    once); the batched and one-query-per-call rates are reported beside it."""
    from gen import configs
    t = configs.cl100k_target()
    w = configs.cl100k(count=n_queries, target=t)
    tid = E.load_target(t)
    pids = [E.load_pattern(p) for p in w.patterns]
    n = len(pids)
    E.count_batch([tid] * 64, pids[:64])
    t0 = time.perf_counter()
    rc, rows = E.count_batch([tid] * n, pids)
    tb = time.perf_counter() - t0
    total_states = int(rows["states"].sum())
    # one query per call, back to back, on an evenly spaced sample
    sample = list(range(0, n, 5))
    t0 = time.perf_counter()
    s_seq = sum(E.count(tid, pids[i])["states"] for i in sample)
    t_seq = time.perf_counter() - t0
    # warm the scheduler threads, then measure saturation
    for tk in [E.serve_submit(tid, pids[i]) for i in range(8)]:
        pass
    E.serve_drain()
    t0 = time.perf_counter()
    sat = [E.serve_submit(tid, pid) for pid in pids]
    E.serve_drain()
    t_sat = time.perf_counter() - t0
    for tk in sat:
        E.serve_poll(tk)
    lam = 0.8 * n / t_sat
    arrivals = configs.cl100k_arrivals(n, lam)
    tickets = []
    start = time.perf_counter()
    for i in range(n):
        due = start + float(arrivals[i])
        while True:
            now = time.perf_counter()
            if now >= due:
                break
            if due - now > 0.0005:
                time.sleep(due - now - 0.0003)
        tickets.append(E.serve_submit(tid, pids[i]))
    E.serve_drain()
    makespan = time.perf_counter() - start
    res = [E.serve_poll(tk) for tk in tickets]
    lat = np.array([r["latency_ms"] for r in res])
    bad = sum(1 for r in res if r["status"] != 0)
    bad_status = sorted({int(r["status"]) for r in res if r["status"] != 0})
    served_states = sum(r["states"] for r in res)
    return {"workload": f"cl100k: Chung-Lu n=100,000 target, first {n} of the 5000 queries (8-128 vertices), RI",
            "queries": n, "arrival": "Poisson", "offered_qps": lam,
            "offered_load": "0.8 x serving saturation throughput", "saturation_qps": n / t_sat,
            "batched_qps": n / tb, "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "errors": bad, "error_statuses": bad_status,
            "served_states_per_s": served_states / makespan,
            "makespan_s": makespan, "batched_states_per_s": total_states / tb,
            "sequential_per_query_states_per_s": s_seq / t_seq,
            "served_vs_sequential": (served_states / makespan) / (s_seq / t_seq)}


def run_ablation(args):
    """The paper's variant comparison (Section 5: RI-DS vs RI-DS-SI vs RI-DS-SI-FC,
    search-space size and time) re-created on the synthetic workloads; one
    JSON line per (workload, variant)."""
    import torch
    import paper_1705_09358_gb300 as sge
    from gen import configs
    sge.build.build()
    E = sge.Context(0)
    names = {0: "RI", 1: "RI-DS", 2: "RI-DS-SI", 3: "RI-DS-SI-FC"}
    t5 = configs.cl100k_target()
    cases = [("er2000", configs.er2000()), ("cl10k", configs.cl10k()),
             ("cl100k-200", configs.cl100k(count=200, target=t5))]
    for wname, w in cases:
        tid = E.load_target(w.targets[0])
        pids = [E.load_pattern(p) for p in w.patterns]
        for algo in range(4):
            E.count_batch([tid] * len(pids), pids, algo=algo)
            best = None
            for _ in range(3):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rc, rows = E.count_batch([tid] * len(pids), pids, algo=algo)
                dt = time.perf_counter() - t0
                if best is None or dt < best[0]:
                    best = (dt, rows)
            dt, rows = best
            print(json.dumps({"ablation": wname, "variant": names[algo], "pairs": len(pids),
                              "states": int(rows["states"].sum()), "nodes": int(rows["nodes"].sum()),
                              "matches": int(rows["matches"].sum()), "seconds": dt,
                              "preprocess_ms": float(rows["preprocess_ms"][0]),
                              "search_kernel_ms": float(rows["search_kernel_ms"][0]),
                              "states_per_s": int(rows["states"].sum()) / dt}), flush=True)
    E.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip the CPU baseline and batched comparison")
    ap.add_argument("--ablation", action="store_true", help="variant comparison instead of the throughput line")
    args = ap.parse_args()
    if args.ablation:
        run_ablation(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        # the oracle runs on the host cores of rank 0 alone; no device, no process group
        world = int(os.environ.get("WORLD_SIZE", "1"))
        rank = int(os.environ.get("RANK", "0"))
        run_reference(args, world, rank)
        return
    world, rank, local = dist_setup()
    run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
