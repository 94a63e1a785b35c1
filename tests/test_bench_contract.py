"""The reference arm of bench.py (the oracle on the host cores): one JSON line
with the contract's keys on rank 0, nothing on the other ranks, no GPU needed."""
from __future__ import annotations

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra: dict) -> subprocess.CompletedProcess:
    env = dict(os.environ)
    env.update(env_extra)
    return subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = _run({"RANK": "0", "WORLD_SIZE": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["unit"] == "states/s" and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 3
    assert d["config"]["workload"].startswith("er2000")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_print_nothing():
    r = _run({"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_clock_samples_are_kept_for_the_timed_region_only():
    import datetime
    import tempfile
    sys.path.insert(0, ROOT)
    import bench
    t0 = datetime.datetime(2026, 1, 2, 3, 4, 5, 0)
    lines = []
    for i in range(20):   # one sample every 100 ms from t0 - 0.5 s
        ts = t0 + datetime.timedelta(milliseconds=100 * i - 500)
        idle = i < 5 or i >= 15
        sm = 1000 if idle else 2070
        thermal = "Active" if i == 18 else "Not Active"
        power = "Active" if i == 9 else "Not Active"
        lines.append(f"{ts.strftime('%Y/%m/%d %H:%M:%S.%f')[:-3]}, {sm}, 2070, 0x0, Not Active, {thermal}, "
                     f"Not Active, {power}")
    fd, path = tempfile.mkstemp(suffix=".csv")
    with os.fdopen(fd, "w") as f:
        f.write("\n".join(lines) + "\n")
    c = bench.Clocks(0)
    c.path = path
    c.t0 = t0
    c.t1 = t0 + datetime.timedelta(milliseconds=900)
    s = c.summary()
    # samples 5..14 lie in [t0, t0 + 0.9 s] (50 ms margin): clocks under load, and only their reasons
    assert s["window"] == "timed region" and s["samples"] == 10
    assert s["sm_mhz"] == 2070 and s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_samples_without_a_window_use_the_whole_run():
    import tempfile
    sys.path.insert(0, ROOT)
    import bench
    fd, path = tempfile.mkstemp(suffix=".csv")
    with os.fdopen(fd, "w") as f:
        f.write("not a time, 1800, 2070, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                "garbage line\n")
    c = bench.Clocks(0)
    c.path = path
    s = c.summary()
    assert s["window"] == "whole run" and s["samples"] == 1 and s["sm_mhz"] == 1800 and s["reasons"] == []


def test_search_roofline_follows_the_capture_record():
    """The roofline names instruction issue as the bound, with the peak from the
    device's SM count and the sampled clock; the ncu counts appear only while the
    sources they were taken on are unchanged."""
    sys.path.insert(0, ROOT)
    import bench
    rec = bench._measured_record()
    r = bench.search_roofline(5e-3, 14e9, 17e6, 1800.0, 152)
    assert r["bound"] == "alu" and r["peak"] == 152 * 4 * 1800e6
    assert abs(r["alg_bytes_frac_of_hbm"] - 14e9 / 5e-3 / 1e9 / r["hbm_peak_gbs"]) < 1e-12
    if not rec:   # sources changed since the last capture: nothing measured is claimed
        assert r["frac"] is None and r["traffic"] is None and r["instructions_per_launch"] is None
        return
    assert r["instructions_per_launch"] == int(rec["warp_instructions_per_launch"])
    assert abs(r["frac"] - r["instructions_per_launch"] / 5e-3 / r["peak"]) < 1e-12
    assert r["traffic"] == int(rec["dram_bytes_per_launch"])
    assert abs(r["instructions_per_search_node"] - r["instructions_per_launch"] / 17e6) < 1e-9


def test_capture_record_belongs_to_these_sources():
    """The ncu counts committed under profiles/ were taken on the kernel and schedule sources as
    they stand (their SHA-256 is recorded with them), so the bench line's roofline carries
    measured instruction and traffic counts rather than none."""
    sys.path.insert(0, ROOT)
    import bench
    rec = bench._measured_record()
    assert rec, "profiles/search_kernel_traffic.txt was captured on other sources"
    assert int(rec["warp_instructions_per_launch"]) > 0 and int(rec["dram_bytes_per_launch"]) > 0
