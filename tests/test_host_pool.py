"""CPU check of the host loop runner that batched calls use for their per-pair host work
(job records, orderings, result rows): the pool of worker threads and parallel_for, compiled
here from the library's own source text into a small stress program.  Every index of every
loop must be visited exactly once, for many loop sizes and thread counts, from several host
threads at once, from inside a loop body, after an exception in a loop body, and in a forked
child (which inherits the pool's memory but not its threads)."""
from __future__ import annotations

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HOST_SRC = os.path.join(ROOT, "paper_1705_09358_gb300", "csrc", "sge_host.cpp")

_HEADERS = """#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <cstdio>
#include <exception>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>
#include <sys/wait.h>
#include <unistd.h>
"""

_MAIN = r"""
static int check_loop(int n, int mpt, int tag, std::vector<int> &hits) {
    std::fill(hits.begin(), hits.begin() + n, 0);
    parallel_for(n, [&](int b, int e) {
        for (int i = b; i < e; ++i) __atomic_add_fetch(&hits[i], tag, __ATOMIC_RELAXED);
    }, mpt);
    for (int i = 0; i < n; ++i)
        if (hits[i] != tag) return 1;
    return 0;
}

int main() {
    std::vector<int> hits(1 << 18);
    // many sizes and grain sizes: inline runs, partial pools, every worker busy
    for (int rep = 0; rep < 2000; ++rep) {
        const int n = (rep * 7919) % (1 << 18);
        const int mpt = 1 + (rep * 104729) % 40000;
        if (check_loop(n, mpt, 1 + rep % 5, hits)) { std::printf("loop %d wrong\n", rep); return 1; }
    }
    // concurrent callers (one gets the pool, the others start threads), each nesting a loop
    std::atomic<int> bad{0};
    std::vector<std::thread> callers;
    for (int c = 0; c < 4; ++c)
        callers.emplace_back([&, c] {
            std::vector<int> v(50000);
            for (int rep = 0; rep < 300; ++rep) {
                parallel_for(50000, [&](int b, int e) {
                    for (int i = b; i < e; ++i) v[i] = i + rep + c;
                    if (b == 0) {
                        std::atomic<int> inner{0};
                        parallel_for(4096, [&](int ib, int ie) { inner += ie - ib; }, 256);
                        if (inner != 4096) bad++;
                    }
                }, 1000);
                for (int i = 0; i < 50000; ++i)
                    if (v[i] != i + rep + c) { bad++; break; }
            }
        });
    for (auto &t : callers) t.join();
    if (bad) { std::printf("concurrent callers wrong: %d\n", bad.load()); return 1; }
    // an exception in the caller's own slice reaches the caller after the workers finish
    try {
        parallel_for(100000, [&](int b, int) { if (b == 0) throw 7; }, 1000);
        std::printf("exception lost\n");
        return 1;
    } catch (int x) {
        if (x != 7) return 1;
    }
    if (check_loop(100000, 1000, 3, hits)) { std::printf("pool unusable after an exception\n"); return 1; }
    // a forked child runs its loops on a pool of its own
    const pid_t pid = fork();
    if (pid == 0) _exit(check_loop(100000, 1000, 2, hits) ? 2 : 0);
    int st = 0;
    waitpid(pid, &st, 0);
    if (!WIFEXITED(st) || WEXITSTATUS(st) != 0) { std::printf("forked child wrong\n"); return 1; }
    std::printf("ok\n");
    return 0;
}
"""


def _pool_source() -> str:
    with open(HOST_SRC) as f:
        text = f.read()
    a = text.index("constexpr int HOST_THREADS_MAX")
    b = text.index("void parallel_for(", a)
    end = "\n}\n"
    return text[a:text.index(end, b) + len(end)]


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_parallel_for_visits_every_index_once(tmp_path):
    src = tmp_path / "pool_check.cpp"
    src.write_text(_HEADERS + _pool_source() + _MAIN)
    exe = tmp_path / "pool_check"
    subprocess.run(["g++", "-std=c++17", "-O2", "-pthread", str(src), "-o", str(exe)], check=True,
                   capture_output=True, timeout=300)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
