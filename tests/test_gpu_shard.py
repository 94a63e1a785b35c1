"""The multi-device form with the engine doing the counting: each shard of the
split frontier (frame i to shard i mod S) is searched through the C ABI and
reduced by shard.count_sharded over a one-rank gloo group, and the shard sums
equal the unsharded counters that the oracle stored (tests/golden)."""
from __future__ import annotations

import os
import socket

import pytest

from gen import configs
from gpu_common import engine, golden

pytestmark = pytest.mark.gpu

KEYS = ("matches", "states", "nodes", "hash")


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


@pytest.fixture(scope="module")
def one_rank_group():
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(_free_port())
    dist.init_process_group("gloo", rank=0, world_size=1)
    yield
    dist.destroy_process_group()


@pytest.mark.parametrize("name,kernel", [("er2000", 2), ("er2000", 1), ("cl10k", 0)])
def test_engine_shards_through_count_sharded(one_rank_group, name, kernel):
    from paper_1705_09358_gb300.shard import count_sharded
    w = configs.BUILDERS[name]()
    g = golden(name)
    E = engine()
    tid = E.load_target(w.targets[0])
    pids = [E.load_pattern(p) for p in w.patterns]
    want = [0, 0, 0, 0]
    for ent in g["patterns"]:
        for i, k in enumerate(KEYS):
            want[i] = (want[i] + int(ent["algos"]["3"][k])) % (1 << 64)

    def count_fn(shard_index, shard_count, split_depth):
        rc, rows = E.count_batch([tid] * len(pids), pids, algo=3, kernel=kernel, shard_index=shard_index,
                                 shard_count=shard_count, split_depth=split_depth)
        return {k: int(rows[k].sum()) % (1 << 64) for k in KEYS}

    for count in (2, 3):
        for depth in (1, 2):
            tot = [0, 0, 0, 0]
            for s in range(count):
                got = count_sharded(count_fn, s, count, split_depth=depth)
                for i, k in enumerate(KEYS):
                    tot[i] = (tot[i] + got[k]) % (1 << 64)
            assert tot == want, (count, depth)
