"""The multi-device path on CPU: two gloo ranks, each counting its shard of
the split frontier, reduce to the unsharded counters.  The per-shard counts
come from the oracle (the GPU test checks the engine's shards against the
same oracle shards), so this exercises the host-side sharding and the
wrapping 64-bit reduction."""
from __future__ import annotations

import os
import socket

import pytest


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, depth, q):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    sys.path.insert(0, os.path.join(root, "tests"))
    import torch.distributed as dist
    import oracle
    from gen import configs
    from paper_1705_09358_gb300.shard import count_sharded
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = configs.er1000()
    t, p = w.targets[0], w.patterns[0]

    def count_fn(shard_index, shard_count, split_depth):
        return oracle.run(t, p, 3, shard=(split_depth, shard_index, shard_count))

    got = count_sharded(count_fn, rank, world, split_depth=depth)
    dist.destroy_process_group()
    q.put((rank, got))


@pytest.mark.parametrize("world,depth", [(2, 1), (2, 3), (3, 2)])
def test_sharded_reduction_equals_whole(world, depth):
    import multiprocessing as mp
    import oracle
    from gen import configs
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, depth, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    results = [q.get(timeout=120) for _ in procs]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    w = configs.er1000()
    whole = oracle.run(w.targets[0], w.patterns[0], 3)
    for rank, got in results:
        assert got == {k: whole[k] for k in ("matches", "states", "nodes", "hash")}, rank


def test_reduction_wraps_like_uint64():
    from paper_1705_09358_gb300.shard import _to_i64, _MASK
    a, b = (1 << 64) - 5, 9
    assert (_to_i64(a) + _to_i64(b)) & _MASK == (a + b) & _MASK
