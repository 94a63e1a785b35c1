"""sge_count_noalloc: counting for callers that cannot allocate device memory.

Such a caller (one whose device memory is owned by its own memory manager,
or whose threads may not call cudaMalloc/cudaFree) keeps the target graph in
device memory it already has and passes it in; the engine carves everything
else from a fixed array in its own device memory.  Here the test allocates
the target with torch, as such a caller's manager would, and checks the
entry point's four counters against sge_count on the same graphs -- exactly,
as every parity test does -- on two calls in a row, since every call reuses
the same fixed array.
"""
from __future__ import annotations

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _device_csr(g):
    """Undirected CSR (rows sorted, each edge in both rows) as device tensors."""
    import torch
    u = np.concatenate([g.src, g.dst]).astype(np.int64)
    v = np.concatenate([g.dst, g.src]).astype(np.int64)
    order = np.lexsort((v, u))
    rowptr = np.zeros(g.n + 1, dtype=np.int64)
    np.add.at(rowptr, u + 1, 1)
    rowptr = np.cumsum(rowptr)
    dev = lambda a: torch.tensor(np.ascontiguousarray(a, dtype=np.int32), device="cuda")
    out = {"rowptr": dev(rowptr), "col": dev(v[order]), "vlabel": dev(g.vlabel)}
    if g.elabel is not None:
        out["elabel"] = dev(np.concatenate([g.elabel, g.elabel])[order])
    return out


def _cases():
    from brute import random_graph, plant_connected
    from gen import configs
    w1 = configs.er1000()
    w3 = configs.cl10k()
    rng = np.random.default_rng(77)
    t = random_graph(rng, 180, 0.08, 3, 3)
    p = plant_connected(rng, t, 6)
    unlab = configs.er1000()
    pl = unlab.patterns[0]
    pl.elabel = np.ones(pl.m, dtype=np.int32)      # labelled pattern, unlabelled target
    return [("er1000", w1.targets[0], w1.patterns[0]), ("cl10k", w3.targets[0], w3.patterns[4]),
            ("labelled", t, p), ("pattern-labels-only", unlab.targets[0], pl)]


@pytest.mark.parametrize("case", range(4))
def test_noalloc_equals_count_on_two_calls(case):
    import torch
    import paper_1705_09358_gb300 as sge
    from gpu_common import engine, counters
    name, t, p = _cases()[case]
    E = engine()
    want = counters(E.count(E.load_target(t), E.load_pattern(p), algo=0))
    d = _device_csr(t)
    eptr = d["elabel"].data_ptr() if "elabel" in d else 0
    stream = torch.cuda.current_stream()
    for call in range(2):
        rc, got = sge.sge_count_noalloc(t.n, d["rowptr"].data_ptr(), d["col"].data_ptr(), d["vlabel"].data_ptr(),
                                        eptr, p, stream=stream)
        assert rc == sge.SGE_OK, (name, call, rc)
        assert counters(got) == want, (name, call)


def test_noalloc_rejects_a_target_beyond_its_fixed_scratch():
    import torch
    import paper_1705_09358_gb300 as sge
    from brute import complete
    n = 2_500_000
    rowptr = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    col = torch.zeros(1, dtype=torch.int32, device="cuda")
    vlabel = torch.zeros(n, dtype=torch.int32, device="cuda")
    rc, got = sge.sge_count_noalloc(n, rowptr.data_ptr(), col.data_ptr(), vlabel.data_ptr(), 0, complete(3))
    assert rc == sge.SGE_ERR_ARG and got["matches"] == 0


def test_noalloc_reads_the_csr_in_order_on_a_nonblocking_stream():
    """A caller that fills its CSR on its own non-blocking stream and calls at once:
    every read the entry point makes of that CSR (including rowptr[n], which a
    labelled pattern on an unlabelled target needs) must wait for the fill.  The
    fill is held back behind a short spin kernel on that stream."""
    import torch
    import paper_1705_09358_gb300 as sge
    from gpu_common import engine, counters
    name, t, p = _cases()[3]          # labelled pattern, unlabelled target
    E = engine()
    want = counters(E.count(E.load_target(t), E.load_pattern(p), algo=0))
    ready = _device_csr(t)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()           # created non-blocking: no implicit order with the legacy stream
    for call in range(2):
        with torch.cuda.stream(s):
            d = {key: torch.full_like(v, -1) for key, v in ready.items()}
            torch.cuda._sleep(20_000_000)             # about 10 ms of device time before the fill
            for key in d:
                d[key].copy_(ready[key])
        rc, got = sge.sge_count_noalloc(t.n, d["rowptr"].data_ptr(), d["col"].data_ptr(), d["vlabel"].data_ptr(),
                                        0, p, stream=s)
        assert rc == sge.SGE_OK, (call, rc)
        assert counters(got) == want, call
        s.synchronize()
