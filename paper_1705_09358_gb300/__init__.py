"""Python binding of the GB300 subgraph-enumeration engine.

Argument marshalling only: every call goes through the C ABI of
``include/sge.h`` into ``_build/libsge.so``, where all enumeration work runs in
sm_103a CUDA kernels.  There is no CPU fallback: if the library is missing or
no CUDA device is present, the calls raise.

The module exposes the C entry points under their C names (``sge_create``,
``sge_load_target``, ``sge_count`` ...) and a small ``Context`` class on top.
PyTorch is optional: a ``torch.cuda.Stream`` may be handed to ``Context`` so
that the engine runs on the caller's stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import LIB as LIB_PATH

SGE_OK = 0
SGE_ERR_ARG, SGE_ERR_OOM, SGE_ERR_CUDA, SGE_ERR_BUDGET = -1, -2, -3, -4
SGE_ERR_TIMEOUT, SGE_ERR_CANCELLED, SGE_ERR_STOPPED, SGE_ERR_NOT_FOUND = -5, -6, -7, -8
SGE_RI, SGE_RIDS, SGE_RIDS_SI, SGE_RIDS_SI_FC = 0, 1, 2, 3
SGE_KERNEL_AUTO, SGE_KERNEL_CSR, SGE_KERNEL_BITSET = 0, 1, 2
SGE_DOMAIN_AUTO, SGE_DOMAIN_SWEEPS, SGE_DOMAIN_BLOCKS = 0, 1, 2

ERROR_NAMES = {0: "OK", -1: "ARG", -2: "OOM", -3: "CUDA", -4: "BUDGET", -5: "TIMEOUT", -6: "CANCELLED",
               -7: "STOPPED", -8: "NOT_FOUND"}

# every entry point declared in include/sge.h
SYMBOLS = ["sge_create", "sge_destroy", "sge_load_target", "sge_load_pattern", "sge_unload_target",
           "sge_unload_pattern", "sge_count", "sge_enumerate", "sge_count_batch", "sge_serve_submit",
           "sge_serve_poll", "sge_serve_drain", "sge_cancel", "sge_last_error", "sge_version", "sge_count_noalloc",
           "sge_count_batch_ckpt", "sge_resume", "sge_ckpt_info", "sge_free"]


class sge_opts(C.Structure):
    _fields_ = [("algo", C.c_int32), ("split_depth", C.c_int32), ("frames_per_warp", C.c_int32),
                ("steal_granularity", C.c_int32), ("state_budget", C.c_int64), ("time_limit_ms", C.c_int64),
                ("kernel", C.c_int32), ("blocks_per_sm", C.c_int32), ("shard_index", C.c_int32),
                ("shard_count", C.c_int32), ("no_donation", C.c_int32), ("donate_every_iters", C.c_int32),
                ("donate_every_us", C.c_int32), ("domain_fixpoint", C.c_int32), ("frontier_kib", C.c_int32),
                ("reserved", C.c_int32 * 1)]


class sge_result(C.Structure):
    _fields_ = [("matches", C.c_uint64), ("states", C.c_uint64), ("nodes", C.c_uint64), ("hash", C.c_uint64),
                ("preprocess_ms", C.c_double), ("match_ms", C.c_double), ("search_kernel_ms", C.c_double),
                ("frames", C.c_int64), ("donations", C.c_int64), ("alg_bytes", C.c_uint64),
                ("launches", C.c_int64), ("latency_ms", C.c_double), ("split_depth", C.c_int32),
                ("status", C.c_int32), ("kernel", C.c_int32), ("split_kernel_ms", C.c_float),
                ("queue_ms", C.c_float), ("split_exec_ms", C.c_float), ("search_exec_ms", C.c_float),
                ("reserved", C.c_int32 * 1)]


# numpy view of sge_result: batched calls write their results straight into such an array
RESULT_DTYPE = np.dtype(sge_result)


def _result_array(n: int):
    """(numpy array of n sge_result rows, pointer to pass to the library)."""
    out = np.zeros(max(n, 1), dtype=RESULT_DTYPE)
    return out, C.c_void_p(out.ctypes.data)


SINK = C.CFUNCTYPE(C.c_int, C.c_void_p, C.POINTER(C.c_int32), C.c_int64, C.c_int32)

_lib = None


class SgeError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


def load_library(path: str = LIB_PATH):
    """Load libsge.so (built by ``paper_1705_09358_gb300.build``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libsge.so not built ({path}); run `python -m paper_1705_09358_gb300.build`")
    lib = C.CDLL(path)
    P, I32, I64 = C.c_void_p, C.c_int32, C.c_int64
    lib.sge_create.argtypes = [C.POINTER(C.c_void_p), I32, P]
    lib.sge_destroy.argtypes = [P]
    lib.sge_destroy.restype = None
    for fn in (lib.sge_load_target, lib.sge_load_pattern):
        fn.argtypes = [P, I32, I64, P, P, P, P, I32, C.POINTER(I32)]
    lib.sge_unload_target.argtypes = [P, I32]
    lib.sge_unload_pattern.argtypes = [P, I32]
    lib.sge_count.argtypes = [P, I32, I32, C.POINTER(sge_opts), C.POINTER(sge_result)]
    lib.sge_enumerate.argtypes = [P, I32, I32, C.POINTER(sge_opts), SINK, P, C.POINTER(sge_result)]
    lib.sge_count_batch.argtypes = [P, I64, P, P, C.POINTER(sge_opts), P]
    lib.sge_serve_submit.argtypes = [P, I32, I32, C.POINTER(sge_opts), C.POINTER(I64)]
    lib.sge_serve_poll.argtypes = [P, I64, C.POINTER(I32), C.POINTER(sge_result)]
    lib.sge_serve_drain.argtypes = [P]
    lib.sge_count_noalloc.argtypes = [I32, P, P, P, P, I32, I64, P, P, P, P, P, I64, P]
    lib.sge_count_batch_ckpt.argtypes = [P, I64, P, P, C.POINTER(sge_opts), P, C.POINTER(C.c_void_p),
                                         C.POINTER(I64)]
    lib.sge_resume.argtypes = [P, P, I64, C.POINTER(sge_opts), P, C.POINTER(C.c_void_p), C.POINTER(I64)]
    lib.sge_ckpt_info.argtypes = [P, I64, C.POINTER(I64), C.POINTER(I64)]
    lib.sge_free.argtypes = [P]
    lib.sge_free.restype = None
    lib.sge_cancel.argtypes = [P]
    lib.sge_last_error.argtypes = [P]
    lib.sge_last_error.restype = C.c_char_p
    lib.sge_version.argtypes = []
    lib.sge_version.restype = C.c_char_p
    for name in SYMBOLS:
        fn = getattr(lib, name)
        if fn.restype is C.c_int and name not in ("sge_destroy", "sge_free"):
            fn.restype = C.c_int32
    _lib = lib
    return lib


def _i32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.int32)


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def make_opts(**kw) -> sge_opts:
    o = sge_opts()
    for k, v in kw.items():
        setattr(o, k, int(v))
    return o


def result_dict(r: sge_result) -> dict:
    return {"matches": int(r.matches), "states": int(r.states), "nodes": int(r.nodes), "hash": int(r.hash),
            "preprocess_ms": float(r.preprocess_ms), "match_ms": float(r.match_ms),
            "search_kernel_ms": float(r.search_kernel_ms), "frames": int(r.frames),
            "donations": int(r.donations), "alg_bytes": int(r.alg_bytes), "launches": int(r.launches),
            "latency_ms": float(r.latency_ms),
            "split_depth": int(r.split_depth), "status": int(r.status),
            "kernel": int(r.kernel), "split_kernel_ms": float(r.split_kernel_ms), "queue_ms": float(r.queue_ms),
            "split_exec_ms": float(r.split_exec_ms), "search_exec_ms": float(r.search_exec_ms)}


# ----------------------------------------------------------- C-named calls
def sge_version() -> str:
    return load_library().sge_version().decode()


def sge_create(device: int = 0, stream=None) -> C.c_void_p:
    lib = load_library()
    h = C.c_void_p()
    sp = None
    if stream is not None:
        sp = C.c_void_p(int(getattr(stream, "cuda_stream", stream)))
    rc = lib.sge_create(C.byref(h), int(device), sp)
    if rc != SGE_OK:
        raise SgeError(rc, "sge_create failed (no CUDA device?)")
    return h


def sge_destroy(ctx) -> None:
    load_library().sge_destroy(ctx)


def sge_last_error(ctx) -> str:
    return load_library().sge_last_error(ctx).decode(errors="replace")


def _check(ctx, rc, what):
    if rc != SGE_OK:
        raise SgeError(rc, f"{what}: {sge_last_error(ctx)}")


def _load(fn, ctx, n, src, dst, vlabel, elabel, directed):
    src, dst, vl, el = _i32(src), _i32(dst), _i32(vlabel), _i32(elabel)
    out = C.c_int32()
    m = 0 if src is None else int(src.shape[0])
    rc = fn(ctx, int(n), m, _p(src), _p(dst), _p(vl), _p(el), int(bool(directed)), C.byref(out))
    return rc, int(out.value)


def sge_load_target(ctx, n, src, dst, vlabel, elabel=None, directed=False) -> int:
    rc, tid = _load(load_library().sge_load_target, ctx, n, src, dst, vlabel, elabel, directed)
    _check(ctx, rc, "sge_load_target")
    return tid


def sge_load_pattern(ctx, n, src, dst, vlabel, elabel=None, directed=False) -> int:
    rc, pid = _load(load_library().sge_load_pattern, ctx, n, src, dst, vlabel, elabel, directed)
    _check(ctx, rc, "sge_load_pattern")
    return pid


def sge_unload_target(ctx, tid: int) -> None:
    _check(ctx, load_library().sge_unload_target(ctx, int(tid)), "sge_unload_target")


def sge_unload_pattern(ctx, pid: int) -> None:
    _check(ctx, load_library().sge_unload_pattern(ctx, int(pid)), "sge_unload_pattern")


def sge_count(ctx, tid: int, pid: int, opts: sge_opts | None = None, check: bool = True) -> dict:
    r = sge_result()
    rc = load_library().sge_count(ctx, int(tid), int(pid), C.byref(opts) if opts is not None else None, C.byref(r))
    d = result_dict(r)
    d["rc"] = int(rc)
    if check:
        _check(ctx, rc, "sge_count")
    return d


def sge_count_batch(ctx, tids, pids, opts: sge_opts | None = None, check: bool = True):
    """Returns (rc, structured numpy array of sge_result rows)."""
    tids, pids = _i32(tids), _i32(pids)
    n = int(tids.shape[0])
    out, ptr = _result_array(n)
    rc = load_library().sge_count_batch(ctx, n, _p(tids), _p(pids), C.byref(opts) if opts is not None else None, ptr)
    if check:
        _check(ctx, rc, "sge_count_batch")
    return int(rc), out[:n]


def _take_blob(ptr: C.c_void_p, nbytes: C.c_int64):
    """Copy a library-allocated checkpoint blob into bytes and free it (None if there is none)."""
    if not ptr.value:
        return None
    try:
        return C.string_at(ptr.value, int(nbytes.value))
    finally:
        load_library().sge_free(ptr)


_STOPS = (-4, -5, -6)   # BUDGET, TIMEOUT, CANCELLED: the search stopped and left a checkpoint


def sge_count_batch_ckpt(ctx, tids, pids, opts: sge_opts | None = None, check: bool = True):
    """As sge_count_batch; returns (rc, rows, checkpoint bytes or None).

    A stop (budget, time limit, cancel) is not an error here: rc says which,
    rows hold the counters so far and the checkpoint the work left."""
    tids, pids = _i32(tids), _i32(pids)
    n = int(tids.shape[0])
    out, optr = _result_array(n)
    ptr, nbytes = C.c_void_p(), C.c_int64(0)
    rc = load_library().sge_count_batch_ckpt(ctx, n, _p(tids), _p(pids),
                                             C.byref(opts) if opts is not None else None,
                                             optr, C.byref(ptr), C.byref(nbytes))
    blob = _take_blob(ptr, nbytes)
    if check and rc not in _STOPS:
        _check(ctx, rc, "sge_count_batch_ckpt")
    return int(rc), out[:n], blob


def sge_ckpt_info(blob: bytes):
    """(pairs, unexplored frames) recorded in a checkpoint."""
    npairs, nframes = C.c_int64(0), C.c_int64(0)
    rc = load_library().sge_ckpt_info(blob, len(blob), C.byref(npairs), C.byref(nframes))
    if rc != 0:
        raise SgeError(int(rc), "malformed checkpoint")
    return int(npairs.value), int(nframes.value)


def sge_resume(ctx, blob: bytes, opts: sge_opts | None = None, check: bool = True):
    """Continue from a checkpoint; returns (rc, rows with the counters so far, next checkpoint or None)."""
    n, _ = sge_ckpt_info(blob)
    out, optr = _result_array(n)
    ptr, nbytes = C.c_void_p(), C.c_int64(0)
    rc = load_library().sge_resume(ctx, blob, len(blob), C.byref(opts) if opts is not None else None,
                                   optr, C.byref(ptr), C.byref(nbytes))
    nxt = _take_blob(ptr, nbytes)
    if check and rc not in _STOPS:
        _check(ctx, rc, "sge_resume")
    return int(rc), out[:n], nxt


def sge_enumerate(ctx, tid: int, pid: int, opts: sge_opts | None = None, check: bool = True):
    """(result dict, list of int32 arrays of shape (count, k) delivered to the sink)."""
    chunks = []

    def sink(user, ptr, count, k):
        chunks.append(np.ctypeslib.as_array(ptr, shape=(int(count) * int(k),)).reshape(int(count), int(k)).copy())
        return 0

    cb = SINK(sink)
    r = sge_result()
    rc = load_library().sge_enumerate(ctx, int(tid), int(pid), C.byref(opts) if opts is not None else None, cb,
                                      None, C.byref(r))
    d = result_dict(r)
    d["rc"] = int(rc)
    if check:
        _check(ctx, rc, "sge_enumerate")
    return d, chunks


def sge_serve_submit(ctx, tid: int, pid: int, opts: sge_opts | None = None) -> int:
    t = C.c_int64()
    rc = load_library().sge_serve_submit(ctx, int(tid), int(pid), C.byref(opts) if opts is not None else None,
                                         C.byref(t))
    _check(ctx, rc, "sge_serve_submit")
    return int(t.value)


def sge_serve_poll(ctx, ticket: int):
    done = C.c_int32()
    r = sge_result()
    rc = load_library().sge_serve_poll(ctx, int(ticket), C.byref(done), C.byref(r))
    _check(ctx, rc, "sge_serve_poll")
    return (result_dict(r) if done.value else None)


def sge_serve_drain(ctx) -> None:
    _check(ctx, load_library().sge_serve_drain(ctx), "sge_serve_drain")


def sge_count_noalloc(n, d_rowptr, d_col, d_vlabel, d_elabel, pattern, stream=None, time_limit_ms=0):
    """Count with no device allocation (see include/sge.h).

    The target arguments are device addresses (ints, e.g. a tensor's
    ``data_ptr()``; ``d_elabel`` may be 0/None); ``pattern`` has ``n``,
    ``src``, ``dst``, ``vlabel``, ``elabel`` as host arrays.  Returns
    (status, dict of the four counters)."""
    src, dst, vl, el = _i32(pattern.src), _i32(pattern.dst), _i32(pattern.vlabel), _i32(pattern.elabel)
    out = np.zeros(4, dtype=np.uint64)
    sp = None if stream is None else C.c_void_p(int(getattr(stream, "cuda_stream", stream)))
    rc = load_library().sge_count_noalloc(int(n), C.c_void_p(int(d_rowptr or 0)), C.c_void_p(int(d_col or 0)),
                                          C.c_void_p(int(d_vlabel or 0)), C.c_void_p(int(d_elabel or 0)),
                                          int(pattern.n), int(src.shape[0]), _p(src), _p(dst), _p(vl), _p(el), sp,
                                          int(time_limit_ms), _p(out))
    return int(rc), {"matches": int(out[0]), "states": int(out[1]), "nodes": int(out[2]), "hash": int(out[3])}


def sge_cancel(ctx) -> None:
    _check(ctx, load_library().sge_cancel(ctx), "sge_cancel")


# ------------------------------------------------------------- convenience
class Context:
    """Owns one engine context (and with it all device memory of its graphs).

    ``count_batch`` runs a batch with the schedule tuned for its workload class
    (see ``autotune``) unless the call sets a schedule option or passes
    ``tuned=False``; ``autotune_cache`` names the user cache consulted before the
    one shipped with the package (None: only the package cache)."""

    def __init__(self, device: int = 0, stream=None, autotune_cache: str | None = None):
        from . import autotune
        self.h = sge_create(device, stream)
        self.device = device
        self.stream = stream
        self.autotune_cache = autotune_cache if autotune_cache is not None else autotune.DEFAULT_PATH
        # per loaded graph, indexed by its id (ids count up from 0 per context): vertices,
        # edge labels present, directed -- the inputs of a batch's workload class
        self._tn = np.zeros(0, np.int64)
        self._tfl = np.zeros(0, np.int8)     # bit 0: edge-labelled, bit 1: directed
        self._pk = np.zeros(0, np.int64)
        self._pfl = np.zeros(0, np.int8)
        self._tuned = {}      # workload class -> schedule options (looked up once)

    def close(self):
        if self.h:
            sge_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _put(arr, i: int, v):
        if i >= arr.shape[0]:
            arr = np.concatenate([arr, np.zeros(max(i + 1 - arr.shape[0], arr.shape[0], 64), arr.dtype)])
        arr[i] = v
        return arr

    def load_target(self, g) -> int:
        tid = sge_load_target(self.h, g.n, g.src, g.dst, g.vlabel, g.elabel, g.directed)
        lab = g.elabel is not None and bool(np.any(np.asarray(g.elabel)))
        self._tn = self._put(self._tn, tid, int(g.n))
        self._tfl = self._put(self._tfl, tid, int(lab) | (2 if g.directed else 0))
        return tid

    def load_pattern(self, g) -> int:
        pid = sge_load_pattern(self.h, g.n, g.src, g.dst, g.vlabel, g.elabel, g.directed)
        lab = g.elabel is not None and bool(np.any(np.asarray(g.elabel)))
        self._pk = self._put(self._pk, pid, int(g.n))
        self._pfl = self._put(self._pfl, pid, int(lab))
        return pid

    def synchronize(self):
        """Wait for all device work (every engine call already returns with its own work done;
        this also covers work the caller queued with PyTorch)."""
        try:
            import torch
            torch.cuda.synchronize(self.device)
        except Exception:
            pass

    def batch_key(self, tids, pids, algo: int = 0) -> str:
        """Workload class of a batch (see autotune.batch_key).  The last batch's class is
        remembered, so a caller that submits the same id arrays again pays nothing."""
        ident = (id(tids), id(pids), len(tids), len(pids), int(algo))
        last = getattr(self, "_last_key", None)
        if last is not None and last[0] == ident:
            return last[1]
        key = self._batch_key(tids, pids, algo)
        self._last_key = (ident, key)
        return key

    def _batch_key(self, tids, pids, algo: int = 0) -> str:
        from . import autotune
        t = np.asarray(tids)
        p = np.asarray(pids)
        if t.dtype.kind not in "iu":
            t = t.astype(np.int64)
        if p.dtype.kind not in "iu":
            p = p.astype(np.int64)
        if t.size == 0 or t.max() >= self._tn.shape[0] or p.max() >= self._pk.shape[0] or t.min() < 0 or p.min() < 0:
            return autotune.batch_key(int(algo), 0, 0, int(t.size))    # ids this context did not load
        # a batch's targets and patterns are usually few distinct graphs repeated: reduce over
        # the per-id tables restricted to the ids present
        tpres = np.zeros(self._tn.shape[0], bool)
        tpres[t] = True
        ppres = np.zeros(self._pk.shape[0], bool)
        ppres[p] = True
        tf = np.bitwise_or.reduce(self._tfl[tpres]) if tpres.any() else 0
        pf = np.bitwise_or.reduce(self._pfl[ppres]) if ppres.any() else 0
        return autotune.batch_key(int(algo), int(self._tn[tpres].max()), int(self._pk[ppres].max()), int(t.size),
                                  bool((tf | pf) & 1), bool(tf & 2))

    def tuned_schedule(self, tids, pids, algo: int = 0) -> dict:
        """Schedule options tuned for this batch's workload class ({} if none)."""
        from . import autotune
        key = self.batch_key(tids, pids, algo)
        if key not in self._tuned:
            self._tuned[key] = autotune.lookup(key, self.autotune_cache, package=True)
        return dict(self._tuned[key])

    def count(self, tid, pid, check=True, **opts) -> dict:
        return sge_count(self.h, tid, pid, make_opts(**opts), check=check)

    def count_batch(self, tids, pids, check=True, tuned=True, **opts):
        from . import autotune
        if tuned and not (set(opts) & autotune.SCHEDULE_KEYS):
            opts = {**self.tuned_schedule(tids, pids, opts.get("algo", 0)), **opts}
        return sge_count_batch(self.h, tids, pids, make_opts(**opts), check=check)

    def count_batch_ckpt(self, tids, pids, check=True, **opts):
        return sge_count_batch_ckpt(self.h, tids, pids, make_opts(**opts), check=check)

    def resume(self, blob, check=True, **opts):
        return sge_resume(self.h, blob, make_opts(**opts), check=check)

    def enumerate(self, tid, pid, check=True, **opts):
        d, chunks = sge_enumerate(self.h, tid, pid, make_opts(**opts), check=check)
        rows = np.concatenate(chunks) if chunks else np.zeros((0, 0), np.int32)
        if rows.shape[0]:
            rows = rows[np.lexsort(rows.T[::-1])]
        d["match_list"] = rows
        return d

    def serve_submit(self, tid, pid, **opts) -> int:
        return sge_serve_submit(self.h, tid, pid, make_opts(**opts))

    def serve_poll(self, ticket):
        return sge_serve_poll(self.h, ticket)

    def serve_drain(self):
        sge_serve_drain(self.h)

    def cancel(self):
        sge_cancel(self.h)
