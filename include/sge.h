/*
 * sge.h -- C ABI of the GB300 subgraph-enumeration engine.
 *
 * The engine lists every non-induced labelled subgraph isomorphism (Kimmig,
 * Meyerhenke, Strash, "Shared Memory Parallel Subgraph Enumeration", arXiv
 * 1705.09358, Section 2.1, Eqs. 1-3): each injection f of the pattern's
 * vertices into the target's vertices such that every pattern edge (u, v)
 * is carried onto a target edge (f(u), f(v)) with an equal edge label and
 * every pattern vertex onto a target vertex with an equal label.  The
 * search is RI (Section "RI": GreatestConstraintFirst ordering, parent map,
 * pruning rules 1-4) or RI-DS (Section 4: per-pattern-vertex target
 * domains pruned by arc consistency), optionally with the paper's stronger
 * pruning (Section 4.2: domain-size tie-break "SI" and forward checking of
 * singleton domains "FC").  All compute runs in sm_103a CUDA kernels.
 *
 * Conventions for every call:
 *  - Return value: SGE_OK (0) or a negative SGE_ERR_* code.  Nothing is
 *    thrown across the ABI.  sge_last_error() gives a message for the last
 *    failing call on that context.
 *  - Host arrays passed in are borrowed for the duration of the call and
 *    copied; the caller keeps ownership.  All device memory is owned by the
 *    context and freed by sge_destroy().
 *  - A context is used by one host thread at a time, except sge_cancel()
 *    (any thread) and the serving calls (internally synchronised).
 *  - Vertex ids are 0..n-1 (int32).  Labels are arbitrary int32 values
 *    compared for equality; a NULL edge-label array means every edge has
 *    label 0.
 */
#ifndef SGE_H
#define SGE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sge_ctx sge_ctx;
typedef int32_t sge_status;

enum {
    SGE_OK = 0,
    SGE_ERR_ARG = -1,       /* invalid argument or input graph */
    SGE_ERR_OOM = -2,       /* host or device allocation failed */
    SGE_ERR_CUDA = -3,      /* a CUDA call failed (message in sge_last_error) */
    SGE_ERR_BUDGET = -4,    /* opts.state_budget reached; counters are partial */
    SGE_ERR_TIMEOUT = -5,   /* opts.time_limit_ms reached; counters are partial */
    SGE_ERR_CANCELLED = -6, /* sge_cancel() was called; counters are partial */
    SGE_ERR_STOPPED = -7,   /* the match sink asked to stop */
    SGE_ERR_NOT_FOUND = -8  /* unknown target / pattern / ticket id */
};

/* Search variants (Section "RI" and Section 4). */
enum {
    SGE_RI = 0,         /* RI: candidates from V_t or the parent's adjacency */
    SGE_RIDS = 1,       /* RI-DS: domains with arc consistency */
    SGE_RIDS_SI = 2,    /* RI-DS + domain-size tie-break in the ordering */
    SGE_RIDS_SI_FC = 3  /* RI-DS-SI + forward checking of singleton domains */
};

/* Kernel family used for the persistent search. */
enum {
    SGE_KERNEL_AUTO = 0,   /* bitset kernel when the target allows it, else CSR */
    SGE_KERNEL_CSR = 1,    /* candidates streamed from sorted CSR rows */
    SGE_KERNEL_BITSET = 2  /* candidates as word-parallel ANDs of adjacency bitsets */
};

/* Options; a zero field takes its default. */
typedef struct {
    int32_t algo;              /* SGE_RI .. SGE_RIDS_SI_FC (default SGE_RI) */
    int32_t split_depth;       /* depth of the breadth-first split; 0 = auto */
    int32_t frames_per_warp;   /* auto split stops at frames_per_warp x resident warps (default 8) */
    int32_t steal_granularity; /* most frames one donation hands out (default 32 for the bitset
                                  kernel, 2 for the CSR kernel) */
    int64_t state_budget;      /* stop after about this many states of one pair (0 = none) */
    int64_t time_limit_ms;     /* stop after about this much search-kernel time (0 = none);
                                  with either limit set the split stops at the frame
                                  target, so the search kernel, which checks them, does
                                  the bulk of the work */
    int32_t kernel;            /* SGE_KERNEL_* */
    int32_t blocks_per_sm;     /* persistent-kernel blocks per SM (0 = occupancy maximum) */
    int32_t shard_index;       /* multi-device form: this device's shard ... */
    int32_t shard_count;       /* ... of the split frontier (0 or 1 = unsharded) */
    int32_t no_donation;       /* 1 = persistent kernel without work donation */
    int32_t donate_every_iters;/* a warp donates at most once per this many search iterations ... */
    int32_t donate_every_us;   /* ... or once per this many microseconds, whichever comes first
                                  (defaults: CSR kernel 1024 / 500, bitset kernel 2^30 / 50) */
    int32_t domain_fixpoint;   /* RI-DS domains (arc consistency with forward checking, Section 4):
                                  SGE_DOMAIN_SWEEPS = sweeps over the whole device under a host
                                  loop; SGE_DOMAIN_BLOCKS = each pair's whole fixpoint in one block
                                  of one launch (targets of at most 16384 vertices: word by word;
                                  larger ones: over candidate lists); 0 = auto: on targets of at
                                  most 16384 vertices word-by-word blocks from half as many RI-DS
                                  pairs as the device has SMs, candidate-list blocks from 32 pairs,
                                  else sweeps; on larger targets candidate-list blocks always.
                                  All reach the same fixpoint. */
    int32_t frontier_kib;      /* size of each of the breadth-first split's two frontier buffers
                                  in KiB (default 524288 = 512 MiB); a split level whose children
                                  do not fit is not taken, and the search starts from the
                                  frontier as it stands */
    int32_t reserved[1];
} sge_opts;

enum { SGE_DOMAIN_AUTO = 0, SGE_DOMAIN_SWEEPS = 1, SGE_DOMAIN_BLOCKS = 2 };

/* Result of one (target, pattern) search.
 *  matches: number of injections found.
 *  states:  (pattern node, target node) pairs considered = sum over expanded
 *           search nodes of the raw candidate-set size (Section 5, "search
 *           space size").
 *  nodes:   accepted pairs (search-tree nodes below the root, matches included).
 *  hash:    sum over matches of h(f) mod 2^64, with
 *           g(u, v) = fmix64(((u64)u << 32 | v) + 0x9E3779B97F4A7C15) and
 *           h(f) = fmix64(sum_u g(u, f(u))), fmix64 the SplitMix64 finaliser.
 * With shard_count > 1 the counters cover this shard only; summing them over
 * all shards gives the unsharded result. */
typedef struct {
    uint64_t matches, states, nodes, hash;
    double preprocess_ms;    /* domains, ordering, table upload (host clock) */
    double match_ms;         /* split + persistent search (host clock) */
    double search_kernel_ms; /* device time of the persistent search kernel (CUDA events) */
    int64_t frames;          /* frontier frames handed to the persistent kernel */
    int64_t donations;       /* frames donated between warps during the search */
    uint64_t alg_bytes;      /* algorithmic bytes of the persistent search: bitset kernel:
                                sum over expanded nodes of (rows ANDed) x ceil(n_t/64) x 8;
                                CSR kernel: 12 per state (4-byte candidate id + 8-byte
                                label/degree record) */
    int64_t launches;        /* CUDA kernels this call launched */
    double latency_ms;       /* serving: from sge_serve_submit to completion (host clock) */
    int32_t split_depth;     /* depth of that frontier */
    int32_t status;          /* SGE_OK or the error of this pair */
    int32_t kernel;          /* SGE_KERNEL_CSR or SGE_KERNEL_BITSET as used */
    float split_kernel_ms;   /* device time of the breadth-first split kernel (CUDA events; 0 if it
                                did not run as one cooperative launch) */
    float queue_ms;          /* serving: from sge_serve_submit to admission into a launch group */
    float split_exec_ms;     /* the split and search kernels' own spans (device clock, first block's */
    float search_exec_ms;    /* start to last block's end); the event times minus these spans are the
                                time the kernels waited for SMs held by other work */
    int32_t reserved[1];
} sge_result;

/* Match sink: receives `count` matches, each k int32 target ids giving the
 * images of pattern vertices 0..k-1.  The buffer is valid only during the
 * call; calls come from the thread that called sge_enumerate.  Return
 * nonzero to stop the enumeration (sge_enumerate then returns
 * SGE_ERR_STOPPED).  Call order is unspecified. */
typedef int (*sge_match_sink)(void *user, const int32_t *matches, int64_t count, int32_t k);

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * to run on (for example the current PyTorch stream), or NULL for a stream
 * the context creates.  Errors: ARG (bad device), CUDA, OOM. */
sge_status sge_create(sge_ctx **out, int32_t device, void *cuda_stream);

/* Free the context and every device buffer it owns.  NULL is allowed. */
void sge_destroy(sge_ctx *ctx);

/* Load a target graph (Section 2.1).  Edge e is (src[e], dst[e]) with label
 * elabel[e] (NULL = all 0).  Undirected (directed = 0): each edge is given
 * once in either orientation.  The graph is validated, repeated edges with an
 * equal label are merged, and it is copied to device memory as sorted CSR
 * rows (plus an adjacency bitset when small enough).
 * Errors: ARG for n < 0, m < 0, an id out of range, a self-loop, a repeated
 * edge with a different label, or more than 2^31 - 1 stored arcs; OOM; CUDA. */
sge_status sge_load_target(sge_ctx *ctx, int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                           const int32_t *vlabel, const int32_t *elabel, int32_t directed,
                           int32_t *target_id);

/* Load a pattern graph; same arguments and errors as sge_load_target.
 * Patterns have at most 128 vertices (ARG otherwise); the pattern and the
 * target of a search must agree on `directed`. */
sge_status sge_load_pattern(sge_ctx *ctx, int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                            const int32_t *vlabel, const int32_t *elabel, int32_t directed,
                            int32_t *pattern_id);

/* Release a loaded graph.  Waits until the device is idle, then keeps the
 * graph's device blocks in the context (up to 1 GiB) for later loads, which
 * take them instead of allocating; sge_destroy frees them.  NOT_FOUND for an
 * unknown id. */
sge_status sge_unload_target(sge_ctx *ctx, int32_t target_id);
sge_status sge_unload_pattern(sge_ctx *ctx, int32_t pattern_id);

/* Count the matches of pattern `pattern_id` in target `target_id`.
 * opts may be NULL (defaults).  A pattern with no vertices or more vertices
 * than the target has no match and no search (all counters 0).  Errors: ARG,
 * NOT_FOUND, OOM, CUDA, BUDGET / TIMEOUT / CANCELLED (out holds partial
 * counters). */
sge_status sge_count(sge_ctx *ctx, int32_t target_id, int32_t pattern_id, const sge_opts *opts,
                     sge_result *out);

/* As sge_count, and also pass every match to `sink` (called after the device
 * search, in chunks).  Errors as sge_count, plus STOPPED. */
sge_status sge_enumerate(sge_ctx *ctx, int32_t target_id, int32_t pattern_id, const sge_opts *opts,
                         sge_match_sink sink, void *user, sge_result *out);

/* Count `npairs` (target, pattern) pairs in one batched launch sequence: all
 * pairs share one split and one persistent search kernel.  out[i] is the
 * result of pair i (caller-owned array of npairs).  The return value is
 * SGE_OK or the first error; per-pair errors are in out[i].status. */
sge_status sge_count_batch(sge_ctx *ctx, int64_t npairs, const int32_t *target_ids,
                           const int32_t *pattern_ids, const sge_opts *opts, sge_result *out);

/* Checkpoint and resume.  The paper's experiments stop a search at a time
 * limit (Section 5) and lose its work; these calls keep it.
 *
 * sge_count_batch_ckpt counts like sge_count_batch.  When the search stops
 * (state budget, time limit or sge_cancel) it returns BUDGET / TIMEOUT /
 * CANCELLED, out[i] holds pair i's counters so far, and *ckpt receives a
 * host blob of *ckpt_bytes bytes, allocated by the library (free it with
 * sge_free), that records the pairs, the counters and every subtree not yet
 * searched.  When the search finishes it returns SGE_OK and sets
 * *ckpt = NULL, *ckpt_bytes = 0.  Other errors as sge_count_batch (no blob).
 *
 * sge_resume continues from such a blob (the caller keeps ownership of it;
 * it may come from another process or context) on a context that has the
 * same targets and patterns loaded under the same ids.  opts may change the
 * schedule, budget and time limit; the variant (algo) and shard come from
 * the blob.  out (npairs entries, see sge_ckpt_info) receives the counters
 * accumulated over the first call and every resume so far, and *next a new
 * blob if the search stopped again.  Calling sge_resume until it returns
 * SGE_OK gives exactly the counters of one uninterrupted sge_count_batch.
 * Errors: ARG (malformed blob, or ids/sizes that do not match the loaded
 * graphs), and as sge_count_batch.
 *
 * Blob layout (little-endian): header {u64 magic "SGECKPT1", i32 version 1,
 * i32 algo, i64 npairs, i32 ngroups, i32 0}; npairs x {i32 target id,
 * i32 pattern id, i32 n_t, i32 k}; npairs x {u64 matches, states, nodes,
 * hash}; per group (the pairs of one directedness) {i32 kmax, i32 npairs_g,
 * i64 nframes}, npairs_g x i32 pair index (padded to even), nframes frames
 * of 4 + kmax i32: [job, depth | 65536 if the range's nodes were already
 * counted, first, end, image of each of the first depth positions of the
 * pair's search order], where [first, end) is a range of the candidate list
 * of position `depth` (first = -1: the whole list). */
sge_status sge_count_batch_ckpt(sge_ctx *ctx, int64_t npairs, const int32_t *target_ids,
                                const int32_t *pattern_ids, const sge_opts *opts, sge_result *out,
                                void **ckpt, int64_t *ckpt_bytes);
sge_status sge_resume(sge_ctx *ctx, const void *ckpt, int64_t ckpt_bytes, const sge_opts *opts,
                      sge_result *out, void **next, int64_t *next_bytes);
/* Pairs and unexplored frames recorded in a blob (ARG if malformed). */
sge_status sge_ckpt_info(const void *ckpt, int64_t ckpt_bytes, int64_t *npairs, int64_t *nframes);
/* Free a blob returned by sge_count_batch_ckpt or sge_resume (NULL is fine). */
void sge_free(void *p);

/* Serving (continuous batching).  sge_serve_submit queues one query and
 * returns at once with a ticket; scheduler threads owned by the context
 * admit queued queries (up to 64, within a device-memory budget) into
 * the next free launch slot, and each slot runs its admitted group through
 * the batched launch sequence on its own stream, so a group's host work and
 * launches overlap with earlier groups still on the device.
 * sge_serve_poll sets *done = 1 and fills *out once the query finished
 * (out->status holds its own error), else *done = 0.  Errors: ARG,
 * NOT_FOUND. */
sge_status sge_serve_submit(sge_ctx *ctx, int32_t target_id, int32_t pattern_id, const sge_opts *opts,
                            int64_t *ticket);
sge_status sge_serve_poll(sge_ctx *ctx, int64_t ticket, int32_t *done, sge_result *out);
/* Block until every submitted query finished. */
sge_status sge_serve_drain(sge_ctx *ctx);

/* Count without allocating: a variant of sge_count for callers that cannot
 * allocate device memory at the time they search (code under a memory
 * manager that owns every device allocation, an allocator at its limit, or
 * a runtime that forbids cudaMalloc/cudaFree on its threads).  The paper has
 * no counterpart; this is an interface for such callers.
 *
 * The caller passes the inputs and the output: an undirected target already
 * in device memory as CSR (d_rowptr[n+1], d_col[d_rowptr[n]] with every
 * edge stored in both rows and each row sorted ascending, d_vlabel[n],
 * d_elabel parallel to d_col or NULL for all 0), the pattern as host arrays
 * (k <= 128 vertices, m edges as for sge_load_pattern), and out[4] in host
 * memory, which receives matches, states, nodes and hash as sge_count
 * defines them for SGE_RI.  The search is RI on the CSR kernel, started
 * from the root with work donation; it runs on `cuda_stream` (NULL = the
 * default stream) and the call returns once the counters are in `out`.
 * time_limit_ms <= 0 means none.
 *
 * Nothing is allocated: every device-side buffer the search needs (its job
 * record, counters, position tables, root frame, a 2048-frame work queue
 * and the per-vertex label/degree records, 8 bytes per target vertex) is
 * carved from one fixed 16 MiB array in the library's device memory, which
 * every GPU that loads the library holds until the process exits.  A
 * target too large for that array (about 1.9 million vertices; fewer if
 * the pattern has edge labels and the target has none) is rejected with
 * SGE_ERR_ARG before any device work.  The first call on each device looks
 * up that device's copy of the array (cudaGetSymbolAddress, with that device
 * current), so that first call should come before any stream capture begins.
 * All calls share the one array, which keeps the last call's contents; each
 * call clears the parts that must start at zero, so calls must not overlap
 * on the GPU: calls that run at the same time (on different streams or host
 * threads) race and corrupt each other's results.
 *
 * Every device access of the call, including the read of d_rowptr[n] that a
 * labelled pattern on an unlabelled target needs, is ordered on cuda_stream,
 * after whatever the caller queued there before.  The pattern's host-side
 * tables (about 200 KB at 128 vertices) go to one host heap block freed
 * before return, so the call needs only a few KB of the calling thread's
 * stack.
 *
 * Returns SGE_OK, SGE_ERR_ARG (bad arguments or sizes), SGE_ERR_OOM (the
 * host block could not be allocated), SGE_ERR_CUDA, or SGE_ERR_TIMEOUT (out
 * holds partial counters).  The caller's CSR is not validated on the device;
 * ids out of range are undefined behaviour. */
sge_status sge_count_noalloc(int32_t n, const int32_t *d_rowptr, const int32_t *d_col, const int32_t *d_vlabel,
                             const int32_t *d_elabel, int32_t k, int64_t m, const int32_t *src, const int32_t *dst,
                             const int32_t *vlabel, const int32_t *elabel, void *cuda_stream, int64_t time_limit_ms,
                             uint64_t *out);

/* Ask the running search(es) to stop; they return SGE_ERR_CANCELLED.
 * Callable from any thread. */
sge_status sge_cancel(sge_ctx *ctx);

/* Message for the last error on this context (never NULL). */
const char *sge_last_error(sge_ctx *ctx);

/* Library version string. */
const char *sge_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SGE_H */
