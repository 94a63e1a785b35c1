// sge_internal.h -- device-side tables shared by the host and kernel units.
//
// Layout in HBM (all owned by the context):
//   target:  CSR rows sorted ascending (int32 offsets `rowptr[n+1]`, int32
//            neighbours `col`, int32 edge labels `elab`), `vld[n]` = {label,
//            out-degree} as one 8-byte gather, in-rows for directed graphs,
//            and for small undirected targets an n x dw adjacency bitset
//            (dw = ceil(n / 64) 64-bit words per row).
//   pattern: vertex-indexed label / degree arrays and CSR rows (used by the
//            domain kernels), plus per-search "position tables" (PosInfo,
//            BackEdge) built on the host from the ordering.
//   filter:  per (job, pattern vertex) a dw-word bitset over target vertices:
//            the RI-DS domain D(v) (Section 4) or, for RI, the label/degree
//            filter of rules 2-3.
//   frames:  int32 records [job, depth, begin, end, M_0 .. M_{depth-1}].
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace sge {

constexpr int KMAX = 128;            // largest pattern handled by the kernels
constexpr int FRAME_HDR = 4;         // job, depth, begin, end
constexpr int POOL_STRIDE = FRAME_HDR + KMAX;
// Flag in a frame's depth word: the frame is the remainder [begin, end) of a
// node's candidate range whose accepted nodes (and the node's states) were
// already counted when the candidates were first tested; it only re-derives
// the survivors to search below them.  Checkpoints write such frames.
constexpr int FRAME_COUNTED = 1 << 16;
constexpr int FRAME_DEPTH_MASK = FRAME_COUNTED - 1;

// PosInfo.flags
constexpr int POS_IN_ROW = 1;        // candidates come from the parent's in-row (directed)

// JobDesc.flags
constexpr int JOB_RIDS = 1;          // test v_t in D(mu_i) for every candidate
constexpr int JOB_ELAB = 2;          // compare edge labels
constexpr int JOB_DIRECTED = 4;
constexpr int JOB_FC = 8;            // forward checking of singleton domains
// Arc-consistency sweep entries {job, pattern vertex (| AC_ENT_DENSE), global vertex, list start}:
// AC_ENT_DENSE marks a vertex whose pattern neighbours' domains are all dense (see k_domain_ac_cand)
constexpr int AC_ENT_DENSE = 1 << 16;
constexpr int AC_DENSE = 8;           // dense: a domain holding at least 1/AC_DENSE of the target
constexpr int JOB_LONG_LISTS = 16;   // some position after the first may have more than SPLIT_RANGE candidates

// The breadth-first split writes a child whose candidate list is longer than
// this as range frames of this many candidates each.
constexpr int SPLIT_RANGE = 256;

// One search position i of a job: pattern vertex mu_i and its constraints.
struct PosInfo {
    int32_t pv;     // mu_i
    int32_t par;    // position of P(mu_i), or -1 when unparented
    int32_t lab;    // lab(mu_i)
    int32_t odeg;   // out-degree of mu_i (undirected: degree)
    int32_t ideg;   // in-degree of mu_i (directed)
    int32_t pel;    // label of the pattern arc joining mu_i and P(mu_i) along the row used
    int32_t bbeg;   // back edges [bbeg, bbeg + bcnt) in the job's BackEdge array
    int32_t bcnt;
    int32_t ucnt;   // unparented RI-DS: |D(mu_i)| raw candidates (RI reads n_t from the target)
    int32_t uoff;   // unparented RI-DS: offset of D(mu_i) in the job's candidate list
    int32_t flags;  // POS_IN_ROW
    int32_t pad;
    uint64_t same[2];   // bit j (j < i): mu_j has lab(mu_i).  Only those positions can already hold a
                        // candidate of mu_i (any other image has another label), so rule 1 checks them alone
};

// A pattern edge from mu_i back to an earlier position j (rule 4).
struct BackEdge {
    int32_t pos;      // j
    int32_t dir;      // bit 0: arc mu_i -> mu_j needed; bit 1: arc mu_j -> mu_i needed
    int32_t lab_out;  // label of mu_i -> mu_j (undirected: the edge label)
    int32_t lab_in;   // label of mu_j -> mu_i
};

struct TargetView {
    int32_t n;
    int32_t dw;                 // 64-bit words per bitset row
    const int32_t *rowptr;      // out-rows (undirected: all neighbours)
    const int32_t *col;
    const int32_t *elab;
    const int32_t *irowptr;     // in-rows (directed)
    const int32_t *icol;
    const int32_t *ielab;
    const int2 *vld;            // {label, out-degree}
    const int32_t *indeg;       // directed
    const uint64_t *adj;        // adjacency bitset rows (undirected, small n) or null
    const int32_t *hub_slot;    // large undirected targets: bitset row of vertex v, or -1
    const uint64_t *hub_bits;   // hub rows, dw words each
    // undirected targets: the distinct vertex labels (ascending, nlab of them) and, per label
    // index l and vertex t, the largest degree among t's neighbours of that label (0: none), in
    // nbmax[l * n + t]; null when not built (directed targets, or n x nlab above 2^26)
    const int32_t *labs;
    const int32_t *nbmax;
    int32_t nlab;
    int32_t maxdeg;             // longest out- or in-row (0: not known)
    // large undirected targets: vertices grouped by label index (bucket l = [lbstart[l],
    // lbstart[l + 1])), descending degree within a bucket, with those degrees in lbdeg; null
    // otherwise.  A pattern vertex's initial domain is a prefix of its label's bucket.
    const int32_t *lbuck;
    const int32_t *lbdeg;
    const int32_t *lbstart;
    // small undirected targets: per label index l and degree threshold d < LDM_DEGREES, the dw-word
    // mask of the vertices with label l and degree at least d, at ldm[(l * LDM_DEGREES + d) * dw];
    // null otherwise.  Domain initialisation without the neighbour-label test copies a row.
    const uint64_t *ldm;
};

constexpr int LDM_DEGREES = 17;          // degree thresholds 0..16 in a target's label-degree masks
constexpr int LDM_MAX_N = 4096;          // targets up to this many vertices get the masks ...
constexpr long long LDM_MAX_WORDS = 1ll << 18;   // ... when they take at most this many words

struct PatternView {
    int32_t k;
    int32_t pad;
    const int32_t *lab;         // vertex-indexed
    const int32_t *odeg;
    const int32_t *ideg;
    const int32_t *rowptr;      // out-rows (undirected: all neighbours)
    const int32_t *col;
    const int32_t *elab;
    const int32_t *irowptr;     // in-rows (directed)
    const int32_t *icol;
    const int32_t *ielab;
};

struct JobDesc {
    TargetView t;
    PatternView p;
    const PosInfo *pos;
    const BackEdge *back;
    uint64_t *filt;             // k x t.dw words: D(v) / label-degree filter, or null
    const int32_t *ulist;       // candidate lists of unparented RI-DS positions
    const int32_t *plidx;       // RI-DS on a target with nbmax: each pattern vertex's label index among
                                // the target's labels (-1: absent), else null
    int32_t k;
    int32_t flags;
    unsigned long long *ctr;    // [4]: matches, states, nodes, hash
    int32_t *mbuf;              // enumerate: match rows (k ints each), or null
    long long mcap;             // rows that fit in mbuf
    unsigned long long *mlen;   // rows produced (may exceed mcap)
    unsigned long long *abytes; // algorithmic bytes of the bitset search
};

// Control block of one persistent search launch.
struct SearchCtl {
    const int32_t *front;       // frontier frames, stride fstride
    long long nfront;           // frames of this shard
    int32_t fstride;
    int32_t shard_index, shard_count;
    int32_t pcap;               // pool cells
    unsigned long long *fnext;  // next frontier index (atomic)
    int32_t *pool;              // pcap x POOL_STRIDE ints
    unsigned long long *pseq;   // per-cell sequence numbers (bounded MPMC queue)
    unsigned long long *phead, *ptail;
    int *outstanding;           // frames not yet finished
    int *idle;                  // warps waiting for work
    int *status;                // first error code (0 = ok)
    unsigned long long *donations;
    int *promised;              // donations decided on but not yet pushed (bounds concurrent donors)
    const volatile int *cancel; // host-mapped cancel word (nonzero = stop), or null
    unsigned long long deadline_ns;  // time limit in ns from each warp's start (%globaltimer), 0 = none
    long long budget;           // states budget per job, 0 = none
    int32_t donate;             // work donation on/off
    int32_t gran;               // most frames per donation
    int32_t donate_iters;       // a warp donates at most once per this many iterations ...
    unsigned long long donate_ns; // ... or per this much device time, whichever comes first
    unsigned long long idle_exit_ns; // a warp idle this long exits (0 = wait for the end)
    uint64_t *slab;             // bitset kernel: per-warp level bitsets (search_slab_bytes)
    int32_t *ckpt;              // checkpoint: on a stop, warps dump their unexplored work here
    long long ckpt_cap;         // ... up to this many frames of ckpt_stride ints
    int32_t ckpt_stride;        // FRAME_HDR + kmax
    unsigned long long *ckpt_n; // frames dumped (may exceed ckpt_cap: then the dump is incomplete)
    unsigned long long *wtrace; // optional per-warp trace records of WTRACE_WORDS words (null: off)
    unsigned long long *span;   // [2]: ~(first block's start), last warp's end (%globaltimer, atomicMax)
};

constexpr int WTRACE_WORDS = 16;   // words of one warp's trace record (see WarpClock)

// The control words of a search launch live in a block of CTL_BYTES bytes,
// each on its own 128-byte line: idle warps poll some of them while busy
// warps update others with atomics, and sharing one line would queue every
// update behind the polls.
constexpr size_t CTL_LINE = 128;
constexpr size_t CTL_BYTES = 9 * CTL_LINE;
inline void bind_control(SearchCtl &C, void *block) {
    char *b = static_cast<char *>(block);
    C.fnext = reinterpret_cast<unsigned long long *>(b + 0 * CTL_LINE);
    C.phead = reinterpret_cast<unsigned long long *>(b + 1 * CTL_LINE);
    C.ptail = reinterpret_cast<unsigned long long *>(b + 2 * CTL_LINE);
    C.donations = reinterpret_cast<unsigned long long *>(b + 3 * CTL_LINE);
    C.outstanding = reinterpret_cast<int *>(b + 4 * CTL_LINE);
    C.idle = reinterpret_cast<int *>(b + 5 * CTL_LINE);
    C.status = reinterpret_cast<int *>(b + 6 * CTL_LINE);
    C.promised = reinterpret_cast<int *>(b + 7 * CTL_LINE);
    C.span = reinterpret_cast<unsigned long long *>(b + 8 * CTL_LINE);
}

// ------------------------------------------------------------ launchers
// (implemented in sge_kernels.cu; all launch on `st`)

// plidx of every job that has one: its pattern vertices' label indices (thread per vertex).
cudaError_t launch_label_index(const JobDesc *jobs, const long long *vert_off, int njobs, long long nverts,
                               cudaStream_t st);
// Initial domains of the jobs whose targets have label buckets (their filter words already
// zeroed): one warp per (job, pattern vertex), setting the bits of the bucket prefix.
cudaError_t launch_domain_init_buckets(const JobDesc *jobs, const long long *vert_off, int njobs, long long nverts,
                                       cudaStream_t st);
cudaError_t launch_domain_init(const JobDesc *jobs, const long long *unit_off, int njobs,
                               long long nunits, cudaStream_t st);
cudaError_t launch_domain_ac_cand(const JobDesc *jobs, const int4 *ent, const long long *eoff, int nent,
                                  long long ncand, int32_t *cand, int *changed, unsigned char *vchanged,
                                  cudaStream_t st);
cudaError_t launch_domain_ac(const JobDesc *jobs, const int4 *ent, const long long *eoff, int nent, long long nunits,
                             int *changed, unsigned char *vchanged, cudaStream_t st);
cudaError_t launch_domain_fc(const JobDesc *jobs, const long long *vert_off, const long long *sizes, int njobs,
                             int *changed, unsigned char *vchanged, cudaStream_t st);
// Arc consistency and forward checking to their joint fixpoint, one block per
// job (for batches of many jobs; no host round trips).  With `cand` null the
// sweeps scan domain words; else they walk each vertex's candidate list
// (slots [cstart[g], cstart[g] + csize[g]), g = vert_off[job] + v).  Blocks
// take jobs from the counter `next_job` (one int of device scratch, zeroed here).
cudaError_t launch_domain_fixpoint(const JobDesc *jobs, int njobs, const long long *vert_off, const long long *cstart,
                                   const long long *csize, int32_t *cand, int *next_job, cudaStream_t st);
cudaError_t launch_domain_sizes(const JobDesc *jobs, const long long *vert_off, int njobs,
                                long long nverts, long long *sizes, cudaStream_t st);
cudaError_t launch_domain_lists(const JobDesc *jobs, const int *task_job, const int *task_vert,
                                const int *task_out, int ntasks, int32_t *lists, cudaStream_t st);

// BFS split of one level: pass 0 counts children per frame, pass 1 writes
// them at `offs` and accumulates the level's counters into the jobs.
cudaError_t launch_split(const JobDesc *jobs, const int32_t *fin, long long nf, int depth,
                         int32_t *counts, const long long *offs, int32_t *fout, int pass,
                         int count_ctr, int directed, cudaStream_t st);
// The whole split as one cooperative launch (see k_split_coop): frames of
// level L have stride FRAME_HDR + L in buffers of cap_ints ints; result[4] =
// {final frame count, final buffer 0/1, levels done, last level's child count, -, -,
// ~(first block's start), last block's end} (device clock; the host zeroes all eight);
// wtot needs one entry per block of the grid (at most wtot_cap).
cudaError_t launch_split_coop(const JobDesc *jobs, long long f0, int32_t *buf0, int32_t *buf1, long long cap_ints,
                              long long target, int max_levels, long long *wtot, long long wtot_cap,
                              unsigned *bar, long long *result, int *status, int count_ctr, int directed,
                              int blocks_per_sm, uint32_t *masks, long long mask_total, int ordered,
                              long long *trace, cudaStream_t st);
cudaError_t launch_scan(const int32_t *in, long long *out, long long n, long long *total,
                        void *tmp, size_t tmp_bytes, cudaStream_t st);
size_t scan_tmp_bytes(long long n);

// Persistent search.  kernel: 1 = CSR, 2 = bitset.  Returns the grid size used.
// The grid is capped at `max_grid` blocks (the blocks the slab was sized for; 0 = no cap).
cudaError_t launch_search(int kernel, const JobDesc *jobs, const SearchCtl &ctl, int kmax, int nwl,
                          int directed, int blocks_per_sm, long long max_grid, int *grid_out, cudaStream_t st);
int search_warps_per_block();
cudaError_t search_blocks_per_sm(int kernel, int kmax, int nwl, int directed, int *occ);
cudaError_t launch_pool_init(unsigned long long *seq, int cap, cudaStream_t st);
size_t search_smem_bytes(int kernel, int kmax, int nwl);
// Global scratch the search kernel needs for a grid of `grid` blocks.
size_t search_slab_bytes(int kernel, int kmax, int nwl, long long grid);

// Adjacency bitset rows of the hub vertices `hubs[0..h)` (rows zeroed first).
cudaError_t launch_build_hubs(const int32_t *rowptr, const int32_t *col, const int32_t *hubs, int h, int dw,
                              uint64_t *bits, cudaStream_t st);

// Fixed scratch of sge_count_noalloc (sge_noalloc.cu): the current device's
// address of the library's static device array, set up once per device.
cudaError_t noalloc_scratch(void **ptr, size_t *bytes);
cudaError_t launch_make_vld(const int32_t *rowptr, const int32_t *vlabel, int2 *vld, int n, cudaStream_t st);

// Target ingest on the device (sge_ingest.cu).  Error bits of the flags word:
constexpr int ING_RANGE = 1;   // an endpoint outside [0, n)
constexpr int ING_LOOP = 2;    // a self-loop
constexpr int ING_LABEL = 4;   // a repeated edge with another label
constexpr int ING_ELAB = 8;    // (not an error) some edge label is nonzero
cudaError_t launch_ingest_count(const int32_t *src, const int32_t *dst, const int32_t *elab, long long m, int n,
                                int directed, int32_t *cnt_out, int32_t *cnt_in, int *flags, cudaStream_t st);
cudaError_t launch_ingest_scatter(const int32_t *src, const int32_t *dst, const int32_t *elab, long long m, int n,
                                  int directed, const long long *off_out, const long long *off_in, int32_t *fill_out,
                                  int32_t *fill_in, uint64_t *key_out, uint64_t *key_in, cudaStream_t st);
cudaError_t launch_ingest_rows(const long long *off, int n, uint64_t *keys, uint64_t *scratch, int32_t *ucnt,
                               int32_t *long_rows, int32_t *nlong, int *flags, int sms, cudaStream_t st);
cudaError_t launch_ingest_compact(const long long *off, const long long *uoff, const int32_t *ucnt,
                                  const long long *utotal, const uint64_t *keys, int n, int32_t *rowptr, int32_t *col,
                                  int32_t *lab, cudaStream_t st);
cudaError_t launch_ingest_degree(const int32_t *rowptr, int n, int32_t *deg, cudaStream_t st);
cudaError_t launch_ingest_maxdeg(const int32_t *rowptr, int n, int32_t *maxdeg, cudaStream_t st);
cudaError_t launch_ingest_bits(const int32_t *rowptr, const int32_t *col, int n, int dw, uint64_t *bits,
                               cudaStream_t st);
// The label-degree masks of TargetView::ldm for the nlab labels labs[] (vld: {label, degree}).
cudaError_t launch_label_degree_masks(const int2 *vld, int n, const int32_t *labs, int nlab, int dw, uint64_t *ldm,
                                      cudaStream_t st);
// nbmax[lidx[y] * n + t] = max deg(y) over the neighbours y of t (nbmax zeroed first).
cudaError_t launch_label_nbmax(const int32_t *rowptr, const int32_t *col, const int2 *vld, const int32_t *lidx, int n,
                               int nlab, int32_t *nbmax, cudaStream_t st);

}  // namespace sge
