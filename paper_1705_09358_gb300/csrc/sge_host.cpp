// sge_host.cpp -- host side of the C ABI declared in include/sge.h.
//
// Graph ingest (validation, CSR build, adjacency bitsets), the GPU-host
// statement of RI's GreatestConstraintFirst ordering (Section "RI") with the
// RI-DS singleton block and SI tie-break (Section 4), the per-search position
// tables, and the launch sequence: domains (RI-DS), breadth-first split,
// persistent search.  All enumeration arithmetic runs in sge_kernels.cu; this
// file only prepares tables and orchestrates launches.
#include "../../include/sge.h"
#include "sge_internal.h"

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <climits>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <exception>
#include <functional>
#include <map>
#include <memory>
#include <new>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <unistd.h>

using namespace sge;

namespace {

constexpr int NO_ARC = INT_MIN;
constexpr int BITSET_MAX_N = 16384;              // adjacency bitset kept for n <= this (<= 32 MB)
constexpr int HUB_MIN_DEGREE = 24;               // larger targets: bitset rows for vertices of this degree+
constexpr long long HUB_BYTES = 512ll << 20;     // ... within this much device memory
constexpr long long FRONTIER_MAX_INTS = 1ll << 27;  // 512 MB per frontier buffer
constexpr int POOL_CELLS = 1 << 15;
constexpr long long CAND_MAX = 1ll << 28;   // most listed domain candidates per launch group (1 GiB)
constexpr int ROOT_CHUNK = 1024;                 // root candidates per root range frame
constexpr int BLOCK_FIXPOINT_MAX_N = 16384;      // auto domain mode: in-block fixpoint for targets up to this
constexpr long long LABEL_TABLE_MAX = 1ll << 26; // most (vertex, label) entries of a target's degree table
constexpr int LIST_FIXPOINT_MIN_JOBS = 32;      // auto domain mode, small targets: in-block fixpoint over lists from
                                                 // this many pairs (large targets: always; on the 100k-vertex target it
                                                 // beat the sweeps from 1 to 32 pairs)

// Opt-in phase trace on stderr (SGE_TRACE=1): sizes and timings of each launch group.
// SGE_TRACE: unset or "0" off; "errors" prints only failures; anything else
// also prints per-launch timings (which adds synchronisation).
bool trace_errors() {
    static const bool on = std::getenv("SGE_TRACE") != nullptr && std::getenv("SGE_TRACE")[0] != '0';
    return on;
}
bool trace_on() {
    static const bool on = trace_errors() && std::strcmp(std::getenv("SGE_TRACE"), "errors") != 0;
    return on;
}

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// ------------------------------------------------------------ device buffers
// Device blocks of unloaded graphs, kept by the context for the next load: a
// load then needs no cudaMalloc and an unload no cudaFree (each cudaFree
// synchronises the device).  Blocks are handed back only after the device is
// idle (sge_unload_*) or when only the context's own stream used them (a
// failed load), so a block is never reused while a kernel still reads it.
struct BlockCache {
    static constexpr size_t LIMIT = size_t(1) << 30;   // cached bytes kept at most
    std::mutex mu;
    std::multimap<size_t, void *> blocks;              // capacity -> block
    size_t bytes = 0;
    // A cached block of at least `want` bytes and at most about twice that.
    void *take(size_t want, size_t *cap) {
        std::lock_guard<std::mutex> g(mu);
        auto it = blocks.lower_bound(want);
        if (it == blocks.end() || it->first > 2 * want + 4096) return nullptr;
        void *q = it->second;
        *cap = it->first;
        bytes -= it->first;
        blocks.erase(it);
        return q;
    }
    void give(void *q, size_t cap) {
        {
            std::lock_guard<std::mutex> g(mu);
            if (bytes + cap <= LIMIT) {
                blocks.emplace(cap, q);
                bytes += cap;
                return;
            }
        }
        cudaFree(q);
    }
    // Free every cached block; returns whether there were any.
    bool clear() {
        std::lock_guard<std::mutex> g(mu);
        const bool had = !blocks.empty();
        for (auto &kv : blocks) cudaFree(kv.second);
        blocks.clear();
        bytes = 0;
        return had;
    }
};

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
    BlockCache *cache = nullptr;   // where released blocks go (null: cudaFree)
    // Stream-ordered mode (launch-group workspaces, each used on one stream): blocks come from
    // and go back to the device's memory pool in the order of `astream` (cudaMallocAsync /
    // cudaFreeAsync), so growing a buffer never synchronises the device -- with several serving
    // groups in flight, a cudaFree waited for every other group's kernels -- and a buffer grows
    // by at least half its size at a time.
    cudaStream_t astream = nullptr;
    bool async = false;
    cudaError_t ensure(size_t bytes) {
        if (bytes <= cap && p) return cudaSuccess;
        size_t nb = bytes < 256 ? 256 : bytes;
        if (async) {
            if (nb < cap + cap / 2) nb = cap + cap / 2;
            release();
            cudaError_t e = cudaMallocAsync(&p, nb, astream);
            if (e != cudaSuccess) {
                (void)cudaGetLastError();
                nb = bytes < 256 ? 256 : bytes;   // retry at the exact size
                e = cudaMallocAsync(&p, nb, astream);
            }
            if (e != cudaSuccess) { p = nullptr; cap = 0; return e; }
            cap = nb;
            return cudaSuccess;
        }
        release();
        if (cache) {
            size_t c = 0;
            if (void *q = cache->take(nb, &c)) {
                p = q;
                cap = c;
                return cudaSuccess;
            }
        }
        cudaError_t e = cudaMalloc(&p, nb);
        if (e == cudaErrorMemoryAllocation && cache && cache->clear()) {
            cudaGetLastError();   // the failed attempt must not surface at a later launch check
            e = cudaMalloc(&p, nb);
        }
        if (e != cudaSuccess) { p = nullptr; return e; }
        cap = nb;
        return cudaSuccess;
    }
    void release() {
        if (p) {
            if (async) cudaFreeAsync(p, astream);
            else if (cache) cache->give(p, cap);
            else cudaFree(p);
        }
        p = nullptr;
        cap = 0;
    }
    // Free at once, whatever the mode (the owner is going away, its stream perhaps with it).
    void free_now() {
        if (p) {
            if (async && astream) cudaStreamSynchronize(astream);
            cudaFree(p);
        }
        p = nullptr;
        cap = 0;
        async = false;
    }
    template <class T> T *as() const { return static_cast<T *>(p); }
};

// -------------------------------------------------------------- graph build
struct Rows {
    std::vector<int32_t> ptr, col, lab;
};

struct Built {
    int n = 0;
    bool directed = false;
    bool any_elab = false;
    Rows out, in;   // in: directed only
    std::vector<int32_t> vlab, odeg, ideg;
};

struct Arc {
    uint64_t key;  // (a << 32) | b
    int32_t lab;
};

// Sort arcs, merge repeats with an equal label; false on a conflicting repeat.
bool rows_from_arcs(int n, std::vector<Arc> &arcs, Rows &r) {
    // two stable counting sorts (by target, then by source) leave every row sorted by
    // target in O(m + n); repeated arcs end up adjacent and are merged
    const size_t m = arcs.size();
    // scratch kept per thread: large temporaries freed after every call cost more in
    // fresh-page faults than the sorting itself
    static thread_local std::vector<Arc> tmp;
    static thread_local std::vector<int64_t> at;
    tmp.resize(m);
    at.assign((size_t)n + 1, 0);
    auto pass = [&](const std::vector<Arc> &from, std::vector<Arc> &to, int shift) {
        std::fill(at.begin(), at.end(), 0);
        for (const Arc &a : from) at[(size_t)((a.key >> shift) & 0xffffffffu) + 1]++;
        for (int v = 0; v < n; ++v) at[(size_t)v + 1] += at[v];
        for (const Arc &a : from) to[(size_t)at[(size_t)((a.key >> shift) & 0xffffffffu)]++] = a;
    };
    pass(arcs, tmp, 0);    // by target
    pass(tmp, arcs, 32);   // by source, stable: rows stay sorted by target
    r.ptr.assign((size_t)n + 1, 0);
    r.col.clear();
    r.lab.clear();
    r.col.reserve(m);
    r.lab.reserve(m);
    for (size_t i = 0; i < m; ++i) {
        if (i > 0 && arcs[i - 1].key == arcs[i].key) {
            if (arcs[i - 1].lab != arcs[i].lab) return false;   // repeated edge, other label
            continue;
        }
        r.ptr[(size_t)(arcs[i].key >> 32) + 1]++;
        r.col.push_back((int32_t)(arcs[i].key & 0xffffffffu));
        r.lab.push_back(arcs[i].lab);
    }
    for (int v = 0; v < n; ++v) r.ptr[(size_t)v + 1] += r.ptr[v];
    return true;
}

bool build_graph(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, const int32_t *vlabel,
                 const int32_t *elabel, int directed, Built &g, std::string &err) {
    if (n < 0 || m < 0) { err = "negative vertex or edge count"; return false; }
    if (m > 0 && (!src || !dst)) { err = "null edge arrays"; return false; }
    if (n > 0 && !vlabel) { err = "null vertex-label array"; return false; }
    if ((directed ? m : 2 * m) > INT32_MAX) { err = "more than 2^31-1 stored arcs"; return false; }
    g.n = n;
    g.directed = directed != 0;
    g.any_elab = false;
    static thread_local std::vector<Arc> out, in;   // per-thread scratch, reused
    out.clear();
    in.clear();
    out.reserve(g.directed ? (size_t)m : 2 * (size_t)m);
    if (g.directed) in.reserve((size_t)m);
    for (int64_t e = 0; e < m; ++e) {
        const int a = src[e], b = dst[e];
        const int l = elabel ? elabel[e] : 0;
        if (a < 0 || a >= n || b < 0 || b >= n) { err = "edge endpoint out of range"; return false; }
        if (a == b) { err = "self-loop"; return false; }
        if (l != 0) g.any_elab = true;
        out.push_back({(uint64_t)(uint32_t)a << 32 | (uint32_t)b, l});
        if (g.directed) in.push_back({(uint64_t)(uint32_t)b << 32 | (uint32_t)a, l});
        else out.push_back({(uint64_t)(uint32_t)b << 32 | (uint32_t)a, l});
    }
    if (!g.directed) {   // no in-rows (and none left from an earlier load through this scratch)
        g.in.ptr.clear();
        g.in.col.clear();
        g.in.lab.clear();
    }
    if (!rows_from_arcs(n, out, g.out) || (g.directed && !rows_from_arcs(n, in, g.in))) {
        err = "repeated edge with a different label";
        return false;
    }
    g.vlab.assign(vlabel, vlabel + n);
    g.odeg.resize(n);
    g.ideg.resize(n);
    for (int v = 0; v < n; ++v) {
        g.odeg[v] = g.out.ptr[v + 1] - g.out.ptr[v];
        g.ideg[v] = g.directed ? g.in.ptr[v + 1] - g.in.ptr[v] : g.odeg[v];
    }
    return true;
}

// --------------------------------------------------------------- contexts
struct TargetRec {
    int n = 0, dw = 0;
    bool directed = false, any_elab = false;
    long long nnz = 0;
    TargetView cached{};   // view(), taken once the record is complete
    DevBuf rowptr, col, elab, irowptr, icol, ielab, vld, indeg, adj, hub_slot, hub_bits, hub_list;
    DevBuf ltab;           // distinct labels, then the per-(label, vertex) largest neighbour degree
    int nlab = 0, ltab_off = 0;
    int maxdeg = 0;                // longest out- or in-row
    std::vector<int32_t> labs_h;   // host copy of the distinct labels (ascending)
    DevBuf lbk;            // large targets: label buckets (vertices, their degrees, bucket starts)
    DevBuf ldm;            // small undirected targets: label-degree masks
    TargetView view() const {
        TargetView v;
        v.n = n;
        v.dw = dw;
        v.rowptr = rowptr.as<int32_t>();
        v.col = col.as<int32_t>();
        v.elab = elab.as<int32_t>();
        // undirected: the in-rows are the rows themselves
        v.irowptr = directed ? irowptr.as<int32_t>() : v.rowptr;
        v.icol = directed ? icol.as<int32_t>() : v.col;
        v.ielab = directed ? ielab.as<int32_t>() : v.elab;
        v.vld = vld.as<int2>();
        v.indeg = directed ? indeg.as<int32_t>() : nullptr;
        v.adj = adj.p ? adj.as<uint64_t>() : nullptr;
        v.hub_slot = hub_slot.p ? hub_slot.as<int32_t>() : nullptr;
        v.hub_bits = hub_bits.p ? hub_bits.as<uint64_t>() : nullptr;
        v.labs = ltab.p ? ltab.as<int32_t>() : nullptr;
        v.nbmax = ltab.p ? ltab.as<int32_t>() + ltab_off : nullptr;
        v.nlab = ltab.p ? nlab : 0;
        v.maxdeg = maxdeg;
        v.lbuck = lbk.p ? lbk.as<int32_t>() : nullptr;
        v.lbdeg = lbk.p ? lbk.as<int32_t>() + n : nullptr;
        v.lbstart = lbk.p ? lbk.as<int32_t>() + 2 * (size_t)n : nullptr;
        v.ldm = ldm.p ? ldm.as<uint64_t>() : nullptr;
        return v;
    }
    void use_cache(BlockCache *c) {
        for (DevBuf *b : {&rowptr, &col, &elab, &irowptr, &icol, &ielab, &vld, &indeg, &adj, &hub_slot, &hub_bits,
                          &hub_list, &ltab, &lbk, &ldm})
            b->cache = c;
    }
    void release() {
        for (DevBuf *b : {&rowptr, &col, &elab, &irowptr, &icol, &ielab, &vld, &indeg, &adj, &hub_slot, &hub_bits,
                          &hub_list, &ltab, &lbk, &ldm})
            b->release();
    }
    ~TargetRec() { release(); }
};

// The host-side facts about a pattern that the ordering and the position
// tables read: labels, degrees, the k x k arc-label matrix and undirected
// neighbourhood bitsets (two words per vertex, k <= 128).
struct PatView {
    int k;
    bool directed;
    const int32_t *lab, *odeg, *ideg;
    const int *amat;       // k x k, NO_ARC if absent
    const uint64_t *nb;    // 2 words per vertex
};

struct PatternRec {
    PatternView cached{};   // view(), taken once the record is complete
    int k = 0;
    bool directed = false, any_elab = false;
    std::vector<int32_t> lab, odeg, ideg;
    std::vector<int> amat;                 // k x k arc labels, NO_ARC if absent
    std::vector<uint64_t> nb;              // undirected neighbourhood bitsets (2 words per vertex)
    std::vector<int> ri_mu, ri_par;        // cached RI ordering
    std::vector<PosInfo> ri_pos;           // ... and its position tables (they depend on the pattern alone)
    std::vector<BackEdge> ri_back;
    // the device arrays, packed into one block (one upload per load) at these
    // int32 offsets, each a multiple of 4 (16-byte aligned)
    DevBuf dall;
    size_t o_lab = 0, o_odeg = 0, o_ideg = 0, o_row = 0, o_col = 0, o_elab = 0, o_irow = 0, o_icol = 0, o_ielab = 0;
    PatView core() const {
        return PatView{k, directed, lab.data(), odeg.data(), ideg.data(), amat.data(), nb.data()};
    }
    PatternView view() const {
        PatternView v;
        v.k = k;
        v.pad = 0;
        const int32_t *b = dall.as<int32_t>();
        v.lab = b + o_lab;
        v.odeg = b + o_odeg;
        v.ideg = directed ? b + o_ideg : v.odeg;
        v.rowptr = b + o_row;
        v.col = b + o_col;
        v.elab = b + o_elab;
        v.irowptr = directed ? b + o_irow : v.rowptr;
        v.icol = directed ? b + o_icol : v.col;
        v.ielab = directed ? b + o_ielab : v.elab;
        return v;
    }
    void use_cache(BlockCache *c) {
        dall.cache = c;
    }
    void release() { dall.release(); }
    ~PatternRec() { release(); }
};

// Scratch of one launch sequence (the serving scheduler has one per slot).
// One (target, pattern) pair of a batched call, as run_group prepares it.
struct Job {
    int pair;        // index into the request
    TargetRec *t;
    PatternRec *p;
    int algo;
    bool active;
    long long filt_off = -1;  // offset (u64 words) of the job's filter block
    long long vert_off = 0;   // offset in the sizes array
    std::vector<int> mu, par;
    const long long *dsize = nullptr;   // |D(v)| of the job's pattern vertices (RI-DS), in the workspace
};

struct Workspace {
    DevBuf jobs, fjobs, ctr, filt, pos, back, ulist, unit_off, vert_off, sizes, task, flag, dent, deoff, vchg, cand,
        ctask;
    DevBuf front[2], counts, offs, scan_tmp, total, splitctl;
    DevBuf pool, pseq, ctl, slab;
    DevBuf mbuf, ckpt, wtrace, smask, plidx, cstart;
    std::vector<Job> hjobs;       // the call's pairs, reused (their vectors keep their capacity)
    std::vector<JobDesc> hdesc;   // host job records, reused
    std::vector<JobDesc> hfdesc;  // host records of the jobs with a filter block, reused
    std::vector<long long> hsizes;  // host copy of the domain sizes, reused
    std::vector<unsigned long long> hctr;  // host copy of the job counters, reused
    std::vector<PosInfo> hpos;             // host position tables and back edges, reused
    std::vector<BackEdge> hback;
    std::vector<std::vector<PosInfo>> hjpos;   // per job: its RI-DS position tables, reused
    std::vector<std::vector<BackEdge>> hjback;
    std::vector<long long> hri_off;        // per pattern id: offsets of its RI tables in this call
    std::vector<int> hri_rep;              // per pattern id: a job of that pattern in this call (-1 after)
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr, ev3 = nullptr;   // search kernel, split kernel
    cudaStream_t bound = nullptr;
#define SGE_WS_BUFFERS                                                                                             \
    &jobs, &fjobs, &ctr, &filt, &pos, &back, &ulist, &unit_off, &vert_off, &sizes, &task, &flag, &dent, &deoff, &vchg, \
        &cand, &ctask, &front[0], &front[1], &counts, &offs, &scan_tmp, &total, &splitctl, &pool, &pseq, &ctl, &slab, \
        &mbuf, &ckpt, &wtrace, &smask, &plidx, &cstart
    // Every buffer of this workspace is used on `st` only: allocate them stream-ordered there.
    void bind(cudaStream_t st) {
        if (bound == st && st != nullptr) return;
        for (DevBuf *b : {SGE_WS_BUFFERS}) {
            if (b->p && b->async && b->astream != st) b->free_now();   // a block of another stream
            b->async = true;
            b->astream = st;
        }
        bound = st;
    }
    void release() {
        for (DevBuf *b : {SGE_WS_BUFFERS}) b->free_now();
#undef SGE_WS_BUFFERS
        bound = nullptr;
        for (cudaEvent_t *e : {&ev0, &ev1, &ev2, &ev3})
            if (*e) cudaEventDestroy(*e);
        ev0 = ev1 = ev2 = ev3 = nullptr;
    }
};

// Device buffers of target ingest, kept by the context and reused by every load.
struct IngestWs {
    DevBuf src, dst, elab, vlab, cnt_out, cnt_in, fill_out, fill_in, off_out, off_in, key_out, key_in, scratch, ucnt,
        uoff, long_rows, small, scan_tmp;
    void release() {
        for (DevBuf *b : {&src, &dst, &elab, &vlab, &cnt_out, &cnt_in, &fill_out, &fill_in, &off_out, &off_in, &key_out,
                          &key_in, &scratch, &ucnt, &uoff, &long_rows, &small, &scan_tmp})
            b->release();
    }
};

struct ServeReq;

}  // namespace

struct sge_ctx {
    int device = 0;
    int sms = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    BlockCache cache;            // device blocks of unloaded graphs (declared before the graphs)
    std::unordered_map<int, std::unique_ptr<TargetRec>> targets;
    std::unordered_map<int, std::unique_ptr<PatternRec>> patterns;
    int next_target = 1, next_pattern = 1;
    std::string err;
    std::mutex mu;               // guards targets / patterns / err for the serving thread
    int *cancel_host = nullptr;  // mapped pinned word
    int *cancel_dev = nullptr;
    Workspace ws;
    IngestWs ing;
    std::mutex ingest_mu;        // one target ingest at a time uses `ing`
    // serving
    std::mutex smu;
    std::condition_variable scv;
    std::deque<std::shared_ptr<ServeReq>> squeue;
    std::map<int64_t, std::shared_ptr<ServeReq>> sreqs;
    int64_t next_ticket = 1;
    std::vector<std::thread> sworkers;
    bool sstop = false;
    int sinflight = 0;
    long long sbytes_in_use = 0;
};

namespace {

struct ServeReq {
    int32_t tid, pid;
    sge_opts opts;
    sge_result res;
    bool done = false;
    long long bytes = 0;
    double t_submit = 0;
};

sge_status fail(sge_ctx *ctx, sge_status code, const std::string &msg) {
    if (ctx) {
        std::lock_guard<std::mutex> g(ctx->mu);
        ctx->err = msg;
    }
    if (trace_errors()) std::fprintf(stderr, "[sge] error %d: %s\n", code, msg.c_str());
    return code;
}

sge_status cuda_fail(sge_ctx *ctx, cudaError_t e, const char *what) {
    return fail(ctx, e == cudaErrorMemoryAllocation ? SGE_ERR_OOM : SGE_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(expr, what)                                   \
    do {                                                 \
        cudaError_t e_ = (expr);                         \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
    } while (0)

template <class T>
cudaError_t upload(DevBuf &b, const std::vector<T> &v, cudaStream_t st) {
    cudaError_t e = b.ensure(std::max<size_t>(v.size() * sizeof(T), 16));
    if (e != cudaSuccess || v.empty()) return e;
    return cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st);
}

// ------------------------------------------------------------- ordering
// GreatestConstraintFirst (Section "RI"): the first vertex has the highest
// degree, then greedily the vertex with most neighbours in mu (w_m), then most
// vertices of mu reachable through one vertex outside mu (w_n), then highest
// degree; RI-DS puts singleton domains first (ascending id) and SI breaks the
// remaining ties by the smaller domain (Section 4.1).  Lower id last.
// Neighbourhoods ignore edge direction.
struct OrderKey {
    long wm, wn, deg;
    long long dsz;
};

void gcf_order_into(const PatView &P, int algo, const long long *dsize, int *mu, int *par) {
    const int k = P.k;
    const bool si = algo == SGE_RIDS_SI || algo == SGE_RIDS_SI_FC;
    uint64_t in[2] = {0, 0};
    auto has = [&](const uint64_t *s, int v) { return (s[v >> 6] >> (v & 63)) & 1ull; };
    auto deg = [&](int v) -> long { return P.odeg[v] + (P.directed ? P.ideg[v] : 0); };
    int len = 0;
    if (algo != SGE_RI)
        for (int v = 0; v < k; ++v)
            if (dsize[v] == 1) { mu[len++] = v; in[v >> 6] |= 1ull << (v & 63); }
    if (len == 0 && k > 0) {
        int best = 0;
        for (int v = 1; v < k; ++v) {
            const long dv = deg(v), db = deg(best);
            if (dv > db || (dv == db && si && dsize[v] < dsize[best])) best = v;
        }
        mu[len++] = best;
        in[best >> 6] |= 1ull << (best & 63);
    }
    while (len < k) {
        int best = -1;
        OrderKey bk{0, 0, 0, 0};
        for (int v = 0; v < k; ++v) {
            if (has(in, v)) continue;
            const uint64_t *nv = P.nb + 2 * v;
            OrderKey key;
            key.wm = __builtin_popcountll(nv[0] & in[0]) + __builtin_popcountll(nv[1] & in[1]);
            // vertices of mu adjacent to some neighbour x of v outside mu
            uint64_t reach[2] = {0, 0};
            for (int h = 0; h < 2; ++h) {
                uint64_t outside = nv[h] & ~in[h];
                while (outside) {
                    const int x = h * 64 + __builtin_ctzll(outside);
                    outside &= outside - 1;
                    reach[0] |= P.nb[2 * x];
                    reach[1] |= P.nb[2 * x + 1];
                }
            }
            key.wn = __builtin_popcountll(reach[0] & in[0]) + __builtin_popcountll(reach[1] & in[1]);
            key.deg = deg(v);
            key.dsz = si ? dsize[v] : 0;
            bool take = best < 0;
            if (!take) {
                if (key.wm != bk.wm) take = key.wm > bk.wm;
                else if (key.wn != bk.wn) take = key.wn > bk.wn;
                else if (key.deg != bk.deg) take = key.deg > bk.deg;
                else if (key.dsz != bk.dsz) take = key.dsz < bk.dsz;
            }
            if (take) { best = v; bk = key; }
        }
        mu[len++] = best;
        in[best >> 6] |= 1ull << (best & 63);
    }
    // parent: the earliest earlier vertex adjacent to mu_i
    for (int i = 0; i < k; ++i) {
        par[i] = -1;
        for (int j = 0; j < i; ++j)
            if (has(P.nb + 2 * mu[i], mu[j])) { par[i] = j; break; }
    }
}

void gcf_order(const PatternRec &P, int algo, const long long *dsize, std::vector<int> &mu, std::vector<int> &par) {
    mu.assign(P.k, -1);
    par.assign(P.k, -1);
    gcf_order_into(P.core(), algo, dsize, mu.data(), par.data());
}

// Position tables of one search from its ordering (rules 2-4 per position),
// written to caller-provided arrays: pos[k] and back[] (at most k(k-1)/2
// entries).  Returns the number of back edges.
int build_positions_into(const PatView &P, const int *mu, const int *par, int algo, const long long *dsize, int n,
                         PosInfo *pos, BackEdge *back) {
    const int k = P.k;
    int nb = 0;
    for (int i = 0; i < k; ++i) {
        const int v = mu[i];
        PosInfo &p = pos[i];
        std::memset(&p, 0, sizeof(p));
        p.pv = v;
        p.par = par[i];
        p.lab = P.lab[v];
        p.odeg = P.odeg[v];
        p.ideg = P.directed ? P.ideg[v] : 0;
        p.uoff = -1;
        if (p.par >= 0) {
            const int u = mu[p.par];
            if (!P.directed || P.amat[(size_t)u * k + v] != NO_ARC) {
                p.pel = P.amat[(size_t)u * k + v];           // arc P -> mu_i: out-row of M(P)
            } else {
                p.flags |= POS_IN_ROW;                         // arc mu_i -> P: in-row of M(P)
                p.pel = P.amat[(size_t)v * k + u];
            }
        } else {
            p.ucnt = algo == SGE_RI ? n : (int)dsize[v];
        }
        for (int j = 0; j < i; ++j)
            if (P.lab[mu[j]] == p.lab) p.same[j >> 6] |= 1ull << (j & 63);
        p.bbeg = nb;
        for (int j = 0; j < i; ++j) {
            const int w = mu[j];
            const int lo = P.amat[(size_t)v * k + w], li = P.amat[(size_t)w * k + v];
            bool need_out = lo != NO_ARC, need_in = li != NO_ARC;
            if (!need_out && !need_in) continue;
            if (j == p.par) {
                if (!P.directed) continue;                      // the row itself is this edge
                if (p.flags & POS_IN_ROW) need_out = false; else need_in = false;
                if (!need_out && !need_in) continue;
            }
            BackEdge &be = back[nb++];
            be.pos = j;
            be.dir = P.directed ? ((need_out ? 1 : 0) | (need_in ? 2 : 0)) : 1;
            be.lab_out = need_out ? lo : 0;
            be.lab_in = need_in ? li : 0;
        }
        p.bcnt = nb - p.bbeg;
    }
    return nb;
}

void build_positions(const PatternRec &P, const std::vector<int> &mu, const std::vector<int> &par, int algo,
                     const long long *dsize, int n, std::vector<PosInfo> &pos, std::vector<BackEdge> &back) {
    const int k = P.k;
    pos.resize(k);
    back.resize((size_t)k * (k > 0 ? k - 1 : 0) / 2 + 1);
    const int nb = build_positions_into(P.core(), mu.data(), par.data(), algo, dsize, n, pos.data(), back.data());
    back.resize(nb);
}


struct PairReq {
    int32_t tid, pid;
    TargetRec *t = nullptr;    // resolved by prepare_pairs
    PatternRec *p = nullptr;
};

constexpr int HOST_THREADS_MAX = 16;  // host threads of one parallel_for, the caller's included

// Host worker threads for parallel_for, started once per process: creating and
// joining threads for every loop cost tens of microseconds per thread, paid several
// times by each large batched call.  One parallel_for at a time runs on the pool
// (`busy`); one that finds it taken, by another host thread or from inside a loop
// body, starts threads of its own.  A forked child, which inherits the pool's
// memory but not its threads, starts a pool of its own.
class HostPool {
  public:
    explicit HostPool(int nworkers) {
        for (int i = 1; i <= nworkers; ++i) std::thread([this, i] { worker(i); }).detach();
    }
    std::atomic<bool> busy{false};
    // runs task(0) on the calling thread and task(1) .. task(nt - 1) on workers
    // 1 .. nt - 1 (nt - 1 <= nworkers), returning when all have finished
    void run(int nt, const std::function<void(int)> &t) {
        {
            std::lock_guard<std::mutex> lk(m_);
            task_ = &t;
            want_ = left_ = nt - 1;
            ++gen_;
        }
        go_.notify_all();
        std::exception_ptr err;   // (the workers still use `t`: wait for them before rethrowing)
        try {
            t(0);
        } catch (...) {
            err = std::current_exception();
        }
        std::unique_lock<std::mutex> lk(m_);
        fin_.wait(lk, [&] { return left_ == 0; });
        if (err) std::rethrow_exception(err);
    }

  private:
    // Worker i takes part in a run if i <= want_.  A run cannot end (left_ > 0) before
    // each of its workers has seen its generation, so none skips one it belongs to.
    void worker(int i) {
        unsigned long long seen = 0;
        std::unique_lock<std::mutex> lk(m_);
        for (;;) {
            go_.wait(lk, [&] { return gen_ != seen; });
            seen = gen_;
            if (i > want_) continue;
            const std::function<void(int)> *t = task_;
            lk.unlock();
            (*t)(i);
            lk.lock();
            if (--left_ == 0) fin_.notify_one();
        }
    }
    std::mutex m_;
    std::condition_variable go_, fin_;
    const std::function<void(int)> *task_ = nullptr;
    int want_ = 0, left_ = 0;
    unsigned long long gen_ = 0;
};

HostPool *host_pool() {
    static std::mutex mk;
    static HostPool *pool = nullptr;   // never destroyed: its detached workers outlive static teardown
    static pid_t owner = 0;
    std::lock_guard<std::mutex> lk(mk);
    if (pool == nullptr || owner != getpid()) {
        pool = new HostPool(HOST_THREADS_MAX - 1);
        owner = getpid();
    }
    return pool;
}

// Runs body(begin, end) over [0, n) split across up to HOST_THREADS_MAX host threads
// (no more than the machine has), each with at least `min_per_thread` items (16384 by
// default: batches of many thousands of cheap pairs), else inline.
template <class F>
void parallel_for(int n, F body, int min_per_thread = 16384) {
    const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
    const int nt = std::min(std::min(HOST_THREADS_MAX, hw), n / min_per_thread);
    if (nt <= 1) {
        body(0, n);
        return;
    }
    const int chunk = (n + nt - 1) / nt;
    const std::function<void(int)> slice = [&](int t) {
        const int b = t * chunk, e = std::min(n, b + chunk);
        if (b < e) body(b, e);
    };
    HostPool *pool = host_pool();
    bool idle = false;
    if (pool->busy.compare_exchange_strong(idle, true)) {
        struct Release {
            std::atomic<bool> &b;
            ~Release() { b.store(false); }
        } release{pool->busy};
        pool->run(nt, slice);
        return;
    }
    std::vector<std::thread> th;
    for (int t = 1; t < nt; ++t) th.emplace_back([&slice, t] { slice(t); });
    slice(0);
    for (auto &x : th) x.join();
}

// With SGE_TRACE=1: wait for the stream and print when a phase of run_group ended.
void trace_phase(cudaStream_t st, const char *what, double t_start) {
    if (!trace_on()) return;
    cudaStreamSynchronize(st);
    std::fprintf(stderr, "[sge] phase %s done at %.3f ms\n", what, now_ms() - t_start);
}

// Kernel span in ms from the words its blocks leave: ~(earliest start), latest end.
float span_ms(unsigned long long inv_start, unsigned long long end) {
    if (inv_start == 0 || end == 0) return 0.f;
    const unsigned long long start = ~inv_start;
    return end > start ? (float)((double)(end - start) * 1e-6) : 0.f;
}

int pow2_at_least(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

// Run a homogeneous group of pairs (same directedness) through the whole
// launch sequence on `st` with workspace `W`.
// Resume input / checkpoint output of run_group (see sge_count_batch_ckpt).
struct Resume {
    const int32_t *frames = nullptr;   // frames of stride FRAME_HDR + kmax
    long long n = 0;
    int kmax = 0;
};

sge_status run_group(sge_ctx *ctx, Workspace &W, cudaStream_t st, const std::vector<PairReq> &reqs,
                     const std::vector<int> &idx, const sge_opts &o, sge_result *out, bool enumerate,
                     std::vector<int32_t> *match_rows, long long match_cap, bool serving,
                     const Resume *resume = nullptr, std::vector<int32_t> *ckpt_frames = nullptr,
                     int *ckpt_kmax = nullptr) {
    const double t_start = now_ms();
    W.bind(st);
    if (ckpt_frames) ckpt_frames->clear();
    long long launches = 0;   // kernels launched by this call
    const int algo = o.algo;
    const int nj = (int)idx.size();
    std::vector<Job> &jobs = W.hjobs;   // kept across calls (no fresh pages)
    if (jobs.size() < (size_t)nj) jobs.resize((size_t)nj);
    bool directed = false, any_elab = false;
    int kmax = 1, nmax = 1, max_pid = 0;
    std::mutex red;   // merges the threads' partial maxima
    parallel_for(nj, [&](int q0, int q1) {
        bool el = false;
        int km = 1, nm = 1, mp = 0;
        for (int q = q0; q < q1; ++q) {
            Job &J = jobs[q];
            J.filt_off = -1;
            J.vert_off = 0;
            J.dsize = nullptr;
            J.pair = idx[q];
            J.t = reqs[J.pair].t;
            J.p = reqs[J.pair].p;
            if (!J.t || !J.p) {
                std::lock_guard<std::mutex> g(ctx->mu);
                J.t = ctx->targets.at(reqs[J.pair].tid).get();
                J.p = ctx->patterns.at(reqs[J.pair].pid).get();
            }
            J.algo = algo;
            J.active = J.p->k > 0 && J.p->k <= J.t->n;
            mp = std::max(mp, reqs[J.pair].pid);
            if (J.active) {
                km = std::max(km, J.p->k);
                nm = std::max(nm, J.t->n);
                el = el || J.t->any_elab || J.p->any_elab;
            }
        }
        std::lock_guard<std::mutex> g(red);
        kmax = std::max(kmax, km);
        nmax = std::max(nmax, nm);
        max_pid = std::max(max_pid, mp);
        any_elab = any_elab || el;
    });
    if (nj > 0) directed = jobs[0].t->directed;   // (a group holds pairs of one directedness)
    // kernel family: the bitset kernel needs undirected, unlabelled edges, an
    // adjacency bitset and at most 4 words per lane with the level stack in
    // shared memory
    bool bits_ok = !directed && !any_elab;
    int nwl = 1;
    for (int q = 0; q < nj; ++q)   // (the workspace's job vector may be longer than this call)
        if (const Job &J = jobs[q]; J.active) {
            if (!J.t->adj.p) bits_ok = false;
            nwl = std::max(nwl, pow2_at_least((J.t->dw + 31) / 32));
        }
    if (nwl > 4 || search_smem_bytes(2, kmax, nwl) > 160 * 1024) bits_ok = false;
    int kernel = SGE_KERNEL_CSR;
    if (o.kernel == SGE_KERNEL_BITSET) {
        if (!bits_ok) return fail(ctx, SGE_ERR_ARG, "bitset kernel requested but a pair does not allow it");
        kernel = SGE_KERNEL_BITSET;
    } else if (o.kernel == SGE_KERNEL_AUTO && bits_ok) {
        kernel = SGE_KERNEL_BITSET;
    }
    const bool need_filt_all = kernel == SGE_KERNEL_BITSET;
    const double t_jobs = now_ms();

    // ---------------------------------------------------------- job tables
    long long filt_words = 0, nverts = 0, nunits = 0;
    std::vector<long long> unit_off, vert_off;
    for (int q = 0; q < nj; ++q) {
        Job &J = jobs[q];
        if (!J.active) continue;
        if (J.algo != SGE_RI || need_filt_all) {
            J.filt_off = filt_words;
            filt_words += (long long)J.p->k * J.t->dw;
        }
    }
    std::vector<JobDesc> &desc = W.hdesc;   // host copy kept across calls (no fresh pages)
    desc.resize((size_t)nj);
    CK(W.filt.ensure(std::max<long long>(filt_words, 1) * 8), "alloc filter");
    // per job: 4 counters, then nj match-row counts, then nj byte counters
    CK(W.ctr.ensure((size_t)nj * 6 * sizeof(unsigned long long)), "alloc counters");
    CK(cudaMemsetAsync(W.ctr.p, 0, (size_t)nj * 6 * sizeof(unsigned long long), st), "clear counters");
    parallel_for(nj, [&](int q0, int q1) {
        for (int q = q0; q < q1; ++q) {
            const Job &J = jobs[q];
            JobDesc &D = desc[q];
            D.t = J.t->cached;
            D.p = J.p->cached;
            D.pos = nullptr;
            D.back = nullptr;
            D.ulist = nullptr;
            D.plidx = nullptr;
            D.mbuf = nullptr;
            D.mcap = 0;
            D.k = J.p->k;
            D.flags = (J.algo != SGE_RI ? JOB_RIDS : 0) | (any_elab ? JOB_ELAB : 0) |
                      (directed ? JOB_DIRECTED : 0) | (J.algo == SGE_RIDS_SI_FC ? JOB_FC : 0);
            D.ctr = W.ctr.as<unsigned long long>() + 4 * (size_t)q;
            D.mlen = W.ctr.as<unsigned long long>() + 4 * (size_t)nj + q;
            D.abytes = W.ctr.as<unsigned long long>() + 5 * (size_t)nj + q;
            D.filt = J.filt_off >= 0 ? W.filt.as<uint64_t>() + J.filt_off : nullptr;
        }
    });
    const double t_desc = now_ms();
    // units of the domain kernels: (job, pattern vertex, 64-target word)
    std::vector<int> fjobs;  // jobs with a filter block, in order
    for (int q = 0; q < nj; ++q)
        if (jobs[q].active && jobs[q].filt_off >= 0) fjobs.push_back(q);
    // RI-DS jobs on targets with a label-degree table (undirected, no edge labels in the batch):
    // their pattern vertices' label indices among the target's labels, written on the device
    // below into one array indexed like the domain sizes (job's vertex offset + vertex)
    bool any_plidx = false;
    if (!any_elab && !directed) {
        long long g = 0;
        for (int q : fjobs) {
            const Job &J = jobs[q];
            if (J.algo != SGE_RI && !J.t->labs_h.empty()) any_plidx = true;
            g += J.p->k;
        }
        if (any_plidx) {
            CK(W.plidx.ensure((size_t)std::max<long long>(g, 1) * 4), "alloc label indices");
            g = 0;
            for (int q : fjobs) {
                const Job &J = jobs[q];
                if (J.algo != SGE_RI && !J.t->labs_h.empty()) desc[q].plidx = W.plidx.as<int32_t>() + g;
                g += J.p->k;
            }
        }
    }
    bool any_buckets = false;
    unit_off.reserve(fjobs.size());
    vert_off.reserve(fjobs.size());
    for (int q : fjobs) {
        unit_off.push_back(nunits);
        vert_off.push_back(nverts);
        jobs[q].vert_off = nverts;
        // (targets with label buckets initialise their domains from the buckets, not word by word)
        if (!jobs[q].t->lbk.p) nunits += (long long)jobs[q].p->k * jobs[q].t->dw;
        else any_buckets = true;
        nverts += jobs[q].p->k;
    }
    const int nf = (int)fjobs.size();
    if (trace_on()) std::fprintf(stderr, "[sge] %d domain pairs laid out at %.3f ms\n", nf, now_ms() - t_start);
    if (nf > 0) {
        if (nf == nj) {
            CK(upload(W.fjobs, desc, st), "upload domain jobs");   // every job has a filter block
        } else {
            std::vector<JobDesc> &fdesc = W.hfdesc;
            fdesc.resize((size_t)nf);
            parallel_for(nf, [&](int x0, int x1) {
                for (int x = x0; x < x1; ++x) fdesc[(size_t)x] = desc[(size_t)fjobs[x]];
            });
            CK(upload(W.fjobs, fdesc, st), "upload domain jobs");
        }
        CK(upload(W.unit_off, unit_off, st), "upload unit offsets");
        CK(upload(W.vert_off, vert_off, st), "upload vertex offsets");
        if (any_plidx) {
            CK(launch_label_index(W.fjobs.as<JobDesc>(), W.vert_off.as<long long>(), nf, nverts, st), "label indices");
            ++launches;
        }
        CK(W.sizes.ensure((size_t)nverts * 8), "alloc sizes");
        CK(W.flag.ensure(64), "alloc flag");
        trace_phase(st, "domain uploads", t_start);
        if (any_buckets) CK(cudaMemsetAsync(W.filt.p, 0, (size_t)filt_words * 8, st), "clear domains");
        CK(launch_domain_init(W.fjobs.as<JobDesc>(), W.unit_off.as<long long>(), nf, nunits, st), "domain init");
        ++launches;
        if (any_buckets) {
            CK(launch_domain_init_buckets(W.fjobs.as<JobDesc>(), W.vert_off.as<long long>(), nf, nverts, st),
               "domain init from buckets");
            ++launches;
        }
        trace_phase(st, "domain init", t_start);
        bool any_rids = false, any_fc = false;
        for (int q : fjobs) {
            any_rids = any_rids || jobs[q].algo != SGE_RI;
            any_fc = any_fc || jobs[q].algo == SGE_RIDS_SI_FC;
        }
        // RI-DS jobs in the batch; with many of them (or on request) the whole
        // fixpoint of each job runs inside one block of one launch, else under the host loop
        // below, whose sweeps spread one job's candidates over the whole device
        // (on small targets the blocks scan domains word by word; large targets' domains are
        // mostly empty words, so there the blocks walk candidate lists, built first, below)
        int nrids = 0;
        bool small_targets = true;
        for (int q : fjobs) {
            nrids += jobs[q].algo != SGE_RI ? 1 : 0;
            small_targets = small_targets && jobs[q].t->n <= BLOCK_FIXPOINT_MAX_N;
        }
        const bool block_fixpoint = any_rids && small_targets &&
                                    (o.domain_fixpoint == SGE_DOMAIN_BLOCKS ||
                                     (o.domain_fixpoint == SGE_DOMAIN_AUTO && nrids >= ctx->sms / 2));
        if (block_fixpoint) {
            CK(launch_domain_fixpoint(W.fjobs.as<JobDesc>(), nf, nullptr, nullptr, nullptr, nullptr,
                                      W.flag.as<int>() + 8, st),
               "domain fixpoint");
            ++launches;
            if (trace_on()) {
                CK(cudaStreamSynchronize(st), "fixpoint sync");
                std::fprintf(stderr, "[sge] domain fixpoint in blocks: %d jobs at %.3f ms\n", nf, now_ms() - t_start);
            }
        } else if (any_rids) {
            // arc consistency to its fixpoint, alternating with forward checking.  A sweep
            // re-checks D(v) only if the domain of a pattern neighbour of v shrank in the
            // previous sweep (the first sweep of a round checks every RI-DS vertex).
            std::vector<int> gjob((size_t)nverts), gv_v((size_t)nverts);
            for (int fj = 0; fj < nf; ++fj) {
                const Job &J = jobs[fjobs[fj]];
                for (int v = 0; v < J.p->k; ++v) {
                    gjob[(size_t)J.vert_off + v] = fj;
                    gv_v[(size_t)J.vert_off + v] = v;
                }
            }
            std::vector<unsigned char> dirty((size_t)nverts, 0), vchg((size_t)nverts, 0);
            auto mark_all = [&]() {
                for (long long g = 0; g < nverts; ++g) dirty[(size_t)g] = jobs[fjobs[gjob[(size_t)g]]].algo != SGE_RI;
            };
            CK(W.vchg.ensure((size_t)std::max<long long>(nverts, 1)), "alloc domain flags");
            // explicit candidate lists of the RI-DS domains, so that a sweep runs one thread per
            // candidate instead of one warp per 64-target word (most words of a large target's
            // domains hold few candidates); word sweeps when the lists would be too large
            std::vector<long long> csize((size_t)nverts, 0), cstart((size_t)nverts, 0);
            long long ncand = 0;
            {
                CK(launch_domain_sizes(W.fjobs.as<JobDesc>(), W.vert_off.as<long long>(), nf, nverts,
                                       W.sizes.as<long long>(), st), "domain sizes");
                ++launches;
                CK(cudaMemcpyAsync(csize.data(), W.sizes.p, (size_t)nverts * 8, cudaMemcpyDeviceToHost, st),
                   "read sizes");
                CK(cudaStreamSynchronize(st), "sizes sync");
                for (long long g = 0; g < nverts; ++g) {
                    if (jobs[fjobs[gjob[(size_t)g]]].algo == SGE_RI) csize[(size_t)g] = 0;
                    cstart[(size_t)g] = ncand;
                    ncand += csize[(size_t)g];
                }
            }
            // SGE_DOMAIN_WORDS=1 forces the word sweeps (they otherwise serve only lists beyond CAND_MAX)
            static const bool force_words = std::getenv("SGE_DOMAIN_WORDS") != nullptr &&
                                            std::getenv("SGE_DOMAIN_WORDS")[0] == '1';
            const bool cand_mode = !force_words && ncand > 0 && ncand <= CAND_MAX;
            if (cand_mode) {
                std::vector<int> tj, tv, to;
                for (long long g = 0; g < nverts; ++g)
                    if (csize[(size_t)g] > 0) {
                        tj.push_back(gjob[(size_t)g]);
                        tv.push_back(gv_v[(size_t)g]);
                        to.push_back((int)cstart[(size_t)g]);
                    }
                std::vector<int> tall(tj);
                tall.insert(tall.end(), tv.begin(), tv.end());
                tall.insert(tall.end(), to.begin(), to.end());
                CK(upload(W.ctask, tall, st), "upload candidate tasks");
                CK(W.cand.ensure((size_t)ncand * 4), "alloc candidate lists");
                const int nt = (int)tj.size();
                CK(launch_domain_lists(W.fjobs.as<JobDesc>(), W.ctask.as<int>(), W.ctask.as<int>() + nt,
                                       W.ctask.as<int>() + 2 * nt, nt, W.cand.as<int32_t>(), st), "candidate lists");
                trace_phase(st, "candidate lists", t_start);
                ++launches;
            }
            // many RI-DS pairs on large targets: each pair's whole fixpoint in one block, walking
            // the candidate lists (no host round trip per sweep)
            const bool list_blocks = cand_mode && (o.domain_fixpoint == SGE_DOMAIN_BLOCKS ||
                                                   (o.domain_fixpoint == SGE_DOMAIN_AUTO &&
                                                    (!small_targets || nrids >= LIST_FIXPOINT_MIN_JOBS)));
            if (list_blocks) {
                std::vector<long long> cs((size_t)nverts * 2);
                std::copy(cstart.begin(), cstart.end(), cs.begin());
                std::copy(csize.begin(), csize.end(), cs.begin() + nverts);
                CK(upload(W.cstart, cs, st), "upload candidate list offsets");
                CK(launch_domain_fixpoint(W.fjobs.as<JobDesc>(), nf, W.vert_off.as<long long>(),
                                          W.cstart.as<long long>(), W.cstart.as<long long>() + nverts,
                                          W.cand.as<int32_t>(), W.flag.as<int>() + 8, st), "domain fixpoint");
                ++launches;
                if (trace_on()) {
                    CK(cudaStreamSynchronize(st), "fixpoint sync");
                    std::fprintf(stderr, "[sge] domain fixpoint over candidate lists in blocks: %d jobs at %.3f ms\n",
                                 nf, now_ms() - t_start);
                }
            }
            // the neighbours of every shrunk domain (vchg) are re-checked next
            auto mark_neighbours = [&]() {
                std::fill(dirty.begin(), dirty.end(), 0);
                for (long long g = 0; g < nverts; ++g) {
                    if (!vchg[(size_t)g]) continue;
                    const Job &J = jobs[fjobs[gjob[(size_t)g]]];
                    if (J.algo == SGE_RI) continue;
                    const int v = gv_v[(size_t)g];
                    for (int w = 0; w < 2; ++w)
                        for (uint64_t b = J.p->nb[(size_t)v * 2 + w]; b; b &= b - 1)
                            dirty[(size_t)J.vert_off + 64 * w + __builtin_ctzll(b)] = 1;
                }
            };
            std::vector<int4> ent;
            std::vector<long long> eoff;
            mark_all();
            for (int outer = 0; outer < (list_blocks ? 0 : 100000); ++outer) {
                for (int sweep = 0; sweep < 1000000; ++sweep) {
                    ent.clear();
                    eoff.clear();
                    long long units = 0;
                    for (long long g = 0; g < nverts; ++g)
                        if (dirty[(size_t)g]) {
                            const int fj = gjob[(size_t)g];
                            if (cand_mode && csize[(size_t)g] == 0) continue;
                            int ey = gv_v[(size_t)g];
                            if (cand_mode) {
                                // every pattern neighbour's domain (as first counted) is dense: the
                                // sweep lets a lane try a long row before the warp
                                const Job &Jq = jobs[fjobs[fj]];
                                bool dense = true;
                                for (int w = 0; w < 2 && dense; ++w)
                                    for (uint64_t b = Jq.p->nb[(size_t)ey * 2 + w]; b && dense; b &= b - 1)
                                        dense = csize[(size_t)Jq.vert_off + 64 * w + __builtin_ctzll(b)] * AC_DENSE >=
                                                Jq.t->n;
                                if (dense) ey |= AC_ENT_DENSE;
                            }
                            ent.push_back(make_int4(fj, ey, (int)g, (int)cstart[(size_t)g]));
                            eoff.push_back(units);
                            units += cand_mode ? csize[(size_t)g] : jobs[fjobs[fj]].t->dw;
                        }
                    if (ent.empty()) break;
                    eoff.push_back(units);
                    const double ts = now_ms();
                    CK(upload(W.dent, ent, st), "upload domain entries");
                    CK(upload(W.deoff, eoff, st), "upload domain entries");
                    CK(cudaMemsetAsync(W.flag.p, 0, sizeof(int), st), "clear flag");
                    CK(cudaMemsetAsync(W.vchg.p, 0, (size_t)nverts, st), "clear domain flags");
                    if (cand_mode)
                        CK(launch_domain_ac_cand(W.fjobs.as<JobDesc>(), W.dent.as<int4>(), W.deoff.as<long long>(),
                                                 (int)ent.size(), units, W.cand.as<int32_t>(), W.flag.as<int>(),
                                                 W.vchg.as<unsigned char>(), st),
                           "domain ac");
                    else
                        CK(launch_domain_ac(W.fjobs.as<JobDesc>(), W.dent.as<int4>(), W.deoff.as<long long>(),
                                            (int)ent.size(), units, W.flag.as<int>(), W.vchg.as<unsigned char>(), st),
                           "domain ac");
                    ++launches;
                    CK(cudaMemcpyAsync(vchg.data(), W.vchg.p, (size_t)nverts, cudaMemcpyDeviceToHost, st),
                       "read domain flags");
                    CK(cudaStreamSynchronize(st), "ac sync");
                    if (trace_on())
                        std::fprintf(stderr, "[sge] ac sweep %d (round %d): %.3f ms, %zu vertices, %lld units\n", sweep,
                                     outer, now_ms() - ts, ent.size(), units);
                    mark_neighbours();
                }
                if (!any_fc) break;
                int fchanged = 0;
                const double tf = now_ms();
                CK(cudaMemsetAsync(W.flag.p, 0, sizeof(int), st), "clear flag");
                CK(cudaMemsetAsync(W.vchg.p, 0, (size_t)nverts, st), "clear domain flags");
                CK(launch_domain_sizes(W.fjobs.as<JobDesc>(), W.vert_off.as<long long>(), nf, nverts,
                                       W.sizes.as<long long>(), st), "domain sizes");
                CK(launch_domain_fc(W.fjobs.as<JobDesc>(), W.vert_off.as<long long>(), W.sizes.as<long long>(), nf,
                                    W.flag.as<int>(), W.vchg.as<unsigned char>(), st), "domain fc");
                launches += 2;
                CK(cudaMemcpyAsync(&fchanged, W.flag.p, sizeof(int), cudaMemcpyDeviceToHost, st), "read flag");
                CK(cudaMemcpyAsync(vchg.data(), W.vchg.p, (size_t)nverts, cudaMemcpyDeviceToHost, st),
                   "read domain flags");
                CK(cudaStreamSynchronize(st), "fc sync");
                if (trace_on()) std::fprintf(stderr, "[sge] fc round %d: %.3f ms\n", outer, now_ms() - tf);
                if (!fchanged) break;
                mark_neighbours();   // only neighbours of domains that forward checking shrank
            }
        }
        CK(launch_domain_sizes(W.fjobs.as<JobDesc>(), W.vert_off.as<long long>(), nf, nverts,
                               W.sizes.as<long long>(), st), "domain sizes");
        ++launches;
        std::vector<long long> &sizes = W.hsizes;   // kept across calls (no fresh pages)
        if (sizes.size() < (size_t)nverts) sizes.resize((size_t)nverts);
        CK(cudaMemcpyAsync(sizes.data(), W.sizes.p, (size_t)nverts * 8, cudaMemcpyDeviceToHost, st), "read sizes");
        CK(cudaStreamSynchronize(st), "sizes sync");
        parallel_for(nf, [&](int x0, int x1) {
            for (int x = x0; x < x1; ++x) {
                Job &J = jobs[fjobs[x]];
                J.dsize = sizes.data() + J.vert_off;
                if (J.algo != SGE_RI)
                    for (int v = 0; v < J.p->k; ++v)
                        if (J.dsize[v] == 0) J.active = false;   // an empty domain: no match, no search
            }
        });
    }
    trace_phase(st, "domains", t_start);
    // orderings and position tables; RI tables depend only on the pattern and
    // are shared by every job of that pattern (n_t of an unparented RI position
    // is read from the job's target at run time)
    std::vector<PosInfo> &pos = W.hpos;     // kept across calls (no fresh pages)
    std::vector<BackEdge> &back = W.hback;
    pos.clear();
    back.clear();
    std::vector<long long> pos_off(nj, 0), back_off(nj, 0);
    std::vector<int> task_job, task_vert, task_out;
    std::vector<int> fidx(nj, -1);
    for (int x = 0; x < nf; ++x) fidx[fjobs[x]] = x;
    // an RI pattern's tables are appended once per call: their offsets, by pattern id
    std::vector<long long> &ri_off = W.hri_off;   // [pid]: pos offset, back offset (-1: not yet)
    if (ri_off.size() < 2 * ((size_t)max_pid + 1)) ri_off.resize(2 * ((size_t)max_pid + 1), -1);
    std::vector<int> ri_seen;
    long long ulist_len = 0;
    // the RI-DS jobs' orderings and tables (each depends on its own domain sizes) on a few host
    // threads, into per-job vectors (kept in the workspace); they are appended in job order below
    std::vector<std::vector<PosInfo>> &jpos = W.hjpos;
    std::vector<std::vector<BackEdge>> &jback = W.hjback;
    const bool any_rids_job = algo != SGE_RI;   // (every pair of a call has the call's variant)
    if (any_rids_job && jpos.size() < (size_t)nj) {
        jpos.resize((size_t)nj);
        jback.resize((size_t)nj);
    }
    parallel_for(nj, [&](int q0, int q1) {
        for (int q = q0; q < q1; ++q) {
            Job &J = jobs[q];
            if (!J.active || J.algo == SGE_RI) continue;
            gcf_order(*J.p, J.algo, J.dsize, J.mu, J.par);
            build_positions(*J.p, J.mu, J.par, J.algo, J.dsize, J.t->n, jpos[(size_t)q], jback[(size_t)q]);
        }
    }, 64);
    if (trace_on()) {
        int act = 0;
        for (int q = 0; q < nj; ++q) act += jobs[q].active && jobs[q].algo != SGE_RI;
        std::fprintf(stderr, "[sge] RI-DS orderings of %d live pairs built at %.3f ms\n", act, now_ms() - t_start);
    }
    if (algo == SGE_RI) {
        // the distinct patterns' tables: a job of each pattern is noted on several threads
        // (any job will do), the tables appended by pattern id, then every job's offsets set
        std::vector<int> &rep = W.hri_rep;   // [pid]: a job of that pattern, or -1
        if (rep.size() < (size_t)max_pid + 1) rep.resize((size_t)max_pid + 1, -1);
        parallel_for(nj, [&](int q0, int q1) {
            for (int q = q0; q < q1; ++q)
                if (jobs[q].active)   // (threads may note different jobs of one pattern: any is valid)
                    __atomic_store_n(&rep[(size_t)reqs[jobs[q].pair].pid], q, __ATOMIC_RELAXED);
        });
        for (int pid = 0; pid <= max_pid; ++pid) {
            const int q = rep[(size_t)pid];
            if (q < 0) continue;
            rep[(size_t)pid] = -1;
            const PatternRec *P = jobs[q].p;
            ri_off[2 * (size_t)pid] = (long long)pos.size();
            ri_off[2 * (size_t)pid + 1] = (long long)back.size();
            pos.insert(pos.end(), P->ri_pos.begin(), P->ri_pos.end());
            back.insert(back.end(), P->ri_back.begin(), P->ri_back.end());
            ri_seen.push_back(pid);
        }
        parallel_for(nj, [&](int q0, int q1) {
            for (int q = q0; q < q1; ++q) {
                if (!jobs[q].active) continue;
                const size_t pid = (size_t)reqs[jobs[q].pair].pid;
                pos_off[q] = ri_off[2 * pid];
                back_off[q] = ri_off[2 * pid + 1];
            }
        });
    }
    for (int q = 0; q < nj && algo != SGE_RI; ++q) {
        Job &J = jobs[q];
        if (!J.active) continue;
        if (J.algo == SGE_RI) {
            const size_t pid = (size_t)reqs[J.pair].pid;
            if (ri_off[2 * pid] < 0) {
                ri_off[2 * pid] = (long long)pos.size();
                ri_off[2 * pid + 1] = (long long)back.size();
                pos.insert(pos.end(), J.p->ri_pos.begin(), J.p->ri_pos.end());
                back.insert(back.end(), J.p->ri_back.begin(), J.p->ri_back.end());
                ri_seen.push_back((int)pid);
            }
            pos_off[q] = ri_off[2 * pid];
            back_off[q] = ri_off[2 * pid + 1];
            continue;
        }
        pos_off[q] = (long long)pos.size();
        back_off[q] = (long long)back.size();
        std::vector<PosInfo> &pq = jpos[(size_t)q];
        std::vector<BackEdge> &bq = jback[(size_t)q];
        for (PosInfo &p : pq) {
            if (p.par < 0) {
                // the D(mu_i) list is written by a kernel below
                p.uoff = (int)ulist_len;
                task_job.push_back(fidx[q]);
                task_vert.push_back(p.pv);
                task_out.push_back((int)ulist_len);
                ulist_len += p.ucnt;
            }
        }
        pos.insert(pos.end(), pq.begin(), pq.end());
        back.insert(back.end(), bq.begin(), bq.end());
    }
    for (int pid : ri_seen) ri_off[2 * (size_t)pid] = ri_off[2 * (size_t)pid + 1] = -1;
    if (ulist_len > INT32_MAX) return fail(ctx, SGE_ERR_OOM, "unparented candidate lists too large");
    if (trace_on())
        std::fprintf(stderr,
                     "[sge] jobs %d kernel %d kmax %d nwl %d filt_words %lld: jobs %.3f, records %.3f, domains and "
                     "orders %.3f ms\n",
                     nj, kernel, kmax, nwl, filt_words, t_jobs - t_start, t_desc - t_jobs, now_ms() - t_desc);
    trace_phase(st, "orderings", t_start);
    CK(upload(W.pos, pos, st), "upload positions");
    CK(upload(W.back, back, st), "upload back edges");
    CK(W.ulist.ensure((size_t)std::max<long long>(ulist_len, 1) * 4), "alloc lists");
    if (!task_job.empty()) {
        std::vector<int> tasks;
        tasks.insert(tasks.end(), task_job.begin(), task_job.end());
        tasks.insert(tasks.end(), task_vert.begin(), task_vert.end());
        tasks.insert(tasks.end(), task_out.begin(), task_out.end());
        CK(upload(W.task, tasks, st), "upload list tasks");
        const int nt = (int)task_job.size();
        CK(launch_domain_lists(W.fjobs.as<JobDesc>(), W.task.as<int>(), W.task.as<int>() + nt,
                               W.task.as<int>() + 2 * nt, nt, W.ulist.as<int32_t>(), st), "domain lists");
        ++launches;
    }
    // enumeration output
    if (enumerate) {
        const long long rows = std::max<long long>(match_cap, 1);
        CK(W.mbuf.ensure((size_t)rows * kmax * 4), "alloc match buffer");
    }
    parallel_for(nj, [&](int q0, int q1) {
        for (int q = q0; q < q1; ++q) {
            JobDesc &D = desc[q];
            D.pos = W.pos.as<PosInfo>() + pos_off[q];
            D.back = W.back.as<BackEdge>() + back_off[q];
            if (jobs[q].active) {
                // can a position after the first have more than SPLIT_RANGE candidates?
                bool longl = jobs[q].t->maxdeg == 0 || jobs[q].t->maxdeg > SPLIT_RANGE;
                for (int i = 1; i < D.k && !longl; ++i) {
                    const PosInfo &P = pos[(size_t)pos_off[q] + i];
                    longl = P.par < 0 && ((D.flags & JOB_RIDS) ? (long long)P.ucnt : jobs[q].t->n) > SPLIT_RANGE;
                }
                if (longl) D.flags |= JOB_LONG_LISTS;
            }
            D.ulist = W.ulist.as<int32_t>();
            if (enumerate) {
                D.mbuf = W.mbuf.as<int32_t>();
                D.mcap = match_cap;
            }
        }
    });
    const double t_up = now_ms();
    CK(upload(W.jobs, desc, st), "upload jobs");
    const double t_pre = now_ms();
    if (trace_on()) std::fprintf(stderr, "[sge] job records uploaded in %.3f ms\n", t_pre - t_up);

    // -------------------------------------------------------- split (BFS)
    const int shard_count = o.shard_count > 1 ? o.shard_count : 1;
    const int shard_index = shard_count > 1 ? o.shard_index : 0;
    const int count_ctr = shard_index == 0 ? 1 : 0;
    int occ = 0;
    CK(search_blocks_per_sm(kernel == SGE_KERNEL_BITSET ? 2 : 1, kmax, nwl, directed ? 1 : 0, &occ), "occupancy");
    if (o.blocks_per_sm > 0 && o.blocks_per_sm < occ) occ = o.blocks_per_sm;
    const long long resident_warps = (long long)ctx->sms * occ * search_warps_per_block();
    const long long fpw = o.frames_per_warp > 0 ? o.frames_per_warp : 8;
    const long long target_frames = fpw * resident_warps * shard_count;
    // roots: one frame per active job, cut into ranges of ROOT_CHUNK candidates
    // when the root has more (a range frame counts the node's states only if it
    // starts at candidate 0)
    std::vector<std::array<int32_t, 4>> roots;
    roots.reserve((size_t)nj);
    for (int q = 0; q < nj; ++q) {
        const Job &J = jobs[q];
        if (!J.active) continue;
        const long long len = J.algo == SGE_RI ? J.t->n : pos[pos_off[q]].ucnt;
        if (len <= ROOT_CHUNK) {
            roots.push_back({q, 0, -1, -1});
        } else {
            for (long long b = 0; b < len; b += ROOT_CHUNK)
                roots.push_back({q, 0, (int32_t)b, (int32_t)std::min<long long>(b + ROOT_CHUNK, len)});
        }
    }
    long long F0 = (long long)roots.size();
    long long F = 0;
    float split_ms = 0.f;   // device time of the cooperative split (CUDA events)
    float split_exec_ms = 0.f, search_exec_ms = 0.f;   // the kernels' own spans (device clock)
    int cur = 0, depth = 0, fstride = FRAME_HDR;
    bool split_done = F0 == 0;
    if (resume != nullptr) {
        // continue from a checkpoint: its frames (mixed depths, stride FRAME_HDR + kmax) are the frontier
        if (resume->kmax != kmax) return fail(ctx, SGE_ERR_ARG, "checkpoint does not match these pairs");
        fstride = FRAME_HDR + kmax;
        F = resume->n;
        if (F > 0) {
            CK(W.front[0].ensure((size_t)F * fstride * 4), "alloc frontier");
            CK(cudaMemcpyAsync(W.front[0].p, resume->frames, (size_t)F * fstride * 4, cudaMemcpyHostToDevice, st),
               "upload checkpoint frames");
        }
        split_done = true;
    }
    const int max_levels = std::max(0, std::min(o.split_depth > 0 ? o.split_depth : INT_MAX, kmax - 1));
    const long long front_ints = o.frontier_kib > 0 ? 256ll * o.frontier_kib : FRONTIER_MAX_INTS;
    if (!split_done && resume == nullptr) {
        // the whole split as one cooperative launch.  Auto depth, CSR kernel: breadth-first
        // for as long as the next level fits the frontier budget (deep, narrow searches are
        // far cheaper level by level than depth-first, and the split tests candidates the way
        // the CSR kernel does).  Bitset kernel: stop at the frame target, since its
        // word-parallel expansion beats the split's per-candidate tests on dense targets.
        // A state budget or time limit is enforced by the search kernel, so with either
        // set the split also stops at the frame target and the search does the bulk.
        const bool limited = o.state_budget > 0 || o.time_limit_ms > 0;
        const long long target = o.split_depth > 0 ? LLONG_MAX
                                 : (kernel == SGE_KERNEL_BITSET || limited) ? target_frames : (long long)INT_MAX;
        const long long cap_ints = std::max<long long>(F0 * FRAME_HDR, front_ints);
        // sharded runs need the children in search order (frame i -> shard i mod S); an
        // unsharded run takes the single-pass form, one pass and one grid barrier per level
        const bool ordered = shard_count > 1 || !count_ctr;
        CK(W.front[0].ensure((size_t)cap_ints * 4), "alloc frontier");
        CK(W.front[1].ensure((size_t)cap_ints * 4), "alloc frontier");
        CK(cudaMemcpyAsync(W.front[0].p, roots.data(), (size_t)F0 * sizeof(roots[0]), cudaMemcpyHostToDevice, st),
           "upload roots");
        const long long wcap = (long long)ctx->sms * 32 * search_warps_per_block();
        const size_t ctl_words = (size_t)wcap + 16 + 2 * KMAX;   // (+ the level trace)
        CK(W.splitctl.ensure(ctl_words * 8), "alloc split control");
        CK(cudaMemsetAsync(W.splitctl.p, 0, ctl_words * 8, st), "clear split control");
        long long *wtot = W.splitctl.as<long long>();
        unsigned *bar = reinterpret_cast<unsigned *>(wtot + wcap);
        long long *res = wtot + wcap + 1;
        int *sstat = reinterpret_cast<int *>(res + 4);
        constexpr long long SPLIT_MASKS = 1ll << 24;   // 64 MiB of replayed candidate ballots
        const bool have_masks = ordered && W.smask.ensure((size_t)SPLIT_MASKS * 4) == cudaSuccess;
        if (!have_masks) (void)cudaGetLastError();   // without the buffer the write pass tests again
        if (!W.ev2) {
            CK(cudaEventCreate(&W.ev2), "event");
            CK(cudaEventCreate(&W.ev3), "event");
        }
        CK(cudaEventRecord(W.ev2, st), "event record");
        const cudaError_t le = launch_split_coop(W.jobs.as<JobDesc>(), F0, W.front[0].as<int32_t>(),
                                                 W.front[1].as<int32_t>(), cap_ints, target, max_levels, wtot,
                                                 wcap, bar, res, sstat, count_ctr, directed ? 1 : 0,
                                                 serving ? 1 : 0, have_masks ? W.smask.as<uint32_t>() : nullptr,
                                                 SPLIT_MASKS, ordered ? 1 : 0,
                                                 trace_on() ? wtot + wcap + 16 : nullptr, st);
        if (le == cudaSuccess) {
            ++launches;
            CK(cudaEventRecord(W.ev3, st), "event record");
            long long r4[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            int ss = 0;
            CK(cudaMemcpyAsync(r4, res, sizeof(r4), cudaMemcpyDeviceToHost, st), "read split result");
            CK(cudaMemcpyAsync(&ss, sstat, sizeof(int), cudaMemcpyDeviceToHost, st), "read split status");
            CK(cudaStreamSynchronize(st), "split sync");
            CK(cudaEventElapsedTime(&split_ms, W.ev2, W.ev3), "event time");
            split_exec_ms = span_ms((unsigned long long)r4[6], (unsigned long long)r4[7]);
            if (ss != 0) return fail(ctx, SGE_ERR_CUDA, "device split barrier timed out");
            F = r4[0];
            cur = (int)r4[1];
            depth = (int)r4[2];
            fstride = FRAME_HDR + depth;
            split_done = true;
            if (trace_on()) {
                std::fprintf(stderr, "[sge] device split: %d levels, %lld frames at %.3f ms\n", depth, F,
                             now_ms() - t_start);
                if (!ordered) {
                    // per level: end time, children, longest candidate list of one frame
                    std::vector<long long> tr((size_t)2 * KMAX), lv((size_t)std::max(depth, 1));
                    CK(cudaMemcpy(tr.data(), wtot + wcap + 16, tr.size() * 8, cudaMemcpyDeviceToHost), "read trace");
                    CK(cudaMemcpy(lv.data(), wtot, lv.size() * 8, cudaMemcpyDeviceToHost), "read trace");
                    long long prev = ~r4[6];
                    for (int l = 0; l < depth; ++l) {
                        std::fprintf(stderr, "[sge]   level %d: %.1f us, %lld children, longest list %lld\n", l,
                                     (tr[(size_t)l] - prev) * 1e-3, lv[(size_t)l], tr[(size_t)KMAX + l]);
                        prev = tr[(size_t)l];
                    }
                }
            }
        } else {
            (void)cudaGetLastError();   // cooperative launch refused: split level by level below
        }
    }
    if (!split_done && resume == nullptr) {
        fstride = FRAME_HDR;
        std::vector<int32_t> f0;
        for (const auto &r : roots) f0.insert(f0.end(), r.begin(), r.end());
        F = F0;
        CK(upload(W.front[0], f0, st), "upload roots");
        while (F > 0 && depth < max_levels) {
            if (o.split_depth <= 0 && F >= target_frames) break;
            CK(W.counts.ensure((size_t)F * 4), "alloc counts");
            CK(W.offs.ensure((size_t)F * 8), "alloc offsets");
            CK(W.scan_tmp.ensure(scan_tmp_bytes(F)), "alloc scan");
            CK(W.total.ensure(16), "alloc total");
            CK(launch_split(W.jobs.as<JobDesc>(), W.front[cur].as<int32_t>(), F, depth, W.counts.as<int32_t>(),
                            nullptr, nullptr, 0, count_ctr, directed ? 1 : 0, st), "split count");
            launches += 4;   // split count + three scan kernels
            CK(launch_scan(W.counts.as<int32_t>(), W.offs.as<long long>(), F, W.total.as<long long>(),
                           W.scan_tmp.p, W.scan_tmp.cap, st), "split scan");
            long long total = 0;
            CK(cudaMemcpyAsync(&total, W.total.p, 8, cudaMemcpyDeviceToHost, st), "read split total");
            CK(cudaStreamSynchronize(st), "split sync");
            const long long need = total * (FRAME_HDR + depth + 1);
            if (need > front_ints) break;   // keep the current frontier
            CK(W.front[cur ^ 1].ensure((size_t)std::max<long long>(need, 1) * 4), "alloc frontier");
            CK(launch_split(W.jobs.as<JobDesc>(), W.front[cur].as<int32_t>(), F, depth, W.counts.as<int32_t>(),
                            W.offs.as<long long>(), W.front[cur ^ 1].as<int32_t>(), 1, count_ctr, directed ? 1 : 0,
                            st), "split write");
            ++launches;
            cur ^= 1;
            F = total;
            ++depth;
            if (trace_on())
                std::fprintf(stderr, "[sge] split depth %d frames %lld at %.3f ms\n", depth, F, now_ms() - t_start);
        }
        fstride = FRAME_HDR + depth;
    }

    // ------------------------------------------------- persistent search
    long long nfront = 0;
    if (F > shard_index) nfront = (F - shard_index + shard_count - 1) / shard_count;
    float kernel_ms = 0.f;
    long long donations = 0;
    int status = 0;
    if (nfront > 0) {
        CK(W.pool.ensure((size_t)POOL_CELLS * POOL_STRIDE * 4), "alloc pool");
        CK(W.pseq.ensure((size_t)POOL_CELLS * 8), "alloc pool seq");
        CK(W.ctl.ensure(CTL_BYTES), "alloc control");
        CK(cudaMemsetAsync(W.ctl.p, 0, CTL_BYTES, st), "clear control");
        CK(launch_pool_init(W.pseq.as<unsigned long long>(), POOL_CELLS, st), "pool init");
        ++launches;
        SearchCtl C;
        std::memset(&C, 0, sizeof(C));
        bind_control(C, W.ctl.p);
        C.front = W.front[cur].as<int32_t>();
        C.nfront = nfront;
        C.fstride = fstride;
        C.shard_index = shard_index;
        C.shard_count = shard_count;
        C.pcap = POOL_CELLS;
        C.pool = W.pool.as<int32_t>();
        C.pseq = W.pseq.as<unsigned long long>();
        const int nf32 = (int)nfront;
        CK(cudaMemcpyAsync(C.outstanding, &nf32, sizeof(int), cudaMemcpyHostToDevice, st), "init outstanding");
        C.cancel = ctx->cancel_dev;
        C.deadline_ns = o.time_limit_ms > 0 ? (unsigned long long)o.time_limit_ms * 1000000ull : 0ull;
        C.budget = o.state_budget;
        C.donate = o.no_donation ? 0 : 1;
        // a bitset-kernel donor hands out up to 16 of its shallowest pending survivors at once:
        // with few, large frontier frames the tail is split fastest that way
        C.gran = o.steal_granularity > 0 ? o.steal_granularity : (kernel == SGE_KERNEL_BITSET ? 32 : 2);
        // donation cadence: a busy warp checks whether idle warps wait for work at most once
        // per this many iterations or this much device time.  Donating costs a few microseconds
        // (two fetch-and-adds and one cell write), so the bitset kernel checks every 50 us; the
        // CSR kernel's searches are mostly finished by the breadth-first split and keep 500 us,
        // except in serving groups: every 20 us there, so that the frames a group's split left
        // (its deepest, heaviest subtrees) are shared before idle warps leave.
        const bool bits_k = kernel == SGE_KERNEL_BITSET;
        C.donate_iters = o.donate_every_iters > 0 ? o.donate_every_iters
                         : (bits_k || serving ? (1 << 30) : 1024);
        C.donate_ns = (unsigned long long)(o.donate_every_us > 0 ? o.donate_every_us
                                           : (bits_k ? 50 : (serving ? 20 : 500))) * 1000ull;
        // serving groups: a warp idle for 200 us (ten donation periods without a frame for it)
        // leaves, so a group's tail frees block slots for the next group's kernels
        C.idle_exit_ns = serving ? 200000ull : 0ull;
        if (!W.ev0) {
            CK(cudaEventCreate(&W.ev0), "event");
            CK(cudaEventCreate(&W.ev1), "event");
        }
        int grid = 0;
        const int kfam = kernel == SGE_KERNEL_BITSET ? 2 : 1;
        const long long max_grid = (long long)ctx->sms * occ;
        const size_t slab_bytes = search_slab_bytes(kfam, kmax, nwl, max_grid);
        if (slab_bytes > 0) {
            CK(W.slab.ensure(slab_bytes), "alloc search slab");
            C.slab = W.slab.as<uint64_t>();
        }
        const int cs = FRAME_HDR + kmax;   // checkpoint frame stride
        if (ckpt_frames != nullptr) {
            // each warp dumps at most two range frames per level
            const long long cap = max_grid * search_warps_per_block() * 2 * kmax;
            const size_t bytes = (size_t)cap * cs * 4;
            CK(W.ckpt.ensure(bytes + 64), "alloc checkpoint");
            C.ckpt = W.ckpt.as<int32_t>();
            C.ckpt_cap = cap;
            C.ckpt_stride = cs;
            C.ckpt_n = reinterpret_cast<unsigned long long *>(W.ckpt.as<char>() + bytes);
            CK(cudaMemsetAsync(C.ckpt_n, 0, 8, st), "clear checkpoint");
        }
        if (trace_on()) {
            CK(W.wtrace.ensure((size_t)max_grid * search_warps_per_block() * WTRACE_WORDS * 8), "alloc warp trace");
            CK(cudaMemsetAsync(W.wtrace.p, 0, (size_t)max_grid * search_warps_per_block() * WTRACE_WORDS * 8, st),
               "clear warp trace");
            C.wtrace = W.wtrace.as<unsigned long long>();
        }
        CK(cudaEventRecord(W.ev0, st), "event record");
        CK(launch_search(kfam, W.jobs.as<JobDesc>(), C, kmax, nwl, directed ? 1 : 0, o.blocks_per_sm, max_grid, &grid,
                         st), "search launch");
        ++launches;
        CK(cudaEventRecord(W.ev1, st), "event record");
        unsigned long long dn = 0, sp[2] = {0, 0};
        CK(cudaMemcpyAsync(&status, C.status, sizeof(int), cudaMemcpyDeviceToHost, st), "read status");
        CK(cudaMemcpyAsync(&dn, C.donations, 8, cudaMemcpyDeviceToHost, st), "read donations");
        CK(cudaMemcpyAsync(sp, C.span, sizeof(sp), cudaMemcpyDeviceToHost, st), "read kernel span");
        CK(cudaStreamSynchronize(st), "search sync");
        CK(cudaEventElapsedTime(&kernel_ms, W.ev0, W.ev1), "event time");
        search_exec_ms = span_ms(sp[0], sp[1]);
        donations = (long long)dn;
        if (trace_on()) {
            std::fprintf(stderr, "[sge] search grid %d frames %lld kernel %.3f ms status %d donations %llu\n", grid,
                         nfront, kernel_ms, status, dn);
            // warp timeline: when warps exit relative to the first start, and their busy share
            const size_t nw = (size_t)grid * search_warps_per_block();
            constexpr int TW = WTRACE_WORDS;   // words per warp record
            std::vector<unsigned long long> wt(nw * TW);
            CK(cudaMemcpy(wt.data(), W.wtrace.p, nw * TW * 8, cudaMemcpyDeviceToHost), "read warp trace");
            unsigned long long t0 = ~0ull;
            for (size_t w = 0; w < nw; ++w)
                if (wt[TW * w]) t0 = std::min(t0, wt[TW * w]);
            std::vector<double> ex, last;
            std::vector<size_t> order;
            double busy = 0, span = 0;
            for (size_t w = 0; w < nw; ++w) {
                if (!wt[TW * w]) continue;
                ex.push_back((wt[TW * w + 1] - t0) * 1e-6);
                last.push_back(wt[TW * w + 3] ? (wt[TW * w + 3] - t0) * 1e-6 : 0.0);
                busy += wt[TW * w + 2] * 1e-6;
                span = std::max(span, ex.back());
                order.push_back(w);
            }
            std::sort(ex.begin(), ex.end());
            std::sort(last.begin(), last.end());
            auto q = [](const std::vector<double> &v, double f) {
                return v.empty() ? 0.0 : v[std::min(v.size() - 1, (size_t)(f * v.size()))];
            };
            std::fprintf(stderr,
                         "[sge] warps %zu: exit at p50 %.3f max %.3f ms; last work at p10 %.3f p50 %.3f p90 %.3f "
                         "p99 %.3f ms; busy %.1f%% of warps x span\n",
                         ex.size(), q(ex, 0.5), span, q(last, 0.1), q(last, 0.5), q(last, 0.9), q(last, 0.99),
                         span > 0 ? 100.0 * busy / (span * ex.size()) : 0.0);
            double don_ms = 0, don_ev = 0, don_fr = 0, don_max = 0;
            for (size_t w : order) {
                don_ms += wt[TW * w + 9] * 1e-6;
                don_ev += (double)wt[TW * w + 10];
                don_fr += (double)wt[TW * w + 11];
                don_max = std::max(don_max, wt[TW * w + 9] * 1e-6);
            }
            {
                double qn = 0, qt = 0, qs = 0;
                for (size_t w : order) {
                    qn += (double)wt[TW * w + 12];
                    qt += wt[TW * w + 13] * 1e-6;
                    qs += (double)wt[TW * w + 14];
                }
                std::fprintf(stderr, "[sge] queue frames %.0f: %.1f warp-ms, %.3g states\n", qn, qt, qs);
            }
            std::fprintf(stderr, "[sge] donation: %.0f events, %.0f frames, %.3f warp-ms in total, %.3f ms at most in "
                         "one warp, %.2f us per event\n", don_ev, don_fr, don_ms, don_max,
                         don_ev > 0 ? 1000.0 * don_ms / don_ev : 0.0);
            std::sort(order.begin(), order.end(), [&](size_t a, size_t b) { return wt[TW * a + 4] > wt[TW * b + 4]; });
            for (size_t r = 0; r < std::min<size_t>(8, order.size()); ++r) {
                const unsigned long long *x = &wt[TW * order[r]];
                std::fprintf(stderr,
                             "[sge]   longest frame %zu: %.3f ms, ended at %.3f ms, job %llu depth %llu from %s, "
                             "states %llu nodes %llu\n",
                             r, x[4] * 1e-6, (x[3] - t0) * 1e-6, x[5] & 0xffff, (x[5] >> 16) & 0x3fff,
                             (x[5] >> 30) == 1 ? "frontier" : "queue", x[6], x[7]);
            }
        }
        if (ckpt_frames != nullptr && (status == SGE_ERR_BUDGET || status == SGE_ERR_TIMEOUT ||
                                       status == SGE_ERR_CANCELLED)) {
            // unexplored work = the warps' dumps + frontier frames never taken + queued frames
            unsigned long long hc[1] = {0}, nd = 0;   // fnext
            CK(cudaMemcpyAsync(&hc[0], C.fnext, 8, cudaMemcpyDeviceToHost, st), "read control");
            CK(cudaMemcpyAsync(&nd, C.ckpt_n, 8, cudaMemcpyDeviceToHost, st), "read checkpoint count");
            CK(cudaStreamSynchronize(st), "checkpoint sync");
            if ((long long)nd > C.ckpt_cap) return fail(ctx, SGE_ERR_OOM, "checkpoint larger than its buffer");
            std::vector<int32_t> &outf = *ckpt_frames;
            outf.clear();
            // n frames of `stride` ints, `pitch` ints apart, into frames of cs ints
            auto take = [&](const int32_t *dev, long long n, int stride, long long pitch) -> cudaError_t {
                if (n <= 0) return cudaSuccess;
                const size_t at = outf.size();
                outf.resize(at + (size_t)n * cs, 0);
                return cudaMemcpy2DAsync(outf.data() + at, (size_t)cs * 4, dev, (size_t)pitch * 4,
                                         (size_t)std::min(stride, cs) * 4, (size_t)n, cudaMemcpyDeviceToHost, st);
            };
            CK(take(C.ckpt, (long long)nd, cs, cs), "read checkpoint frames");
            // frontier frames of this shard never taken (frame i of the shard is frame i*count+index)
            const long long taken = std::min<long long>((long long)hc[0], nfront);
            CK(take(C.front + (taken * shard_count + shard_index) * (long long)fstride, nfront - taken, fstride,
                    (long long)fstride * shard_count), "read frontier");
            // queued frames never taken: the cells left published (sequence word = ticket + 1)
            std::vector<unsigned long long> seq(POOL_CELLS);
            CK(cudaMemcpyAsync(seq.data(), C.pseq, (size_t)POOL_CELLS * 8, cudaMemcpyDeviceToHost, st), "read queue");
            CK(cudaStreamSynchronize(st), "checkpoint sync");
            for (int cell = 0; cell < POOL_CELLS; ++cell) {
                const unsigned long long sv = seq[cell];
                if (sv >= 1 && (sv >> 63) == 0 && (sv - 1) % POOL_CELLS == (unsigned long long)cell)
                    CK(take(C.pool + (size_t)cell * POOL_STRIDE, 1, POOL_STRIDE, POOL_STRIDE), "read queue");
            }
            CK(cudaStreamSynchronize(st), "checkpoint sync");
            if (ckpt_kmax) *ckpt_kmax = kmax;
        }
    }
    std::vector<unsigned long long> &ctr = W.hctr;   // kept across calls (no fresh pages)
    if (ctr.size() < (size_t)nj * 6) ctr.resize((size_t)nj * 6);
    CK(cudaMemcpyAsync(ctr.data(), W.ctr.p, (size_t)nj * 6 * 8, cudaMemcpyDeviceToHost, st), "read counters");
    CK(cudaStreamSynchronize(st), "counter sync");
    const double t_end = now_ms();
    parallel_for(nj, [&](int q0, int q1) {
        for (int q = q0; q < q1; ++q) {
            sge_result &r = out[jobs[q].pair];
            std::memset(&r, 0, sizeof(r));
            r.matches = ctr[4 * (size_t)q + 0];
            r.states = ctr[4 * (size_t)q + 1];
            r.nodes = ctr[4 * (size_t)q + 2];
            r.hash = ctr[4 * (size_t)q + 3];
            r.preprocess_ms = t_pre - t_start;
            r.match_ms = t_end - t_pre;
            r.search_kernel_ms = kernel_ms;
            r.split_kernel_ms = split_ms;
            r.split_exec_ms = split_exec_ms;
            r.search_exec_ms = search_exec_ms;
            r.frames = F;
            r.donations = donations;
            r.alg_bytes = kernel == SGE_KERNEL_BITSET ? ctr[5 * (size_t)nj + q] : 12ull * r.states;
            r.launches = launches;
            r.split_depth = depth;
            r.status = status;
            r.kernel = kernel;
        }
    });
    if (enumerate && match_rows && nj == 1) {
        const long long produced = (long long)ctr[4 * (size_t)nj + 0];
        const long long rows = std::min(produced, match_cap);
        match_rows->resize((size_t)rows * jobs[0].p->k);
        if (rows > 0)
            CK(cudaMemcpy(match_rows->data(), W.mbuf.p, (size_t)rows * jobs[0].p->k * 4, cudaMemcpyDeviceToHost),
               "read matches");
    }
    if (status != 0) {
        const char *why = status == SGE_ERR_BUDGET ? "state budget reached"
                          : status == SGE_ERR_TIMEOUT ? "time limit reached"
                          : status == SGE_ERR_CANCELLED ? "cancelled" : "search error";
        return fail(ctx, status, why);
    }
    return SGE_OK;
}

// Options with defaults applied, checked, and the pairs split by directedness.
sge_status prepare_pairs(sge_ctx *ctx, std::vector<PairReq> &reqs, const sge_opts *opts, sge_opts &o,
                         std::vector<int> &und, std::vector<int> &dir) {
    std::memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    if (o.time_limit_ms <= 0) {
        // a process-wide default limit (SGE_TIME_LIMIT_MS) when the call sets none
        const char *env = std::getenv("SGE_TIME_LIMIT_MS");
        if (env) o.time_limit_ms = std::atoll(env);
    }
    if (o.algo < SGE_RI || o.algo > SGE_RIDS_SI_FC) return fail(ctx, SGE_ERR_ARG, "unknown algo");
    if (o.kernel < 0 || o.kernel > 2) return fail(ctx, SGE_ERR_ARG, "unknown kernel family");
    if (o.domain_fixpoint < SGE_DOMAIN_AUTO || o.domain_fixpoint > SGE_DOMAIN_BLOCKS)
        return fail(ctx, SGE_ERR_ARG, "unknown domain fixpoint mode");
    if (o.frontier_kib < 0) return fail(ctx, SGE_ERR_ARG, "negative frontier size");
    if (o.shard_count > 1 && (o.shard_index < 0 || o.shard_index >= o.shard_count))
        return fail(ctx, SGE_ERR_ARG, "shard index out of range");
    und.clear();
    dir.clear();
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        // ids are handed out in sequence, so a call resolves each distinct id once through the
        // maps and every pair through a table indexed by id (large batches repeat few ids)
        std::vector<TargetRec *> tt((size_t)std::max(ctx->next_target, 1), nullptr);
        std::vector<PatternRec *> pt((size_t)std::max(ctx->next_pattern, 1), nullptr);
        std::vector<unsigned char> tseen(tt.size(), 0), pseen(pt.size(), 0);
        und.reserve(reqs.size());
        for (size_t i = 0; i < reqs.size(); ++i) {
            const int32_t tid = reqs[i].tid, pid = reqs[i].pid;
            TargetRec *T = nullptr;
            PatternRec *P = nullptr;
            if (tid >= 0 && (size_t)tid < tt.size()) {
                if (!tseen[(size_t)tid]) {
                    auto ti = ctx->targets.find(tid);
                    tt[(size_t)tid] = ti == ctx->targets.end() ? nullptr : ti->second.get();
                    tseen[(size_t)tid] = 1;
                }
                T = tt[(size_t)tid];
            }
            if (pid >= 0 && (size_t)pid < pt.size()) {
                if (!pseen[(size_t)pid]) {
                    auto pi = ctx->patterns.find(pid);
                    pt[(size_t)pid] = pi == ctx->patterns.end() ? nullptr : pi->second.get();
                    pseen[(size_t)pid] = 1;
                }
                P = pt[(size_t)pid];
            }
            if (!T || !P) {
                ctx->err = "unknown target or pattern id";
                return SGE_ERR_NOT_FOUND;
            }
            if (T->directed != P->directed) {
                ctx->err = "target and pattern disagree on directedness";
                return SGE_ERR_ARG;
            }
            reqs[i].t = T;
            reqs[i].p = P;
            (T->directed ? dir : und).push_back((int)i);
        }
    }
    return SGE_OK;
}

sge_status run_pairs(sge_ctx *ctx, Workspace &W, cudaStream_t st, std::vector<PairReq> &reqs,
                     const sge_opts *opts, sge_result *out, bool enumerate, std::vector<int32_t> *rows,
                     long long cap, bool serving = false) {
    sge_opts o;
    std::vector<int> und, dir;
    sge_status rc = prepare_pairs(ctx, reqs, opts, o, und, dir);
    if (rc != SGE_OK) return rc;
    if (!und.empty()) rc = run_group(ctx, W, st, reqs, und, o, out, enumerate, rows, cap, serving);
    if (rc == SGE_OK && !dir.empty()) rc = run_group(ctx, W, st, reqs, dir, o, out, enumerate, rows, cap, serving);
    return rc;
}

// ------------------------------------------------------------ checkpoints
//
// A checkpoint is one host blob (little-endian, all fields naturally aligned):
//   header   u64 magic, i32 version, i32 algo, i64 npairs, i32 ngroups, i32 0
//   pairs    npairs x {i32 target id, i32 pattern id, i32 n_t, i32 k}
//   counters npairs x {u64 matches, states, nodes, hash}   (so far, all calls)
//   groups   ngroups x {i32 kmax, i32 npairs_g, i64 nframes,
//                       npairs_g x i32 pair index (+ one i32 pad if odd),
//                       nframes x (4 + kmax) i32 frames}
// A frame is [job, depth (| FRAME_COUNTED), begin, end, M_0 .. M_{depth-1}]:
// job indexes the group's pair list, M the images of the first depth
// positions of the pair's search order.
constexpr uint64_t CKPT_MAGIC = 0x3154504B43454753ull;   // "SGECKPT1"
constexpr int32_t CKPT_VERSION = 1;

struct CkptGroup {
    std::vector<int> idx;          // pair indices, in job order
    int kmax = 0;
    std::vector<int32_t> frames;   // stride FRAME_HDR + kmax
};

struct CkptState {
    int algo = 0;
    std::vector<PairReq> reqs;
    std::vector<int32_t> nt, k;
    std::vector<uint64_t> ctr;     // 4 per pair
    std::vector<CkptGroup> groups;
};

template <class T>
void put(std::vector<unsigned char> &b, const T &v) {
    const unsigned char *p = reinterpret_cast<const unsigned char *>(&v);
    b.insert(b.end(), p, p + sizeof(T));
}

std::vector<unsigned char> ckpt_write(const CkptState &S) {
    std::vector<unsigned char> b;
    put(b, CKPT_MAGIC);
    put(b, CKPT_VERSION);
    put(b, (int32_t)S.algo);
    put(b, (int64_t)S.reqs.size());
    put(b, (int32_t)S.groups.size());
    put(b, (int32_t)0);
    for (size_t i = 0; i < S.reqs.size(); ++i) {
        put(b, S.reqs[i].tid);
        put(b, S.reqs[i].pid);
        put(b, S.nt[i]);
        put(b, S.k[i]);
    }
    for (uint64_t v : S.ctr) put(b, v);
    for (const CkptGroup &g : S.groups) {
        const int stride = FRAME_HDR + g.kmax;
        put(b, (int32_t)g.kmax);
        put(b, (int32_t)g.idx.size());
        put(b, (int64_t)(g.frames.size() / stride));
        for (int i : g.idx) put(b, (int32_t)i);
        if (g.idx.size() & 1) put(b, (int32_t)0);
        const unsigned char *p = reinterpret_cast<const unsigned char *>(g.frames.data());
        b.insert(b.end(), p, p + g.frames.size() * 4);
    }
    return b;
}

// Parses and checks a blob against the context (ids loaded, sizes unchanged,
// every frame within its pair's pattern and target).  Returns an error
// message, empty on success.
std::string ckpt_read(sge_ctx *ctx, const unsigned char *b, long long bytes, CkptState &S) {
    long long at = 0;
    auto get = [&](void *dst, long long n) {
        if (n < 0 || at + n > bytes) return false;
        std::memcpy(dst, b + at, (size_t)n);
        at += n;
        return true;
    };
    uint64_t magic = 0;
    int32_t version = 0, algo = 0, ngroups = 0, pad = 0;
    int64_t npairs = 0;
    if (!get(&magic, 8) || magic != CKPT_MAGIC) return "not a checkpoint";
    if (!get(&version, 4) || version != CKPT_VERSION) return "unsupported checkpoint version";
    if (!get(&algo, 4) || algo < SGE_RI || algo > SGE_RIDS_SI_FC) return "bad algo in checkpoint";
    if (!get(&npairs, 8) || npairs < 0 || npairs > bytes / 48) return "bad pair count in checkpoint";
    if (!get(&ngroups, 4) || ngroups < 0 || ngroups > 2 || !get(&pad, 4)) return "bad group count in checkpoint";
    S.algo = algo;
    S.reqs.resize((size_t)npairs);
    S.nt.resize((size_t)npairs);
    S.k.resize((size_t)npairs);
    S.ctr.resize((size_t)npairs * 4);
    std::vector<char> dir((size_t)npairs, 0);
    for (int64_t i = 0; i < npairs; ++i) {
        int32_t f[4];
        if (!get(f, 16)) return "truncated checkpoint";
        S.reqs[i] = {f[0], f[1]};
        S.nt[i] = f[2];
        S.k[i] = f[3];
        std::lock_guard<std::mutex> g(ctx->mu);
        auto ti = ctx->targets.find(f[0]);
        auto pi = ctx->patterns.find(f[1]);
        if (ti == ctx->targets.end() || pi == ctx->patterns.end()) return "checkpoint names an unknown target or pattern";
        if (ti->second->n != f[2] || pi->second->k != f[3]) return "checkpoint target or pattern size differs";
        dir[i] = ti->second->directed ? 1 : 0;
    }
    if (!get(S.ctr.data(), npairs * 32)) return "truncated checkpoint";
    std::vector<char> seen((size_t)npairs, 0);
    for (int32_t g = 0; g < ngroups; ++g) {
        CkptGroup G;
        int32_t kmax = 0, np = 0;
        int64_t nf = 0;
        if (!get(&kmax, 4) || !get(&np, 4) || !get(&nf, 8)) return "truncated checkpoint";
        if (kmax < 1 || kmax > KMAX || np < 1 || np > npairs || nf < 0) return "bad checkpoint group";
        G.kmax = kmax;
        G.idx.resize((size_t)np);
        if (!get(G.idx.data(), 4ll * np)) return "truncated checkpoint";
        if (np & 1) { int32_t z; if (!get(&z, 4)) return "truncated checkpoint"; }
        int gk = 1;
        for (int q = 0; q < np; ++q) {
            const int i = G.idx[q];
            if (i < 0 || i >= npairs || seen[i]) return "bad checkpoint group";
            if (dir[i] != dir[G.idx[0]]) return "checkpoint group mixes directedness";
            seen[i] = 1;
            if (S.k[i] <= S.nt[i]) gk = std::max(gk, S.k[i]);
        }
        if (gk != kmax) return "checkpoint group kmax differs from its pairs";
        const int stride = FRAME_HDR + kmax;
        if (nf > (bytes - at) / (4ll * stride)) return "truncated checkpoint";
        G.frames.resize((size_t)nf * stride);
        if (!get(G.frames.data(), nf * 4ll * stride)) return "truncated checkpoint";
        for (int64_t f = 0; f < nf; ++f) {
            const int32_t *fr = G.frames.data() + f * stride;
            const int j = fr[0];
            if (j < 0 || j >= np) return "checkpoint frame names no pair";
            const int i = G.idx[j];
            const int depth = fr[1] & FRAME_DEPTH_MASK;
            // (a counted range never lies on the last position: its matches are counted at once)
            if ((fr[1] & ~(FRAME_DEPTH_MASK | FRAME_COUNTED)) != 0 || S.k[i] > S.nt[i] || depth >= S.k[i] ||
                ((fr[1] & FRAME_COUNTED) && (depth >= S.k[i] - 1 || fr[2] < 0)))
                return "bad checkpoint frame depth";
            if (fr[2] < -1 || (fr[2] >= 0 && fr[3] < fr[2])) return "bad checkpoint frame range";
            for (int t = 0; t < depth; ++t)
                if (fr[FRAME_HDR + t] < 0 || fr[FRAME_HDR + t] >= S.nt[i]) return "bad checkpoint frame image";
        }
        S.groups.push_back(std::move(G));
    }
    if (at != bytes) return "checkpoint has trailing bytes";
    return std::string();
}

bool stop_status(sge_status rc) {
    return rc == SGE_ERR_BUDGET || rc == SGE_ERR_TIMEOUT || rc == SGE_ERR_CANCELLED;
}

// Runs S's groups (all of them from the start, or each group's frames when
// resuming), adds the counters to S.ctr, and leaves in each group the frames
// still unexplored.  Returns OK when nothing is left, else the first stop
// status (other errors end the call at once).
sge_status run_ckpt(sge_ctx *ctx, const sge_opts &o, CkptState &S, bool resume, sge_result *out) {
    sge_status first_stop = SGE_OK;
    std::vector<sge_result> tmp(S.reqs.size());
    for (size_t i = 0; i < S.reqs.size(); ++i) {
        std::memset(&out[i], 0, sizeof(sge_result));
        out[i].status = 0;
    }
    for (CkptGroup &G : S.groups) {
        if (G.kmax == 0) {   // the group's largest searchable pattern, as run_group sizes frames
            G.kmax = 1;
            for (int i : G.idx)
                if (S.k[i] <= S.nt[i]) G.kmax = std::max(G.kmax, (int)S.k[i]);
        }
        if (resume && G.frames.empty()) continue;
        Resume R;
        R.frames = G.frames.data();
        R.n = (long long)(G.frames.size() / (FRAME_HDR + G.kmax));
        R.kmax = G.kmax;
        std::vector<int32_t> left;
        int kmax = G.kmax;
        sge_status rc = run_group(ctx, ctx->ws, ctx->stream, S.reqs, G.idx, o, tmp.data(), false, nullptr, 0, false,
                                  resume ? &R : nullptr, &left, &kmax);
        if (rc != SGE_OK && !stop_status(rc)) return rc;
        if (rc != SGE_OK && first_stop == SGE_OK) first_stop = rc;
        for (int i : G.idx) {
            out[i] = tmp[i];
            S.ctr[4 * (size_t)i + 0] += tmp[i].matches;
            S.ctr[4 * (size_t)i + 1] += tmp[i].states;
            S.ctr[4 * (size_t)i + 2] += tmp[i].nodes;
            S.ctr[4 * (size_t)i + 3] += tmp[i].hash;
        }
        G.kmax = kmax;
        G.frames.swap(left);   // empty when the group finished
    }
    for (size_t i = 0; i < S.reqs.size(); ++i) {
        out[i].matches = S.ctr[4 * i + 0];
        out[i].states = S.ctr[4 * i + 1];
        out[i].nodes = S.ctr[4 * i + 2];
        out[i].hash = S.ctr[4 * i + 3];
    }
    if (first_stop != SGE_OK) {
        // a stop with nothing left to do (all the work fit before it) is a finished search
        bool left = false;
        for (const CkptGroup &G : S.groups) left = left || !G.frames.empty();
        if (!left) first_stop = SGE_OK;
    }
    return first_stop;
}

sge_status ckpt_hand_out(sge_ctx *ctx, const CkptState &S, sge_status rc, void **ckpt, int64_t *ckpt_bytes) {
    *ckpt = nullptr;
    *ckpt_bytes = 0;
    if (rc == SGE_OK) return SGE_OK;
    const std::vector<unsigned char> b = ckpt_write(S);
    void *p = std::malloc(b.size());
    if (!p) return fail(ctx, SGE_ERR_OOM, "checkpoint blob allocation failed");
    std::memcpy(p, b.data(), b.size());
    *ckpt = p;
    *ckpt_bytes = (int64_t)b.size();
    return rc;
}

sge_status load_graph_common(sge_ctx *ctx, int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                             const int32_t *vlabel, const int32_t *elabel, int32_t directed, Built &g) {
    if (!ctx) return SGE_ERR_ARG;
    std::string err;
    if (!build_graph(n, m, src, dst, vlabel, elabel, directed, g, err)) return fail(ctx, SGE_ERR_ARG, err);
    return SGE_OK;
}

void serve_worker(sge_ctx *ctx);

}  // namespace

// =================================================================== C ABI

extern "C" {

const char *sge_version(void) { return "sge-gb300 1.0 (sm_103a)"; }

sge_status sge_create(sge_ctx **out, int32_t device, void *cuda_stream) {
    if (!out) return SGE_ERR_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) return SGE_ERR_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return SGE_ERR_CUDA;
    sge_ctx *ctx = new (std::nothrow) sge_ctx();
    if (!ctx) return SGE_ERR_OOM;
    ctx->device = device;
    cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, device);
    {
        // workspaces allocate stream-ordered from the device's default pool: let the pool keep
        // what they free for their next growth instead of returning it at every synchronisation
        cudaMemPool_t mp;
        if (cudaDeviceGetDefaultMemPool(&mp, device) == cudaSuccess) {
            uint64_t keep = UINT64_MAX;
            cudaMemPoolSetAttribute(mp, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        (void)cudaGetLastError();
    }
    if (cuda_stream) {
        ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) { delete ctx; return SGE_ERR_CUDA; }
        ctx->own_stream = true;
    }
    if (cudaHostAlloc(reinterpret_cast<void **>(&ctx->cancel_host), sizeof(int), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer(reinterpret_cast<void **>(&ctx->cancel_dev), ctx->cancel_host, 0) != cudaSuccess) {
        if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
        delete ctx;
        return SGE_ERR_CUDA;
    }
    *ctx->cancel_host = 0;
    *out = ctx;
    return SGE_OK;
}

void sge_destroy(sge_ctx *ctx) {
    if (!ctx) return;
    {
        std::lock_guard<std::mutex> g(ctx->smu);
        ctx->sstop = true;
    }
    ctx->scv.notify_all();
    for (std::thread &t : ctx->sworkers) t.join();
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (auto &kv : ctx->targets) kv.second->release();
    for (auto &kv : ctx->patterns) kv.second->release();
    ctx->cache.clear();
    ctx->ws.release();
    ctx->ing.release();
    if (ctx->cancel_host) cudaFreeHost(ctx->cancel_host);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

sge_status sge_load_target(sge_ctx *ctx, int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                           const int32_t *vlabel, const int32_t *elabel, int32_t directed, int32_t *target_id) {
    if (!ctx || !target_id) return SGE_ERR_ARG;
    if (n < 0 || m < 0) return fail(ctx, SGE_ERR_ARG, "negative vertex or edge count");
    if (m > 0 && (!src || !dst)) return fail(ctx, SGE_ERR_ARG, "null edge arrays");
    if (n > 0 && !vlabel) return fail(ctx, SGE_ERR_ARG, "null vertex-label array");
    const long long arcs = directed ? m : 2 * m;   // stored arcs before repeats merge
    if (arcs > INT32_MAX) return fail(ctx, SGE_ERR_ARG, "more than 2^31-1 stored arcs");
    const double t_in = now_ms();
    cudaSetDevice(ctx->device);
    cudaStream_t st = ctx->stream;
    std::lock_guard<std::mutex> ig(ctx->ingest_mu);
    IngestWs &I = ctx->ing;
    auto T = std::make_unique<TargetRec>();
    T->use_cache(&ctx->cache);
    T->n = n;
    T->directed = directed != 0;
    T->dw = std::max(1, (n + 63) / 64);
    const size_t n1 = (size_t)n + 1;
    // the caller's arrays, once
    CK(I.src.ensure(std::max<long long>(m, 1) * 4), "alloc ingest");
    CK(I.dst.ensure(std::max<long long>(m, 1) * 4), "alloc ingest");
    CK(I.vlab.ensure(std::max<size_t>(n, 1) * 4), "alloc ingest");
    if (m > 0) {
        CK(cudaMemcpyAsync(I.src.p, src, (size_t)m * 4, cudaMemcpyHostToDevice, st), "upload edges");
        CK(cudaMemcpyAsync(I.dst.p, dst, (size_t)m * 4, cudaMemcpyHostToDevice, st), "upload edges");
    }
    if (n > 0) CK(cudaMemcpyAsync(I.vlab.p, vlabel, (size_t)n * 4, cudaMemcpyHostToDevice, st), "upload labels");
    const int32_t *d_elab = nullptr;
    if (elabel && m > 0) {
        CK(I.elab.ensure((size_t)m * 4), "alloc ingest");
        CK(cudaMemcpyAsync(I.elab.p, elabel, (size_t)m * 4, cudaMemcpyHostToDevice, st), "upload edge labels");
        d_elab = I.elab.as<int32_t>();
    }
    // scratch: per-vertex counters and offsets, arc keys
    const size_t nv = std::max<size_t>(n, 1);
    for (DevBuf *b : {&I.cnt_out, &I.cnt_in, &I.fill_out, &I.fill_in, &I.ucnt, &I.long_rows})
        CK(b->ensure(nv * 4), "alloc ingest");
    for (DevBuf *b : {&I.off_out, &I.off_in, &I.uoff}) CK(b->ensure(n1 * 8), "alloc ingest");
    CK(I.key_out.ensure((size_t)std::max<long long>(arcs, 1) * 8), "alloc ingest");
    CK(I.scratch.ensure((size_t)std::max<long long>(arcs, 1) * 8), "alloc ingest");
    if (directed) CK(I.key_in.ensure((size_t)std::max<long long>(m, 1) * 8), "alloc ingest");
    CK(I.small.ensure(64), "alloc ingest");
    CK(I.scan_tmp.ensure(scan_tmp_bytes(n)), "alloc ingest");
    int *flags = I.small.as<int>();
    int32_t *nlong = I.small.as<int32_t>() + 1;   // [1] out rows, [2] in rows
    CK(cudaMemsetAsync(I.small.p, 0, 64, st), "clear ingest");
    for (DevBuf *b : {&I.cnt_out, &I.cnt_in, &I.fill_out, &I.fill_in})
        CK(cudaMemsetAsync(b->p, 0, nv * 4, st), "clear ingest");
    CK(launch_ingest_count(I.src.as<int32_t>(), I.dst.as<int32_t>(), d_elab, m, n, directed ? 1 : 0,
                           I.cnt_out.as<int32_t>(), I.cnt_in.as<int32_t>(), flags, st), "ingest count");
    CK(launch_scan(I.cnt_out.as<int32_t>(), I.off_out.as<long long>(), n, I.off_out.as<long long>() + n,
                   I.scan_tmp.p, I.scan_tmp.cap, st), "ingest scan");
    if (directed)
        CK(launch_scan(I.cnt_in.as<int32_t>(), I.off_in.as<long long>(), n, I.off_in.as<long long>() + n,
                       I.scan_tmp.p, I.scan_tmp.cap, st), "ingest scan");
    CK(launch_ingest_scatter(I.src.as<int32_t>(), I.dst.as<int32_t>(), d_elab, m, n, directed ? 1 : 0,
                             I.off_out.as<long long>(), I.off_in.as<long long>(), I.fill_out.as<int32_t>(),
                             I.fill_in.as<int32_t>(), I.key_out.as<uint64_t>(), I.key_in.as<uint64_t>(), st),
       "ingest scatter");
    // sort and merge the rows of one direction, then compact them into the target's CSR
    auto rows = [&](DevBuf &off, DevBuf &keys, int32_t *nl, DevBuf &rowptr, DevBuf &colb, DevBuf &labb,
                    long long cap) -> cudaError_t {
        cudaError_t e = launch_ingest_rows(off.as<long long>(), n, keys.as<uint64_t>(), I.scratch.as<uint64_t>(),
                                           I.ucnt.as<int32_t>(), I.long_rows.as<int32_t>(), nl, flags, ctx->sms, st);
        if (e == cudaSuccess)
            e = launch_scan(I.ucnt.as<int32_t>(), I.uoff.as<long long>(), n, I.uoff.as<long long>() + n,
                            I.scan_tmp.p, I.scan_tmp.cap, st);
        if (e == cudaSuccess) e = rowptr.ensure(n1 * 4);
        if (e == cudaSuccess) e = colb.ensure((size_t)std::max<long long>(cap, 1) * 4);
        if (e == cudaSuccess) e = labb.ensure((size_t)std::max<long long>(cap, 1) * 4);
        if (e == cudaSuccess)
            e = launch_ingest_compact(off.as<long long>(), I.uoff.as<long long>(), I.ucnt.as<int32_t>(),
                                      I.uoff.as<long long>() + n, keys.as<uint64_t>(), n, rowptr.as<int32_t>(),
                                      colb.as<int32_t>(), labb.as<int32_t>(), st);
        return e;
    };
    long long nnz[2] = {0, 0};
    CK(rows(I.off_out, I.key_out, nlong, T->rowptr, T->col, T->elab, arcs), "ingest rows");
    CK(cudaMemcpyAsync(&nnz[0], I.uoff.as<long long>() + n, 8, cudaMemcpyDeviceToHost, st), "read arc count");
    if (directed) {
        CK(rows(I.off_in, I.key_in, nlong + 1, T->irowptr, T->icol, T->ielab, m), "ingest in-rows");
        CK(cudaMemcpyAsync(&nnz[1], I.uoff.as<long long>() + n, 8, cudaMemcpyDeviceToHost, st), "read arc count");
        CK(T->indeg.ensure(nv * 4), "alloc in-degree");
        CK(launch_ingest_degree(T->irowptr.as<int32_t>(), n, T->indeg.as<int32_t>(), st), "in-degree");
    }
    CK(T->vld.ensure(nv * sizeof(int2)), "alloc vertex info");
    CK(launch_make_vld(T->rowptr.as<int32_t>(), I.vlab.as<int32_t>(), T->vld.as<int2>(), n, st), "vertex info");
    int32_t *d_maxdeg = I.small.as<int32_t>() + 3;   // (zeroed with the ingest flags)
    CK(launch_ingest_maxdeg(T->rowptr.as<int32_t>(), n, d_maxdeg, st), "longest row");
    if (directed) CK(launch_ingest_maxdeg(T->irowptr.as<int32_t>(), n, d_maxdeg, st), "longest row");
    if (!directed && n > 0) {
        // the largest neighbour degree per (vertex, label): domain initialisation reads it to
        // drop, at once, the candidates that have no neighbour able to carry some pattern edge
        std::vector<int32_t> labs(vlabel, vlabel + n);
        std::sort(labs.begin(), labs.end());
        labs.erase(std::unique(labs.begin(), labs.end()), labs.end());
        const long long L = (long long)labs.size();
        if ((long long)n * L <= LABEL_TABLE_MAX) {
            std::vector<int32_t> lidx((size_t)n);
            for (int v = 0; v < n; ++v)
                lidx[(size_t)v] = (int32_t)(std::lower_bound(labs.begin(), labs.end(), vlabel[v]) - labs.begin());
            T->nlab = (int)L;
            T->labs_h = labs;
            T->ltab_off = (int)((L + 3) & ~3LL);
            CK(T->ltab.ensure(((size_t)T->ltab_off + (size_t)n * L) * 4), "alloc label table");
            CK(cudaMemcpyAsync(T->ltab.p, labs.data(), (size_t)L * 4, cudaMemcpyHostToDevice, st), "upload labels");
            CK(cudaMemcpyAsync(I.fill_out.p, lidx.data(), (size_t)n * 4, cudaMemcpyHostToDevice, st),
               "upload label indices");
            CK(launch_label_nbmax(T->rowptr.as<int32_t>(), T->col.as<int32_t>(), T->vld.as<int2>(),
                                  I.fill_out.as<int32_t>(), n, (int)L, T->ltab.as<int32_t>() + T->ltab_off, st),
               "label table");
            const long long ldm_words = L * LDM_DEGREES * T->dw;
            if (n <= LDM_MAX_N && ldm_words <= LDM_MAX_WORDS) {
                CK(T->ldm.ensure((size_t)ldm_words * 8), "alloc label-degree masks");
                CK(launch_label_degree_masks(T->vld.as<int2>(), n, T->ltab.as<int32_t>(), (int)L, T->dw,
                                             T->ldm.as<uint64_t>(), st),
                   "label-degree masks");
            }
            if (n > BITSET_MAX_N) {
                // label buckets: vertices by label index, descending degree within a label, so that
                // a pattern vertex's initial domain is one bucket prefix (domain initialisation then
                // touches its candidates only, not all n vertices)
                std::vector<int2> vld_h((size_t)n);
                CK(cudaMemcpyAsync(vld_h.data(), T->vld.p, (size_t)n * sizeof(int2), cudaMemcpyDeviceToHost, st),
                   "read vertex records");
                CK(cudaStreamSynchronize(st), "read vertex records");
                std::vector<int32_t> ord((size_t)n);
                for (int v = 0; v < n; ++v) ord[(size_t)v] = v;
                std::sort(ord.begin(), ord.end(), [&](int a, int b) {
                    if (lidx[(size_t)a] != lidx[(size_t)b]) return lidx[(size_t)a] < lidx[(size_t)b];
                    if (vld_h[(size_t)a].y != vld_h[(size_t)b].y) return vld_h[(size_t)a].y > vld_h[(size_t)b].y;
                    return a < b;
                });
                std::vector<int32_t> bk((size_t)n * 2 + (size_t)L + 1);
                for (int x = 0; x < n; ++x) {
                    bk[(size_t)x] = ord[(size_t)x];
                    bk[(size_t)n + x] = vld_h[(size_t)ord[(size_t)x]].y;
                }
                int32_t *start = bk.data() + 2 * (size_t)n;
                for (long long l = 0; l <= L; ++l) start[l] = 0;
                for (int v = 0; v < n; ++v) ++start[lidx[(size_t)v] + 1];
                for (long long l = 0; l < L; ++l) start[l + 1] += start[l];
                CK(upload(T->lbk, bk, st), "upload label buckets");
            }
        }
    }
    if (!directed && n > 0 && n <= BITSET_MAX_N) {
        CK(T->adj.ensure((size_t)n * T->dw * 8), "alloc adjacency bitset");
        CK(cudaMemsetAsync(T->adj.p, 0, (size_t)n * T->dw * 8, st), "clear adjacency bitset");
        CK(launch_ingest_bits(T->rowptr.as<int32_t>(), T->col.as<int32_t>(), n, T->dw, T->adj.as<uint64_t>(), st),
           "adjacency bitset");
    }
    int32_t hsmall[4] = {0, 0, 0, 0};   // flags, long out-rows, long in-rows, longest row
    CK(cudaMemcpyAsync(hsmall, flags, sizeof(hsmall), cudaMemcpyDeviceToHost, st), "read ingest flags");
    CK(cudaStreamSynchronize(st), "target ingest");
    const int hflags = hsmall[0];
    T->maxdeg = hsmall[3];
    const char *bad = (hflags & ING_RANGE) ? "edge endpoint out of range"
                      : (hflags & ING_LOOP) ? "self-loop"
                      : (hflags & ING_LABEL) ? "repeated edge with a different label" : nullptr;
    if (bad) {
        T->release();
        return fail(ctx, SGE_ERR_ARG, bad);
    }
    T->any_elab = (hflags & ING_ELAB) != 0;
    T->nnz = nnz[0];
    if (!directed && n > BITSET_MAX_N) {
        // hub rows: the highest-degree vertices get a bitset row (rule 4 becomes one bit test)
        std::vector<int32_t> ptr(n1);
        CK(cudaMemcpy(ptr.data(), T->rowptr.p, n1 * 4, cudaMemcpyDeviceToHost), "read row offsets");
        std::vector<int32_t> order;
        for (int v = 0; v < n; ++v)
            if (ptr[v + 1] - ptr[v] >= HUB_MIN_DEGREE) order.push_back(v);
        std::sort(order.begin(), order.end(), [&](int a, int b) {
            const int da = ptr[a + 1] - ptr[a], db = ptr[b + 1] - ptr[b];
            return da != db ? da > db : a < b;
        });
        const long long max_hubs = HUB_BYTES / ((long long)T->dw * 8);
        if ((long long)order.size() > max_hubs) order.resize((size_t)max_hubs);
        if (!order.empty()) {
            std::vector<int32_t> slot((size_t)n, -1);
            for (size_t i = 0; i < order.size(); ++i) slot[order[i]] = (int32_t)i;
            CK(upload(T->hub_slot, slot, st), "upload hub slots");
            CK(upload(T->hub_list, order, st), "upload hub list");
            CK(T->hub_bits.ensure(order.size() * (size_t)T->dw * 8), "alloc hub rows");
            CK(launch_build_hubs(T->rowptr.as<int32_t>(), T->col.as<int32_t>(), T->hub_list.as<int32_t>(),
                                 (int)order.size(), T->dw, T->hub_bits.as<uint64_t>(), st), "hub rows");
            CK(cudaStreamSynchronize(st), "hub rows");
        }
    }
    if (trace_on()) std::fprintf(stderr, "[sge] target n %d: ingested on the device in %.3f ms\n", n, now_ms() - t_in);
    std::lock_guard<std::mutex> gd(ctx->mu);
    const int id = ctx->next_target++;
    T->cached = T->view();
    ctx->targets[id] = std::move(T);
    *target_id = id;
    return SGE_OK;
}

sge_status sge_load_pattern(sge_ctx *ctx, int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                            const int32_t *vlabel, const int32_t *elabel, int32_t directed, int32_t *pattern_id) {
    if (!ctx || !pattern_id) return SGE_ERR_ARG;
    if (n > KMAX) return fail(ctx, SGE_ERR_ARG, "pattern has more than 128 vertices");
    Built g;
    sge_status rc = load_graph_common(ctx, n, m, src, dst, vlabel, elabel, directed, g);
    if (rc != SGE_OK) return rc;
    cudaSetDevice(ctx->device);
    cudaStream_t st = ctx->stream;
    auto P = std::make_unique<PatternRec>();
    P->use_cache(&ctx->cache);
    P->k = n;
    P->directed = g.directed;
    P->any_elab = g.any_elab;
    P->lab = g.vlab;
    P->odeg = g.odeg;
    P->ideg = g.ideg;
    P->amat.assign((size_t)n * n, NO_ARC);
    P->nb.assign(2 * (size_t)n, 0);
    for (int v = 0; v < n; ++v)
        for (int e = g.out.ptr[v]; e < g.out.ptr[v + 1]; ++e) {
            const int w = g.out.col[e];
            P->amat[(size_t)v * n + w] = g.out.lab[e];
            P->nb[2 * v + (w >> 6)] |= 1ull << (w & 63);
            P->nb[2 * w + (v >> 6)] |= 1ull << (v & 63);
        }
    gcf_order(*P, SGE_RI, nullptr, P->ri_mu, P->ri_par);
    build_positions(*P, P->ri_mu, P->ri_par, SGE_RI, nullptr, 0, P->ri_pos, P->ri_back);
    std::vector<int32_t> img;   // the host image of P->dall
    auto put = [&img](const std::vector<int32_t> &v) {
        const size_t at = img.size();
        img.insert(img.end(), v.begin(), v.end());
        img.resize((img.size() + 3) & ~size_t(3), 0);
        return at;
    };
    P->o_lab = put(g.vlab);
    P->o_odeg = put(g.odeg);
    P->o_row = put(g.out.ptr);
    P->o_col = put(g.out.col);
    P->o_elab = put(g.out.lab);
    if (g.directed) {
        P->o_ideg = put(g.ideg);
        P->o_irow = put(g.in.ptr);
        P->o_icol = put(g.in.col);
        P->o_ielab = put(g.in.lab);
    }
    CK(upload(P->dall, img, st), "upload pattern");
    CK(cudaStreamSynchronize(st), "pattern upload");
    std::lock_guard<std::mutex> gd(ctx->mu);
    const int id = ctx->next_pattern++;
    P->cached = P->view();
    ctx->patterns[id] = std::move(P);
    *pattern_id = id;
    return SGE_OK;
}

sge_status sge_unload_target(sge_ctx *ctx, int32_t target_id) {
    if (!ctx) return SGE_ERR_ARG;
    std::lock_guard<std::mutex> g(ctx->mu);
    auto it = ctx->targets.find(target_id);
    if (it == ctx->targets.end()) return SGE_ERR_NOT_FOUND;
    // the blocks go back to the context's cache: wait until no kernel on any stream reads them
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    it->second->release();
    ctx->targets.erase(it);
    return SGE_OK;
}

sge_status sge_unload_pattern(sge_ctx *ctx, int32_t pattern_id) {
    if (!ctx) return SGE_ERR_ARG;
    std::lock_guard<std::mutex> g(ctx->mu);
    auto it = ctx->patterns.find(pattern_id);
    if (it == ctx->patterns.end()) return SGE_ERR_NOT_FOUND;
    // the blocks go back to the context's cache: wait until no kernel on any stream reads them
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    it->second->release();
    ctx->patterns.erase(it);
    return SGE_OK;
}

sge_status sge_count(sge_ctx *ctx, int32_t target_id, int32_t pattern_id, const sge_opts *opts, sge_result *out) {
    if (!ctx || !out) return SGE_ERR_ARG;
    cudaSetDevice(ctx->device);
    *ctx->cancel_host = 0;
    std::vector<PairReq> reqs{{target_id, pattern_id}};
    return run_pairs(ctx, ctx->ws, ctx->stream, reqs, opts, out, false, nullptr, 0);
}

sge_status sge_count_batch(sge_ctx *ctx, int64_t npairs, const int32_t *target_ids, const int32_t *pattern_ids,
                           const sge_opts *opts, sge_result *out) {
    if (!ctx || !out || npairs < 0 || (npairs > 0 && (!target_ids || !pattern_ids))) return SGE_ERR_ARG;
    if (npairs > INT32_MAX / 8) return fail(ctx, SGE_ERR_ARG, "too many pairs");
    cudaSetDevice(ctx->device);
    *ctx->cancel_host = 0;
    std::vector<PairReq> reqs((size_t)npairs);
    for (int64_t i = 0; i < npairs; ++i) reqs[i] = {target_ids[i], pattern_ids[i]};
    if (npairs == 0) return SGE_OK;
    return run_pairs(ctx, ctx->ws, ctx->stream, reqs, opts, out, false, nullptr, 0);
}

sge_status sge_count_batch_ckpt(sge_ctx *ctx, int64_t npairs, const int32_t *target_ids, const int32_t *pattern_ids,
                                const sge_opts *opts, sge_result *out, void **ckpt, int64_t *ckpt_bytes) {
    if (!ctx || !out || !ckpt || !ckpt_bytes || npairs < 0 || (npairs > 0 && (!target_ids || !pattern_ids)))
        return SGE_ERR_ARG;
    *ckpt = nullptr;
    *ckpt_bytes = 0;
    if (npairs > INT32_MAX / 8) return fail(ctx, SGE_ERR_ARG, "too many pairs");
    if (npairs == 0) return SGE_OK;
    cudaSetDevice(ctx->device);
    *ctx->cancel_host = 0;
    CkptState S;
    S.reqs.resize((size_t)npairs);
    for (int64_t i = 0; i < npairs; ++i) S.reqs[i] = {target_ids[i], pattern_ids[i]};
    sge_opts o;
    std::vector<int> und, dir;
    sge_status rc = prepare_pairs(ctx, S.reqs, opts, o, und, dir);
    if (rc != SGE_OK) return rc;
    S.algo = o.algo;
    S.nt.resize((size_t)npairs);
    S.k.resize((size_t)npairs);
    S.ctr.assign((size_t)npairs * 4, 0);
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        for (int64_t i = 0; i < npairs; ++i) {
            S.nt[i] = ctx->targets.at(S.reqs[i].tid)->n;
            S.k[i] = ctx->patterns.at(S.reqs[i].pid)->k;
        }
    }
    for (std::vector<int> *grp : {&und, &dir})
        if (!grp->empty()) {
            CkptGroup G;
            G.idx = *grp;
            S.groups.push_back(std::move(G));
        }
    rc = run_ckpt(ctx, o, S, false, out);
    return ckpt_hand_out(ctx, S, rc, ckpt, ckpt_bytes);
}

sge_status sge_resume(sge_ctx *ctx, const void *ckpt, int64_t ckpt_bytes, const sge_opts *opts, sge_result *out,
                      void **next, int64_t *next_bytes) {
    if (!ctx || !ckpt || ckpt_bytes <= 0 || !out || !next || !next_bytes) return SGE_ERR_ARG;
    *next = nullptr;
    *next_bytes = 0;
    cudaSetDevice(ctx->device);
    *ctx->cancel_host = 0;
    CkptState S;
    const std::string err = ckpt_read(ctx, static_cast<const unsigned char *>(ckpt), ckpt_bytes, S);
    if (!err.empty()) return fail(ctx, SGE_ERR_ARG, err);
    sge_opts o;
    std::vector<int> und, dir;
    sge_opts oi;
    std::memset(&oi, 0, sizeof(oi));
    if (opts) oi = *opts;
    oi.algo = S.algo;          // the frames follow the checkpoint's variant
    oi.shard_count = 0;        // and hold only this shard's work already
    oi.shard_index = 0;
    sge_status rc = prepare_pairs(ctx, S.reqs, &oi, o, und, dir);
    if (rc != SGE_OK) return rc;
    rc = run_ckpt(ctx, o, S, true, out);
    return ckpt_hand_out(ctx, S, rc, next, next_bytes);
}

sge_status sge_ckpt_info(const void *ckpt, int64_t ckpt_bytes, int64_t *npairs, int64_t *nframes) {
    if (!ckpt || ckpt_bytes < 32 || !npairs || !nframes) return SGE_ERR_ARG;
    const unsigned char *b = static_cast<const unsigned char *>(ckpt);
    uint64_t magic = 0;
    int32_t version = 0, ngroups = 0;
    int64_t np = 0;
    std::memcpy(&magic, b, 8);
    std::memcpy(&version, b + 8, 4);
    std::memcpy(&np, b + 16, 8);
    std::memcpy(&ngroups, b + 24, 4);
    if (magic != CKPT_MAGIC || version != CKPT_VERSION || np < 0 || ngroups < 0 || ngroups > 2) return SGE_ERR_ARG;
    long long at = 32 + np * 48;
    long long frames = 0;
    for (int g = 0; g < ngroups; ++g) {
        int32_t kmax = 0, n = 0;
        int64_t nf = 0;
        if (at + 16 > ckpt_bytes) return SGE_ERR_ARG;
        std::memcpy(&kmax, b + at, 4);
        std::memcpy(&n, b + at + 4, 4);
        std::memcpy(&nf, b + at + 8, 8);
        if (kmax < 1 || kmax > KMAX || n < 0 || nf < 0) return SGE_ERR_ARG;
        at += 16 + 4ll * (n + (n & 1)) + nf * 4ll * (FRAME_HDR + kmax);
        frames += nf;
    }
    if (at != ckpt_bytes) return SGE_ERR_ARG;
    *npairs = np;
    *nframes = frames;
    return SGE_OK;
}

void sge_free(void *p) { std::free(p); }

sge_status sge_enumerate(sge_ctx *ctx, int32_t target_id, int32_t pattern_id, const sge_opts *opts,
                         sge_match_sink sink, void *user, sge_result *out) {
    if (!ctx || !out || !sink) return SGE_ERR_ARG;
    cudaSetDevice(ctx->device);
    *ctx->cancel_host = 0;
    std::vector<PairReq> reqs{{target_id, pattern_id}};
    // count first to size the match buffer exactly, then enumerate
    sge_result first;
    sge_status rc = run_pairs(ctx, ctx->ws, ctx->stream, reqs, opts, &first, false, nullptr, 0);
    if (rc != SGE_OK) { *out = first; return rc; }
    int k = 0;
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        k = ctx->patterns.at(pattern_id)->k;
    }
    if ((long long)first.matches * std::max(k, 1) * 4 > (1ll << 32))
        return fail(ctx, SGE_ERR_OOM, "match list larger than 4 GiB; use sge_count");
    std::vector<int32_t> rows;
    rc = run_pairs(ctx, ctx->ws, ctx->stream, reqs, opts, out, true, &rows, (long long)first.matches);
    if (rc != SGE_OK) return rc;
    const long long n = k > 0 ? (long long)rows.size() / k : 0;
    const long long chunk = 1 << 16;
    for (long long i = 0; i < n; i += chunk) {
        const long long c = std::min(chunk, n - i);
        if (sink(user, rows.data() + i * k, c, k) != 0) return fail(ctx, SGE_ERR_STOPPED, "sink stopped");
    }
    return SGE_OK;
}

// No device allocation: see include/sge.h.  The pattern's host-side tables
// (about 200 KB at 128 vertices) live in one host heap block freed on return,
// so the call needs little stack; all device-side data lives in the library's
// fixed scratch array (sge_noalloc.cu).
namespace {
struct NoallocHost {
    int amat[KMAX * KMAX];
    uint64_t nbits[2 * KMAX];
    int32_t lab[KMAX], odeg[KMAX];
    int mu[KMAX], par[KMAX];
    PosInfo pos[KMAX];
    BackEdge back[KMAX * (KMAX - 1) / 2 + 1];
};
}  // namespace

sge_status sge_count_noalloc(int32_t n, const int32_t *d_rowptr, const int32_t *d_col, const int32_t *d_vlabel,
                             const int32_t *d_elabel, int32_t k, int64_t m, const int32_t *src, const int32_t *dst,
                             const int32_t *vlabel, const int32_t *elabel, void *cuda_stream, int64_t time_limit_ms,
                             uint64_t *out) {
    if (!out || n < 0 || k < 0 || m < 0) return SGE_ERR_ARG;
    out[0] = out[1] = out[2] = out[3] = 0;
    if (k > KMAX) return SGE_ERR_ARG;
    if (n > 0 && (!d_rowptr || !d_vlabel)) return SGE_ERR_ARG;
    if (m > 0 && (!src || !dst)) return SGE_ERR_ARG;
    if (k > 0 && !vlabel) return SGE_ERR_ARG;
    if (k == 0 || k > n) return SGE_OK;                  // no match and no search
    // the pattern, validated into fixed-size host tables
    std::unique_ptr<NoallocHost> hbuf(new (std::nothrow) NoallocHost);
    if (!hbuf) return SGE_ERR_OOM;
    int *amat = hbuf->amat;
    uint64_t *nbits = hbuf->nbits;
    int32_t *lab = hbuf->lab, *odeg = hbuf->odeg;
    bool any_elab = d_elabel != nullptr;
    for (int i = 0; i < k * k; ++i) amat[i] = NO_ARC;
    for (int i = 0; i < 2 * k; ++i) nbits[i] = 0;
    for (int64_t e = 0; e < m; ++e) {
        const int a = src[e], b = dst[e], l = elabel ? elabel[e] : 0;
        if (a < 0 || a >= k || b < 0 || b >= k || a == b) return SGE_ERR_ARG;
        if (amat[a * k + b] != NO_ARC && amat[a * k + b] != l) return SGE_ERR_ARG;
        amat[a * k + b] = amat[b * k + a] = l;
        nbits[2 * a + (b >> 6)] |= 1ull << (b & 63);
        nbits[2 * b + (a >> 6)] |= 1ull << (a & 63);
        if (l != 0) any_elab = true;
    }
    for (int v = 0; v < k; ++v) {
        lab[v] = vlabel[v];
        odeg[v] = __builtin_popcountll(nbits[2 * v]) + __builtin_popcountll(nbits[2 * v + 1]);
    }
    const PatView P{k, false, lab, odeg, odeg, amat, nbits};
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int *mu = hbuf->mu, *par = hbuf->par;
    gcf_order_into(P, SGE_RI, nullptr, mu, par);
    PosInfo *pos = hbuf->pos;
    BackEdge *back = hbuf->back;
    const int nb = build_positions_into(P, mu, par, SGE_RI, nullptr, n, pos, back);

    void *base = nullptr;
    size_t cap = 0;
    if (noalloc_scratch(&base, &cap) != cudaSuccess) return SGE_ERR_CUDA;
    int32_t nnz = 0;
    const bool zero_elab = any_elab && d_elabel == nullptr;   // labelled pattern, unlabelled target
    if (zero_elab) {
        // rowptr[n] read on the caller's stream, after whatever the caller queued there to fill it
        if (cudaMemcpyAsync(&nnz, d_rowptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return SGE_ERR_CUDA;
        if (nnz < 0) return SGE_ERR_ARG;
    }
    // carve the scratch (256-byte aligned pieces)
    constexpr int POOL = 2048;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = (off + bytes + 255) & ~(size_t)255;
        return static_cast<unsigned char *>(base) + at;
    };
    JobDesc *djob = reinterpret_cast<JobDesc *>(take(sizeof(JobDesc)));
    unsigned long long *dctr = reinterpret_cast<unsigned long long *>(take(6 * 8));
    unsigned char *dctl = take(CTL_BYTES);
    int32_t *dfront = reinterpret_cast<int32_t *>(take(FRAME_HDR * 4));
    PosInfo *dpos = reinterpret_cast<PosInfo *>(take((size_t)k * sizeof(PosInfo)));
    BackEdge *dback = reinterpret_cast<BackEdge *>(take((size_t)(nb > 0 ? nb : 1) * sizeof(BackEdge)));
    unsigned long long *dseq = reinterpret_cast<unsigned long long *>(take((size_t)POOL * 8));
    int32_t *dpool = reinterpret_cast<int32_t *>(take((size_t)POOL * POOL_STRIDE * 4));
    int2 *dvld = reinterpret_cast<int2 *>(take((size_t)n * sizeof(int2)));
    int32_t *delab = zero_elab ? reinterpret_cast<int32_t *>(take((size_t)nnz * 4)) : nullptr;
    if (off > cap) return SGE_ERR_ARG;   // target too large for the fixed scratch

    JobDesc D;
    std::memset(&D, 0, sizeof(D));
    D.t.n = n;
    D.t.dw = (n + 63) / 64;
    D.t.rowptr = D.t.irowptr = d_rowptr;
    D.t.col = D.t.icol = d_col;
    D.t.elab = D.t.ielab = zero_elab ? delab : d_elabel;
    D.t.vld = dvld;
    D.pos = dpos;
    D.back = dback;
    D.k = k;
    D.flags = any_elab ? JOB_ELAB : 0;
    D.ctr = dctr;
    D.mlen = dctr + 4;
    D.abytes = dctr + 5;
    const int32_t root[FRAME_HDR] = {0, 0, -1, -1};
    const int one = 1;
    SearchCtl C;
    std::memset(&C, 0, sizeof(C));
    bind_control(C, dctl);
    cudaError_t e = cudaSuccess;
    auto ok = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
    ok(launch_make_vld(d_rowptr, d_vlabel, dvld, n, st));
    if (zero_elab) ok(cudaMemsetAsync(delab, 0, (size_t)nnz * 4, st));
    // every call shares the array: clear what must start at zero
    ok(cudaMemsetAsync(dctr, 0, 6 * 8, st));
    ok(cudaMemsetAsync(dctl, 0, CTL_BYTES, st));
    ok(cudaMemcpyAsync(djob, &D, sizeof(D), cudaMemcpyHostToDevice, st));
    ok(cudaMemcpyAsync(dpos, pos, (size_t)k * sizeof(PosInfo), cudaMemcpyHostToDevice, st));
    if (nb > 0) ok(cudaMemcpyAsync(dback, back, (size_t)nb * sizeof(BackEdge), cudaMemcpyHostToDevice, st));
    ok(cudaMemcpyAsync(dfront, root, sizeof(root), cudaMemcpyHostToDevice, st));
    ok(cudaMemcpyAsync(C.outstanding, &one, sizeof(int), cudaMemcpyHostToDevice, st));
    ok(launch_pool_init(dseq, POOL, st));
    if (e != cudaSuccess) return SGE_ERR_CUDA;
    C.front = dfront;
    C.nfront = 1;
    C.fstride = FRAME_HDR;
    C.shard_index = 0;
    C.shard_count = 1;
    C.pcap = POOL;
    C.pool = dpool;
    C.pseq = dseq;
    if (time_limit_ms <= 0) {
        const char *env = std::getenv("SGE_TIME_LIMIT_MS");
        if (env) time_limit_ms = std::atoll(env);
    }
    C.deadline_ns = time_limit_ms > 0 ? (unsigned long long)time_limit_ms * 1000000ull : 0ull;
    C.donate = 1;
    C.gran = 2;
    C.donate_iters = 1024;
    C.donate_ns = 500000ull;
    int grid = 0;
    ok(launch_search(1, djob, C, k, 1, 0, 0, 0, &grid, st));
    unsigned long long hc[4] = {0, 0, 0, 0};
    int status = 0;
    ok(cudaMemcpyAsync(hc, dctr, sizeof(hc), cudaMemcpyDeviceToHost, st));
    ok(cudaMemcpyAsync(&status, C.status, sizeof(int), cudaMemcpyDeviceToHost, st));
    ok(cudaStreamSynchronize(st));
    if (e != cudaSuccess) return SGE_ERR_CUDA;
    for (int i = 0; i < 4; ++i) out[i] = hc[i];
    return status;
}

sge_status sge_cancel(sge_ctx *ctx) {
    if (!ctx || !ctx->cancel_host) return SGE_ERR_ARG;
    *reinterpret_cast<volatile int *>(ctx->cancel_host) = 1;
    return SGE_OK;
}

const char *sge_last_error(sge_ctx *ctx) {
    if (!ctx) return "null context";
    return ctx->err.c_str();
}

}  // extern "C"

// ================================================================ serving

namespace {

constexpr int SERVE_SLOTS = 4;               // concurrent launch groups (one stream each)
constexpr int SERVE_GROUP_MAX = 64;          // queries admitted into one launch (a group ends with its slowest query)
constexpr long long SERVE_BYTES = 2ll << 30; // device memory budget for admitted queries

long long query_bytes(const TargetRec &t, const PatternRec &p) {
    // filter block + frontier estimate + pool share
    return (long long)p.k * t.dw * 8 + (1ll << 20);
}

void serve_worker(sge_ctx *ctx) {
    cudaSetDevice(ctx->device);
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return;
    Workspace W;
    for (;;) {
        std::vector<std::shared_ptr<ServeReq>> group;
        long long bytes = 0;
        {
            std::unique_lock<std::mutex> lk(ctx->smu);
            ctx->scv.wait(lk, [&] { return ctx->sstop || !ctx->squeue.empty(); });
            if (ctx->sstop && ctx->squeue.empty()) break;
            // admit queued queries while they fit the memory budget
            while (!ctx->squeue.empty() && (int)group.size() < SERVE_GROUP_MAX) {
                auto &r = ctx->squeue.front();
                if (!group.empty() && (ctx->sbytes_in_use + bytes + r->bytes > SERVE_BYTES ||
                                       std::memcmp(&r->opts, &group[0]->opts, sizeof(sge_opts)) != 0))
                    break;
                bytes += r->bytes;
                group.push_back(r);
                ctx->squeue.pop_front();
            }
            ctx->sbytes_in_use += bytes;
            ctx->sinflight += (int)group.size();
        }
        const double t_admit = now_ms();
        std::vector<PairReq> reqs;
        for (auto &r : group) reqs.push_back({r->tid, r->pid});
        std::vector<sge_result> res(group.size());
        const sge_opts o = group[0]->opts;
        // a serving group: idle warps exit early and the split runs one block per SM
        sge_status rc = run_pairs(ctx, W, st, reqs, &o, res.data(), false, nullptr, 0, true);
        const double t_done = now_ms();
        {
            std::lock_guard<std::mutex> lk(ctx->smu);
            for (size_t i = 0; i < group.size(); ++i) {
                group[i]->res = res[i];
                group[i]->res.latency_ms = t_done - group[i]->t_submit;
                group[i]->res.queue_ms = (float)(t_admit - group[i]->t_submit);
                if (rc != SGE_OK && res[i].status == 0) group[i]->res.status = rc;
                group[i]->done = true;
            }
            ctx->sbytes_in_use -= bytes;
            ctx->sinflight -= (int)group.size();
        }
        ctx->scv.notify_all();
    }
    W.release();
    cudaStreamDestroy(st);
}

}  // namespace

extern "C" {

sge_status sge_serve_submit(sge_ctx *ctx, int32_t target_id, int32_t pattern_id, const sge_opts *opts,
                            int64_t *ticket) {
    if (!ctx || !ticket) return SGE_ERR_ARG;
    auto r = std::make_shared<ServeReq>();
    r->tid = target_id;
    r->pid = pattern_id;
    std::memset(&r->opts, 0, sizeof(sge_opts));
    if (opts) r->opts = *opts;
    std::memset(&r->res, 0, sizeof(r->res));
    r->t_submit = now_ms();
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        auto ti = ctx->targets.find(target_id);
        auto pi = ctx->patterns.find(pattern_id);
        if (ti == ctx->targets.end() || pi == ctx->patterns.end()) {
            ctx->err = "unknown target or pattern id";
            return SGE_ERR_NOT_FOUND;
        }
        r->bytes = query_bytes(*ti->second, *pi->second);
    }
    {
        std::lock_guard<std::mutex> lk(ctx->smu);
        if (ctx->sworkers.empty())
            for (int i = 0; i < SERVE_SLOTS; ++i) ctx->sworkers.emplace_back(serve_worker, ctx);
        *ticket = ctx->next_ticket++;
        ctx->sreqs[*ticket] = r;
        ctx->squeue.push_back(r);
    }
    ctx->scv.notify_all();
    return SGE_OK;
}

sge_status sge_serve_poll(sge_ctx *ctx, int64_t ticket, int32_t *done, sge_result *out) {
    if (!ctx || !done) return SGE_ERR_ARG;
    std::lock_guard<std::mutex> lk(ctx->smu);
    auto it = ctx->sreqs.find(ticket);
    if (it == ctx->sreqs.end()) return SGE_ERR_NOT_FOUND;
    *done = it->second->done ? 1 : 0;
    if (*done) {
        if (out) *out = it->second->res;
        ctx->sreqs.erase(it);
    }
    return SGE_OK;
}

sge_status sge_serve_drain(sge_ctx *ctx) {
    if (!ctx) return SGE_ERR_ARG;
    std::unique_lock<std::mutex> lk(ctx->smu);
    ctx->scv.wait(lk, [&] { return ctx->squeue.empty() && ctx->sinflight == 0; });
    return SGE_OK;
}

}  // extern "C"
