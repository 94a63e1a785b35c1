// sge_kernels.cu -- sm_103a kernels of the subgraph-enumeration engine.
//
// Method (arXiv 1705.09358): RI backtracking search (Section "RI": static
// GreatestConstraintFirst order, candidates from the adjacency of the
// parent's image, pruning rules 1-4) and RI-DS (Section 4: domains D(v)
// pruned by arc consistency, forward checking of singleton domains).
//
// GPU design (not the paper's CPU work-stealing runtime):
//  * domain kernels: one warp per 64-target bitset word; arc consistency and
//    forward checking iterate to their joint fixpoint under a host loop;
//  * split: breadth-first expansion of the search tree, one warp per frame,
//    until the frontier holds enough frames for every resident warp;
//  * persistent search: one warp owns one depth-first search.  The CSR kernel
//    scans the candidate row 32 candidates at a time (one per lane), tests
//    rules 1-4 per lane and compacts survivors with a ballot; the bitset kernel
//    computes a whole candidate set as the AND of the parent's adjacency row,
//    the back-neighbours' rows and the filter D(mu_i), one 64-bit word per
//    lane.  Idle warps take frames from the frontier, then from a bounded
//    lock-free queue into which busy warps donate their shallowest unexplored
//    work (the paper's "steal from the back of the deque" idea without deques).
//  * every wait is bounded; cancellation, deadline and state budget are
//    checked periodically and reported through a status word.
#include "sge_internal.h"

#include <cuda/atomic>

#include <algorithm>

namespace sge {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int WARPS_PER_BLOCK = 8;
constexpr int BLOCK = WARPS_PER_BLOCK * 32;
constexpr unsigned long long CHECK_NS = 20000;         // device time between donation / abort checks
// (the timer is read every 8 iterations of the CSR kernel and every 64 of the bitset kernel,
// whose iterations are an order of magnitude cheaper)
constexpr unsigned long long CANCEL_CHECK_NS = 1000000; // device time between reads of the host cancel word
constexpr int DONATE_MIN_LEVELS = 2;     // a donated node keeps at least this many levels below it
constexpr unsigned long long IDLE_GUARD_NS = 60ull * 1000000000ull;   // 60 s idle: internal error
constexpr long long RESERVE_SPIN_LIMIT = 1 << 20;   // bounded wait for a queue cell's previous lap
constexpr int RESERVE_TICKETS = 64;                  // producer tickets tried before keeping the work
// Idle back-off caps (ns): one warp per block polls for work at short
// intervals, the others at longer ones.  A waiting consumer polls only its own
// queue cell, so short intervals cost little and hand donated work over fast
// (measured: 256 ns / 4 us beat 1 us / 32 us by ~2.5% on the dense workload).
constexpr unsigned IDLE_BACKOFF_FAST = 256;
constexpr unsigned IDLE_BACKOFF_SLOW = 4096;

__device__ __forceinline__ uint64_t fmix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// g(u, v) of the per-match hash h(f) = fmix64(sum_u g(u, f(u))).
__device__ __forceinline__ uint64_t gterm(int u, int v) {
    return fmix64(((uint64_t)(uint32_t)u << 32 | (uint64_t)(uint32_t)v) + 0x9E3779B97F4A7C15ull);
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
    return x;
}

__device__ __forceinline__ int warp_max(int x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = max(x, __shfl_xor_sync(FULL, x, o));
    return x;
}

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Strong (gpu-scope) loads and stores of the words warps poll and publish:
// they are ordered and always see the latest value at the point of coherence
// (L2), never a copy left in a streaming multiprocessor's L1.
__device__ __forceinline__ unsigned long long load_acquire(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void store_release(unsigned long long *p, unsigned long long v) {
    asm volatile("st.release.gpu.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ int load_relaxed(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void set_status(int *status, int code) { atomicCAS(status, 0, code); }

// Is `c` in the sorted row of `x` (with edge label `lab` when `chk`)?
__device__ __forceinline__ bool row_has(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                                        const int32_t *__restrict__ elab, int x, int c, int lab, bool chk) {
    int lo = __ldg(rowptr + x), hi = __ldg(rowptr + x + 1);
    const int end = hi;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (__ldg(col + mid) < c) lo = mid + 1; else hi = mid;
    }
    if (lo >= end || __ldg(col + lo) != c) return false;
    return !chk || __ldg(elab + lo) == lab;
}

// Candidate source of position i (Section "RI": neighbours of M(P(mu_i));
// all of V_t, or D(mu_i) for RI-DS, when mu_i has no parent).
struct Src {
    const int32_t *ptr;   // null: candidate j is vertex j
    long long base;
    int len;
};

__device__ __forceinline__ Src cand_source(const JobDesc &J, const PosInfo &P, const int *M) {
    Src s;
    if (P.par >= 0) {
        int a = M[P.par];
        if (P.flags & POS_IN_ROW) {
            int b = __ldg(J.t.irowptr + a);
            s.ptr = J.t.icol; s.base = b; s.len = __ldg(J.t.irowptr + a + 1) - b;
        } else {
            int b = __ldg(J.t.rowptr + a);
            s.ptr = J.t.col; s.base = b; s.len = __ldg(J.t.rowptr + a + 1) - b;
        }
    } else if (J.flags & JOB_RIDS) {
        s.ptr = J.ulist; s.base = P.uoff; s.len = P.ucnt;
    } else {
        s.ptr = nullptr; s.base = 0; s.len = J.t.n;
    }
    return s;
}

// Rules 1-4 (Section "RI", pruning rules) and the RI-DS domain test for
// mapping mu_i onto candidate c.  `eidx` is c's index in the parent's row
// (for the parent-arc label), or -1.  M holds the images of positions 0..i-1.
template <bool DIR>
__device__ __forceinline__ bool feasible(const JobDesc &J, const PosInfo &P, int i, int c, long long eidx,
                                         const int *M) {
    const int2 v = __ldg(J.t.vld + c);
    if (v.x != P.lab || v.y < P.odeg) return false;                       // rules 2, 3
    if (DIR && __ldg(J.t.indeg + c) < P.ideg) return false;              // rule 3 (in)
    if (J.flags & JOB_RIDS) {                                             // v_t in D(mu_i)
        const uint64_t w = J.filt[(size_t)P.pv * J.t.dw + (c >> 6)];
        if (!((w >> (c & 63)) & 1ull)) return false;
    }
    const bool chk = (J.flags & JOB_ELAB) != 0;
    if (chk && eidx >= 0) {                                               // parent arc label
        const int l = (P.flags & POS_IN_ROW) ? __ldg(J.t.ielab + eidx) : __ldg(J.t.elab + eidx);
        if (l != P.pel) return false;
    }
    for (int b = 0; b < P.bcnt; ++b) {                                    // rule 4
        const BackEdge be = J.back[P.bbeg + b];
        const int x = M[be.pos];
        if (!DIR) {
            if (J.t.adj != nullptr && !chk) {
                const uint64_t w = __ldg(J.t.adj + (size_t)x * J.t.dw + (c >> 6));
                if (!((w >> (c & 63)) & 1ull)) return false;
            } else if (J.t.hub_slot != nullptr && !chk && __ldg(J.t.hub_slot + x) >= 0) {
                const uint64_t w = __ldg(J.t.hub_bits + (size_t)__ldg(J.t.hub_slot + x) * J.t.dw + (c >> 6));
                if (!((w >> (c & 63)) & 1ull)) return false;
            } else if (!row_has(J.t.rowptr, J.t.col, J.t.elab, x, c, be.lab_out, chk)) {
                return false;
            }
        } else {
            // arc c -> x: c is in the in-row of x; arc x -> c: c is in the out-row of x
            if ((be.dir & 1) && !row_has(J.t.irowptr, J.t.icol, J.t.ielab, x, c, be.lab_out, chk)) return false;
            if ((be.dir & 2) && !row_has(J.t.rowptr, J.t.col, J.t.elab, x, c, be.lab_in, chk)) return false;
        }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h)                                           // rule 1 (same-label positions)
        for (uint64_t m = P.same[h]; m; m &= m - 1)
            if (M[64 * h + __ffsll((long long)m) - 1] == c) return false;
    return true;
}

__device__ __forceinline__ int find_job(const long long *off, int njobs, long long u) {
    int lo = 0, hi = njobs;  // largest j with off[j] <= u
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (off[mid] <= u) lo = mid; else hi = mid;
    }
    return lo;
}

// Write one match row (images of pattern vertices 0..k-1) for enumeration.
__device__ __forceinline__ void emit_match(const JobDesc &J, const int *M, int last_pos, int c) {
    unsigned long long slot = atomicAdd(J.mlen, 1ull);
    if ((long long)slot >= J.mcap) return;
    int32_t *row = J.mbuf + (size_t)slot * J.k;
    for (int t = 0; t < last_pos; ++t) row[J.pos[t].pv] = M[t];
    row[J.pos[last_pos].pv] = c;
}

// ================================================================ domains

// D(v) initialisation (Section 4): equal label, in/out-degree at least v's.
// For RI it is exactly the rule 2-3 filter.  One warp per 32 consecutive 64-bit words.
// Each pattern vertex's label index among its job's target labels (-1: absent),
// for the jobs that read the label-degree table; one thread per (job, vertex).
__global__ void __launch_bounds__(BLOCK) k_label_index(const JobDesc *jobs, const long long *vert_off, int njobs,
                                                       long long nverts) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nverts) return;
    const int j = find_job(vert_off, njobs, g);
    const JobDesc &J = jobs[j];
    if (J.plidx == nullptr) return;
    const int u = (int)(g - vert_off[j]);
    const int lab = J.p.lab[u];
    int lo = 0, hi = J.t.nlab;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(J.t.labs + mid) < lab) lo = mid + 1; else hi = mid;
    }
    const_cast<int32_t *>(J.plidx)[u] = lo < J.t.nlab && __ldg(J.t.labs + lo) == lab ? lo : -1;
}

// Initial domain of pattern vertex v on a target with label buckets: the prefix of
// lab(v)'s bucket with degree at least v's (descending order), then, for RI-DS, the
// label-degree support test of k_domain_init; bits set with atomicOr into the zeroed filter.
__global__ void __launch_bounds__(BLOCK) k_domain_init_buckets(const JobDesc *jobs, const long long *vert_off,
                                                               int njobs, long long nverts) {
    const long long g = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (g >= nverts) return;
    const int j = find_job(vert_off, njobs, g);
    const JobDesc &J = jobs[j];
    if (J.filt == nullptr || J.t.lbuck == nullptr) return;
    const int v = (int)(g - vert_off[j]);
    const int lab = J.p.lab[v], od = J.p.odeg[v];
    int lo = 0, hi = J.t.nlab;   // lab(v)'s bucket
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(J.t.labs + mid) < lab) lo = mid + 1; else hi = mid;
    }
    if (lo >= J.t.nlab || __ldg(J.t.labs + lo) != lab) return;   // label absent: empty domain
    const int b0 = __ldg(J.t.lbstart + lo), b1 = __ldg(J.t.lbstart + lo + 1);
    int e = b0, f = b1;          // first bucket position with degree below od (degrees descend)
    while (e < f) {
        const int mid = (e + f) >> 1;
        if (__ldg(J.t.lbdeg + mid) >= od) e = mid + 1; else f = mid;
    }
    const bool nbcheck = (J.flags & JOB_RIDS) && !(J.flags & JOB_ELAB) && J.t.nbmax != nullptr && J.plidx != nullptr;
    uint64_t *Fv = J.filt + (size_t)v * J.t.dw;
    for (int x = b0 + lane; x < e; x += 32) {
        const int t = __ldg(J.t.lbuck + x);
        bool ok = true;
        if (nbcheck) {
            for (int pe = J.p.rowptr[v]; pe < J.p.rowptr[v + 1] && ok; ++pe) {
                const int pu = J.p.col[pe];
                const int li = J.plidx[pu];
                ok = li >= 0 && __ldg(J.t.nbmax + (size_t)li * J.t.n + t) >= J.p.odeg[pu];
            }
        }
        if (ok) atomicOr((unsigned long long *)(Fv + (t >> 6)), 1ull << (t & 63));
    }
}

constexpr int INIT_WORDS_PER_WARP = 32;   // most consecutive filter words one warp of k_domain_init writes
static_assert(INIT_WORDS_PER_WARP <= 32, "k_domain_init copies a warp's words one per lane");

__global__ void __launch_bounds__(BLOCK) k_domain_init(const JobDesc *jobs, const long long *unit_off, int njobs,
                                                       long long nunits, int wpw) {
    const long long u0 = (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * wpw;
    const int lane = threadIdx.x & 31;
    if (u0 >= nunits) return;
    // the warp's words are consecutive units: find the job once, then step over its
    // boundaries; (v, q) = (pattern vertex, word) steps along with u (a job holds
    // k x dw < 2^15 units, so 32-bit arithmetic).  The job's fields are read once per job
    // and the vertex's once per vertex, not once per word.
    int j = find_job(unit_off, njobs, u0);
    {
        // when every word of the warp's range is a copy of a label-degree mask row (see
        // below), the lanes copy one word each at once instead of the warp stepping word by word
        const long long u = u0 + lane;
        bool copyable = true;
        uint64_t *dst = nullptr;
        uint64_t word = 0;
        if (u < nunits && u < u0 + wpw) {
            int jl = j;
            while (jl + 1 < njobs && unit_off[jl + 1] <= u) ++jl;
            const JobDesc &J = jobs[jl];
            if (J.filt != nullptr && J.t.lbuck == nullptr) {
                const bool nbc = (J.flags & JOB_RIDS) && !(J.flags & JOB_ELAB) && J.t.nbmax != nullptr &&
                                 J.plidx != nullptr;
                const int dwl = J.t.dw, local = (int)(u - unit_off[jl]);
                const int vl = local / dwl, ql = local - vl * dwl;
                const int odl = J.p.odeg[vl];
                if (nbc || (J.flags & JOB_DIRECTED) || J.t.ldm == nullptr || odl >= LDM_DEGREES) {
                    copyable = false;
                } else {
                    const int labl = J.p.lab[vl];
                    int lo = 0, hi = J.t.nlab;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (__ldg(J.t.labs + mid) < labl) lo = mid + 1; else hi = mid;
                    }
                    if (lo < J.t.nlab && __ldg(J.t.labs + lo) == labl)
                        word = __ldg(J.t.ldm + ((size_t)lo * LDM_DEGREES + odl) * dwl + ql);
                    dst = J.filt + (size_t)vl * dwl + ql;
                }
            }
        }
        if (__all_sync(FULL, copyable)) {
            if (dst != nullptr) *dst = word;
            return;
        }
    }
    int jcur = -1, v = -1, q = 0, vcur = -1;
    bool skip = true, DIR = false, nbcheck = false;
    int dw = 1, n = 0, lab = 0, od = 0, id = 0;
    const int2 *vld = nullptr;
    const int32_t *indeg = nullptr;
    uint64_t *filt = nullptr;
    // without the neighbour test, D(v) initialised = the target's label-degree mask row of
    // (lab(v), deg(v)) when it has one: a copy (mrow null and mempty: lab(v) absent)
    const uint64_t *mrow = nullptr;
    bool mempty = false;
    for (long long u = u0; u < u0 + wpw && u < nunits; ++u) {
        while (j + 1 < njobs && unit_off[j + 1] <= u) ++j;
        const JobDesc &J = jobs[j];
        if (j != jcur) {
            jcur = j;
            skip = J.filt == nullptr || J.t.lbuck != nullptr;   // (bucket targets: k_domain_init_buckets)
            DIR = (J.flags & JOB_DIRECTED) != 0;
            // RI-DS on an undirected target without edge labels: a candidate t also needs, for
            // every pattern neighbour u of v, a neighbour of its own with u's label and at least
            // u's degree.  That is arc consistency's test against the domains as initialised, so
            // dropping the failures here removes only candidates the first sweep would remove;
            // their rows, which the sweep would scan to the end, are never read.
            nbcheck = (J.flags & JOB_RIDS) && !(J.flags & JOB_ELAB) && !DIR && J.t.nbmax != nullptr &&
                      J.plidx != nullptr;
            dw = J.t.dw;
            n = J.t.n;
            vld = J.t.vld;
            indeg = J.t.indeg;
            filt = J.filt;
            const int local = (int)(u - unit_off[j]);
            v = local / dw;
            q = local - v * dw;
            vcur = -1;
        } else if (++q == dw) {
            q = 0;
            ++v;
        }
        if (skip) continue;
        if (v != vcur) {
            vcur = v;
            lab = J.p.lab[v];
            od = J.p.odeg[v];
            id = DIR ? J.p.ideg[v] : 0;
            mrow = nullptr;
            mempty = false;
            if (!nbcheck && !DIR && J.t.ldm != nullptr && od < LDM_DEGREES) {
                int lo = 0, hi = J.t.nlab;   // lab(v)'s index among the target's labels
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (__ldg(J.t.labs + mid) < lab) lo = mid + 1; else hi = mid;
                }
                if (lo < J.t.nlab && __ldg(J.t.labs + lo) == lab)
                    mrow = J.t.ldm + ((size_t)lo * LDM_DEGREES + od) * dw;
                else
                    mempty = true;
            }
        }
        if (mrow != nullptr || mempty) {
            if (lane == 0) filt[(size_t)v * dw + q] = mempty ? 0ull : __ldg(mrow + q);
            continue;
        }
        unsigned long long word = 0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int t = q * 64 + h * 32 + lane;
            bool ok = false;
            if (t < n) {
                const int2 x = __ldg(vld + t);
                ok = x.x == lab && x.y >= od && (!DIR || __ldg(indeg + t) >= id);
            }
            if (nbcheck && __any_sync(FULL, ok)) {
                for (int e = J.p.rowptr[v]; e < J.p.rowptr[v + 1]; ++e) {
                    const int pu = J.p.col[e];
                    const int li = J.plidx[pu];   // lab(pu)'s index among the target's labels, -1 if absent
                    if (ok) ok = li >= 0 && __ldg(J.t.nbmax + (size_t)li * n + t) >= J.p.odeg[pu];
                }
            }
            word |= (unsigned long long)__ballot_sync(FULL, ok) << (32 * h);
        }
        if (lane == 0) filt[(size_t)v * dw + q] = word;
    }
}

// Arc consistency of one candidate (Section 4): does target vertex t keep,
// for every pattern edge at v, a compatible target edge into the other
// endpoint's domain?
__device__ __forceinline__ bool ac_supported(const JobDesc &J, int v, int t, bool DIR, bool chk) {
    const int dw = J.t.dw;
    for (int e = J.p.rowptr[v]; e < J.p.rowptr[v + 1]; ++e) {
        const int uu = J.p.col[e], bl = chk ? J.p.elab[e] : 0;
        const uint64_t *Du = J.filt + (size_t)uu * dw;
        bool found = false;
        for (int f = __ldg(J.t.rowptr + t), fe = __ldg(J.t.rowptr + t + 1); f < fe; ++f) {
            const int y = __ldg(J.t.col + f);
            if ((!chk || __ldg(J.t.elab + f) == bl) && ((Du[y >> 6] >> (y & 63)) & 1ull)) { found = true; break; }
        }
        if (!found) return false;
    }
    if (DIR) {
        for (int e = J.p.irowptr[v]; e < J.p.irowptr[v + 1]; ++e) {
            const int uu = J.p.icol[e], bl = chk ? J.p.ielab[e] : 0;
            const uint64_t *Du = J.filt + (size_t)uu * dw;
            bool found = false;
            for (int f = __ldg(J.t.irowptr + t), fe = __ldg(J.t.irowptr + t + 1); f < fe; ++f) {
                const int y = __ldg(J.t.icol + f);
                if ((!chk || __ldg(J.t.ielab + f) == bl) && ((Du[y >> 6] >> (y & 63)) & 1ull)) { found = true; break; }
            }
            if (!found) return false;
        }
    }
    return true;
}

// Warp-collective form of ac_supported for a candidate with a long row: for each
// pattern edge the 32 lanes stride t's row and a ballot says whether any of them
// found a compatible neighbour in the other endpoint's domain.
__device__ __forceinline__ bool ac_supported_warp(const JobDesc &J, int v, int t, bool DIR, bool chk) {
    const int lane = threadIdx.x & 31;
    const int dw = J.t.dw;
    for (int pass = 0; pass < (DIR ? 2 : 1); ++pass) {
        const int32_t *prow = pass ? J.p.irowptr : J.p.rowptr;
        const int32_t *pcol = pass ? J.p.icol : J.p.col;
        const int32_t *pel = pass ? J.p.ielab : J.p.elab;
        const int32_t *trow = pass ? J.t.irowptr : J.t.rowptr;
        const int32_t *tcol = pass ? J.t.icol : J.t.col;
        const int32_t *tel = pass ? J.t.ielab : J.t.elab;
        const int fb = __ldg(trow + t), fe = __ldg(trow + t + 1);
        for (int e = prow[v]; e < prow[v + 1]; ++e) {
            const int uu = pcol[e], bl = chk ? pel[e] : 0;
            const uint64_t *Du = J.filt + (size_t)uu * dw;
            bool found = false;
            for (int f0 = fb; f0 < fe && !found; f0 += 32) {
                const int f = f0 + lane;
                bool ok = false;
                if (f < fe) {
                    const int y = __ldg(tcol + f);
                    ok = (!chk || __ldg(tel + f) == bl) && ((Du[y >> 6] >> (y & 63)) & 1ull);
                }
                found = __any_sync(FULL, ok);
            }
            if (!found) return false;
        }
    }
    return true;
}

// A candidate whose row (out- plus in-row) is longer than AC_WARP_ROW is searched
// by the whole warp (ac_supported_warp) -- unless the domains at the other ends of
// its pattern edges are dense (each at least 1/AC_DENSE of the target), where a
// row scan finds support within a few entries: then its own lane scans at most
// AC_LANE_SCAN entries per pattern edge first, and only an edge left open sends
// it to the warp.  Rows longer than AC_WARP_ROW_DIRECT always go to the warp.
constexpr int AC_WARP_ROW = 48;
constexpr int AC_LANE_SCAN = 32;
constexpr int AC_WARP_ROW_DIRECT = 512;

// ac_supported with each row scan cut after `bound` entries: returns false if
// some pattern edge has no support (its whole row scanned), true if every edge
// found one, and sets `open` (result then true) when no edge failed but some
// scan stopped at the bound.
__device__ __forceinline__ bool ac_supported_bounded(const JobDesc &J, int v, int t, bool DIR, bool chk, int bound, bool &open) {
    const int dw = J.t.dw;
    open = false;
    for (int pass = 0; pass < (DIR ? 2 : 1); ++pass) {
        const int32_t *prow = pass ? J.p.irowptr : J.p.rowptr;
        const int32_t *pcol = pass ? J.p.icol : J.p.col;
        const int32_t *pel = pass ? J.p.ielab : J.p.elab;
        const int32_t *trow = pass ? J.t.irowptr : J.t.rowptr;
        const int32_t *tcol = pass ? J.t.icol : J.t.col;
        const int32_t *tel = pass ? J.t.ielab : J.t.elab;
        const int f0 = __ldg(trow + t), fe = __ldg(trow + t + 1);
        const int fb = min(fe, f0 + bound);
        for (int e = prow[v]; e < prow[v + 1]; ++e) {
            const int uu = pcol[e], bl = chk ? pel[e] : 0;
            const uint64_t *Du = J.filt + (size_t)uu * dw;
            bool found = false;
            for (int f = f0; f < fb; ++f) {
                const int y = __ldg(tcol + f);
                if ((!chk || __ldg(tel + f) == bl) && ((Du[y >> 6] >> (y & 63)) & 1ull)) { found = true; break; }
            }
            if (!found) {
                if (fb == fe) return false;
                open = true;
            }
        }
    }
    return true;
}

// Lane-local part of the arc-consistency test of candidate t of D(v) with a row of
// `len` entries: whether to drop it, or (`heavy`) to leave it to the warp.
__device__ __forceinline__ bool ac_lane_check(const JobDesc &J, int v, int t, bool DIR, bool chk, int len,
                                              bool dense, bool &heavy) {
    heavy = false;
    if (len <= AC_WARP_ROW) return !ac_supported(J, v, t, DIR, chk);
    if (!dense || len > AC_WARP_ROW_DIRECT) {
        heavy = true;
        return false;
    }
    bool open = false;
    const bool sup = ac_supported_bounded(J, v, t, DIR, chk, AC_LANE_SCAN, open);
    heavy = open;
    return !sup;
}

// The same sweep over explicit candidate lists: one lane per listed candidate of
// the listed entries {job, pattern vertex, global vertex, list start}; a removed
// candidate is cleared from D(v) and its list slot.  A lane tests a candidate with
// a short row itself; the warp then takes its lanes' long-row candidates one at a
// time together, so a hub's row is read 32 entries per step instead of one.
__global__ void __launch_bounds__(BLOCK, 1) k_domain_ac_cand(const JobDesc *jobs, const int4 *ent, const long long *eoff,
                                                          int nent, long long ncand, int32_t *cand, int *changed,
                                                          unsigned char *vchanged) {
    const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if ((x & ~31ll) >= ncand) return;   // warp-uniform: a warp with any candidate stays whole
    const int lane = threadIdx.x & 31;
    int jidx = 0, v = 0, g = 0, t = -1;
    bool dense_v = false;
    int32_t *slot = nullptr;
    if (x < ncand) {
        const int i = find_job(eoff, nent, x);
        const int4 E = ent[i];
        jidx = E.x; v = E.y & (AC_ENT_DENSE - 1); g = E.z;
        dense_v = (E.y & AC_ENT_DENSE) != 0;
        slot = cand + (long long)E.w + (x - eoff[i]);
        t = *slot;
    }
    bool drop = false, heavy = false;
    if (t >= 0) {
        const JobDesc &J = jobs[jidx];
        uint64_t *wp = J.filt + (size_t)v * J.t.dw + (t >> 6);
        if (!(*wp & (1ull << (t & 63)))) {
            *slot = -1;                                  // removed by forward checking
        } else {
            const bool DIR = (J.flags & JOB_DIRECTED) != 0;
            const int len = __ldg(J.t.rowptr + t + 1) - __ldg(J.t.rowptr + t) +
                            (DIR ? __ldg(J.t.irowptr + t + 1) - __ldg(J.t.irowptr + t) : 0);
            drop = ac_lane_check(J, v, t, DIR, (J.flags & JOB_ELAB) != 0, len, dense_v, heavy);
        }
    }
    unsigned hv = __ballot_sync(FULL, heavy);
    while (hv) {
        const int L = __ffs(hv) - 1;
        hv &= hv - 1;
        const int jl = __shfl_sync(FULL, jidx, L), vl = __shfl_sync(FULL, v, L), tl = __shfl_sync(FULL, t, L);
        const JobDesc &J = jobs[jl];
        const bool sup = ac_supported_warp(J, vl, tl, (J.flags & JOB_DIRECTED) != 0, (J.flags & JOB_ELAB) != 0);
        if (lane == L) drop = !sup;
    }
    if (drop) {                                          // unsupported: remove t from D(v)
        const JobDesc &J = jobs[jidx];
        atomicAnd((unsigned long long *)(J.filt + (size_t)v * J.t.dw + (t >> 6)), ~(1ull << (t & 63)));
        *slot = -1;
        *changed = 1;
        vchanged[g] = 1;
    }
}

// One arc-consistency sweep (Section 4): drop t from D(v) when a pattern
// edge at v has no compatible target edge at t into the other endpoint's
// domain.  Removals are applied in place (monotone), so sweeping until no
// word changes reaches the unique greatest fixpoint.  A sweep visits only
// the listed (job, pattern vertex) entries -- those with a neighbour whose
// domain shrank in the previous sweep -- one warp per 64-target word, and
// marks every domain it shrinks in vchanged.
__global__ void __launch_bounds__(BLOCK, 1) k_domain_ac(const JobDesc *jobs, const int4 *ent, const long long *eoff,
                                                     int nent, long long nunits, int *changed,
                                                     unsigned char *vchanged) {
    const long long u = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (u >= nunits) return;
    const int i = find_job(eoff, nent, u);
    const int4 E = ent[i];   // {job, pattern vertex, global vertex index, 0}
    const JobDesc &J = jobs[E.x];
    if (J.filt == nullptr || !(J.flags & JOB_RIDS)) return;
    const bool DIR = (J.flags & JOB_DIRECTED) != 0;
    const int v = E.y & (AC_ENT_DENSE - 1), q = (int)(u - eoff[i]);
    uint64_t *wp = J.filt + (size_t)v * J.t.dw + q;
    const uint64_t word = *wp;
    if (word == 0) return;
    const bool chk = (J.flags & JOB_ELAB) != 0;
    const int dw = J.t.dw;
    unsigned long long keep = 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int bit = h * 32 + lane;
        const int t = q * 64 + bit;
        bool ok = (word >> bit) & 1ull;
        if (ok) {
            for (int e = J.p.rowptr[v]; ok && e < J.p.rowptr[v + 1]; ++e) {
                const int uu = J.p.col[e], bl = chk ? J.p.elab[e] : 0;
                const uint64_t *Du = J.filt + (size_t)uu * dw;
                bool found = false;
                for (int f = __ldg(J.t.rowptr + t), fe = __ldg(J.t.rowptr + t + 1); f < fe; ++f) {
                    const int y = __ldg(J.t.col + f);
                    if ((!chk || __ldg(J.t.elab + f) == bl) && ((Du[y >> 6] >> (y & 63)) & 1ull)) { found = true; break; }
                }
                ok = found;
            }
            if (DIR) {
                for (int e = J.p.irowptr[v]; ok && e < J.p.irowptr[v + 1]; ++e) {
                    const int uu = J.p.icol[e], bl = chk ? J.p.ielab[e] : 0;
                    const uint64_t *Du = J.filt + (size_t)uu * dw;
                    bool found = false;
                    for (int f = __ldg(J.t.irowptr + t), fe = __ldg(J.t.irowptr + t + 1); f < fe; ++f) {
                        const int y = __ldg(J.t.icol + f);
                        if ((!chk || __ldg(J.t.ielab + f) == bl) && ((Du[y >> 6] >> (y & 63)) & 1ull)) { found = true; break; }
                    }
                    ok = found;
                }
            }
        }
        keep |= (unsigned long long)__ballot_sync(FULL, ok) << (32 * h);
    }
    if (lane == 0 && keep != word) {
        atomicAnd((unsigned long long *)wp, keep);
        *changed = 1;
        vchanged[E.z] = 1;
    }
}

// Forward checking (Section 4.2): the target node of a singleton domain is
// removed from every other domain, repeated until no new singleton appears.
// One block per job, starting from the domain sizes: each round takes the
// singletons not yet propagated, finds each one's element (one warp scans
// its words), and clears that element's word in every other domain,
// counting the sizes down (all singletons of a round propagate together).
__global__ void __launch_bounds__(BLOCK) k_domain_fc(const JobDesc *jobs, const long long *vert_off,
                                                     const long long *sizes, int *changed, unsigned char *vchanged) {
    __shared__ int size[KMAX];
    __shared__ int elem[KMAX];
    __shared__ unsigned char done[KMAX];
    __shared__ int newu[KMAX];
    __shared__ int nnew;
    const JobDesc &J = jobs[blockIdx.x];
    if (J.filt == nullptr || !(J.flags & JOB_FC)) return;
    const int k = J.k, dw = J.t.dw;
    const long long vo = vert_off[blockIdx.x];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int v = threadIdx.x; v < k; v += blockDim.x) {
        size[v] = (int)sizes[vo + v];   // exact, counted down on every removal
        done[v] = 0;
    }
    __syncthreads();
    for (int round = 0; round <= k; ++round) {
        if (threadIdx.x == 0) nnew = 0;
        __syncthreads();
        for (int v = threadIdx.x; v < k; v += blockDim.x)
            if (size[v] == 1 && !done[v]) {
                done[v] = 1;
                newu[atomicAdd(&nnew, 1)] = v;
            }
        __syncthreads();
        const int nn = nnew;
        if (nn == 0) break;
        for (int s = wid; s < nn; s += nwarps) {
            const int u = newu[s];
            int found = -1;
            for (int q0 = 0; q0 < dw && found < 0; q0 += 32) {
                const int q = q0 + lane;
                const uint64_t w = q < dw ? J.filt[(size_t)u * dw + q] : 0ull;
                const unsigned b = __ballot_sync(FULL, w != 0);
                if (b) {
                    const int L = __ffs(b) - 1;
                    const uint64_t wl = __shfl_sync(FULL, w, L);
                    found = (q0 + L) * 64 + __ffsll((long long)wl) - 1;
                }
            }
            if (lane == 0) elem[u] = found;
        }
        __syncthreads();
        for (int x = threadIdx.x; x < nn * k; x += blockDim.x) {
            const int u = newu[x / k], v = x % k, t = elem[u];
            if (v == u || t < 0) continue;
            unsigned long long *wp = reinterpret_cast<unsigned long long *>(J.filt + (size_t)v * dw + (t >> 6));
            const unsigned long long bit = 1ull << (t & 63);
            if (atomicAnd(wp, ~bit) & bit) {
                atomicSub(&size[v], 1);
                vchanged[vo + v] = 1;
                *changed = 1;
            }
        }
        __syncthreads();
    }
}

// Arc consistency alternating with forward checking to their joint fixpoint
// (Section 4, Section 4.2), all of one job inside one block: no host round
// trip between sweeps, so a batch of many small jobs costs one launch.  A
// sweep re-checks D(v) only for the vertices whose pattern neighbours' domains
// shrank in the previous sweep (all vertices first); when arc consistency
// holds, one forward-checking round clears the element of every new singleton
// from the other domains, and the loop goes on until neither changes anything.
// Removals are monotone deletions, so this schedule reaches the same unique
// greatest fixpoint as any other.  A forward-checking round that finds an
// empty domain ends the job (it has no match).  Blocks take jobs from a counter.
// A sweep visits a dirty vertex's candidates either word by word (small
// targets: `cand` null) or through its candidate list (large targets, whose
// domain words are mostly empty: slots [cstart[g], cstart[g] + csize[g]) of
// `cand`, g = vert_off[job] + v, a removed candidate's slot set to -1), 32
// slots per warp step so that a candidate with a long row is checked by the
// whole warp.
constexpr int FIXPOINT_BIG_BLOCK = 1024;   // threads per block of k_domain_fixpoint when pairs are few
constexpr int FIXPOINT_SMALL_BLOCK = 128;  // ... and when they are many
constexpr int FP_CHUNK = 1024;             // domain words scanned at once by k_domain_fixpoint
static_assert(FP_CHUNK % FIXPOINT_BIG_BLOCK == 0 && FP_CHUNK % FIXPOINT_SMALL_BLOCK == 0,
              "a fixpoint block scans FP_CHUNK words in whole rounds of one word per thread");

// Exclusive scan of one int per thread over the block (up to 1024 threads);
// `total` receives the block's sum.  wsum: 32 ints of shared memory.
__device__ __forceinline__ int block_scan_int(int x, int *wsum, int &total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int s = lane < nw ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) wsum[lane] = s;
    }
    __syncthreads();
    total = wsum[nw - 1];
    const int before = wid ? wsum[wid - 1] : 0;
    __syncthreads();   // wsum may be reused at once
    return before + incl - x;
}

// Position of the r-th (0-based) set bit of w (r < popcount(w)): the window that
// holds it is halved six times, each step comparing r with the low half's popcount.
__device__ __forceinline__ int select_bit(uint64_t w, int r) {
    int base = 0;
    uint32_t h = (uint32_t)w;
    int c = __popc(h);
    if (r >= c) {
        r -= c;
        h = (uint32_t)(w >> 32);
        base = 32;
    }
#pragma unroll
    for (int half = 16; half >= 1; half >>= 1) {
        c = __popc(h & ((1u << half) - 1u));
        if (r >= c) {
            r -= c;
            h >>= half;
            base += half;
        }
    }
    return base;
}

__global__ void __launch_bounds__(FIXPOINT_BIG_BLOCK, 1) k_domain_fixpoint(const JobDesc *jobs, int njobs,
                                                                        const long long *vert_off,
                                                           const long long *cstart, const long long *csize,
                                                           int32_t *cand, int *next_job) {
    __shared__ unsigned char dirty[KMAX], chg[KMAX], done[KMAX], dns[KMAX];
    __shared__ int dl[KMAX], size[KMAX], elem[KMAX], newu[KMAX];
    __shared__ long long pre[KMAX + 1];
    __shared__ int nd, any, nnew, empty;
    __shared__ uint64_t wsnap[FP_CHUNK];
    __shared__ int wpre[FP_CHUNK + 1], wsum[32];
    __shared__ int jnext;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nwarps = blockDim.x >> 5;
    for (;;) {
        // the next job, taken dynamically: pairs differ widely in cost
        if (tid == 0) jnext = atomicAdd(next_job, 1);
        __syncthreads();
        const int jb = jnext;
        __syncthreads();
        if (jb >= njobs) break;
        const JobDesc &J = jobs[jb];
        if (J.filt == nullptr || !(J.flags & JOB_RIDS)) continue;
        const bool DIR = (J.flags & JOB_DIRECTED) != 0, chk = (J.flags & JOB_ELAB) != 0;
        const bool FC = (J.flags & JOB_FC) != 0;
        const int k = J.k, dw = J.t.dw;
        for (int v = tid; v < k; v += blockDim.x) { dirty[v] = 1; done[v] = 0; }
        if (tid == 0) empty = 0;
        __syncthreads();
        // |D(v)|, kept exact below: every removal counts it down, and the first domain to
        // empty ends the pair (it has no match, so the rest of its fixpoint is never needed)
        for (int v = wid; v < k; v += nwarps) {
            unsigned long long c = 0;
            for (int q = lane; q < dw; q += 32) c += __popcll(J.filt[(size_t)v * dw + q]);
            c = warp_sum(c);
            if (lane == 0) {
                size[v] = (int)c;
                if (c == 0) empty = 1;
            }
        }
        __syncthreads();
        while (!empty) {
            // ---- arc consistency over the dirty vertices, to its fixpoint
            for (;;) {
                if (tid == 0) { nd = 0; any = 0; }
                __syncthreads();
                for (int v = tid; v < k; v += blockDim.x) {
                    chg[v] = 0;
                    if (dirty[v]) { dl[atomicAdd(&nd, 1)] = v; dirty[v] = 0; }
                }
                __syncthreads();
                const int n_d = nd;
                if (n_d == 0) break;
                if (cand == nullptr) {
                    // the dirty domains' words, FP_CHUNK at a time: snapshot them, scan their
                    // popcounts, and give each thread the next set bit, so the candidates of a
                    // dense word are checked in parallel rather than by one thread in turn
                    const long long units = (long long)n_d * dw;
                    for (long long u0 = 0; u0 < units; u0 += FP_CHUNK) {
                        const int nw_c = (int)min((long long)FP_CHUNK, units - u0);
                        // words per thread in the scan: as few as the chunk needs (FP_CHUNK is a
                        // multiple of the block size, so tid * ipt + r stays below FP_CHUNK)
                        const int ipt = (nw_c + (int)blockDim.x - 1) / (int)blockDim.x;
                        int cnt = 0;
                        for (int r = 0; r < ipt; ++r) {
                            const int iw = tid * ipt + r;
                            uint64_t w = 0;
                            if (iw < nw_c) {
                                const long long x = u0 + iw;
                                const int i = (int)x / dw, q = (int)x - i * dw;
                                w = J.filt[(size_t)dl[i] * dw + q];
                            }
                            wsnap[iw] = w;
                            cnt += __popcll(w);
                        }
                        int total;
                        int ex = block_scan_int(cnt, wsum, total);
                        for (int r = 0; r < ipt; ++r) {
                            const int iw = tid * ipt + r;
                            wpre[iw] = ex;
                            ex += __popcll(wsnap[iw]);
                        }
                        if (tid == 0) wpre[FP_CHUNK] = total;
                        __syncthreads();
                        for (int x = tid; x < total; x += blockDim.x) {
                            int lo = 0, hi = nw_c;   // the word holding set bit x: wpre[lo] <= x < wpre[lo + 1]
                            while (hi - lo > 1) {
                                const int mid = (lo + hi) >> 1;
                                if (wpre[mid] <= x) lo = mid; else hi = mid;
                            }
                            const long long ux = u0 + lo;
                            const int i = (int)ux / dw, q = (int)ux - i * dw, v = dl[i];
                            const int b = select_bit(wsnap[lo], x - wpre[lo]);
                            if (!ac_supported(J, v, q * 64 + b, DIR, chk)) {
                                atomicAnd((unsigned long long *)(J.filt + (size_t)v * dw + q), ~(1ull << b));
                                chg[v] = 1;
                                any = 1;
                                if (atomicSub(&size[v], 1) == 1) empty = 1;
                            }
                        }
                        __syncthreads();   // wsnap and wpre are refilled for the next chunk
                    }
                } else {
                    const long long g0 = vert_off[jb];
                    // dense: every pattern neighbour's domain holds at least 1/AC_DENSE of the target
                    for (int i = tid; i < n_d; i += blockDim.x) {
                        const int dv = dl[i];
                        bool d = true;
                        for (int e = J.p.rowptr[dv]; d && e < J.p.rowptr[dv + 1]; ++e)
                            d = (long long)size[J.p.col[e]] * AC_DENSE >= J.t.n;
                        for (int e = DIR ? J.p.irowptr[dv] : 0; d && DIR && e < J.p.irowptr[dv + 1]; ++e)
                            d = (long long)size[J.p.icol[e]] * AC_DENSE >= J.t.n;
                        dns[dv] = d;
                    }
                    if (tid == 0) {
                        long long acc = 0;
                        for (int i = 0; i < n_d; ++i) {
                            pre[i] = acc;
                            acc += csize[g0 + dl[i]];
                        }
                        pre[n_d] = acc;
                    }
                    __syncthreads();
                    const long long units = pre[n_d];
                    for (long long x0 = (long long)wid * 32; x0 < units; x0 += (long long)nwarps * 32) {
                        const long long x = x0 + lane;
                        int v = 0, t = -1;
                        int32_t *slot = nullptr;
                        if (x < units) {
                            int lo = 0, hi = n_d;   // the dirty vertex whose slots hold unit x
                            while (hi - lo > 1) {
                                const int mid = (lo + hi) >> 1;
                                if (pre[mid] <= x) lo = mid; else hi = mid;
                            }
                            v = dl[lo];
                            slot = cand + cstart[g0 + v] + (x - pre[lo]);
                            t = *slot;
                        }
                        bool drop = false, heavy = false;
                        if (t >= 0) {
                            if (!((J.filt[(size_t)v * dw + (t >> 6)] >> (t & 63)) & 1ull)) {
                                *slot = -1;                      // removed by forward checking
                            } else {
                                const int len = __ldg(J.t.rowptr + t + 1) - __ldg(J.t.rowptr + t) +
                                                (DIR ? __ldg(J.t.irowptr + t + 1) - __ldg(J.t.irowptr + t) : 0);
                                drop = ac_lane_check(J, v, t, DIR, chk, len, dns[v] != 0, heavy);
                            }
                        }
                        unsigned hv = __ballot_sync(FULL, heavy);
                        while (hv) {
                            const int L = __ffs(hv) - 1;
                            hv &= hv - 1;
                            const int vl = __shfl_sync(FULL, v, L), tl = __shfl_sync(FULL, t, L);
                            const bool sup = ac_supported_warp(J, vl, tl, DIR, chk);
                            if (lane == L) drop = !sup;
                        }
                        if (drop) {
                            atomicAnd((unsigned long long *)(J.filt + (size_t)v * dw + (t >> 6)), ~(1ull << (t & 63)));
                            *slot = -1;
                            chg[v] = 1;
                            any = 1;
                            if (atomicSub(&size[v], 1) == 1) empty = 1;
                        }
                    }
                }
                __syncthreads();
                if (empty || !any) break;
                // the pattern neighbours of every shrunk domain are checked again
                for (int v = tid; v < k; v += blockDim.x) {
                    if (!chg[v]) continue;
                    for (int e = J.p.rowptr[v]; e < J.p.rowptr[v + 1]; ++e) dirty[J.p.col[e]] = 1;
                    if (DIR)
                        for (int e = J.p.irowptr[v]; e < J.p.irowptr[v + 1]; ++e) dirty[J.p.icol[e]] = 1;
                }
                __syncthreads();
            }
            if (empty || !FC) break;
            // ---- one forward-checking round on the new singletons
            if (tid == 0) nnew = 0;
            __syncthreads();
            for (int v = tid; v < k; v += blockDim.x) {
                chg[v] = 0;
                if (size[v] == 1 && !done[v]) {
                    done[v] = 1;
                    newu[atomicAdd(&nnew, 1)] = v;
                }
            }
            __syncthreads();
            const int nn = nnew;
            if (nn == 0) break;   // both fixpoints hold
            for (int sgl = wid; sgl < nn; sgl += nwarps) {
                const int u = newu[sgl];
                int found = -1;
                for (int q0 = 0; q0 < dw && found < 0; q0 += 32) {
                    const int q = q0 + lane;
                    const uint64_t w = q < dw ? J.filt[(size_t)u * dw + q] : 0ull;
                    const unsigned bal = __ballot_sync(FULL, w != 0);
                    if (bal) {
                        const int L = __ffs(bal) - 1;
                        const uint64_t wl = __shfl_sync(FULL, w, L);
                        found = (q0 + L) * 64 + __ffsll((long long)wl) - 1;
                    }
                }
                if (lane == 0) elem[u] = found;
            }
            if (tid == 0) any = 0;
            __syncthreads();
            for (int x = tid; x < nn * k; x += blockDim.x) {
                const int u = newu[x / k], v = x % k, t = elem[u];
                if (v == u || t < 0) continue;
                unsigned long long *wp = reinterpret_cast<unsigned long long *>(J.filt + (size_t)v * dw + (t >> 6));
                const unsigned long long bit = 1ull << (t & 63);
                if (atomicAnd(wp, ~bit) & bit) {
                    chg[v] = 1;
                    any = 1;
                    if (atomicSub(&size[v], 1) == 1) empty = 1;
                }
            }
            __syncthreads();
            if (empty || !any) break;
            for (int v = tid; v < k; v += blockDim.x) {
                if (!chg[v]) continue;
                for (int e = J.p.rowptr[v]; e < J.p.rowptr[v + 1]; ++e) dirty[J.p.col[e]] = 1;
                if (DIR)
                    for (int e = J.p.irowptr[v]; e < J.p.irowptr[v + 1]; ++e) dirty[J.p.icol[e]] = 1;
            }
            __syncthreads();
        }
        __syncthreads();   // the shared arrays are reused by the next job
    }
}

// |D(v)| for every (job, pattern vertex); one warp each.
__global__ void __launch_bounds__(BLOCK) k_domain_sizes(const JobDesc *jobs, const long long *vert_off, int njobs,
                                                        long long nverts, long long *sizes) {
    const long long u = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (u >= nverts) return;
    const int j = find_job(vert_off, njobs, u);
    const JobDesc &J = jobs[j];
    const int v = (int)(u - vert_off[j]);
    unsigned long long c = 0;
    for (int q = lane; q < J.t.dw; q += 32) c += __popcll(J.filt[(size_t)v * J.t.dw + q]);
    c = warp_sum(c);
    if (lane == 0) sizes[u] = (long long)c;
}

// List D(v) in ascending id order at `out` (one block per task).
__global__ void __launch_bounds__(BLOCK) k_domain_lists(const JobDesc *jobs, const int *task_job, const int *task_vert,
                                                        const int *task_out, int32_t *lists) {
    __shared__ int wsum[WARPS_PER_BLOCK];
    __shared__ int carry;
    const JobDesc &J = jobs[task_job[blockIdx.x]];
    const int v = task_vert[blockIdx.x];
    int32_t *out = lists + task_out[blockIdx.x];
    const uint64_t *row = J.filt + (size_t)v * J.t.dw;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < J.t.dw; base += blockDim.x) {
        const int q = base + threadIdx.x;
        const uint64_t word = q < J.t.dw ? row[q] : 0;
        const int c = __popcll(word);
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wsum[w] = incl;
        __syncthreads();
        int before = carry;
        for (int i = 0; i < w; ++i) before += wsum[i];
        int pos = before + incl - c;
        uint64_t x = word;
        while (x) {
            const int b = __ffsll((long long)x) - 1;
            out[pos++] = q * 64 + b;
            x &= x - 1;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int i = 0; i < WARPS_PER_BLOCK; ++i) tot += wsum[i];
            carry += tot;
        }
        __syncthreads();
    }
}

// ================================================================== split

// One level of the breadth-first split.  Each frame [job, depth, -1, -1, M]
// is a search node whose positions 0..depth-1 are assigned; its candidates
// for position `depth` are tested, and in pass 1 each survivor becomes a
// frame of depth + 1 (or, at the last position, a match).
template <bool DIR>
__global__ void __launch_bounds__(BLOCK) k_split(const JobDesc *jobs, const int32_t *fin, long long nf, int depth,
                                                 int32_t *counts, const long long *offs, int32_t *fout, int pass,
                                                 int count_ctr) {
    __shared__ int Msh[WARPS_PER_BLOCK][KMAX];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int *M = Msh[wib];
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const int in_stride = FRAME_HDR + depth, out_stride = FRAME_HDR + depth + 1;
    for (long long f = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; f < nf; f += nwarps) {
        const int32_t *fr = fin + f * in_stride;
        const int j = fr[0];
        const JobDesc &J = jobs[j];
        for (int t = lane; t < depth; t += 32) M[t] = fr[FRAME_HDR + t];
        __syncwarp();
        const int k = J.k;
        const bool leaf = depth + 1 == k;
        const PosInfo &P = J.pos[depth];
        const Src S = cand_source(J, P, M);
        // a range frame scans candidates [beg, end); the node's states are counted by its first range
        const int rbeg = fr[2], rend = fr[3];
        const int c_lo = rbeg >= 0 ? rbeg : 0, c_hi = rbeg >= 0 ? min(rend, S.len) : S.len;
        const bool count_states = rbeg <= 0;
        unsigned long long psum = 0;
        if (pass == 1 && leaf) {
            for (int t = lane; t < depth; t += 32) psum += gterm(J.pos[t].pv, M[t]);
            psum = warp_sum(psum);
        }
        const long long obase = (pass == 1 && !leaf) ? offs[f] : 0;
        long long child = 0;
        unsigned long long nodes = 0, hs = 0;
        for (int c0 = c_lo; c0 < c_hi; c0 += 32) {
            const int idx = c0 + lane;
            bool ok = false;
            int c = -1;
            if (idx < c_hi) {
                c = S.ptr ? __ldg(S.ptr + S.base + idx) : idx;
                ok = feasible<DIR>(J, P, depth, c, (S.ptr && P.par >= 0) ? S.base + idx : -1, M);
            }
            const unsigned bal = __ballot_sync(FULL, ok);
            const int cnt = __popc(bal);
            if (pass == 1) {
                nodes += cnt;
                if (leaf) {
                    if (ok && count_ctr) {
                        hs += fmix64(psum + gterm(P.pv, c));
                        if (J.mbuf) emit_match(J, M, depth, c);
                    }
                } else if (ok) {
                    const long long o = obase + child + __popc(bal & ((1u << lane) - 1u));
                    int32_t *dst = fout + o * out_stride;
                    dst[0] = j; dst[1] = depth + 1; dst[2] = -1; dst[3] = -1;
                    for (int t = 0; t < depth; ++t) dst[FRAME_HDR + t] = M[t];
                    dst[FRAME_HDR + depth] = c;
                }
            }
            child += cnt;
        }
        if (pass == 0) {
            if (lane == 0) counts[f] = leaf ? 0 : (int32_t)child;
        } else if (count_ctr) {
            hs = warp_sum(hs);
            if (lane == 0) {
                if (count_states) atomicAdd(J.ctr + 1, (unsigned long long)S.len);
                atomicAdd(J.ctr + 2, nodes);
                if (leaf) {
                    atomicAdd(J.ctr + 0, nodes);
                    atomicAdd(J.ctr + 3, hs);
                }
            }
        }
        __syncwarp();
    }
}

// ========================================================= device split
//
// The breadth-first split as one cooperative launch.  Two forms:
//  * ordered (k_split_coop): every level is a count pass, a scan of the
//    warps' child counts and a write pass, so the children of a level come out
//    in search order -- the order that frame i -> shard i mod S relies on;
//  * single-pass (k_split_once, unsharded runs): every frame is tested once
//    and each 32-candidate chunk appends its children at an offset reserved
//    with one fetch-and-add, so a level costs one pass and one grid barrier.
// The loop stops when the frontier reaches `target` frames, is empty, would
// overflow `cap`, or `max_levels` levels are done.  All frames of a level
// share its depth, so a level-L frame has stride FRAME_HDR + L.

__device__ __forceinline__ long long block_excl_scan(long long x, long long *total);

constexpr unsigned long long BARRIER_GUARD_NS = 60ull * 1000000000ull;   // hang guard of one barrier

// Grid barrier for a cooperative launch (all blocks co-resident).  The wait
// is bounded: after BARRIER_GUARD_NS the block records an error and goes on.
__device__ __forceinline__ void grid_barrier(unsigned *count, unsigned *gen, int *status) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = gen;
        const unsigned g = *vgen;
        __threadfence();
        if (atomicAdd(count, 1u) == gridDim.x - 1) {
            *count = 0;
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            const unsigned long long t0 = globaltimer();
            unsigned backoff = 32;
            while (*vgen == g) {
                __nanosleep(backoff);
                if (backoff < 1024) backoff <<= 1;
                if (globaltimer() - t0 > BARRIER_GUARD_NS) { set_status(status, -3); break; }
            }
        }
        __threadfence();
    }
    __syncthreads();
}

struct SplitCtl {
    int32_t *buf0, *buf1;       // frame buffers of `cap_ints` ints each; a level-L frame has stride FRAME_HDR + L
    long long cap_ints;
    long long target;           // stop once the frontier has this many frames
    int max_levels;
    long long *wtot;            // [blocks]: children per block, then the blocks' exclusive offsets
    unsigned *bar;              // [2]: barrier count, generation (zeroed by the host)
    long long *result;          // [4]: final frame count, final buffer (0/1), levels done, last total
    int *status;
    int count_ctr;              // 0 in shards other than 0: levels above the frontier are counted once
    uint32_t *masks;            // candidate ballots of the count pass, replayed by the write pass
    long long mask_total;       // masks in the buffer (each warp owns mask_total / warps of them)
    long long *trace;           // single-pass split, tracing only (else null): [0, KMAX) each level's end
                                // (device clock), [KMAX, 2 KMAX) its longest candidate list of one frame
};

// One frame of a split level: count its children (pass 0) or write them from
// `out` on in candidate order and add its counters (pass 1).  Returns the
// number of children.
// The count pass stores each chunk's ballot in the warp's mask buffer (wm,
// mcap masks, position mp) and the write pass replays it instead of testing
// the candidates again (frames with at least 16 candidates); leaf frames have
// no children, so the count pass skips them and only the write pass tests
// them.  Past mcap masks the write pass tests again.
template <bool DIR>
__device__ __forceinline__ long long split_frame(const JobDesc *jobs, const int32_t *fr, int *M, int pass,
                                                 int32_t *fout, long long out, int stride, int count_ctr,
                                                 uint32_t *wm, long long mcap, long long &mp) {
    const int lane = threadIdx.x & 31;
    const int j = fr[0], depth = fr[1], rbeg = fr[2], rend = fr[3];
    const JobDesc &J = jobs[j];
    const bool leaf = depth + 1 == J.k;
    if (pass == 0 && leaf) return 0;
    for (int t = lane; t < depth; t += 32) M[t] = fr[FRAME_HDR + t];
    __syncwarp();
    const PosInfo P = J.pos[depth];
    const Src src = cand_source(J, P, M);
    const int c_lo = rbeg >= 0 ? rbeg : 0, c_hi = rbeg >= 0 ? min(rend, src.len) : src.len;
    unsigned long long psum = 0, nodes = 0, hs = 0;
    long long child = 0;
    if (pass == 1 && leaf && count_ctr) {
        for (int t = lane; t < depth; t += 32) psum += gterm(J.pos[t].pv, M[t]);
        psum = warp_sum(psum);
    }
    // short rows are cheaper to test twice than to store and reload
    const bool masked = !leaf && c_hi - c_lo >= 16;
    for (int c0 = c_lo; c0 < c_hi; c0 += 32) {
        const int idx = c0 + lane;
        bool ok = false;
        int c = -1;
        const bool replay = pass == 1 && masked && mp < mcap;
        if (idx < c_hi) {
            c = src.ptr ? __ldg(src.ptr + src.base + idx) : idx;
            if (replay) ok = (wm[mp] >> lane) & 1u;
            else ok = feasible<DIR>(J, P, depth, c, (src.ptr && P.par >= 0) ? src.base + idx : -1, M);
        }
        const unsigned bal = __ballot_sync(FULL, ok);
        if (masked) {
            if (pass == 0 && mp < mcap && lane == 0) wm[mp] = bal;
            ++mp;
        }
        const int cnt = __popc(bal);
        if (pass == 1) {
            nodes += cnt;
            if (leaf) {
                if (ok && count_ctr) {
                    hs += fmix64(psum + gterm(P.pv, c));
                    if (J.mbuf) emit_match(J, M, depth, c);
                }
            } else if (ok) {
                int32_t *dst = fout + (out + child + __popc(bal & ((1u << lane) - 1u))) * stride;
                dst[0] = j; dst[1] = depth + 1; dst[2] = -1; dst[3] = -1;
                for (int t = 0; t < depth; ++t) dst[FRAME_HDR + t] = M[t];
                dst[FRAME_HDR + depth] = c;
            }
        }
        if (!leaf) child += cnt;
    }
    if (pass == 1 && count_ctr) {
        hs = warp_sum(hs);
        if (lane == 0) {
            if (rbeg <= 0) atomicAdd(J.ctr + 1, (unsigned long long)src.len);
            atomicAdd(J.ctr + 2, nodes);
            if (leaf) {
                atomicAdd(J.ctr + 0, nodes);
                atomicAdd(J.ctr + 3, hs);
            }
        }
    }
    __syncwarp();
    return child;
}

template <bool DIR>
__global__ void __launch_bounds__(BLOCK) k_split_coop(const JobDesc *jobs, long long f0, SplitCtl S) {
    __shared__ int Msh[WARPS_PER_BLOCK][KMAX];
    __shared__ long long carry;
    __shared__ long long woff[WARPS_PER_BLOCK];   // a level's child offsets of this block's warps
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int *M = Msh[wib];
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    long long F = f0, total = 0;
    int cur = 0, level = 0;
    if (threadIdx.x == 0) atomicMax(reinterpret_cast<unsigned long long *>(S.result + 6), ~globaltimer());
    const long long mcap = S.masks ? S.mask_total / nw : 0;
    uint32_t *wm = S.masks ? S.masks + w * mcap : nullptr;
    for (; level < S.max_levels; ++level) {
        if (F == 0 || F >= S.target) break;
        const int32_t *fin = cur ? S.buf1 : S.buf0;
        int32_t *fout = cur ? S.buf0 : S.buf1;
        const int sin = FRAME_HDR + level, sout = FRAME_HDR + level + 1;   // all frames of a level share a depth
        // each warp owns a contiguous slice of the frontier, so children come out in search order
        const long long lo = F * w / nw, hi = F * (w + 1) / nw;
        long long mine = 0, mp = 0;
        for (long long f = lo; f < hi; ++f)
            mine += split_frame<DIR>(jobs, fin + f * sin, M, 0, fout, 0, sout, S.count_ctr, wm, mcap, mp);
        // children offsets: warps within the block here, blocks across the grid in block 0
        if (lane == 0) woff[wib] = mine;
        __syncthreads();
        if (threadIdx.x == 0) {
            long long acc = 0;
            for (int i = 0; i < WARPS_PER_BLOCK; ++i) {
                const long long x = woff[i];
                woff[i] = acc;
                acc += x;
            }
            S.wtot[blockIdx.x] = acc;
        }
        grid_barrier(S.bar, S.bar + 1, S.status);
        if (blockIdx.x == 0) {
            // exclusive scan of the per-block counts (one block, chunk by chunk)
            if (threadIdx.x == 0) carry = 0;
            __syncthreads();
            for (long long b = 0; b < gridDim.x; b += BLOCK) {
                const long long i = b + threadIdx.x;
                const long long x = i < gridDim.x ? S.wtot[i] : 0;
                long long tot;
                const long long ex = block_excl_scan(x, &tot);
                if (i < gridDim.x) S.wtot[i] = carry + ex;
                __syncthreads();
                if (threadIdx.x == 0) carry += tot;
                __syncthreads();
            }
            if (threadIdx.x == 0) S.result[3] = carry;
        }
        grid_barrier(S.bar, S.bar + 1, S.status);
        total = *(volatile long long *)(S.result + 3);
        if (total * sout > S.cap_ints) break;   // the next level does not fit: keep this frontier
        const long long out = *(volatile long long *)(S.wtot + blockIdx.x) + woff[wib];
        long long written = 0;
        mp = 0;
        for (long long f = lo; f < hi; ++f)
            written += split_frame<DIR>(jobs, fin + f * sin, M, 1, fout, out + written, sout, S.count_ctr, wm,
                                        mcap, mp);
        grid_barrier(S.bar, S.bar + 1, S.status);
        F = total;
        cur ^= 1;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        S.result[0] = F;
        S.result[1] = cur;
        S.result[2] = level;
    }
    if (threadIdx.x == 0) atomicMax(reinterpret_cast<unsigned long long *>(S.result + 7), globaltimer());
}

// Counters of the single-pass split, summed per warp while consecutive frames
// belong to one job and added to the job's counters on a job change or at the
// end of the warp's slice (lane 0), so a level of many frames does not queue
// thousands of atomics on one job's four words.
struct SplitAcc {
    int job;
    unsigned long long st, nd, mt, hs;
};

// (lane 0 only; the warp's SplitAcc lives in shared memory)
__device__ __forceinline__ void split_acc_flush(const JobDesc *jobs, SplitAcc &A) {
    if (A.job >= 0) {
        unsigned long long *ctr = jobs[A.job].ctr;
        if (A.st) atomicAdd(ctr + 1, A.st);
        if (A.nd) atomicAdd(ctr + 2, A.nd);
        if (A.mt) atomicAdd(ctr + 0, A.mt);
        if (A.hs) atomicAdd(ctr + 3, A.hs);
    }
    A.job = -1;
    A.st = A.nd = A.mt = A.hs = 0;
}

// One frame of a single-pass split level: test its candidates once, add its
// counters to A, and append the children of each chunk at offsets reserved on
// the level's child counter `lvl_ctr`.  A reservation that ends past
// `cap_frames` raises `full` and writes nothing (the level is then abandoned,
// see below).  Returns the frame's candidate range length.
template <bool DIR>
__device__ __forceinline__ int split_frame_once(const JobDesc *jobs, const int32_t *fr, int *M, int32_t *fout,
                                                int stride, long long cap_frames, unsigned long long *lvl_ctr,
                                                long long *full, SplitAcc &A) {
    const int lane = threadIdx.x & 31;
    const int j = fr[0], depth = fr[1], rbeg = fr[2], rend = fr[3];
    const JobDesc &J = jobs[j];
    const bool leaf = depth + 1 == J.k;
    for (int t = lane; t < depth; t += 32) M[t] = fr[FRAME_HDR + t];
    __syncwarp();
    const PosInfo &P = J.pos[depth];
    const Src src = cand_source(J, P, M);
    const int c_lo = rbeg >= 0 ? rbeg : 0, c_hi = rbeg >= 0 ? min(rend, src.len) : src.len;
    unsigned long long psum = 0, nodes = 0, hs = 0;
    if (leaf) {
        for (int t = lane; t < depth; t += 32) psum += gterm(J.pos[t].pv, M[t]);
        psum = warp_sum(psum);
    }
    // the children's position: where its candidates come from
    // a child whose own candidate list is longer than SPLIT_RANGE is written as range
    // frames, so that no warp of the next level scans a hub's whole row while the
    // others wait at the level's barrier (JOB_LONG_LISTS: such a list can occur)
    PosInfo Q;
    const int32_t *qrow = nullptr;
    bool ranges = false;
    if (!leaf && (J.flags & JOB_LONG_LISTS)) {
        Q = J.pos[depth + 1];
        if (Q.par >= 0) {
            qrow = (Q.flags & POS_IN_ROW) ? J.t.irowptr : J.t.rowptr;
            ranges = J.t.maxdeg == 0 || J.t.maxdeg > SPLIT_RANGE;
        } else {
            ranges = ((J.flags & JOB_RIDS) ? Q.ucnt : J.t.n) > SPLIT_RANGE;
        }
    }
    for (int c0 = c_lo; c0 < c_hi; c0 += 32) {
        const int idx = c0 + lane;
        bool ok = false;
        int c = -1;
        if (idx < c_hi) {
            c = src.ptr ? __ldg(src.ptr + src.base + idx) : idx;
            ok = feasible<DIR>(J, P, depth, c, (src.ptr && P.par >= 0) ? src.base + idx : -1, M);
        }
        const unsigned bal = __ballot_sync(FULL, ok);
        const int cnt = __popc(bal);
        nodes += cnt;
        if (leaf) {
            if (ok) {
                hs += fmix64(psum + gterm(P.pv, c));
                if (J.mbuf) emit_match(J, M, depth, c);
            }
        } else if (cnt > 0) {
            // frames per child: one, or one per SPLIT_RANGE candidates of a long list
            int r = ok ? 1 : 0;
            if (ok && ranges) {
                int len;
                if (qrow) {
                    const int a = Q.par == depth ? c : M[Q.par];
                    len = __ldg(qrow + a + 1) - __ldg(qrow + a);
                } else {
                    len = (J.flags & JOB_RIDS) ? Q.ucnt : J.t.n;
                }
                r = len > SPLIT_RANGE ? (len + SPLIT_RANGE - 1) / SPLIT_RANGE : 1;
            }
            int incl, total;
            if (ranges) {
                incl = r;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(FULL, incl, o);
                    if (lane >= o) incl += y;
                }
                total = __shfl_sync(FULL, incl, 31);
            } else {
                incl = __popc(bal & (0xffffffffu >> (31 - lane)));   // survivors up to this lane
                total = cnt;
            }
            unsigned long long at = 0;
            if (lane == 0) at = atomicAdd(lvl_ctr, (unsigned long long)total);
            at = __shfl_sync(FULL, at, 0);
            if ((long long)(at + total) <= cap_frames) {
                for (int q = 0; q < r; ++q) {
                    int32_t *dst = fout + (long long)(at + incl - r + q) * stride;
                    dst[0] = j;
                    dst[1] = depth + 1;
                    dst[2] = r == 1 ? -1 : q * SPLIT_RANGE;
                    dst[3] = r == 1 ? -1 : (q + 1 == r ? 0x7fffffff : (q + 1) * SPLIT_RANGE);
                    for (int t = 0; t < depth; ++t) dst[FRAME_HDR + t] = M[t];
                    dst[FRAME_HDR + depth] = c;
                }
            } else if (lane == 0) {
                *(volatile long long *)full = 1;
            }
        }
    }
    hs = warp_sum(hs);
    if (lane == 0) {
        if (A.job != j) {
            split_acc_flush(jobs, A);
            A.job = j;
        }
        if (rbeg <= 0) A.st += (unsigned long long)src.len;
        A.nd += nodes;
        if (leaf) {
            A.mt += nodes;
            A.hs += hs;
        }
    }
    __syncwarp();
    return c_hi - c_lo;
}

// A split frame with at most this many candidates is expanded by one lane.
constexpr int SPLIT_LANE_MAX = 8;
static_assert(SPLIT_LANE_MAX <= 32, "a lane keeps its frame's survivors in one 32-bit mask");

// Frames of candidates a child of position depth + 1 takes: one, or one per
// SPLIT_RANGE candidates when its list is longer (JOB_LONG_LISTS pairs only).
__device__ __forceinline__ int split_child_frames(const JobDesc &J, int depth, int c, const int *M) {
    if (!(J.flags & JOB_LONG_LISTS)) return 1;
    const PosInfo &Q = J.pos[depth + 1];
    long long len;
    if (Q.par >= 0) {
        if (J.t.maxdeg != 0 && J.t.maxdeg <= SPLIT_RANGE) return 1;
        const int32_t *rp = (Q.flags & POS_IN_ROW) ? J.t.irowptr : J.t.rowptr;
        const int a = Q.par == depth ? c : M[Q.par];
        len = __ldg(rp + a + 1) - __ldg(rp + a);
    } else {
        len = (J.flags & JOB_RIDS) ? Q.ucnt : J.t.n;
    }
    return len > SPLIT_RANGE ? (int)((len + SPLIT_RANGE - 1) / SPLIT_RANGE) : 1;
}

// The next 32 frames of a warp's slice [f0, hi) of a single-pass split level,
// one per lane where a frame has at most 32 candidates: the lane tests them in
// turn (a warp on such a frame would leave most lanes idle), reading the
// frame's images straight from the frontier.  Children are appended at offsets
// from one fetch-and-add per warp; counters are summed over runs of lanes with
// the same job and added with one atomic per run.  Returns the lanes whose
// frames have longer ranges (the caller expands them a warp at a time) and
// raises `longest` to the longest range seen.
template <bool DIR>
__device__ unsigned split_lane_frames(const JobDesc *jobs, const int32_t *fin, long long f0, long long hi, int depth,
                                      int32_t *fout, long long cap_frames, unsigned long long *lvl_ctr,
                                      long long *full, int &longest) {
    const int lane = threadIdx.x & 31;
    const int sin = FRAME_HDR + depth, sout = sin + 1;
    const long long f = f0 + lane;
    const bool have = f < hi;
    const int32_t *fr = fin + (have ? f : f0) * sin;
    const int *Mg = fr + FRAME_HDR;
    int j = 0, rbeg = -1, c_lo = 0, c_hi = 0;
    Src src;
    src.ptr = nullptr; src.base = 0; src.len = 0;
    if (have) {
        j = fr[0];
        rbeg = fr[2];
        const int rend = fr[3];
        src = cand_source(jobs[j], jobs[j].pos[depth], Mg);
        c_lo = rbeg >= 0 ? rbeg : 0;
        c_hi = rbeg >= 0 ? min(rend, src.len) : src.len;
        longest = max(longest, c_hi - c_lo);
    }
    const bool mine = have && c_hi - c_lo <= SPLIT_LANE_MAX;
    const unsigned longm = __ballot_sync(FULL, have && !mine);
    if (!__any_sync(FULL, mine)) return longm;
    const JobDesc &J = jobs[j];
    const PosInfo &P = J.pos[depth];   // (read where used: a copy would hold 16 registers)
    const bool leaf = depth + 1 == J.k;
    unsigned mask = 0;   // the lane's survivors, bit i for candidate c_lo + i
    int nch = 0;         // frames its children take
    unsigned long long st = 0, nd = 0, mt = 0, hs = 0;
    if (mine) {
        for (int i = 0; i < c_hi - c_lo; ++i) {
            const int idx = c_lo + i;
            const int c = src.ptr ? __ldg(src.ptr + src.base + idx) : idx;
            if (feasible<DIR>(J, P, depth, c, (src.ptr && P.par >= 0) ? src.base + idx : -1, Mg)) mask |= 1u << i;
        }
        nd = __popc(mask);
        if (rbeg <= 0) st = (unsigned long long)src.len;
        if (leaf) {
            mt = nd;
            if (mask) {
                unsigned long long psum = 0;
                for (int t = 0; t < depth; ++t) psum += gterm(J.pos[t].pv, Mg[t]);
                for (unsigned m = mask; m; m &= m - 1) {
                    const int idx = c_lo + __ffs(m) - 1;
                    const int c = src.ptr ? __ldg(src.ptr + src.base + idx) : idx;
                    hs += fmix64(psum + gterm(P.pv, c));
                    if (J.mbuf) emit_match(J, Mg, depth, c);
                }
            }
        } else {
            for (unsigned m = mask; m; m &= m - 1) {
                const int idx = c_lo + __ffs(m) - 1;
                const int c = src.ptr ? __ldg(src.ptr + src.base + idx) : idx;
                nch += split_child_frames(J, depth, c, Mg);
            }
        }
    }
    // children: one reservation for the warp
    int incl = nch;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(FULL, incl, 31);
    if (total > 0) {
        unsigned long long at = 0;
        if (lane == 0) at = atomicAdd(lvl_ctr, (unsigned long long)total);
        at = __shfl_sync(FULL, at, 0);
        if ((long long)(at + total) <= cap_frames) {
            long long o = (long long)at + incl - nch;
            for (unsigned m = nch ? mask : 0u; m; m &= m - 1) {
                const int idx = c_lo + __ffs(m) - 1;
                const int c = src.ptr ? __ldg(src.ptr + src.base + idx) : idx;
                const int r = split_child_frames(J, depth, c, Mg);
                for (int q = 0; q < r; ++q, ++o) {
                    int32_t *dst = fout + o * sout;
                    dst[0] = j;
                    dst[1] = depth + 1;
                    dst[2] = r == 1 ? -1 : q * SPLIT_RANGE;
                    dst[3] = r == 1 ? -1 : (q + 1 == r ? 0x7fffffff : (q + 1) * SPLIT_RANGE);
                    for (int t = 0; t < depth; ++t) dst[FRAME_HDR + t] = Mg[t];
                    dst[FRAME_HDR + depth] = c;
                }
            }
        } else if (lane == 0) {
            *(volatile long long *)full = 1;
        }
    }
    // counters: segmented sums over runs of consecutive lanes with the same job
    const int key = mine ? j : -1;
    const int prev = __shfl_up_sync(FULL, key, 1);
    const unsigned heads = __ballot_sync(FULL, lane == 0 || key != prev);
    const int head = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long a = __shfl_up_sync(FULL, st, o), b = __shfl_up_sync(FULL, nd, o),
                                 c = __shfl_up_sync(FULL, mt, o), d = __shfl_up_sync(FULL, hs, o);
        if (lane - o >= head) {
            st += a;
            nd += b;
            mt += c;
            hs += d;
        }
    }
    const bool tail = lane == 31 || ((heads >> (lane + 1)) & 1u);
    if (tail && key >= 0) {
        unsigned long long *ctr = J.ctr;
        if (st) atomicAdd(ctr + 1, st);
        if (nd) atomicAdd(ctr + 2, nd);
        if (mt) atomicAdd(ctr + 0, mt);
        if (hs) atomicAdd(ctr + 3, hs);
    }
    return longm;
}

// Single-pass split (unsharded runs; the caller's shard counts the levels).
// The children of level L are counted on wtot[L] (zeroed by the host).  A
// level whose children do not all fit is abandoned after its barrier: its
// frames stay the frontier, rewritten so that the search does not count the
// level again -- a frame with children becomes a counted range (over its
// whole candidate list if it had none; the search re-derives its children
// and counts from the next level on), a frame on the last position becomes
// the empty range [1, 1).
template <bool DIR>
__global__ void __launch_bounds__(BLOCK, 4) k_split_once(const JobDesc *jobs, long long f0, SplitCtl S) {
    __shared__ int Msh[WARPS_PER_BLOCK][KMAX];
    __shared__ SplitAcc Ash[WARPS_PER_BLOCK];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int *M = Msh[wib];
    SplitAcc &A = Ash[wib];
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    unsigned long long *lvl_ctr = reinterpret_cast<unsigned long long *>(S.wtot);
    long long F = f0;
    int cur = 0, level = 0;
    if (lane == 0) {
        A.job = -1;
        A.st = A.nd = A.mt = A.hs = 0;
    }
    if (threadIdx.x == 0) atomicMax(reinterpret_cast<unsigned long long *>(S.result + 6), ~globaltimer());
    for (; level < S.max_levels; ++level) {
        if (F == 0 || F >= S.target) break;
        int32_t *fin = cur ? S.buf1 : S.buf0;
        int32_t *fout = cur ? S.buf0 : S.buf1;
        const int sin = FRAME_HDR + level, sout = FRAME_HDR + level + 1;
        const long long lo = F * w / nw, hi = F * (w + 1) / nw;
        int longest = 0;
        for (long long f0 = lo; f0 < hi; f0 += 32) {
            // frames of at most 32 candidates one per lane, longer ones a warp at a time
            unsigned longm = split_lane_frames<DIR>(jobs, fin, f0, hi, level, fout, S.cap_ints / sout,
                                                    lvl_ctr + level, S.result + 5, longest);
            while (longm) {
                const int L = __ffs(longm) - 1;
                longm &= longm - 1;
                longest = max(longest, split_frame_once<DIR>(jobs, fin + (f0 + L) * sin, M, fout, sout,
                                                             S.cap_ints / sout, lvl_ctr + level, S.result + 5, A));
            }
        }
        longest = warp_max(longest);
        if (lane == 0) split_acc_flush(jobs, A);
        if (S.trace && lane == 0 && longest > 0)
            atomicMax(reinterpret_cast<unsigned long long *>(S.trace + KMAX + level), (unsigned long long)longest);
        grid_barrier(S.bar, S.bar + 1, S.status);
        if (S.trace && blockIdx.x == 0 && threadIdx.x == 0) S.trace[level] = (long long)globaltimer();
        if (*(volatile long long *)(S.result + 5) != 0) {
            for (long long f = lo; f < hi; ++f) {
                int32_t *fr = fin + f * sin;
                if (lane == 0) {
                    const bool leaf = fr[1] + 1 == jobs[fr[0]].k;
                    if (leaf) { fr[2] = 1; fr[3] = 1; }
                    else {
                        fr[1] |= FRAME_COUNTED;
                        if (fr[2] < 0) { fr[2] = 0; fr[3] = 0x7fffffff; }
                    }
                }
            }
            break;
        }
        F = (long long)*(volatile unsigned long long *)(lvl_ctr + level);
        cur ^= 1;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        S.result[0] = F;
        S.result[1] = cur;
        S.result[2] = level;
    }
    if (threadIdx.x == 0) atomicMax(reinterpret_cast<unsigned long long *>(S.result + 7), globaltimer());
}

// =================================================================== scan

constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = BLOCK * SCAN_ITEMS;

__device__ __forceinline__ long long block_excl_scan(long long x, long long *total) {
    __shared__ long long ws[WARPS_PER_BLOCK];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) ws[w] = incl;
    __syncthreads();
    long long before = 0, tot = 0;
    for (int i = 0; i < WARPS_PER_BLOCK; ++i) {
        if (i < w) before += ws[i];
        tot += ws[i];
    }
    __syncthreads();
    *total = tot;
    return before + incl - x;
}

__global__ void __launch_bounds__(BLOCK) k_scan_tiles(const int32_t *in, long long *out, long long n, long long *tile_sum) {
    const long long base = (long long)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    long long v[SCAN_ITEMS], s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        v[i] = (base + i < n) ? in[base + i] : 0;
        s += v[i];
    }
    long long tot;
    long long ex = block_excl_scan(s, &tot);
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        if (base + i < n) out[base + i] = ex;
        ex += v[i];
    }
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(BLOCK) k_scan_sums(long long *tile_sum, long long ntiles, long long *total) {
    __shared__ long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (long long b = 0; b < ntiles; b += BLOCK) {
        const long long i = b + threadIdx.x;
        const long long x = i < ntiles ? tile_sum[i] : 0;
        long long tot;
        const long long ex = block_excl_scan(x, &tot);
        if (i < ntiles) tile_sum[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(BLOCK) k_scan_add(long long *out, long long n, const long long *tile_sum) {
    const long long base = (long long)blockIdx.x * SCAN_TILE;
    const long long add = tile_sum[blockIdx.x];
    for (int i = threadIdx.x; i < SCAN_TILE; i += BLOCK)
        if (base + i < n) out[base + i] += add;
}

// ========================================================= frame queue

// Ticket queue of donated frames.  Producers (donating warps) and consumers
// (idle warps) each draw tickets from their own counter with one
// fetch-and-add; ticket t of either side meets at cell t mod cap, whose
// sequence word walks through
//     t  (free for ticket t)  ->  t | CELL_LOCK  (producer t writing)
//        ->  t + 1  (published)  ->  t + cap  (consumed: free for t + cap)
// or, if consumer t leaves before producer t arrives,  t -> t + cap
// (abandoned; producer t then draws another ticket).  A consumer waits on
// its own cell only, so no line is fought over however many warps are idle,
// and every frame reaches exactly one consumer.  Lane 0 only.
constexpr unsigned long long CELL_LOCK = 1ull << 63;

// Producer: a ticket whose cell is locked for writing, or -1 (the caller keeps its work).
__device__ long long queue_reserve(const SearchCtl &C) {
    const unsigned long long cap = (unsigned long long)C.pcap;
    for (int a = 0; a < RESERVE_TICKETS; ++a) {
        const unsigned long long t = atomicAdd(C.ptail, 1ull);
        unsigned long long *seq = C.pseq + t % cap;
        for (long long spin = 0;; ++spin) {
            const unsigned long long sv = load_acquire(seq);
            if (sv == t) {
                if (atomicCAS(seq, t, t | CELL_LOCK) == t) return (long long)t;
                continue;                                   // consumer t left meanwhile: look again
            }
            if ((sv & ~CELL_LOCK) > t) break;               // consumer t left: draw another ticket
            if (spin > RESERVE_SPIN_LIMIT) {                // the cell's previous lap never ended
                set_status(C.status, -3);
                return -1;
            }
            __nanosleep(128);
        }
    }
    return -1;
}

// Consumer holding ticket t: is its frame published?
__device__ __forceinline__ bool queue_ready(const SearchCtl &C, unsigned long long t) {
    return load_acquire(C.pseq + t % (unsigned long long)C.pcap) == t + 1;
}

// Consumer holding ticket t wants to leave: true if it left (no frame will
// come to it), false if its frame is published (the caller takes it) or, when
// not stopping, if the cell is still in its previous lap (the caller stays).
// A stopping consumer leaves a cell in its previous lap as it is: a frame
// published there later is found among the unconsumed cells after the launch.
__device__ bool queue_leave(const SearchCtl &C, unsigned long long t, bool stopping) {
    const unsigned long long cap = (unsigned long long)C.pcap;
    unsigned long long *seq = C.pseq + t % cap;
    for (long long spin = 0;; ++spin) {
        const unsigned long long sv = load_acquire(seq);
        if (sv == t + 1) return false;
        if (sv == t) {
            if (atomicCAS(seq, t, t + cap) == t) return true;
            continue;
        }
        if (!(sv & CELL_LOCK) && sv < t) return stopping;   // previous lap still in use
        // locked by producer t, which publishes within a few instructions: wait
        if (spin > RESERVE_SPIN_LIMIT) {
            set_status(C.status, -3);
            return true;
        }
        __nanosleep(128);
    }
}

// Warp-collective: push frame [j, depth, beg, end, M[0..mlen-1] (+ last)]
// (`last` >= 0 appends one more image).  Returns false if the queue is full.
__device__ bool push_frame(const SearchCtl &C, int j, int depth, int beg, int end, const int *M, int mlen, int last) {
    const int lane = threadIdx.x & 31;
    long long t = -1;
    if (lane == 0) {
        atomicAdd(C.outstanding, 1);
        t = queue_reserve(C);
        if (t < 0) atomicSub(C.outstanding, 1);
    }
    t = __shfl_sync(FULL, t, 0);
    if (t < 0) return false;
    int32_t *cell = C.pool + (size_t)(t % C.pcap) * POOL_STRIDE;
    if (lane == 0) { cell[0] = j; cell[1] = depth; cell[2] = beg; cell[3] = end; }
    for (int i = lane; i < mlen; i += 32) cell[FRAME_HDR + i] = M[i];
    if (last >= 0 && lane == 0) cell[FRAME_HDR + mlen] = last;
    __syncwarp();
    if (lane == 0) {
        __threadfence();
        store_release(C.pseq + (t % C.pcap), (unsigned long long)t + 1);   // publish (clears the lock)
        atomicAdd(C.donations, 1ull);
    }
    __syncwarp();
    return true;
}

struct Frame {
    int job, depth, beg, end;
    bool counted;   // FRAME_COUNTED: the range's accepted nodes and states are already counted
};

// Optional per-warp timing, kept in the warp's own trace record (no registers):
// {start, exit, busy, last frame end, longest frame's duration, its
// job | depth << 16 | origin << 30 (1 frontier, 2 queue), its states, its
// nodes, origin of the current frame, ns spent donating, donation events,
// frames donated, frames taken from the queue, ns and states in them, 0}
// (WTRACE_WORDS words).
struct WarpClock {
    __device__ static unsigned long long *rec(const SearchCtl &C) {
        return C.wtrace + WTRACE_WORDS * ((size_t)blockIdx.x * WARPS_PER_BLOCK + (threadIdx.x >> 5));
    }
    __device__ static void begin(const SearchCtl &C) {
        if (C.wtrace && (threadIdx.x & 31) == 0) rec(C)[0] = globaltimer();
    }
    __device__ static void origin(const SearchCtl &C, int kind) {
        if (C.wtrace && (threadIdx.x & 31) == 0) rec(C)[8] = (unsigned long long)kind;
    }
    __device__ static void frame_in(const SearchCtl &C) {
        if (C.wtrace && (threadIdx.x & 31) == 0) rec(C)[3] = globaltimer();
    }
    __device__ static void frame_out(const SearchCtl &C, const Frame &fr, unsigned long long st,
                                     unsigned long long nd) {
        if (C.wtrace && (threadIdx.x & 31) == 0) {
            unsigned long long *w = rec(C);
            const unsigned long long now = globaltimer(), dur = now - w[3];
            w[2] += dur;
            w[3] = now;   // after the last frame: when the warp last held work
            if (w[8] == 2) { w[12] += 1; w[13] += dur; w[14] += st; }
            if (dur > w[4]) {
                w[4] = dur;
                w[5] = (unsigned long long)fr.job | ((unsigned long long)fr.depth << 16) | (w[8] << 30);
                w[6] = st;
                w[7] = nd;
            }
        }
    }
    __device__ static void finish(const SearchCtl &C) {
        if (C.wtrace && (threadIdx.x & 31) == 0) rec(C)[1] = globaltimer();
    }
    __device__ static unsigned long long don_begin(const SearchCtl &C) {
        return (C.wtrace && (threadIdx.x & 31) == 0) ? globaltimer() : 0ull;
    }
    __device__ static void don_end(const SearchCtl &C, unsigned long long t, int given) {
        if (C.wtrace && (threadIdx.x & 31) == 0) {
            unsigned long long *w = rec(C);
            w[9] += globaltimer() - t;
            w[10] += 1;
            w[11] += (unsigned long long)given;
        }
    }
};


// Warp-collective: append range frame [j, depth (| FRAME_COUNTED), beg, end,
// M[0..depth-1]] to the checkpoint.  Every warp dumps at most two frames per
// level, so a buffer of 2 * kmax frames per warp never overflows.
__device__ void ckpt_push(const SearchCtl &C, int j, int depth, bool counted, int beg, int end, const int *M) {
    const int lane = threadIdx.x & 31;
    unsigned long long slot = 0;
    if (lane == 0) slot = atomicAdd(C.ckpt_n, 1ull);
    slot = __shfl_sync(FULL, slot, 0);
    if ((long long)slot >= C.ckpt_cap) return;
    int32_t *cell = C.ckpt + (size_t)slot * C.ckpt_stride;
    if (lane == 0) { cell[0] = j; cell[1] = depth | (counted ? FRAME_COUNTED : 0); cell[2] = beg; cell[3] = end; }
    for (int i = lane; i < depth; i += 32) cell[FRAME_HDR + i] = M[i];
    __syncwarp();
}

// First index in ascending a[0..n) whose value is >= x (lane 0 searches, all lanes get it).
__device__ int lower_bound_warp(const int32_t *a, int n, int x) {
    int lo = 0;
    if ((threadIdx.x & 31) == 0) {
        int hi = n;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(a + mid) < x) lo = mid + 1; else hi = mid;
        }
    }
    return __shfl_sync(FULL, lo, 0);
}

// Warp-collective: take the next frame (frontier first, then the queue) and
// copy its images into M.  Waits (bounded) while other warps still hold work.
// Returns false when the search is over or stopped.
__device__ bool acquire_frame(const SearchCtl &C, int *M, Frame &fr, unsigned long long deadline) {
    const int lane = threadIdx.x & 31;
    bool idle = false;
    long long spins = 0;
    unsigned backoff = 64;
    unsigned long long idle_since = 0;
    int kind = 0;        // 1 frontier, 2 queue, 0 stop
    long long idx = -1;
    long long ticket = -1;   // consumer ticket held (lane 0)
    for (;;) {
        kind = -1;
        if (lane == 0) {
            if (load_relaxed(C.status) != 0) {
                // stopping: leave the ticket, or take the frame already sent to it
                if (ticket >= 0 && !queue_leave(C, (unsigned long long)ticket, true)) { kind = 2; idx = ticket; }
                else kind = 0;
            } else {
                if (ticket < 0 && load_acquire(C.fnext) < (unsigned long long)C.nfront) {
                    const unsigned long long f = atomicAdd(C.fnext, 1ull);
                    if ((long long)f < C.nfront) { kind = 1; idx = (long long)f; }
                }
                if (kind < 0) {
                    if (ticket < 0) ticket = (long long)atomicAdd(C.phead, 1ull);
                    if (queue_ready(C, (unsigned long long)ticket)) { kind = 2; idx = ticket; }
                }
                // all work done: no frame can come to the ticket any more
                if (kind < 0 && load_relaxed(C.outstanding) == 0) kind = 0;
            }
            if (kind < 0) {
                if (!idle) { atomicAdd(C.idle, 1); idle = true; idle_since = globaltimer(); }
                // optional early exit of a warp that found no work for a while (it leaves its
                // ticket first; a frame already sent to it is taken instead), so the freed block
                // slots serve kernels launched on other streams
                else if (C.idle_exit_ns != 0 && globaltimer() - idle_since > C.idle_exit_ns) {
                    if (queue_leave(C, (unsigned long long)ticket, false)) kind = 0;
                    else if (queue_ready(C, (unsigned long long)ticket)) { kind = 2; idx = ticket; }
                    else idle_since = globaltimer();   // previous lap still in use: stay a while
                }
                if (kind < 0 && (++spins & 1023) == 0) {
                    // the stop paths set the status; the next round leaves the ticket.  A warp idle
                    // far longer than any search leaves a frame to wait ends the launch with an error.
                    const unsigned long long now = globaltimer();
                    if ((C.cancel != nullptr && *C.cancel != 0)) set_status(C.status, -6);
                    else if (deadline != 0 && now > deadline) set_status(C.status, -5);
                    else if (now - idle_since > IDLE_GUARD_NS) set_status(C.status, -3);
                }
            }
        }
        kind = __shfl_sync(FULL, kind, 0);
        if (kind >= 0) break;
        // exponential backoff: one warp per block polls often, the others rarely
        __nanosleep(backoff);
        if (backoff < ((threadIdx.x >> 5) == 0 ? IDLE_BACKOFF_FAST : IDLE_BACKOFF_SLOW)) backoff <<= 1;
    }
    if (lane == 0 && idle) atomicSub(C.idle, 1);
    if (kind == 0) return false;
    WarpClock::origin(C, kind);
    idx = __shfl_sync(FULL, idx, 0);
    const int32_t *src;
    if (kind == 1) {
        const long long g = idx * (long long)C.shard_count + C.shard_index;
        src = C.front + g * C.fstride;
    } else {
        if (lane == 0) __threadfence();
        __syncwarp();
        src = C.pool + (size_t)(idx % C.pcap) * POOL_STRIDE;
    }
    const int dw = src[1];
    fr.job = src[0]; fr.depth = dw & FRAME_DEPTH_MASK; fr.counted = (dw & FRAME_COUNTED) != 0;
    fr.beg = src[2]; fr.end = src[3];
    for (int i = lane; i < fr.depth; i += 32) M[i] = src[FRAME_HDR + i];
    __syncwarp();
    if (kind == 2 && lane == 0) {
        __threadfence();
        store_release(C.pseq + (idx % C.pcap), (unsigned long long)idx + C.pcap);
    }
    return true;
}

// Periodic checks by lane 0: cancellation, deadline, budget, other warps'
// errors.  Returns nonzero (warp-uniform) when the warp must stop.
__device__ __forceinline__ int must_stop(const SearchCtl &C, const JobDesc &J, unsigned long long local_states,
                                         unsigned long long deadline, unsigned long long now,
                                         unsigned long long &last_cancel) {
    int stop = 0;
    if ((threadIdx.x & 31) == 0) {
        const bool read_cancel = C.cancel != nullptr && now - last_cancel >= CANCEL_CHECK_NS;
        if (read_cancel) last_cancel = now;
        if (load_relaxed(C.status) != 0) stop = 1;
        else if (read_cancel && *C.cancel != 0) { set_status(C.status, -6); stop = 1; }
        else if (deadline != 0 && globaltimer() > deadline) { set_status(C.status, -5); stop = 1; }
        else if (C.budget > 0 && (long long)(*(volatile unsigned long long *)(J.ctr + 1) + local_states) > C.budget) {
            set_status(C.status, -4); stop = 1;
        }
    }
    return __shfl_sync(FULL, stop, 0);
}

// Warp-uniform: has CHECK_NS of device time passed since the last check?
__device__ __forceinline__ bool time_to_check(unsigned long long &last) {
    unsigned long long now = 0;
    if ((threadIdx.x & 31) == 0) now = globaltimer();
    now = __shfl_sync(FULL, now, 0);
    if (now - last < CHECK_NS) return false;
    last = now;
    return true;
}

// Warp-uniform: should this warp donate now?  Donation is wanted while more
// warps are idle than frames wait in the queue; a donor first takes one of
// those (idle - queued) slots, so a few donors, not every busy warp, answer
// one idle warp.  A true result must be paired with donation_done().
__device__ __forceinline__ bool donation_claim(const SearchCtl &C) {
    int ok = 0;
    if ((threadIdx.x & 31) == 0 && C.donate) {
        // consumer tickets not yet matched by a producer = idle warps waiting for a frame
        const long long waiting = (long long)(load_acquire(C.phead) - load_acquire(C.ptail));
        if (waiting > 0 && atomicAdd(C.promised, 1) < waiting) ok = 1;
        else if (waiting > 0) atomicSub(C.promised, 1);
    }
    return __shfl_sync(FULL, ok, 0) != 0;
}

__device__ __forceinline__ void donation_done(const SearchCtl &C) {
    if ((threadIdx.x & 31) == 0) atomicSub(C.promised, 1);
    __syncwarp();
}

// ===================================================== search: CSR kernel
//
// One warp owns one depth-first search.  A level's candidates are the row of
// M(P(mu_i)) (or V_t / D(mu_i) when mu_i is unparented), scanned 32 at a time,
// one candidate per lane; each lane tests rules 1-4 and the domain bit, and a
// ballot compacts the chunk's survivors.  Per warp, shared memory holds M,
// the level records and a compact copy of the job's position table; the
// job's pointers stay in registers.

__host__ __device__ __forceinline__ size_t round16(size_t x) { return (x + 15) & ~(size_t)15; }

struct PosC {                // hot fields of one position
    int16_t pv, par, bb, bc;
    int32_t lab, odeg, ideg, pel, flags;
};

struct LvCsr {
    int base;                // offset of the level's candidate list in its array
    int cur, end;            // unscanned candidates [cur, end)
    unsigned mask;           // survivors of the last scanned chunk, not yet descended
    int cbase;               // index of that chunk's first candidate
    int len;                 // the node's raw candidate count (its states, counted at index 0)
};

__host__ __device__ __forceinline__ size_t csr_smem_per_warp(int kmax) {
    return round16((size_t)kmax * sizeof(LvCsr) + (size_t)kmax * sizeof(int) + (size_t)kmax * sizeof(PosC));
}

struct CsrJob {
    const int32_t *rowptr, *col, *elab, *irowptr, *icol, *ielab, *indeg, *ulist, *hub_slot;
    const int2 *vld;
    const uint64_t *filt, *adj, *hub_bits;
    const BackEdge *back;
    const PosInfo *pos;
    int n, dw, k, flags;
};

// Candidate array of a position: the parent's out- or in-row, D(mu_i), or
// null for "candidate j is vertex j".
__device__ __forceinline__ const int32_t *csr_src(const CsrJob &B, const PosC &p) {
    if (p.par >= 0) return (p.flags & POS_IN_ROW) ? B.icol : B.col;
    return (B.flags & JOB_RIDS) ? B.ulist : nullptr;
}

// Rules 1-4 (Section "RI") and the RI-DS domain test for candidate c of
// position i; eidx is c's index in the parent's row (parent-arc label) or -1.
template <bool DIR>
__device__ __forceinline__ bool csr_feasible(const CsrJob &B, const PosC &p, int i, int c, int eidx, const int *M) {
    const int2 v = __ldg(B.vld + c);
    if (v.x != p.lab || v.y < p.odeg) return false;                           // rules 2, 3
    if (DIR && __ldg(B.indeg + c) < p.ideg) return false;                    // rule 3 (in)
    if (B.flags & JOB_RIDS) {                                                 // v_t in D(mu_i)
        const uint64_t w = B.filt[(size_t)p.pv * B.dw + (c >> 6)];
        if (!((w >> (c & 63)) & 1ull)) return false;
    }
    const bool chk = (B.flags & JOB_ELAB) != 0;
    if (chk && eidx >= 0) {                                                   // parent arc label
        const int l = (p.flags & POS_IN_ROW) ? __ldg(B.ielab + eidx) : __ldg(B.elab + eidx);
        if (l != p.pel) return false;
    }
    for (int b = 0; b < p.bc; ++b) {                                          // rule 4
        const BackEdge be = B.back[p.bb + b];
        const int x = M[be.pos];
        if (!DIR) {
            if (B.adj != nullptr && !chk) {
                const uint64_t w = __ldg(B.adj + (size_t)x * B.dw + (c >> 6));
                if (!((w >> (c & 63)) & 1ull)) return false;
            } else if (B.hub_slot != nullptr && !chk && __ldg(B.hub_slot + x) >= 0) {
                const uint64_t w = __ldg(B.hub_bits + (size_t)__ldg(B.hub_slot + x) * B.dw + (c >> 6));
                if (!((w >> (c & 63)) & 1ull)) return false;
            } else if (!row_has(B.rowptr, B.col, B.elab, x, c, be.lab_out, chk)) {
                return false;
            }
        } else {
            if ((be.dir & 1) && !row_has(B.irowptr, B.icol, B.ielab, x, c, be.lab_out, chk)) return false;
            if ((be.dir & 2) && !row_has(B.rowptr, B.col, B.elab, x, c, be.lab_in, chk)) return false;
        }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h)                                               // rule 1 (same-label positions)
        for (uint64_t m = B.pos[i].same[h]; m; m &= m - 1)
            if (M[64 * h + __ffsll((long long)m) - 1] == c) return false;
    return true;
}

template <bool DIR>
__global__ void __launch_bounds__(BLOCK) k_search_csr(const JobDesc *jobs, SearchCtl C, int kmax) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    unsigned char *base = smem + wib * csr_smem_per_warp(kmax);
    LvCsr *lv = reinterpret_cast<LvCsr *>(base);
    int *M = reinterpret_cast<int *>(lv + kmax);
    PosC *tab = reinterpret_cast<PosC *>(M + kmax);

    const unsigned long long deadline = C.deadline_ns ? globaltimer() + C.deadline_ns : 0ull;
    Frame fr;
    unsigned iter = 0, last_don_iter = 0;
    unsigned long long last_check = 0, last_don_ns = 0, last_cancel = 0;
    int cur_job = -1;
    CsrJob B;
    WarpClock::begin(C);
    if (threadIdx.x == 0) atomicMax(C.span, ~globaltimer());
    while (acquire_frame(C, M, fr, deadline)) {
        WarpClock::frame_in(C);
        const JobDesc &J = jobs[fr.job];
        if (fr.job != cur_job) {
            cur_job = fr.job;
            B.rowptr = J.t.rowptr; B.col = J.t.col; B.elab = J.t.elab;
            B.irowptr = J.t.irowptr; B.icol = J.t.icol; B.ielab = J.t.ielab; B.indeg = J.t.indeg;
            B.ulist = J.ulist; B.vld = J.t.vld; B.filt = J.filt; B.adj = J.t.adj; B.back = J.back; B.pos = J.pos;
            B.hub_slot = J.t.hub_slot; B.hub_bits = J.t.hub_bits;
            B.n = J.t.n; B.dw = J.t.dw; B.k = J.k; B.flags = J.flags;
            for (int t = lane; t < B.k; t += 32) {
                const PosInfo P = J.pos[t];
                PosC q;
                q.pv = (int16_t)P.pv; q.par = (int16_t)P.par; q.bb = (int16_t)P.bbeg; q.bc = (int16_t)P.bcnt;
                q.lab = P.lab; q.odeg = P.odeg; q.ideg = P.ideg; q.pel = P.pel; q.flags = P.flags;
                tab[t] = q;
            }
            __syncwarp();
        }
        const int k = B.k, d0 = fr.depth;
        // a counted frame re-tests its range at level d0 without counting it again
        const int quiet = fr.counted ? d0 : -1;
        unsigned long long st = 0, nd = 0, mt = 0, hs = 0;   // the frame's totals
        // since the last fold (every 64 iterations): an iteration adds at most 32 nodes and a
        // candidate list below 2^24 states (longer lists go straight to the 64-bit total)
        unsigned st32 = 0, nd32 = 0, mt32 = 0;
        // set up level `l` (positions 0..l-1 assigned)
        auto setup = [&](int l, int beg, int endv) {
            const PosC p = tab[l];
            int b0, len;
            if (p.par >= 0) {
                const int a = M[p.par];
                const int32_t *rp = (p.flags & POS_IN_ROW) ? B.irowptr : B.rowptr;
                b0 = __ldg(rp + a);
                len = __ldg(rp + a + 1) - b0;
            } else if (B.flags & JOB_RIDS) {
                const PosInfo &P = J.pos[l];
                b0 = P.uoff;
                len = P.ucnt;
            } else {
                b0 = 0;
                len = B.n;
            }
            int cur = 0, end = len;
            if (beg >= 0) { cur = beg; end = min(endv, len); }
            __syncwarp();
            if (lane == 0) {
                lv[l].base = b0; lv[l].cur = cur; lv[l].end = end; lv[l].mask = 0; lv[l].cbase = 0; lv[l].len = len;
            }
            __syncwarp();
        };
        // a node's states are counted when its candidate 0 is scanned, so every split of
        // its candidate range (range frames, donations, checkpoints) counts them exactly once
        setup(d0, fr.beg, fr.end);
        int lvl = d0;
        bool stopped = false;
        for (;;) {
            if (((++iter) & 63) == 0) {
                st += st32; nd += nd32; mt += mt32;
                st32 = nd32 = mt32 = 0;
            }
            if ((iter & 7) == 0 && time_to_check(last_check)) {
                if (C.budget > 0) {
                    st += st32;
                    st32 = 0;
                    if (lane == 0) atomicAdd(J.ctr + 1, st);
                    st = 0;
                }
                if (must_stop(C, J, st, deadline, last_check, last_cancel)) { stopped = true; break; }
                if ((iter - last_don_iter >= (unsigned)C.donate_iters || last_check - last_don_ns >= C.donate_ns) &&
                    donation_claim(C)) {
                    // donate the shallowest unexplored work: half of an unscanned
                    // range, else up to `gran` pending survivors as new search nodes
                    last_don_iter = iter;
                    last_don_ns = last_check;
                    for (int l = d0; l <= lvl && l + 1 + DONATE_MIN_LEVELS <= k; ++l) {
                        LvCsr &L = lv[l];
                        const int rem = L.end - L.cur;
                        if (rem >= 64) {
                            const int mid = L.cur + ((rem / 2 + 31) & ~31);
                            if (push_frame(C, fr.job, l | (l == quiet ? FRAME_COUNTED : 0), mid, L.end, M, l,
                                           -1)) {
                                __syncwarp();
                                if (lane == 0) L.end = mid;
                                __syncwarp();
                            }
                            break;
                        }
                        if (L.mask != 0) {
                            const int32_t *src = csr_src(B, tab[l]);
                            int given = 0;
                            while (L.mask != 0 && given < C.gran) {
                                const unsigned m = L.mask;
                                const int b = __ffs(m) - 1;
                                const int c = src ? __ldg(src + L.base + L.cbase + b) : L.cbase + b;
                                if (!push_frame(C, fr.job, l + 1, -1, -1, M, l, c)) break;
                                __syncwarp();
                                if (lane == 0) L.mask = m & (m - 1);
                                __syncwarp();
                                ++given;
                            }
                            break;
                        }
                    }
                    donation_done(C);
                }
            }
            LvCsr &L = lv[lvl];
            const unsigned mask = L.mask;
            const PosC p = tab[lvl];
            const int32_t *src = csr_src(B, p);
            if (mask == 0) {
                const int cur = L.cur, end = L.end;
                if (cur >= end) {
                    if (lvl == d0) break;
                    --lvl;
                    continue;
                }
                const int cnt = min(32, end - cur);
                if (cur == 0 && lvl != quiet) {
                    if (L.len < (1 << 24)) st32 += (unsigned)L.len;
                    else st += (unsigned long long)L.len;
                }
                bool ok = false;
                int c = -1;
                if (lane < cnt) {
                    const int e = L.base + cur + lane;
                    c = src ? __ldg(src + e) : cur + lane;
                    ok = csr_feasible<DIR>(B, p, lvl, c, (src && p.par >= 0) ? e : -1, M);
                }
                unsigned bal = __ballot_sync(FULL, ok);
                if (lvl != quiet) nd32 += __popc(bal);
                if (lvl == k - 1) {
                    mt32 += __popc(bal);
                    if (bal) {
                        // hash prefix sum_{t < lvl} g(mu_t, M_t), only when this chunk has matches
                        unsigned long long ps = 0;
                        for (int t = lane; t < lvl; t += 32) ps += gterm(tab[t].pv, M[t]);
                        ps = warp_sum(ps);
                        if (ok) {
                            hs += fmix64(ps + gterm(p.pv, c));
                            if (J.mbuf) emit_match(J, M, lvl, c);
                        }
                    }
                    bal = 0;
                }
                __syncwarp();
                if (lane == 0) { L.cur = cur + cnt; L.mask = bal; L.cbase = cur; }
                __syncwarp();
                continue;
            }
            // descend into the lowest pending survivor
            const int b = __ffs(mask) - 1;
            const int c = src ? __ldg(src + L.base + L.cbase + b) : L.cbase + b;
            __syncwarp();
            if (lane == 0) {
                L.mask = mask & (mask - 1);
                M[lvl] = c;
            }
            __syncwarp();
            ++lvl;
            setup(lvl, -1, 0);
        }
        if (stopped && C.ckpt != nullptr) {
            // checkpoint, per level: the part of the current chunk from its lowest pending
            // survivor on (already counted; survivors are taken lowest first), then the
            // unscanned rest of the range (counted only if the frame itself was)
            for (int l = d0; l <= lvl; ++l) {
                const LvCsr L = lv[l];
                const int cb = L.mask ? L.cbase + __ffs(L.mask) - 1 : L.cur;
                if (l == quiet) {
                    if (cb < L.end) ckpt_push(C, fr.job, l, true, cb, L.end, M);
                } else {
                    if (cb < L.cur) ckpt_push(C, fr.job, l, true, cb, L.cur, M);
                    if (L.cur < L.end) ckpt_push(C, fr.job, l, false, L.cur, L.end, M);
                }
            }
        }
        st += st32; nd += nd32; mt += mt32;
        hs = warp_sum(hs);
        if (lane == 0) {
            atomicAdd(J.ctr + 0, mt);
            atomicAdd(J.ctr + 1, st);
            atomicAdd(J.ctr + 2, nd);
            atomicAdd(J.ctr + 3, hs);
            if (!stopped) atomicSub(C.outstanding, 1);
        }
        __syncwarp();
        WarpClock::frame_out(C, fr, st, nd);
        if (stopped) break;
    }
    WarpClock::finish(C);
    if ((threadIdx.x & 31) == 0) atomicMax(C.span + 1, globaltimer());
}

// ================================================== search: bitset kernel
//
// Candidate set of position i as one AND over bitset rows (dense targets):
//   S_i = D(mu_i) & A[M(P(mu_i))] & AND_j A[M(mu_j)] & ~used
// where D is the domain (RI-DS) or the label/degree filter (RI), A the
// adjacency bitset and `used` the images M_0..M_{i-1} (rule 1).  Lane l owns
// words l, l + 32, ... (NWL per lane).
//
// Per warp, registers hold the used-vertex bitset (lane l: words l + 32 w) and
// shared memory holds M, a compact copy of the job's position table, and for
// every level a list of up to BitsLayout<KM>::LCAP pending survivors; a level with
// more survivors keeps its
// bitset in the warp's slab of global scratch (`SearchCtl::slab`) instead.

// Capacity of a level's survivor list in shared memory: 64 for patterns of up
// to 32 vertices (measured fastest on the dense workload), 16 beyond so that
// four blocks of eight warps still fit an SM.  (The length byte reserves 0xff.)
constexpr uint8_t LIST_SPILLED = 0xff;

// Pattern-size class of a bitset-kernel launch: its per-warp shared layout is
// fixed at compile time for patterns of at most KM vertices.
// (A smaller class keeps shared memory, and so the L1 left beside it for the adjacency rows,
// no larger than the patterns need: 24 vertices take 31 KB per block, 32 take 42 KB.)
__host__ __device__ constexpr int bits_km(int kmax) {
    return kmax <= 24 ? 24 : (kmax <= 32 ? 32 : (kmax <= 64 ? 64 : KMAX));
}

struct __align__(16) PosB {
    int16_t pv, par, bb, bc;  // pattern vertex, parent position, back edges [bb, bb + bc) other than
                              // one to position i - 1 (that one, if any, is stored right after them)
    int32_t ucnt;             // raw candidates of an unparented position
    int32_t abf;              // algorithmic bytes of one expansion (rows ANDed x dw x 8, low 28 bits),
                              // flags PREV_ADJ / PREV_PAR above them
};
constexpr int32_t PREV_ADJ = 1 << 28;   // mu_{i-1} is adjacent to mu_i (as parent or back edge)
constexpr int32_t PREV_PAR = 1 << 29;   // ... and is its parent
constexpr int32_t ABYTES_MASK = (1 << 28) - 1;

// Per-warp shared memory of the bitset kernel, at offsets fixed by KM: the
// position table (16-byte records), the frame's range (for checkpoints), M,
// the survivor lists and their lengths, and the back-edge positions.
template <int KM>
struct BitsLayout {
    static constexpr int LCAP = KM <= 32 ? 64 : 16;   // (KM 24 and 32: 64 entries)
    static constexpr size_t TAB = 0;
    static constexpr size_t FRANGE = TAB + (size_t)KM * 16;
    static constexpr size_t MOFF = FRANGE + 8;
    static constexpr size_t LST = MOFF + (size_t)KM * 4;
    static constexpr size_t LCNT = LST + (size_t)KM * LCAP * 2;
    static constexpr size_t TBACK = LCNT + (size_t)KM;
    static constexpr size_t BYTES = (TBACK + (size_t)KM * (KM - 1) / 2 + 16 + 15) & ~(size_t)15;
};

__host__ __device__ __forceinline__ size_t bits_smem_per_warp(int kmax, int nwl) {
    switch (bits_km(kmax)) {
        case 24: return BitsLayout<24>::BYTES;
        case 32: return BitsLayout<32>::BYTES;
        case 64: return BitsLayout<64>::BYTES;
        default: return BitsLayout<KMAX>::BYTES;
    }
}

__host__ __device__ __forceinline__ size_t bits_slab_words_per_warp(int kmax, int nwl) {
    return (size_t)bits_km(kmax) * nwl * 32;
}

struct BitsJob {
    const uint64_t *filt, *adj;
    const int2 *vld;
    int dw, k;
};

// One warp's state: its shared-memory block (offsets from BitsLayout<KM>) and
// its slab of global scratch (level bitsets of more survivors than a list holds).
template <int KM>
struct BitsWarp {
    using L = BitsLayout<KM>;
    static constexpr int LCAP = L::LCAP;
    unsigned char *base;
    uint64_t *slab;    // global: [KM][NWL * 32]
    // Level l's list length (LIST_SPILLED: its survivors are a slab bitset).  Patterns of up
    // to 32 vertices keep the lengths in a register, lane l holding level l's, so a pop
    // reads it with one shuffle and writes it with one select, no shared-memory store or
    // warp sync; larger ones keep them in shared memory.
    int lcr;
    __device__ __forceinline__ int lc(int l) const {
        if constexpr (KM <= 32) return __shfl_sync(FULL, lcr, l);
        else return lcnt()[l];
    }
    __device__ __forceinline__ void set_lc(int l, int v) {
        if constexpr (KM <= 32) {
            lcr = (threadIdx.x & 31) == l ? v : lcr;
        } else {
            __syncwarp();
            if ((threadIdx.x & 31) == 0) lcnt()[l] = (uint8_t)v;
            __syncwarp();
        }
    }
    __device__ __forceinline__ PosB *tab() const { return reinterpret_cast<PosB *>(base + L::TAB); }
    __device__ __forceinline__ int *frange() const { return reinterpret_cast<int *>(base + L::FRANGE); }
    __device__ __forceinline__ int *M() const { return reinterpret_cast<int *>(base + L::MOFF); }
    __device__ __forceinline__ uint16_t *lst() const { return reinterpret_cast<uint16_t *>(base + L::LST); }
    __device__ __forceinline__ uint8_t *lcnt() const { return base + L::LCNT; }
    __device__ __forceinline__ uint8_t *tback() const { return base + L::TBACK; }
};

template <int NWL>
__device__ __forceinline__ void used_flip(uint64_t (&used)[NWL], int v) {
    // lane (q mod 32) holds word q of the used bitset in register used[q / 32]
    const int q = v >> 6;
    if ((threadIdx.x & 31) == (q & 31)) {
        const uint64_t bit = 1ull << (v & 63);
        if (NWL == 1) {
            used[0] ^= bit;   // v < 64 * 32: q < 32
        } else {
#pragma unroll
            for (int w = 0; w < NWL; ++w)
                if (w == (q >> 5)) used[w] ^= bit;
        }
    }
}

// This lane's words of row x of the adjacency bitset, ANDed into s.
template <int NWL>
__device__ __forceinline__ void and_row(const uint64_t *adj, int dw, int x, uint64_t (&s)[NWL]) {
    const uint64_t *X = adj + (size_t)x * dw;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int w = 0; w < NWL; ++w) {
        const int q = lane + 32 * w;
        if (q < dw) s[w] &= __ldg(X + q);
    }
}

// The part of position i's candidate set that does not depend on M[i-1]:
//   P_i = D(mu_i) & A[M(P(mu_i))] (unless the parent is position i - 1)
//         & AND over the other back-neighbours j < i - 1 of A[M_j] & ~used
// (`used` = images of positions 0..i-2).  With `with_prev` the rows of
// position i - 1 are ANDed too (then `used` must hold M_{i-1} as well), which
// gives the whole candidate set S_i.  `len` receives the raw candidate count
// when it does not depend on M[i-1] (else 0).
template <int NWL, int KM>
__device__ __forceinline__ void bits_rows(const BitsJob &B, const BitsWarp<KM> &W, const PosB &p, int i, bool with_prev,
                                          const uint64_t (&used)[NWL], uint64_t (&s)[NWL], int &len) {
    const int lane = threadIdx.x & 31;
    const int dw = B.dw;
    const uint64_t *F = B.filt + (size_t)p.pv * dw;
    const int *M = W.M();
#pragma unroll
    for (int w = 0; w < NWL; ++w) {
        const int q = lane + 32 * w;
        s[w] = q < dw ? F[q] : 0ull;
    }
    len = p.ucnt;
    if (p.par >= 0) {
        if (with_prev || !(p.abf & PREV_PAR)) {
            const int a = M[p.par];
            and_row<NWL>(B.adj, dw, a, s);
            len = __ldg(B.vld + a).y;
        } else {
            len = 0;
        }
    }
#pragma unroll 2
    for (int b = 0; b < p.bc; ++b) and_row<NWL>(B.adj, dw, M[W.tback()[p.bb + b]], s);
    if (with_prev && (p.abf & PREV_ADJ) && !(p.abf & PREV_PAR)) and_row<NWL>(B.adj, dw, M[i - 1], s);
#pragma unroll
    for (int w = 0; w < NWL; ++w) s[w] &= ~used[w];
}

// Count the survivors of position i's candidate set s (the accepted nodes) and
// either hash them as matches (leaf) or keep them as level i's pending
// survivors: a short list in shared memory, else the bitset in the slab.
// With none, level i's list is left as it was: the caller does not descend.
// `st` and `ab` are 32-bit: one expansion adds at most n_t <= 8192 states and
// (k_max + 1) x 128 x 8 bytes, and the caller folds them into 64-bit totals
// every 64 expansions.  M[0..i-1] must be in shared memory when the set has
// matches (the hash and the match rows read them).
template <int NWL, int KM, bool RANGE = false>
__device__ __forceinline__ int bits_finish(const JobDesc &J, BitsWarp<KM> &W, uint64_t (&s)[NWL], int i, int pv,
                                           bool leaf, unsigned long long &hs, int vlo = 0, int vhi = 0x7fffffff) {
    const int lane = threadIdx.x & 31;
    int cnt = 0;
#pragma unroll
    for (int w = 0; w < NWL; ++w) {
        if (RANGE) {
            // a range frame: keep the candidates with vertex ids in [vlo, vhi]
            const int b0 = (lane + 32 * w) * 64;
            if (vhi < b0 || vlo > b0 + 63) {
                s[w] = 0;
            } else {
                const int lo = vlo > b0 ? vlo - b0 : 0, hi = vhi < b0 + 63 ? vhi - b0 : 63;
                s[w] &= (~0ull << lo) & (~0ull >> (63 - hi));
            }
        }
        cnt += __popcll(s[w]);
    }
    const int total = __reduce_add_sync(FULL, (unsigned)cnt);
    if (total == 0) return 0;
    if (leaf) {
        // hash prefix sum_{t < i} g(mu_t, M_t), computed only when matches exist
        const int *M = W.M();
        unsigned long long ps = 0;
        for (int t = lane; t < i; t += 32) ps += gterm(W.tab()[t].pv, M[t]);
        ps = warp_sum(ps);
#pragma unroll
        for (int w = 0; w < NWL; ++w) {
            const int q = lane + 32 * w;
            uint64_t y = s[w];
            while (y) {
                const int bit = __ffsll((long long)y) - 1;
                const int vtx = q * 64 + bit;
                hs += fmix64(ps + gterm(pv, vtx));
                if (J.mbuf) emit_match(J, M, i, vtx);
                y &= y - 1;
            }
        }
        return total;
    }
    if (total <= W.LCAP) {
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += y;
        }
        uint16_t *L = W.lst() + i * W.LCAP;
        int o = incl - cnt;
#pragma unroll
        for (int w = 0; w < NWL; ++w) {
            const int q = lane + 32 * w;
            uint64_t y = s[w];
            while (y) {
                L[o++] = (uint16_t)(q * 64 + __ffsll((long long)y) - 1);
                y &= y - 1;
            }
        }
        __syncwarp();
        W.set_lc(i, total);
    } else {
        uint64_t *Sl = W.slab + (size_t)i * NWL * 32;
#pragma unroll
        for (int w = 0; w < NWL; ++w) Sl[w * 32 + lane] = s[w];
        __syncwarp();
        W.set_lc(i, LIST_SPILLED);
    }
    return total;
}

// Next pending survivor of level l (warp-uniform, -1 if none); removes it.
template <int NWL, int KM>
__device__ __forceinline__ int bits_next(BitsWarp<KM> &W, int l) {
    const int lane = threadIdx.x & 31;
    const int c = W.lc(l);
    if (c != LIST_SPILLED) {
        if (c == 0) return -1;
        const int v = W.lst()[l * W.LCAP + c - 1];
        W.set_lc(l, c - 1);
        return v;
    }
    uint64_t *S = W.slab + (size_t)l * NWL * 32;
#pragma unroll
    for (int w = 0; w < NWL; ++w) {
        const uint64_t m = S[w * 32 + lane];
        const unsigned bal = __ballot_sync(FULL, m != 0);
        if (bal) {
            const int L = __ffs(bal) - 1;
            const uint64_t mw = __shfl_sync(FULL, m, L);
            const int bit = __ffsll((long long)mw) - 1;
            __syncwarp();
            if (lane == L) S[w * 32 + lane] = mw & (mw - 1);
            __syncwarp();
            return ((L + 32 * w) << 6) + bit;
        }
    }
    return -1;
}

// Put a survivor back at level l (the donation queue was full).
template <int NWL, int KM>
__device__ __forceinline__ void bits_unnext(BitsWarp<KM> &W, int l, int v) {
    const int lane = threadIdx.x & 31;
    const int c = W.lc(l);
    __syncwarp();
    if (c != LIST_SPILLED) {
        if (lane == 0) W.lst()[l * W.LCAP + c] = (uint16_t)v;
        __syncwarp();
        W.set_lc(l, c + 1);
    } else {
        const int q = v >> 6;
        if (lane == (q & 31)) W.slab[(size_t)l * NWL * 32 + (q >> 5) * 32 + lane] |= 1ull << (v & 63);
        __syncwarp();
    }
}

template <int NWL, int KM>
__global__ void __launch_bounds__(BLOCK, 4) k_search_bits(const JobDesc *jobs, SearchCtl C, int kmax) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    BitsWarp<KM> W;
    W.base = smem + wib * BitsLayout<KM>::BYTES;
    W.slab = C.slab + ((size_t)blockIdx.x * WARPS_PER_BLOCK + wib) * ((size_t)KM * NWL * 32);
    W.lcr = 0;
    int *M = W.M();
    uint64_t used[NWL];   // this lane's words of the used-vertex bitset (word lane + 32 w)

    const unsigned long long deadline = C.deadline_ns ? globaltimer() + C.deadline_ns : 0ull;
    Frame fr;
    unsigned iter = 0, last_don_iter = 0;
    unsigned long long last_check = 0, last_don_ns = 0, last_cancel = 0;
    int cur_job = -1;
    BitsJob B;
    WarpClock::begin(C);
    if (threadIdx.x == 0) atomicMax(C.span, ~globaltimer());
    while (acquire_frame(C, M, fr, deadline)) {
        WarpClock::frame_in(C);
        const JobDesc &J = jobs[fr.job];
        if (fr.job != cur_job) {
            // cache the job's pointers in registers and its position table in shared memory
            cur_job = fr.job;
            B.filt = J.filt; B.adj = J.t.adj; B.vld = J.t.vld; B.dw = J.t.dw; B.k = J.k;
            for (int t = lane; t < B.k; t += 32) {
                const PosInfo P = J.pos[t];
                PosB q;
                // back edges come in ascending position order, so one to position t - 1 is the last
                const bool prev_back = P.bcnt > 0 && J.back[P.bbeg + P.bcnt - 1].pos == t - 1;
                const bool prev_par = t > 0 && P.par == t - 1;
                q.pv = (int16_t)P.pv; q.par = (int16_t)P.par; q.bb = (int16_t)P.bbeg;
                q.bc = (int16_t)(P.bcnt - (prev_back ? 1 : 0));
                q.ucnt = (J.flags & JOB_RIDS) ? P.ucnt : J.t.n;   // RI: all of V_t
                q.abf = ((P.par >= 0 ? 2 : 1) + P.bcnt) * J.t.dw * 8 | (prev_back || prev_par ? PREV_ADJ : 0) |
                        (prev_par ? PREV_PAR : 0);
                W.tab()[t] = q;
            }
            __syncwarp();
            const int nb = J.pos[B.k - 1].bbeg + J.pos[B.k - 1].bcnt;
            for (int b = lane; b < nb; b += 32) W.tback()[b] = (uint8_t)J.back[b].pos;
            __syncwarp();
        }
        const int k = B.k, d0 = fr.depth;
        unsigned long long st = 0, nd = 0, mt = 0, hs = 0, ab = 0;   // the frame's totals
        unsigned st32 = 0, nd32 = 0, mt32 = 0, ab32 = 0;               // since the last fold
        {
#pragma unroll
            for (int w = 0; w < NWL; ++w) used[w] = 0ull;
            __syncwarp();
            for (int t = 0; t < d0; ++t) used_flip<NWL>(used, M[t]);
            if (lane == 0) M[d0] = -1;
            __syncwarp();
        }
        bool stopped = false;
        // a range frame covers candidates [beg, end) of its node: as the candidate
        // lists are ascending, that is the vertex-id interval [first, last]
        int vlo = 0, vhi = 0x7fffffff;
        if (fr.beg >= 0) {
            const PosB p = W.tab()[d0];
            const int32_t *lst = nullptr;
            int b0 = 0, len = 0;
            if (p.par >= 0) {
                const int a = M[p.par];
                lst = J.t.col;
                b0 = __ldg(J.t.rowptr + a);
                len = __ldg(J.t.rowptr + a + 1) - b0;
            } else if (J.flags & JOB_RIDS) {
                lst = J.ulist;
                b0 = J.pos[d0].uoff;
                len = J.pos[d0].ucnt;
            } else {
                len = J.t.n;
            }
            const int e = min(fr.end, len);
            if (fr.beg >= e) { vlo = 1; vhi = 0; }
            else if (lst) { vlo = __ldg(lst + b0 + fr.beg); vhi = __ldg(lst + b0 + e - 1); }
            else { vlo = fr.beg; vhi = e - 1; }
        }
        if (lane == 0) { W.frange()[0] = fr.beg; W.frange()[1] = fr.end; }   // read back only by a checkpoint
        const bool count_len = fr.beg <= 0 && !fr.counted;
        const bool leaf0 = d0 == k - 1;
        int c0;
        {
            // the frame's first expansion: position d0 with M[0..d0-1] given and all in `used`
            const PosB p = W.tab()[d0];
            uint64_t s[NWL];
            int len;
            bits_rows<NWL, KM>(B, W, p, d0, true, used, s, len);
            if (count_len) st32 += (unsigned)len;
            ab32 += (unsigned)(p.abf & ABYTES_MASK);
            c0 = fr.beg >= 0 ? bits_finish<NWL, KM, true>(J, W, s, d0, p.pv, leaf0, hs, vlo, vhi)
                             : bits_finish<NWL, KM>(J, W, s, d0, p.pv, leaf0, hs);
        }
        if (!fr.counted) nd += c0;
        if (leaf0) {
            mt += c0;
        } else if (c0 > 0) {
            // Levels d0..lvl hold pending survivors; `used` holds M_0..M_{lvl-1} (not the
            // choice at lvl).  Pv is the part of position lvl + 1's candidate set that does
            // not depend on M[lvl] (see bits_rows), valid while `pok`: consecutive siblings
            // at one level share it, and a descent or ascent invalidates it.  An expansion
            // that finds no survivors does not descend, so a level's list is read only
            // after an expansion filled it.
            int lvl = d0;
            bool pok = false;
            uint64_t Pv[NWL];
            int plen = 0;
#pragma unroll
            for (int w = 0; w < NWL; ++w) Pv[w] = 0ull;
            for (;;) {
                if (((++iter) & 63) == 0) {
                  st += st32; nd += nd32; mt += mt32; ab += ab32;
                  st32 = nd32 = mt32 = ab32 = 0;
                  if (time_to_check(last_check)) {
                    if (C.budget > 0) {
                        if (lane == 0) atomicAdd(J.ctr + 1, st);
                        st = 0;
                    }
                    if (must_stop(C, J, st, deadline, last_check, last_cancel)) { stopped = true; break; }
                    if ((iter - last_don_iter >= (unsigned)C.donate_iters || last_check - last_don_ns >= C.donate_ns) &&
                        donation_claim(C)) {
                        // donate up to `gran` pending survivors of the shallowest level that has some
                        last_don_iter = iter;
                        last_don_ns = last_check;
                        const unsigned long long tdon = WarpClock::don_begin(C);
                        int given = 0;
                        for (int l = d0; l <= lvl && l + 1 + DONATE_MIN_LEVELS <= k; ++l) {
                            given = 0;
                            while (given < C.gran) {
                                const int v = bits_next<NWL, KM>(W, l);
                                if (v < 0) break;
                                if (!push_frame(C, fr.job, l + 1, -1, -1, M, l, v)) {
                                    bits_unnext<NWL, KM>(W, l, v);
                                    given = C.gran;
                                    break;
                                }
                                ++given;
                            }
                            if (given > 0) break;
                        }
                        WarpClock::don_end(C, tdon, given);
                        donation_done(C);
                    }
                  }
                }
                const int v = bits_next<NWL, KM>(W, lvl);
                if (v < 0) {
                    if (lvl == d0) break;
                    --lvl;
                    used_flip<NWL>(used, M[lvl]);   // the choice at the new current level leaves `used`
                    pok = false;
                    continue;
                }
                const int i = lvl + 1;
                const PosB p = W.tab()[i];
                if (!pok) {
                    bits_rows<NWL, KM>(B, W, p, i, false, used, Pv, plen);
                    pok = true;
                }
                uint64_t s[NWL];
#pragma unroll
                for (int w = 0; w < NWL; ++w) s[w] = Pv[w];
                int len = plen;
                if (p.abf & PREV_ADJ) {
                    and_row<NWL>(B.adj, B.dw, v, s);   // A[v] never holds v itself
                    if (p.abf & PREV_PAR) len = __ldg(B.vld + v).y;
                } else {
                    uint64_t nv[NWL];
#pragma unroll
                    for (int w = 0; w < NWL; ++w) nv[w] = ~0ull;
                    used_flip<NWL>(nv, v);
#pragma unroll
                    for (int w = 0; w < NWL; ++w) s[w] &= nv[w];
                }
                st32 += (unsigned)len;
                ab32 += (unsigned)(p.abf & ABYTES_MASK);
                const bool leaf = i == k - 1;
                if (leaf) {
                    // the match rows and the hash read M[0..i-1]: store the choice first when
                    // the set is not empty
                    int any = 0;
#pragma unroll
                    for (int w = 0; w < NWL; ++w) any |= s[w] != 0ull;
                    if (__any_sync(FULL, any)) {
                        if (lane == 0) M[lvl] = v;
                        __syncwarp();
                    }
                    const int c = bits_finish<NWL, KM>(J, W, s, i, p.pv, true, hs);
                    nd32 += c;
                    mt32 += c;
                } else {
                    const int c = bits_finish<NWL, KM>(J, W, s, i, p.pv, false, hs);
                    nd32 += c;
                    if (c > 0) {
                        if (lane == 0) M[lvl] = v;
                        __syncwarp();
                        used_flip<NWL>(used, v);
                        lvl = i;
                        pok = false;
                        continue;
                    }
                }
                // no descent: when that was the last survivor of its list, go up at once
                // (levels whose lists ran out) instead of finding out on the next iteration
                if (lvl > d0 && W.lc(lvl) == 0) {
                    do {
                        --lvl;
                        used_flip<NWL>(used, M[lvl]);
                    } while (lvl > d0 && W.lc(lvl) == 0);
                    pok = false;
                }
            }
            if (stopped && C.ckpt != nullptr) {
                // checkpoint: the pending survivors of each level as one counted range frame.
                // They are a contiguous run of the level's ascending survivors (a short list is
                // taken from its top, a spilled bitset from its lowest bit), so one index range
                // of the level's candidate list holds exactly them among the feasible candidates.
                for (int l = d0; l <= lvl; ++l) {
                    const PosB p = W.tab()[l];
                    const int32_t *lst = nullptr;
                    int len = J.t.n;
                    if (p.par >= 0) {
                        const int a = M[p.par];
                        const int b0 = __ldg(J.t.rowptr + a);
                        lst = J.t.col + b0;
                        len = __ldg(J.t.rowptr + a + 1) - b0;
                    } else if (J.flags & JOB_RIDS) {
                        lst = J.ulist + J.pos[l].uoff;
                        len = J.pos[l].ucnt;
                    }
                    int lo = 0, hi = len;   // the level's own range
                    if (l == d0 && W.frange()[0] >= 0) { lo = W.frange()[0]; hi = min(W.frange()[1], len); }
                    const int c = W.lc(l);
                    if (c == 0) continue;
                    if (c != LIST_SPILLED) {
                        const int vmax = W.lst()[l * W.LCAP + c - 1];
                        hi = lst ? lower_bound_warp(lst, len, vmax + 1) : vmax + 1;
                    } else {
                        const int vmin = bits_next<NWL, KM>(W, l);
                        if (vmin < 0) continue;
                        lo = lst ? lower_bound_warp(lst, len, vmin) : vmin;
                    }
                    if (lo < hi) ckpt_push(C, fr.job, l, true, lo, hi, M);
                }
            }
        }
        st += st32; nd += nd32; mt += mt32; ab += ab32;
        hs = warp_sum(hs);
        if (lane == 0) {
            atomicAdd(J.ctr + 0, mt);
            atomicAdd(J.ctr + 1, st);
            atomicAdd(J.ctr + 2, nd);
            atomicAdd(J.ctr + 3, hs);
            atomicAdd(J.abytes, ab);
            if (!stopped) atomicSub(C.outstanding, 1);
        }
        __syncwarp();
        WarpClock::frame_out(C, fr, st, nd);
        if (stopped) break;
    }
    WarpClock::finish(C);
    if ((threadIdx.x & 31) == 0) atomicMax(C.span + 1, globaltimer());
}

unsigned grid_for(long long warps) {
    long long blocks = (warps + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK;
    if (blocks < 1) blocks = 1;
    return (unsigned)blocks;
}

}  // namespace

// ================================================================ launchers

cudaError_t launch_domain_init_buckets(const JobDesc *jobs, const long long *vert_off, int njobs, long long nverts,
                                       cudaStream_t st) {
    if (nverts <= 0) return cudaSuccess;
    k_domain_init_buckets<<<grid_for(nverts), BLOCK, 0, st>>>(jobs, vert_off, njobs, nverts);
    return cudaGetLastError();
}

cudaError_t launch_label_index(const JobDesc *jobs, const long long *vert_off, int njobs, long long nverts,
                               cudaStream_t st) {
    if (nverts <= 0) return cudaSuccess;
    k_label_index<<<(unsigned)((nverts + BLOCK - 1) / BLOCK), BLOCK, 0, st>>>(jobs, vert_off, njobs, nverts);
    return cudaGetLastError();
}

cudaError_t launch_domain_init(const JobDesc *jobs, const long long *unit_off, int njobs, long long nunits,
                               cudaStream_t st) {
    if (nunits <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    // words per warp: up to 32 (a warp steps along its words reading each job's and vertex's
    // fields once), fewer when that would leave the device short of warps (64 per SM)
    const long long want = nunits / ((long long)sms * 64);
    const int wpw = (int)std::max<long long>(1, std::min<long long>(INIT_WORDS_PER_WARP, want));
    k_domain_init<<<grid_for((nunits + wpw - 1) / wpw), BLOCK, 0, st>>>(jobs, unit_off, njobs, nunits, wpw);
    return cudaGetLastError();
}

cudaError_t launch_domain_ac(const JobDesc *jobs, const int4 *ent, const long long *eoff, int nent, long long nunits,
                             int *changed, unsigned char *vchanged, cudaStream_t st) {
    if (nunits <= 0) return cudaSuccess;
    k_domain_ac<<<grid_for(nunits), BLOCK, 0, st>>>(jobs, ent, eoff, nent, nunits, changed, vchanged);
    return cudaGetLastError();
}

cudaError_t launch_domain_ac_cand(const JobDesc *jobs, const int4 *ent, const long long *eoff, int nent,
                                  long long ncand, int32_t *cand, int *changed, unsigned char *vchanged,
                                  cudaStream_t st) {
    if (ncand <= 0) return cudaSuccess;
    const long long blocks = (ncand + BLOCK - 1) / BLOCK;
    k_domain_ac_cand<<<(unsigned)blocks, BLOCK, 0, st>>>(jobs, ent, eoff, nent, ncand, cand, changed, vchanged);
    return cudaGetLastError();
}

cudaError_t launch_domain_fc(const JobDesc *jobs, const long long *vert_off, const long long *sizes, int njobs,
                             int *changed, unsigned char *vchanged, cudaStream_t st) {
    if (njobs <= 0) return cudaSuccess;
    k_domain_fc<<<njobs, BLOCK, 0, st>>>(jobs, vert_off, sizes, changed, vchanged);
    return cudaGetLastError();
}

cudaError_t launch_domain_fixpoint(const JobDesc *jobs, int njobs, const long long *vert_off, const long long *cstart,
                                   const long long *csize, int32_t *cand, int *next_job, cudaStream_t st) {
    if (njobs <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    // few pairs: one large block each, so that they still fill the device; many pairs:
    // blocks of four warps (eight pairs in flight per SM; 256 threads measured 3% slower and
    // 64 threads 15% slower on 196,000 molecule pairs), as many as are resident at once,
    // each taking pairs from the counter
    const int threads = njobs < sms * 4 ? FIXPOINT_BIG_BLOCK : FIXPOINT_SMALL_BLOCK;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_domain_fixpoint, threads, 0);
    if (e != cudaSuccess) return e;
    const long long wave = (long long)sms * std::max(occ, 1);
    const int grid = (int)std::min<long long>(njobs, wave);
    e = cudaMemsetAsync(next_job, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    k_domain_fixpoint<<<grid, threads, 0, st>>>(jobs, njobs, vert_off, cstart, csize, cand, next_job);
    return cudaGetLastError();
}

cudaError_t launch_domain_sizes(const JobDesc *jobs, const long long *vert_off, int njobs, long long nverts,
                                long long *sizes, cudaStream_t st) {
    if (nverts <= 0) return cudaSuccess;
    k_domain_sizes<<<grid_for(nverts), BLOCK, 0, st>>>(jobs, vert_off, njobs, nverts, sizes);
    return cudaGetLastError();
}

cudaError_t launch_domain_lists(const JobDesc *jobs, const int *task_job, const int *task_vert, const int *task_out,
                                int ntasks, int32_t *lists, cudaStream_t st) {
    if (ntasks <= 0) return cudaSuccess;
    k_domain_lists<<<ntasks, BLOCK, 0, st>>>(jobs, task_job, task_vert, task_out, lists);
    return cudaGetLastError();
}

cudaError_t launch_split(const JobDesc *jobs, const int32_t *fin, long long nf, int depth, int32_t *counts,
                         const long long *offs, int32_t *fout, int pass, int count_ctr, int directed,
                         cudaStream_t st) {
    if (nf <= 0) return cudaSuccess;
    long long warps = nf;
    if (warps > 152LL * 64) warps = 152LL * 64;
    if (directed)
        k_split<true><<<grid_for(warps), BLOCK, 0, st>>>(jobs, fin, nf, depth, counts, offs, fout, pass, count_ctr);
    else
        k_split<false><<<grid_for(warps), BLOCK, 0, st>>>(jobs, fin, nf, depth, counts, offs, fout, pass, count_ctr);
    return cudaGetLastError();
}

cudaError_t launch_split_coop(const JobDesc *jobs, long long f0, int32_t *buf0, int32_t *buf1, long long cap_ints,
                              long long target, int max_levels, long long *wtot, long long wtot_cap,
                              unsigned *bar, long long *result, int *status, int count_ctr, int directed,
                              int blocks_per_sm, uint32_t *masks, long long mask_total, int ordered,
                              long long *trace, cudaStream_t st) {
    SplitCtl S;
    S.trace = ordered ? nullptr : trace;
    S.buf0 = buf0; S.buf1 = buf1; S.cap_ints = cap_ints; S.target = target; S.max_levels = max_levels;
    S.wtot = wtot; S.bar = bar; S.result = result; S.status = status; S.count_ctr = count_ctr;
    S.masks = masks; S.mask_total = masks ? mask_total : 0;
    int dev = 0, sms = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    void *fn = ordered ? (directed ? (void *)k_split_coop<true> : (void *)k_split_coop<false>)
                       : (directed ? (void *)k_split_once<true> : (void *)k_split_once<false>);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, BLOCK, 0);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    if (blocks_per_sm > 0 && blocks_per_sm < occ) occ = blocks_per_sm;
    if ((long long)sms * occ * WARPS_PER_BLOCK > wtot_cap) occ = (int)(wtot_cap / ((long long)sms * WARPS_PER_BLOCK));
    if (occ < 1) return cudaErrorInvalidConfiguration;
    // all blocks must be co-resident for the grid barrier: a cooperative launch guarantees it
    dim3 grid(sms * occ), block(BLOCK);
    void *args[] = {(void *)&jobs, (void *)&f0, (void *)&S};
    return cudaLaunchCooperativeKernel(fn, grid, block, args, 0, st);
}

size_t scan_tmp_bytes(long long n) {
    const long long tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    return (size_t)(tiles + 1) * sizeof(long long);
}

cudaError_t launch_scan(const int32_t *in, long long *out, long long n, long long *total, void *tmp, size_t tmp_bytes,
                        cudaStream_t st) {
    const long long tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if ((size_t)(tiles + 1) * sizeof(long long) > tmp_bytes) return cudaErrorInvalidValue;
    long long *tile_sum = static_cast<long long *>(tmp);
    if (n <= 0) {
        return cudaMemsetAsync(total, 0, sizeof(long long), st);
    }
    k_scan_tiles<<<(unsigned)tiles, BLOCK, 0, st>>>(in, out, n, tile_sum);
    k_scan_sums<<<1, BLOCK, 0, st>>>(tile_sum, tiles, total);
    k_scan_add<<<(unsigned)tiles, BLOCK, 0, st>>>(out, n, tile_sum);
    return cudaGetLastError();
}

int search_warps_per_block() { return WARPS_PER_BLOCK; }

namespace {
// One block per hub: set the bit of every neighbour in the hub's row.
__global__ void k_build_hubs(const int32_t *rowptr, const int32_t *col, const int32_t *hubs, int dw, uint64_t *bits) {
    const int x = hubs[blockIdx.x];
    uint64_t *row = bits + (size_t)blockIdx.x * dw;
    for (int e = rowptr[x] + threadIdx.x; e < rowptr[x + 1]; e += blockDim.x) {
        const int y = col[e];
        atomicOr((unsigned long long *)(row + (y >> 6)), 1ull << (y & 63));
    }
}
}  // namespace

cudaError_t launch_build_hubs(const int32_t *rowptr, const int32_t *col, const int32_t *hubs, int h, int dw,
                              uint64_t *bits, cudaStream_t st) {
    if (h <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(bits, 0, (size_t)h * dw * sizeof(uint64_t), st);
    if (e != cudaSuccess) return e;
    k_build_hubs<<<h, BLOCK, 0, st>>>(rowptr, col, hubs, dw, bits);
    return cudaGetLastError();
}

namespace {
__global__ void k_pool_init(unsigned long long *seq, int cap) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += gridDim.x * blockDim.x)
        seq[i] = (unsigned long long)i;
}
}  // namespace

cudaError_t launch_pool_init(unsigned long long *seq, int cap, cudaStream_t st) {
    k_pool_init<<<(cap + BLOCK - 1) / BLOCK, BLOCK, 0, st>>>(seq, cap);
    return cudaGetLastError();
}

size_t search_smem_bytes(int kernel, int kmax, int nwl) {
    return WARPS_PER_BLOCK * (kernel == 2 ? bits_smem_per_warp(kmax, nwl) : csr_smem_per_warp(kmax));
}

size_t search_slab_bytes(int kernel, int kmax, int nwl, long long grid) {
    if (kernel != 2) return 0;
    return (size_t)grid * WARPS_PER_BLOCK * bits_slab_words_per_warp(kmax, nwl) * sizeof(uint64_t);
}

// Let kernel `kern` take `smem` bytes of dynamic shared memory.  The limit is
// a property of the kernel shared by every host thread that launches it, so
// it is always raised to the device maximum, never set to one launch's need:
// concurrent launches of different sizes (serving groups) cannot lower it
// under one another.
template <typename K>
static cudaError_t allow_dynamic_smem(K kern, size_t smem) {
    if (smem <= 48 * 1024) return cudaSuccess;
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    if ((long long)smem > optin) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
}

template <typename K>
static cudaError_t occupancy_of(K kern, size_t smem, int *occ) {
    cudaError_t e = allow_dynamic_smem(kern, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, kern, BLOCK, smem);
}

cudaError_t search_blocks_per_sm(int kernel, int kmax, int nwl, int directed, int *occ) {
    const size_t smem = search_smem_bytes(kernel, kmax, nwl);
    if (kernel == 2) {
        switch (nwl) {
            case 1:
                return kmax <= 24 ? occupancy_of(k_search_bits<1, 24>, smem, occ)
                       : kmax <= 32 ? occupancy_of(k_search_bits<1, 32>, smem, occ)
                       : kmax <= 64 ? occupancy_of(k_search_bits<1, 64>, smem, occ)
                                    : occupancy_of(k_search_bits<1, KMAX>, smem, occ);
            case 2:
                return kmax <= 24 ? occupancy_of(k_search_bits<2, 24>, smem, occ)
                       : kmax <= 32 ? occupancy_of(k_search_bits<2, 32>, smem, occ)
                       : kmax <= 64 ? occupancy_of(k_search_bits<2, 64>, smem, occ)
                                    : occupancy_of(k_search_bits<2, KMAX>, smem, occ);
            case 4:
                return kmax <= 24 ? occupancy_of(k_search_bits<4, 24>, smem, occ)
                       : kmax <= 32 ? occupancy_of(k_search_bits<4, 32>, smem, occ)
                       : kmax <= 64 ? occupancy_of(k_search_bits<4, 64>, smem, occ)
                                    : occupancy_of(k_search_bits<4, KMAX>, smem, occ);
            default: return cudaErrorInvalidValue;
        }
    }
    if (directed) return occupancy_of(k_search_csr<true>, smem, occ);
    return occupancy_of(k_search_csr<false>, smem, occ);
}

template <typename K>
static cudaError_t launch_persistent(K kern, const JobDesc *jobs, const SearchCtl &ctl, int kmax, size_t smem,
                                     int blocks_per_sm, long long max_grid, int *grid_out, cudaStream_t st) {
    int dev = 0, sms = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = allow_dynamic_smem(kern, smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, BLOCK, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    int per_sm = (blocks_per_sm > 0 && blocks_per_sm < occ) ? blocks_per_sm : occ;
    long long g = (long long)sms * per_sm;
    if (max_grid > 0 && g > max_grid) g = max_grid;   // never more blocks than the scratch slab covers
    const int grid = (int)g;
    if (grid_out) *grid_out = grid;
    kern<<<grid, BLOCK, smem, st>>>(jobs, ctl, kmax);
    return cudaGetLastError();
}

cudaError_t launch_search(int kernel, const JobDesc *jobs, const SearchCtl &ctl, int kmax, int nwl, int directed,
                          int blocks_per_sm, long long max_grid, int *grid_out, cudaStream_t st) {
    const size_t smem = search_smem_bytes(kernel, kmax, nwl);
    if (kernel == 2) {
        switch (nwl) {
            case 1:
                return kmax <= 24 ? launch_persistent(k_search_bits<1, 24>, jobs, ctl, kmax, smem, blocks_per_sm,
                                                      max_grid, grid_out, st)
                       : kmax <= 32 ? launch_persistent(k_search_bits<1, 32>, jobs, ctl, kmax, smem, blocks_per_sm,
                                                      max_grid, grid_out, st)
                       : kmax <= 64 ? launch_persistent(k_search_bits<1, 64>, jobs, ctl, kmax, smem, blocks_per_sm,
                                                        max_grid, grid_out, st)
                                    : launch_persistent(k_search_bits<1, KMAX>, jobs, ctl, kmax, smem, blocks_per_sm,
                                                        max_grid, grid_out, st);
            case 2:
                return kmax <= 24 ? launch_persistent(k_search_bits<2, 24>, jobs, ctl, kmax, smem, blocks_per_sm,
                                                      max_grid, grid_out, st)
                       : kmax <= 32 ? launch_persistent(k_search_bits<2, 32>, jobs, ctl, kmax, smem, blocks_per_sm,
                                                      max_grid, grid_out, st)
                       : kmax <= 64 ? launch_persistent(k_search_bits<2, 64>, jobs, ctl, kmax, smem, blocks_per_sm,
                                                        max_grid, grid_out, st)
                                    : launch_persistent(k_search_bits<2, KMAX>, jobs, ctl, kmax, smem, blocks_per_sm,
                                                        max_grid, grid_out, st);
            case 4:
                return kmax <= 24 ? launch_persistent(k_search_bits<4, 24>, jobs, ctl, kmax, smem, blocks_per_sm,
                                                      max_grid, grid_out, st)
                       : kmax <= 32 ? launch_persistent(k_search_bits<4, 32>, jobs, ctl, kmax, smem, blocks_per_sm,
                                                      max_grid, grid_out, st)
                       : kmax <= 64 ? launch_persistent(k_search_bits<4, 64>, jobs, ctl, kmax, smem, blocks_per_sm,
                                                        max_grid, grid_out, st)
                                    : launch_persistent(k_search_bits<4, KMAX>, jobs, ctl, kmax, smem, blocks_per_sm,
                                                        max_grid, grid_out, st);
            default: return cudaErrorInvalidValue;
        }
    }
    if (directed) return launch_persistent(k_search_csr<true>, jobs, ctl, kmax, smem, blocks_per_sm, max_grid, grid_out, st);
    return launch_persistent(k_search_csr<false>, jobs, ctl, kmax, smem, blocks_per_sm, max_grid, grid_out, st);
}

}  // namespace sge
