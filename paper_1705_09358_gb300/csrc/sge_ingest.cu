// sge_ingest.cu -- target ingest on the device.
//
// The caller's edge list (Section 2.1: labelled vertices, optional edge
// labels, an undirected edge stored in both directions) becomes the engine's
// CSR -- every row sorted by neighbour id and free of repeats -- after one
// upload of the raw arrays: count the arcs of each row, scan, scatter, sort
// and merge each row, compact.  Repeated edges with equal labels merge; a
// repeated edge with another label, a self-loop or an endpoint outside
// [0, n) set an error bit that the host turns into SGE_ERR_ARG.
#include "sge_internal.h"

#include <algorithm>

namespace sge {
namespace {

constexpr int IB = 256;                       // threads per block
constexpr unsigned FULLMASK = 0xffffffffu;
constexpr uint64_t PAD = ~0ull;               // sorts after every arc key
constexpr int LONG_SMEM_KEYS = 4096;          // a long row up to this length is ranked in shared memory

// An arc of a row as one sortable key: neighbour id above, label below.
__device__ __forceinline__ uint64_t arc_key(int v, int lab) {
    return ((uint64_t)(uint32_t)v << 32) | (uint32_t)lab;
}

unsigned blocks_for(long long items, long long per_block) {
    const long long b = (items + per_block - 1) / per_block;
    return (unsigned)std::min<long long>(std::max<long long>(b, 1), 1 << 16);   // grid-stride beyond
}

__device__ __forceinline__ void flag_warp(int *flags, int f) {
    f = (int)__reduce_or_sync(FULLMASK, (unsigned)f);
    if ((threadIdx.x & 31) == 0 && f) atomicOr(flags, f);
}

// 1. Validate every edge and count the arcs of each row (out-rows; in-rows
//    of a directed graph in cnt_in).
__global__ void __launch_bounds__(IB) k_ing_count(const int32_t *src, const int32_t *dst, const int32_t *elab,
                                                  long long m, int n, int directed, int32_t *cnt_out,
                                                  int32_t *cnt_in, int *flags) {
    int f = 0;
    for (long long e = blockIdx.x * (long long)IB + threadIdx.x; e < m; e += (long long)gridDim.x * IB) {
        const int a = src[e], b = dst[e];
        if (a < 0 || a >= n || b < 0 || b >= n) { f |= ING_RANGE; continue; }
        if (a == b) { f |= ING_LOOP; continue; }
        if (elab != nullptr && elab[e] != 0) f |= ING_ELAB;
        atomicAdd(cnt_out + a, 1);
        atomicAdd((directed ? cnt_in : cnt_out) + b, 1);
    }
    flag_warp(flags, f);
}

// 2. Scatter the arcs into their rows (unordered within a row).
__global__ void __launch_bounds__(IB) k_ing_scatter(const int32_t *src, const int32_t *dst, const int32_t *elab,
                                                    long long m, int n, int directed, const long long *off_out,
                                                    const long long *off_in, int32_t *fill_out, int32_t *fill_in,
                                                    uint64_t *key_out, uint64_t *key_in) {
    for (long long e = blockIdx.x * (long long)IB + threadIdx.x; e < m; e += (long long)gridDim.x * IB) {
        const int a = src[e], b = dst[e];
        if (a < 0 || a >= n || b < 0 || b >= n || a == b) continue;
        const int l = elab != nullptr ? elab[e] : 0;
        key_out[off_out[a] + atomicAdd(fill_out + a, 1)] = arc_key(b, l);
        if (directed) key_in[off_in[b] + atomicAdd(fill_in + b, 1)] = arc_key(a, l);
        else key_out[off_out[b] + atomicAdd(fill_out + b, 1)] = arc_key(a, l);
    }
}

// 3a. Rows of at most 32 arcs: one warp per row sorts them with a bitonic
//     network across its lanes, merges repeats and writes the row back
//     compacted; longer rows are listed for 3b.
__global__ void __launch_bounds__(IB) k_ing_rows_short(const long long *off, int n, uint64_t *keys, int32_t *ucnt,
                                                       int32_t *long_rows, int32_t *nlong, int *flags) {
    const int lane = threadIdx.x & 31;
    const long long w0 = (blockIdx.x * (long long)IB + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * IB) >> 5;
    int f = 0;
    for (long long v = w0; v < n; v += nw) {
        const long long b = off[v], len = off[v + 1] - b;
        if (len > 32) {
            if (lane == 0) long_rows[atomicAdd(nlong, 1)] = (int32_t)v;
            continue;
        }
        uint64_t x = lane < len ? keys[b + lane] : PAD;
        for (int k = 2; k <= 32; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                const uint64_t y = __shfl_xor_sync(FULLMASK, x, j);
                const bool keep_min = ((lane & k) == 0) == ((lane & j) == 0);
                x = keep_min ? (x < y ? x : y) : (x < y ? y : x);
            }
        const uint64_t prev = __shfl_up_sync(FULLMASK, x, 1);
        const bool real = x != PAD;
        const bool dup = real && lane > 0 && (prev >> 32) == (x >> 32);
        if (dup && prev != x) f |= ING_LABEL;   // the same neighbour twice, with two labels
        const unsigned keep = __ballot_sync(FULLMASK, real && !dup);
        if (real && !dup) keys[b + __popc(keep & ((1u << lane) - 1u))] = x;
        if (lane == 0) ucnt[v] = __popc(keep);
    }
    flag_warp(flags, f);
}

// Exclusive scan of one int per thread across the block; *total gets the sum.
__device__ int block_scan_excl(int x, int *total) {
    __shared__ int warp_sums[IB / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULLMASK, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_sums[wid] = incl;
    __syncthreads();
    int base = 0, tot = 0;
    for (int w = 0; w < IB / 32; ++w) {
        if (w < wid) base += warp_sums[w];
        tot += warp_sums[w];
    }
    __syncthreads();
    *total = tot;
    return base + incl - x;
}

// 3b. Longer rows: one block per row ranks every arc (its position is the
//     number of smaller keys plus the number of equal keys before it, so the
//     order is total and stable), then merges repeats and compacts.
__global__ void __launch_bounds__(IB) k_ing_rows_long(const long long *off, uint64_t *keys, uint64_t *scratch,
                                                      const int32_t *long_rows, const int32_t *nlong, int32_t *ucnt,
                                                      int *flags) {
    __shared__ uint64_t sk[LONG_SMEM_KEYS];
    const int nl = *nlong;
    int f = 0;
    for (int r = blockIdx.x; r < nl; r += gridDim.x) {
        const int v = long_rows[r];
        const long long b = off[v], len = off[v + 1] - b;
        const bool in_smem = len <= LONG_SMEM_KEYS;
        if (in_smem)
            for (long long i = threadIdx.x; i < len; i += IB) sk[i] = keys[b + i];
        __syncthreads();
        const uint64_t *row = in_smem ? sk : keys + b;
        for (long long i = threadIdx.x; i < len; i += IB) {
            const uint64_t x = row[i];
            long long rank = 0;
            for (long long j = 0; j < len; ++j) {
                const uint64_t y = row[j];
                rank += (y < x) || (y == x && j < i);
            }
            scratch[b + rank] = x;
        }
        __syncthreads();
        long long out = 0;
        for (long long c = 0; c < len; c += IB) {
            const long long i = c + threadIdx.x;
            uint64_t x = 0;
            int keep = 0;
            if (i < len) {
                x = scratch[b + i];
                const bool dup = i > 0 && (scratch[b + i - 1] >> 32) == (x >> 32);
                if (dup && scratch[b + i - 1] != x) f |= ING_LABEL;
                keep = !dup;
            }
            int tot = 0;
            const int pos = block_scan_excl(keep, &tot);
            if (keep) keys[b + out + pos] = x;
            out += tot;
        }
        if (threadIdx.x == 0) ucnt[v] = (int32_t)out;
        __syncthreads();
    }
    flag_warp(flags, f);
}

// 4. Compact the merged rows into the final CSR (one warp per row).
__global__ void __launch_bounds__(IB) k_ing_compact(const long long *off, const long long *uoff, const int32_t *ucnt,
                                                    const long long *utotal, const uint64_t *keys, int n,
                                                    int32_t *rowptr, int32_t *col, int32_t *lab) {
    const int lane = threadIdx.x & 31;
    const long long w0 = (blockIdx.x * (long long)IB + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * IB) >> 5;
    for (long long v = w0; v < n; v += nw) {
        const long long b = off[v], o = uoff[v];
        const int c = ucnt[v];
        for (int i = lane; i < c; i += 32) {
            const uint64_t x = keys[b + i];
            col[o + i] = (int32_t)(x >> 32);
            lab[o + i] = (int32_t)(uint32_t)x;
        }
        if (lane == 0) rowptr[v] = (int32_t)o;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) rowptr[n] = (int32_t)*utotal;
}

// Degree of every vertex from a CSR offset array.
__global__ void __launch_bounds__(IB) k_ing_degree(const int32_t *rowptr, int n, int32_t *deg) {
    for (long long v = blockIdx.x * (long long)IB + threadIdx.x; v < n; v += (long long)gridDim.x * IB)
        deg[v] = rowptr[v + 1] - rowptr[v];
}

// The longest row, folded into *maxdeg with one atomicMax per warp.
__global__ void __launch_bounds__(IB) k_ing_maxdeg(const int32_t *rowptr, int n, int32_t *maxdeg) {
    int m = 0;
    for (long long v = blockIdx.x * (long long)IB + threadIdx.x; v < n; v += (long long)gridDim.x * IB)
        m = max(m, rowptr[v + 1] - rowptr[v]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(maxdeg, m);
}

// Adjacency bitset rows (undirected, n <= the bitset limit): one warp per row.
__global__ void __launch_bounds__(IB) k_ing_bits(const int32_t *rowptr, const int32_t *col, int n, int dw,
                                                 uint64_t *bits) {
    const int lane = threadIdx.x & 31;
    const long long w0 = (blockIdx.x * (long long)IB + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * IB) >> 5;
    for (long long v = w0; v < n; v += nw)
        for (int e = rowptr[v] + lane; e < rowptr[v + 1]; e += 32) {
            const int w = col[e];
            atomicOr(reinterpret_cast<unsigned long long *>(bits + (size_t)v * dw + (w >> 6)), 1ull << (w & 63));
        }
}

// Largest neighbour degree per (label, vertex), label-major so that a warp reading consecutive
// vertices of one label reads consecutive words: one warp per vertex, lanes over its row.
__global__ void __launch_bounds__(IB) k_label_nbmax(const int32_t *rowptr, const int32_t *col, const int2 *vld,
                                                    const int32_t *lidx, int n, int nlab, int32_t *nbmax) {
    const int lane = threadIdx.x & 31;
    const long long w0 = (blockIdx.x * (long long)IB + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * IB) >> 5;
    for (long long v = w0; v < n; v += nw)
        for (int e = rowptr[v] + lane; e < rowptr[v + 1]; e += 32) {
            const int y = col[e];
            atomicMax(nbmax + (size_t)lidx[y] * n + v, vld[y].y);
        }
}

// Label-degree masks: one warp per (label index, degree threshold, 64-vertex word), two
// ballots over the word's vertices.
__global__ void __launch_bounds__(IB) k_label_degree_masks(const int2 *vld, int n, const int32_t *labs, long long units,
                                                           int dw, uint64_t *ldm) {
    const int lane = threadIdx.x & 31;
    const long long u = (blockIdx.x * (long long)IB + threadIdx.x) >> 5;
    if (u >= units) return;
    const int q = (int)(u % dw);
    const long long ld = u / dw;
    const int d = (int)(ld % LDM_DEGREES), l = (int)(ld / LDM_DEGREES);
    const int lab = labs[l];
    unsigned long long word = 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int t = q * 64 + h * 32 + lane;
        bool ok = false;
        if (t < n) {
            const int2 x = vld[t];
            ok = x.x == lab && x.y >= d;
        }
        word |= (unsigned long long)__ballot_sync(0xffffffffu, ok) << (32 * h);
    }
    if (lane == 0) ldm[u] = word;
}

}  // namespace

cudaError_t launch_label_degree_masks(const int2 *vld, int n, const int32_t *labs, int nlab, int dw, uint64_t *ldm,
                                      cudaStream_t st) {
    const long long units = (long long)nlab * LDM_DEGREES * dw;
    if (units <= 0) return cudaSuccess;
    k_label_degree_masks<<<blocks_for(units * 32, IB), IB, 0, st>>>(vld, n, labs, units, dw, ldm);
    return cudaGetLastError();
}

cudaError_t launch_label_nbmax(const int32_t *rowptr, const int32_t *col, const int2 *vld, const int32_t *lidx, int n,
                               int nlab, int32_t *nbmax, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(nbmax, 0, (size_t)n * nlab * sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    k_label_nbmax<<<blocks_for((long long)n * 32, IB), IB, 0, st>>>(rowptr, col, vld, lidx, n, nlab, nbmax);
    return cudaGetLastError();
}

cudaError_t launch_ingest_count(const int32_t *src, const int32_t *dst, const int32_t *elab, long long m, int n,
                                int directed, int32_t *cnt_out, int32_t *cnt_in, int *flags, cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    k_ing_count<<<blocks_for(m, IB), IB, 0, st>>>(src, dst, elab, m, n, directed, cnt_out, cnt_in, flags);
    return cudaGetLastError();
}

cudaError_t launch_ingest_scatter(const int32_t *src, const int32_t *dst, const int32_t *elab, long long m, int n,
                                  int directed, const long long *off_out, const long long *off_in, int32_t *fill_out,
                                  int32_t *fill_in, uint64_t *key_out, uint64_t *key_in, cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    k_ing_scatter<<<blocks_for(m, IB), IB, 0, st>>>(src, dst, elab, m, n, directed, off_out, off_in, fill_out,
                                                   fill_in, key_out, key_in);
    return cudaGetLastError();
}

cudaError_t launch_ingest_rows(const long long *off, int n, uint64_t *keys, uint64_t *scratch, int32_t *ucnt,
                               int32_t *long_rows, int32_t *nlong, int *flags, int sms, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_ing_rows_short<<<blocks_for((long long)n * 32, IB), IB, 0, st>>>(off, n, keys, ucnt, long_rows, nlong, flags);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_ing_rows_long<<<(unsigned)std::max(1, sms * 4), IB, 0, st>>>(off, keys, scratch, long_rows, nlong, ucnt, flags);
    return cudaGetLastError();
}

cudaError_t launch_ingest_compact(const long long *off, const long long *uoff, const int32_t *ucnt,
                                  const long long *utotal, const uint64_t *keys, int n, int32_t *rowptr, int32_t *col,
                                  int32_t *lab, cudaStream_t st) {
    k_ing_compact<<<blocks_for((long long)std::max(n, 1) * 32, IB), IB, 0, st>>>(off, uoff, ucnt, utotal, keys, n,
                                                                                rowptr, col, lab);
    return cudaGetLastError();
}

cudaError_t launch_ingest_degree(const int32_t *rowptr, int n, int32_t *deg, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_ing_degree<<<blocks_for(n, IB), IB, 0, st>>>(rowptr, n, deg);
    return cudaGetLastError();
}

cudaError_t launch_ingest_maxdeg(const int32_t *rowptr, int n, int32_t *maxdeg, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_ing_maxdeg<<<blocks_for(n, IB), IB, 0, st>>>(rowptr, n, maxdeg);
    return cudaGetLastError();
}

cudaError_t launch_ingest_bits(const int32_t *rowptr, const int32_t *col, int n, int dw, uint64_t *bits,
                               cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_ing_bits<<<blocks_for((long long)n * 32, IB), IB, 0, st>>>(rowptr, col, n, dw, bits);
    return cudaGetLastError();
}

}  // namespace sge
