// sge_noalloc.cu -- fixed device scratch for sge_count_noalloc() and the
// small kernel that fills part of it.
//
// Some callers cannot allocate device memory while they search: code that
// runs under a memory manager that owns every device allocation, a process
// whose allocator is locked down or already at its limit, or a runtime that
// forbids cudaMalloc/cudaFree on its threads.  sge_count_noalloc() serves
// them: everything its persistent search needs beyond the caller's inputs
// and output (job record, counters, position tables, root frame, work queue,
// per-vertex label/degree records) is carved out of the one array below
// (16 MiB), which lives in the library's own device memory on every GPU that
// loads the library, until the process exits.  No call allocates or frees
// device memory.
#include "sge_internal.h"

#include <mutex>

namespace sge {

constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)16 << 20;   // 16 MiB, fixed

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Device address and size of the scratch array on the current device.  In
// host code the array's name is only a host-side stand-in, so the address is
// taken once per device with cudaGetSymbolAddress (with that device
// current) and cached.
cudaError_t noalloc_scratch(void **ptr, size_t *bytes) {
    constexpr int MAX_DEVICES = 64;
    static std::mutex mu;
    static void *addr[MAX_DEVICES] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(mu);
    if (addr[dev] == nullptr) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        addr[dev] = p;
    }
    *ptr = addr[dev];
    *bytes = NOALLOC_SCRATCH_BYTES;
    return cudaSuccess;
}

namespace {
// {label, degree} record of every target vertex, from the caller's CSR.
__global__ void k_make_vld(const int32_t *rowptr, const int32_t *vlabel, int2 *vld, int n) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        vld[v] = make_int2(vlabel[v], rowptr[v + 1] - rowptr[v]);
}
}  // namespace

cudaError_t launch_make_vld(const int32_t *rowptr, const int32_t *vlabel, int2 *vld, int n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int blocks = (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096;
    k_make_vld<<<blocks, 256, 0, st>>>(rowptr, vlabel, vld, n);
    return cudaGetLastError();
}

}  // namespace sge
