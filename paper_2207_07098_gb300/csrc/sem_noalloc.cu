// Unique-node inner product that allocates nothing (sem_dot_noalloc).
//
// Some callers cannot call cudaMalloc when they need the inner product: code
// that is recording a CUDA graph by stream capture (allocation is refused
// while a capture is active), applications whose device memory is reserved
// up front by their own pool allocator (an allocation outside the pool may
// fail or fragment it), and latency-critical loops (cudaMalloc and cudaFree
// can synchronise the device).  This entry point keeps its scratch -- one
// FP64 partial sum per CTA plus a ticket counter -- in the file-scope device
// array below instead of memory owned by the handle or allocated per call.
//
// The array is part of the library image: every GPU that loads libsem holds
// it (kNoAllocPartials * 8 + 256 bytes) until the process exits.  All calls
// share it and it keeps the previous call's contents, so each call clears the
// counter first, and calls that overlap on the GPU (e.g. on two streams
// without ordering between them) race on it and give wrong results.
#include <mutex>

#include "sem_device.cuh"
#include "sem_internal.h"

namespace sem {

// Each CTA reduces one fixed chunk of kNoAllocChunk points, so a part of a
// handle may hold at most kNoAllocPartials * kNoAllocChunk local points.
constexpr int kNoAllocPartials = 4096;
constexpr int64_t kNoAllocChunk = 32768;
constexpr int kNoAllocCounterSlot = kNoAllocPartials;  // counter lives after the partials

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocPartials + 32];

constexpr int kMaxDevices = 64;
static double* g_scratch_addr[kMaxDevices] = {};
static std::mutex g_scratch_mutex;

// Device address of g_noalloc_scratch on the current device.  The first call
// on a device looks it up; in host code the array's name is only a host-side
// stand-in and must not be passed to a kernel.
static int scratch_address(double** out) {
    int dev = 0;
    SEM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(SEM_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[dev];
    return SEM_OK;
}

__global__ void __launch_bounds__(256) dot_chunk_kernel(const double* __restrict__ a, const double* __restrict__ b,
                                                        const uint8_t* __restrict__ mult, int64_t n,
                                                        double* scratch, double* out) {
    __shared__ double inv[256];
    __shared__ double red[32];
    __shared__ int is_last;
    for (int m = threadIdx.x; m < 256; m += blockDim.x) inv[m] = m ? 1.0 / m : 0.0;
    __syncthreads();
    const int64_t c0 = (int64_t)blockIdx.x * kNoAllocChunk;
    const int64_t c1 = c0 + kNoAllocChunk < n ? c0 + kNoAllocChunk : n;
    double v[1] = {0.0};
    for (int64_t L = c0 + threadIdx.x; L < c1; L += blockDim.x) v[0] = fma(a[L] * b[L], inv[mult[L]], v[0]);
    block_sum<1>(v, red);
    unsigned int* counter = reinterpret_cast<unsigned int*>(scratch + kNoAllocCounterSlot);
    if (threadIdx.x == 0) {
        scratch[blockIdx.x] = v[0];
        __threadfence();
        is_last = (atomicAdd(counter, 1u) == gridDim.x - 1) ? 1 : 0;
    }
    __syncthreads();
    if (is_last) {
        __threadfence();
        double acc[1] = {0.0};
        for (int q = threadIdx.x; q < (int)gridDim.x; q += blockDim.x) acc[0] += __ldcg(&scratch[q]);
        block_sum<1>(acc, red);
        if (threadIdx.x == 0) {
            *out = acc[0];
            *counter = 0u;
        }
    }
}

}  // namespace sem

using namespace sem;

extern "C" {

SEM_API int sem_dot_noalloc(const sem_handle* h, const double* a, const double* b, double* result,
                            cudaStream_t s) {
    if (!h || !a || !b || !result) return fail(SEM_EINVAL, "null argument");
    for (int q = 0; q < h->nsolve; q++)
        if (h->parts[q].n_local > (int64_t)kNoAllocPartials * kNoAllocChunk)
            return fail(SEM_EINVAL, "sem_dot_noalloc: a mesh has more than 134217728 local points "
                                    "(4096 partial sums of 32768 points each); use sem_dot");
    double* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc) return rc;
    for (int q = 0; q < h->nsolve; q++) {
        const MeshPart& p = h->parts[q];
        if (p.n_local == 0) {  // no launch for an empty mesh: its product is 0
            SEM_CUDA_TRY(cudaMemsetAsync(result + q, 0, sizeof(double), s));
            continue;
        }
        // the ticket counter must start at zero whatever an earlier call left there
        SEM_CUDA_TRY(cudaMemsetAsync(scratch + kNoAllocCounterSlot, 0, sizeof(unsigned int), s));
        const int grid = (int)((p.n_local + kNoAllocChunk - 1) / kNoAllocChunk);
        dot_chunk_kernel<<<grid, 256, 0, s>>>(a + p.loc_off, b + p.loc_off, h->mult + p.loc_off, p.n_local,
                                              scratch, result + q);
        SEM_LAUNCH_CHECK("dot_chunk_kernel");
    }
    return SEM_OK;
}

}  // extern "C"
