// Systematic resampling of one belief without any device allocation.
//
// Some callers cannot allocate device memory: code running inside a CUDA
// graph capture, real-time loops that forbid allocator calls, and host
// applications whose device memory is owned by another allocator.  For them
// this file provides bp_resample_noalloc: the same systematic resampler the
// filter uses after each update, with its FP64 cumulative-weight scratch in a
// file-scope static device array instead of a cudaMalloc'ed buffer.
//
// The array holds NOALLOC_MAX_P doubles (8 MiB) and stays resident on every
// GPU that loads the library until the process exits.  Every call shares it
// and it keeps the previous call's contents; the kernel overwrites the first
// P entries before reading them, so nothing needs clearing.  Calls whose
// kernels overlap on the GPU (different streams, or different host threads
// on one device) race on the array and must be serialised by the caller.
#include <mutex>

#include "bp_internal.cuh"
#include "bp_kernels.cuh"

namespace bp {

constexpr int NOALLOC_MAX_P = 1 << 20;

static __device__ __align__(256) double g_noalloc_cdf[NOALLOC_MAX_P];

// One block of 1024 threads: per-thread chunk sums, block scan (FP64), then the
// first index whose normalised cumulative weight reaches u_i = (U + i)/P.
__global__ void __launch_bounds__(1024) k_resample_noalloc(const double* __restrict__ w, int P, uint32_t k0,
                                                            uint32_t k1, uint32_t n, uint32_t item,
                                                            double* cdf, int* __restrict__ idx) {
    const int per = (P + blockDim.x - 1) / blockDim.x;
    const int p0 = threadIdx.x * per, p1 = min(P, p0 + per);
    double loc = 0.0;
    for (int p = p0; p < p1; ++p) loc += w[p];
    __shared__ double scan[1024];
    __shared__ double total;
    scan[threadIdx.x] = loc;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        const double t = (threadIdx.x >= (unsigned)off) ? scan[threadIdx.x - off] : 0.0;
        __syncthreads();
        scan[threadIdx.x] += t;
        __syncthreads();
    }
    if (threadIdx.x == blockDim.x - 1) total = scan[threadIdx.x];
    __syncthreads();
    double run = scan[threadIdx.x] - loc;
    for (int p = p0; p < p1; ++p) { run += w[p]; cdf[p] = run; }
    __syncthreads();
    const double tot = total;
    for (int p = p0; p < p1; ++p) cdf[p] = (tot > 0) ? cdf[p] / tot : (double)(p + 1) / P;
    __syncthreads();
    if (threadIdx.x == 0) cdf[P - 1] = 1.0;
    __syncthreads();
    const U4 r = philox(item, n, (RNG_RESAMPLE << 16), 0u, k0, k1);
    const double U = u32d(r.x);
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const double u = (U + (double)i) / (double)P;
        int lo = 0, hi = P - 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (cdf[mid] >= u) hi = mid; else lo = mid + 1;
        }
        idx[i] = lo;
    }
}

static std::mutex g_noalloc_mu;
static double* g_noalloc_ptr[64] = {nullptr};

}  // namespace bp

using namespace bp;

extern "C" {

bp_status bp_resample_noalloc(const double* w_dev, int P, uint64_t seed, int n, int kind, int index, int* idx_dev,
                              void* cuda_stream) {
    if (!w_dev || !idx_dev || P < 1 || kind < 0 || kind > 2 || index < 0 || index > 0xFFFF || n < 0)
        return BP_ERR_INVALID_ARG;
    if (P > NOALLOC_MAX_P) return BP_ERR_CAPACITY;   // beyond the static scratch: nothing launched
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return BP_ERR_CUDA;
    double* cdf = nullptr;
    {
        // set-up once per device, with that device current: the device address of
        // the static array (its host-side symbol is not a device address)
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_cdf) != cudaSuccess) return BP_ERR_CUDA;
            g_noalloc_ptr[dev] = static_cast<double*>(p);
        }
        cdf = g_noalloc_ptr[dev];
    }
    // an error left pending by earlier work is not this call's: report it without
    // launching, and leave it for its owner to read
    if (cudaPeekAtLastError() != cudaSuccess) return BP_ERR_CUDA;
    const uint32_t item = ((uint32_t)kind << 16) | (uint32_t)index;
    k_resample_noalloc<<<1, 1024, 0, static_cast<cudaStream_t>(cuda_stream)>>>(
        w_dev, P, (uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32), (uint32_t)n, item, cdf, idx_dev);
    return cudaGetLastError() == cudaSuccess ? BP_OK : BP_ERR_CUDA;
}

}  // extern "C"
