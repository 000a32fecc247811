// Self-test of the bounded waits (failure detection without a GPU fault): one thread
// waits on an mbarrier phase that nothing completes, with the same bounded poll loop
// the tensor-core kernels use, and reports that the wait gave up.  Nothing else is in
// flight (no copies, no MMAs, no tensor memory), so the kernel ends normally and the
// context stays usable.
#include "bp_handle.cuh"
#include "tc_sm100.cuh"

namespace bp {

__global__ void k_wait_selftest(int limit, int* status) {
    __shared__ uint64_t mbar;
    const uint32_t mb = tc::smem_u32(&mbar);
    if (threadIdx.x == 0) { tc::mbar_init(mb, 1); tc::mbar_init_fence(); }
    __syncthreads();
    if (threadIdx.x == 0) {
        // phase 0 of a fresh barrier with an expected count of 1 and no arrival
        const bool done = tc::mbar_wait(mb, 0u, limit);
        *status = done ? 0 : 1;
    }
}

}  // namespace bp

extern "C" bp_status bp_selftest_wait(int limit, void* cuda_stream) {
    if (limit < 1 || limit > (1 << 20)) return BP_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int* d = nullptr;
    int h = -1;
    if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return BP_ERR_CUDA;
    bp::k_wait_selftest<<<1, 32, 0, st>>>(limit, d);
    const bool ok = cudaGetLastError() == cudaSuccess &&
                    cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
                    cudaStreamSynchronize(st) == cudaSuccess;
    cudaFree(d);
    if (!ok) return BP_ERR_CUDA;
    return h == 1 ? BP_ERR_TIMEOUT : BP_OK;
}
