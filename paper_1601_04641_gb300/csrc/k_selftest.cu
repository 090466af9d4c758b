// k_selftest.cu -- failure-detection self-test of the bounded device waits
// and the allocation-failure hook (the paper has no counterpart).
#include "gp.h"
#include "gp_sweep_tma.cuh"

namespace gpcn {
namespace {

// One warp: a bounded wait on an mbarrier whose phase completes (lane 0
// arrives first) and one on an mbarrier that nothing arrives at.  Nothing is
// copied, so the second wait can only run out; it gives up after `cycles`.
__global__ void bounded_wait_kernel(long long cycles, unsigned *result) {
    __shared__ __align__(8) unsigned long long bars[2];
    const unsigned done = smem_u32(&bars[0]), never = smem_u32(&bars[1]);
    if (threadIdx.x == 0) {
        mbar_init(done, 1);
        mbar_init(never, 1);
        mbar_init_fence();
        mbar_arrive(done);
    }
    __syncwarp();
    const bool completed = mbar_wait_bounded(done, 0, true, cycles);
    const bool expired = !mbar_wait_bounded(never, 0, true, cycles);
    if (threadIdx.x == 0) {
        result[0] = completed ? 1u : 0u;
        result[1] = expired ? 1u : 0u;
    }
}

}  // namespace
}  // namespace gpcn

using namespace gpcn;

extern "C" gp_status gp_selftest_bounded_wait(long long cycles, void *cuda_stream, int *completed, int *expired) {
    if (cycles < 1 || cycles > (1LL << 34) || !completed || !expired) {
        set_thread_error("need 1 <= cycles <= 2^34 and both outputs");
        return GP_ERR_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    unsigned *d = nullptr;
    if (dev_malloc(&d, 2 * sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        set_thread_error("cudaMalloc failed");
        return GP_ERR_NOMEM;
    }
    unsigned h[2] = {0, 0};
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(h), s);
    if (e == cudaSuccess) {
        bounded_wait_kernel<<<1, 32, 0, s>>>(cycles, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_thread_error(cudaGetErrorString(e));
        return GP_ERR_CUDA;
    }
    *completed = (int)h[0];
    *expired = (int)h[1];
    return GP_OK;
}

extern "C" void gp_debug_fail_alloc(int n) { set_fail_alloc(n); }
