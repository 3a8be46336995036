// Failure-path self-test of the bounded device waits (lbm_selftest_wait_timeout
// in include/lbm.h).  The paper has no counterpart: this exercises, without any
// GPU fault, the path a step kernel takes when one of its mbarrier waits runs
// out: the wait gives up, the error word gets ERR_TIMEOUT, and the host reads
// LBM_ETIMEOUT while the context stays usable.
#include <cuda_runtime.h>

#include "lbm.h"
#include "lbm_kernels.cuh"

namespace {

// One CTA waits, with the step kernels' bounded wait, on an mbarrier phase
// that can never complete (an expected transaction that no copy delivers).
__global__ void k_wait_selftest(long long limit, uint32_t* __restrict__ err) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        sc::mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) sc::mbar_expect_tx(&bar, 16u);   // the phase's only arrival; 16 bytes never come
    if (!sc::mbar_wait(&bar, 0u, limit) && threadIdx.x == 0) atomicOr(err, sc::ERR_TIMEOUT);
}

}  // namespace

extern "C" int lbm_selftest_wait_timeout(long long cycles, void* stream) {
    if (cycles < 1000 || cycles > 4000000000LL) return LBM_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t* d_err = nullptr;
    if (cudaMalloc(&d_err, sizeof(uint32_t)) != cudaSuccess) return LBM_ENOMEM;
    uint32_t h_err = 0;
    cudaError_t e = cudaMemsetAsync(d_err, 0, sizeof(uint32_t), s);
    if (e == cudaSuccess) {
        k_wait_selftest<<<1, 32, 0, s>>>(cycles, d_err);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_err);
    if (e != cudaSuccess) return LBM_ECUDA;
    return (h_err & sc::ERR_TIMEOUT) ? LBM_ETIMEOUT : LBM_OK;
}
