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

namespace {

// FP64 fused multiply-add throughput: every thread runs 8 independent chains
// of `iters` dependent DFMAs (enough independent work per warp to fill the
// FP64 pipe); the result is written so that nothing is optimised away.
__global__ void k_fp64_fma_rate(int iters, double seed, double* __restrict__ sink) {
    double a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = seed + 1e-3 * (threadIdx.x + j);
    const double m = 0.999999, c = 1e-9;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) a[j] = fma(a[j], m, c);
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += a[j];
    if (s == 12345.0) sink[blockIdx.x] = s;   // never true for these inputs; keeps the work live
}

}  // namespace

extern "C" int lbm_selftest_fp64_rate(double* flops_per_s, void* stream) {
    if (!flops_per_s) return LBM_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess) {
        cudaGetLastError();
        return LBM_ECUDA;
    }
    double* d_sink = nullptr;
    if (cudaMalloc(&d_sink, sizeof(double) * 16 * sms) != cudaSuccess) return LBM_ENOMEM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int blocks = 16 * sms, threads = 256, iters = 4096;
    float ms = 0.f;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {   // the first launch warms up
        e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) {
            k_fp64_fma_rate<<<blocks, threads, 0, s>>>(iters, 1.0 + rep, d_sink);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(d_sink);
    if (e != cudaSuccess || ms <= 0.f) return LBM_ECUDA;
    *flops_per_s = 2.0 * 8.0 * iters * (double)blocks * threads / (ms * 1e-3);
    return LBM_OK;
}
