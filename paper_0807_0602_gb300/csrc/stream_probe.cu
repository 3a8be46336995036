// Streaming probes (include/lbm_probe.h): the step kernel's memory access
// pattern without its arithmetic, to measure what the pattern itself can
// reach on this GPU.  Populations use the step's layout: 18 planes of
// ny rows of `pitch` elements (FP32), interior nodes only (no wrap).
#include <cuda_runtime.h>

#include "lbm.h"
#include "lbm_kernels.cuh"
#include "lbm_probe.h"

namespace {

__constant__ int kDx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__constant__ int kDy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

// one thread per node: the 18 pulled loads, then 18 stores
__global__ void k_probe_pull(const float* __restrict__ src, float* __restrict__ dst, int nx, int ny, int pitch,
                             long long plane) {
    extern __shared__ float occupancy_pad[];   // dynamic size only limits CTAs per SM
    (void)occupancy_pad;
    const int x = blockIdx.x * blockDim.x + threadIdx.x + 1, y = blockIdx.y + 1;
    if (x >= nx - 1 || y >= ny - 1) return;
    float v[18];
#pragma unroll
    for (int q = 0; q < 18; ++q) {
        const int i = q % 9;
        v[q] = __ldg(src + q * plane + (long long)(y - kDy[i]) * pitch + (x - kDx[i]));
    }
#pragma unroll
    for (int q = 0; q < 18; ++q) dst[q * plane + (long long)y * pitch + x] = v[q];
}

// one thread per node, unshifted: a plain copy of 18 planes
__global__ void k_probe_copy(const float* __restrict__ src, float* __restrict__ dst, int nx, int ny, int pitch,
                             long long plane) {
    extern __shared__ float occupancy_pad[];
    (void)occupancy_pad;
    const int x = blockIdx.x * blockDim.x + threadIdx.x + 1, y = blockIdx.y + 1;
    if (x >= nx - 1 || y >= ny - 1) return;
    float v[18];
#pragma unroll
    for (int q = 0; q < 18; ++q) v[q] = __ldg(src + q * plane + (long long)y * pitch + x);
#pragma unroll
    for (int q = 0; q < 18; ++q) dst[q * plane + (long long)y * pitch + x] = v[q];
}

// one thread per column, marching `rows` rows: the step kernels' march
__global__ void k_probe_march(const float* __restrict__ src, float* __restrict__ dst, int nx, int ny, int pitch,
                              long long plane, int rows) {
    extern __shared__ float occupancy_pad[];
    (void)occupancy_pad;
    const int x = blockIdx.x * blockDim.x + threadIdx.x + 1, y0 = blockIdx.y * rows + 1;
    if (x >= nx - 1) return;
    for (int y = y0; y < y0 + rows && y < ny - 1; ++y) {
        float v[18];
#pragma unroll
        for (int q = 0; q < 18; ++q) {
            const int i = q % 9;
            v[q] = __ldg(src + q * plane + (long long)(y - kDy[i]) * pitch + (x - kDx[i]));
        }
#pragma unroll
        for (int q = 0; q < 18; ++q) dst[q * plane + (long long)y * pitch + x] = v[q];
    }
}

// Blocked layout: 32 columns of all 18 planes contiguous, element (q, y, x)
// at ((y nb + x / 32) 18 + q) 32 + x % 32 with nb = pitch / 32 blocks per row.
__device__ __forceinline__ long long blocked(int q, int y, int x, int nb) {
    return ((long long)(y * nb + (x >> 5)) * 18 + q) * 32 + (x & 31);
}

// one thread per node (columns 32 .. nx - 33): pull or copy in the blocked layout
template <bool PULL>
__global__ void k_probe_blocked(const float* __restrict__ src, float* __restrict__ dst, int nx, int ny, int nb) {
    extern __shared__ float occupancy_pad[];
    (void)occupancy_pad;
    const int x = blockIdx.x * blockDim.x + threadIdx.x + 32, y = blockIdx.y + 1;
    if (x >= nx - 32 || y >= ny - 1) return;
    float v[18];
#pragma unroll
    for (int q = 0; q < 18; ++q) {
        const int i = q % 9;
        v[q] = PULL ? __ldg(src + blocked(q, y - kDy[i], x - kDx[i], nb)) : __ldg(src + blocked(q, y, x, nb));
    }
#pragma unroll
    for (int q = 0; q < 18; ++q) dst[blocked(q, y, x, nb)] = v[q];
}

}  // namespace

extern "C" int lbm_probe_stream(int pattern, const float* src, float* dst, int nx, int ny, int pitch, int rows,
                                int block, int smem_bytes, void* stream) {
    if (!src || !dst || nx < 3 || ny < 3 || pitch < nx || block < 32 || block > 1024 || block % 32 ||
        smem_bytes < 0 || smem_bytes > 227 * 1024 || (pattern == LBM_PROBE_MARCH && rows < 1) ||
        pattern < LBM_PROBE_PULL || pattern > LBM_PROBE_COPY_BLOCKED ||
        (pattern >= LBM_PROBE_PULL_BLOCKED && (pitch % 32 || nx < 66)))
        return 1;
    const long long plane = (long long)ny * pitch;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    const void* fn = pattern == LBM_PROBE_PULL          ? (const void*)k_probe_pull
                     : pattern == LBM_PROBE_COPY        ? (const void*)k_probe_copy
                     : pattern == LBM_PROBE_MARCH       ? (const void*)k_probe_march
                     : pattern == LBM_PROBE_PULL_BLOCKED ? (const void*)k_probe_blocked<true>
                                                         : (const void*)k_probe_blocked<false>;
    if (smem_bytes > 48 * 1024) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e != cudaSuccess) return 3;
    const dim3 blk(block);
    if (pattern >= LBM_PROBE_PULL_BLOCKED) {
        const dim3 g((nx - 64 + block - 1) / block, ny - 2);
        if (pattern == LBM_PROBE_PULL_BLOCKED)
            k_probe_blocked<true><<<g, blk, smem_bytes, s>>>(src, dst, nx, ny, pitch / 32);
        else
            k_probe_blocked<false><<<g, blk, smem_bytes, s>>>(src, dst, nx, ny, pitch / 32);
    } else if (pattern == LBM_PROBE_MARCH) {
        const dim3 g((nx - 2 + block - 1) / block, (ny - 2 + rows - 1) / rows);
        k_probe_march<<<g, blk, smem_bytes, s>>>(src, dst, nx, ny, pitch, plane, rows);
    } else {
        const dim3 g((nx - 2 + block - 1) / block, ny - 2);
        if (pattern == LBM_PROBE_PULL) k_probe_pull<<<g, blk, smem_bytes, s>>>(src, dst, nx, ny, pitch, plane);
        else k_probe_copy<<<g, blk, smem_bytes, s>>>(src, dst, nx, ny, pitch, plane);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

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
