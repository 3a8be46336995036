// Launchers of the kernels in lbm_kernels.cuh; Launch<S> is instantiated per
// storage type by kernels_f64.cu, kernels_f32.cu and kernels_f16.cu, and
// Step<S, GEN> by those and by the kernels_gen_*.cu units (GEN = true).
#pragma once

#include <atomic>

#include "lbm_kernels.cuh"
#include "lbm_ring.cuh"

namespace sc {

// Raises the dynamic shared-memory limit of kernel `fn` to `bytes` once per
// device (one bit per device in `done`); two threads racing on a first launch
// both set the same attribute, which is harmless.
static inline cudaError_t ensure_dynamic_smem(const void* fn, int bytes, std::atomic<unsigned long long>& done) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = dev < 64 ? (1ull << dev) : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_release);
    return e;
}

static inline int clamp_grid(long long want, int cap) {
    if (want < 1) return 1;
    return want > cap ? cap : (int)want;
}

template <typename S>
cudaError_t Launch<S>::init(const RunDesc* d_runs, int nruns, int max_nodes, cudaStream_t s) {
    if (nruns <= 0) return cudaSuccess;
    dim3 grid(clamp_grid((max_nodes + 255) / 256, 2048), nruns);
    k_init<S><<<grid, 256, 0, s>>>(d_runs);
    return cudaGetLastError();
}

template <typename S, bool G>
cudaError_t Step<S, G>::step(int W, const RunDesc* d_runs, const Tile* d_tiles, int ntiles, int parity,
                            cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    MomOut none{nullptr, nullptr, 0};
    switch (W) {
        case 64: k_step<S, 64, 0, false, G><<<ntiles, 64, 0, s>>>(d_runs, d_tiles, parity, none); break;
        case 128: k_step<S, 128, 0, false, G><<<ntiles, 128, 0, s>>>(d_runs, d_tiles, parity, none); break;
        case 256: k_step<S, 256, 0, false, G><<<ntiles, 256, 0, s>>>(d_runs, d_tiles, parity, none); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename S, int W, int D, bool G>
static cudaError_t launch_async(const RunDesc* d_runs, const Tile* d_tiles, int ntiles, int parity, cudaStream_t s) {
    constexpr size_t smem = async_smem_bytes<S, W, D>();
    static std::atomic<unsigned long long> configured{0};   // per instantiation, one bit per device
    const cudaError_t e = ensure_dynamic_smem((const void*)k_step_async<S, W, D, G>, (int)smem, configured);
    if (e != cudaSuccess) return e;
    k_step_async<S, W, D, G><<<ntiles, W, smem, s>>>(d_runs, d_tiles, parity);
    return cudaGetLastError();
}

template <typename S, bool G>
cudaError_t Step<S, G>::step_async(int W, int D, const RunDesc* d_runs, const Tile* d_tiles, int ntiles, int parity,
                                  cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    if constexpr (sizeof(S) == 2) {
        return cudaErrorInvalidValue;   // cp.async moves 4 or 8 bytes: FP16 storage uses k_step
    } else {
        const int key = W * 10 + D;
        switch (key) {
            case 643: return launch_async<S, 64, 3, G>(d_runs, d_tiles, ntiles, parity, s);
            case 644: return launch_async<S, 64, 4, G>(d_runs, d_tiles, ntiles, parity, s);
            case 1283: return launch_async<S, 128, 3, G>(d_runs, d_tiles, ntiles, parity, s);
            case 1284: return launch_async<S, 128, 4, G>(d_runs, d_tiles, ntiles, parity, s);
            case 2563: return launch_async<S, 256, 3, G>(d_runs, d_tiles, ntiles, parity, s);
            case 2564: return launch_async<S, 256, 4, G>(d_runs, d_tiles, ntiles, parity, s);
            default: return cudaErrorInvalidValue;
        }
    }
}

template <typename S, int W, int D, bool G>
static cudaError_t launch_tma(const RunDesc* d_runs, const Tile* d_tiles, int ntiles, int parity, uint32_t* err,
                              cudaStream_t s) {
    constexpr size_t smem = TmaGeom<S, W, D>::smem_bytes();
    if constexpr (smem > kMaxSmemPerCta) {
        return cudaErrorInvalidValue;
    } else {
        static std::atomic<unsigned long long> configured{0};   // per instantiation, one bit per device
        const cudaError_t e = ensure_dynamic_smem((const void*)k_step_tma<S, W, D, G>, (int)smem, configured);
        if (e != cudaSuccess) return e;
        k_step_tma<S, W, D, G><<<ntiles, W, smem, s>>>(d_runs, d_tiles, parity, err);
        return cudaGetLastError();
    }
}

template <typename S, bool G>
cudaError_t Step<S, G>::step_tma(int W, int D, const RunDesc* d_runs, const Tile* d_tiles, int ntiles, int parity,
                                uint32_t* err, cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    switch (W * 10 + D) {
        case 644: return launch_tma<S, 64, 4, G>(d_runs, d_tiles, ntiles, parity, err, s);
        case 646: return launch_tma<S, 64, 6, G>(d_runs, d_tiles, ntiles, parity, err, s);
        case 648: return launch_tma<S, 64, 8, G>(d_runs, d_tiles, ntiles, parity, err, s);
        case 1284: return launch_tma<S, 128, 4, G>(d_runs, d_tiles, ntiles, parity, err, s);
        case 1286: return launch_tma<S, 128, 6, G>(d_runs, d_tiles, ntiles, parity, err, s);
        case 1288: return launch_tma<S, 128, 8, G>(d_runs, d_tiles, ntiles, parity, err, s);
        case 2564: return launch_tma<S, 256, 4, G>(d_runs, d_tiles, ntiles, parity, err, s);
        case 2566: return launch_tma<S, 256, 6, G>(d_runs, d_tiles, ntiles, parity, err, s);
        default: return cudaErrorInvalidValue;
    }
}

template <typename S, bool G>
cudaError_t Step<S, G>::step_pf(int W, const RunDesc* d_runs, const Tile* d_tiles, int ntiles, int parity,
                               cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    switch (W) {
        case 64: k_step_pf<S, 64, G><<<ntiles, 64, 0, s>>>(d_runs, d_tiles, parity); break;
        case 128:
            if constexpr (sizeof(typename Prec<S>::C) == 8) return cudaErrorInvalidValue;
            else k_step_pf<S, 128, G><<<ntiles, 128, 0, s>>>(d_runs, d_tiles, parity);
            break;

        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename S, bool G>
cudaError_t Step<S, G>::step_split(int W, const RunDesc* d_runs, const Tile* d_tiles, int ntiles, int parity,
                                  cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    switch (W) {
        case 64: k_step_split<S, 64, G><<<ntiles, 128, 0, s>>>(d_runs, d_tiles, parity); break;
        case 128: k_step_split<S, 128, G><<<ntiles, 256, 0, s>>>(d_runs, d_tiles, parity); break;
        case 256: k_step_split<S, 256, G><<<ntiles, 512, 0, s>>>(d_runs, d_tiles, parity); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename S, bool G>
cudaError_t Step<S, G>::step_l2pf(int W, const RunDesc* d_runs, const Tile* d_tiles, int ntiles, int parity,
                                 cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    MomOut none{nullptr, nullptr, 0};
    switch (W) {
        case 64: k_step<S, 64, 0, true, G><<<ntiles, 64, 0, s>>>(d_runs, d_tiles, parity, none); break;
        case 128: k_step<S, 128, 0, true, G><<<ntiles, 128, 0, s>>>(d_runs, d_tiles, parity, none); break;
        case 256: k_step<S, 256, 0, true, G><<<ntiles, 256, 0, s>>>(d_runs, d_tiles, parity, none); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename S, bool G>
cudaError_t Step<S, G>::step_smem(int W, const RunDesc* d_runs, const Tile* d_tiles, int ntiles, int parity,
                                 cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    switch (W) {
        case 64: k_step_smem<S, 64, G><<<ntiles, 64, 0, s>>>(d_runs, d_tiles, parity); break;
        case 128: k_step_smem<S, 128, G><<<ntiles, 128, 0, s>>>(d_runs, d_tiles, parity); break;
        case 256:
            if constexpr (sizeof(typename Prec<S>::C) == 8) return cudaErrorInvalidValue;
            else k_step_smem<S, 256, G><<<ntiles, 256, 0, s>>>(d_runs, d_tiles, parity);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename S, bool G>
cudaError_t Step<S, G>::step_pair(int W, const RunDesc* d_runs, const Tile* d_tiles, int ntiles, int parity,
                                 cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    switch (W) {
        case 64: k_step_pair<S, 64, G><<<ntiles, 64, 0, s>>>(d_runs, d_tiles, parity); break;
        case 128:
            if constexpr (sizeof(typename Prec<S>::C) == 8) return cudaErrorInvalidValue;
            else k_step_pair<S, 128, G><<<ntiles, 128, 0, s>>>(d_runs, d_tiles, parity);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename S, bool G>
cudaError_t Step<S, G>::step_tile(int W, int R, const RunDesc* d_runs, const Tile* d_tiles, int ntiles, int parity,
                                 cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    // R = collided rows per tile: TY = R + 2 thread rows
    switch (W * 100 + R) {
        case 3206: k_step_tile<S, 32, 8, G><<<ntiles, 256, 0, s>>>(d_runs, d_tiles, parity); break;
        case 3214: k_step_tile<S, 32, 16, G><<<ntiles, 512, 0, s>>>(d_runs, d_tiles, parity); break;
        case 3230: k_step_tile<S, 32, 32, G><<<ntiles, 1024, 0, s>>>(d_runs, d_tiles, parity); break;
        case 6406: k_step_tile<S, 64, 8, G><<<ntiles, 512, 0, s>>>(d_runs, d_tiles, parity); break;
        case 6414: k_step_tile<S, 64, 16, G><<<ntiles, 1024, 0, s>>>(d_runs, d_tiles, parity); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename S, bool G>
cudaError_t Step<S, G>::step_bidir(int W, const RunDesc* d_runs, const Tile* d_tiles, int ntiles, int parity,
                                  cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    switch (W) {
        case 64: k_step_bidir<S, 64, G><<<ntiles, 128, 0, s>>>(d_runs, d_tiles, parity); break;
        case 128:
            if constexpr (sizeof(typename Prec<S>::C) == 8) return cudaErrorInvalidValue;
            else k_step_bidir<S, 128, G><<<ntiles, 256, 0, s>>>(d_runs, d_tiles, parity);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename S, int D, bool G>
static cudaError_t ring_fn(const void** fn, int* smem, int* threads) {
    if constexpr (sizeof(S) == 8) {
        return cudaErrorInvalidValue;   // FP64 is arithmetic-bound: it keeps the register kernels
    } else {
        using RG = RingGeom<S, D>;
        constexpr size_t bytes = RG::smem_bytes();
        static_assert(bytes <= kMaxSmemPerCta, "ring slots exceed the shared memory of a CTA");
        static std::atomic<unsigned long long> configured{0};   // per instantiation, one bit per device
        const cudaError_t e = ensure_dynamic_smem((const void*)k_step_ring<S, D, G>, (int)bytes, configured);
        if (e != cudaSuccess) return e;
        *fn = (const void*)k_step_ring<S, D, G>;
        *smem = (int)bytes;
        *threads = RG::THREADS;
        return cudaSuccess;
    }
}

template <typename S, bool G>
static cudaError_t ring_lookup(int D, const void** fn, int* smem, int* threads) {
    switch (D) {
        case 3: return ring_fn<S, 3, G>(fn, smem, threads);
        case 4: return ring_fn<S, 4, G>(fn, smem, threads);
        case 5: return ring_fn<S, 5, G>(fn, smem, threads);
        default: return cudaErrorInvalidValue;
    }
}

template <typename S, bool G>
cudaError_t Step<S, G>::ring_ctas_per_sm(int D, int* out) {
    *out = 0;
    const void* fn = nullptr;
    int smem = 0, threads = 0;
    cudaError_t e = ring_lookup<S, G>(D, &fn, &smem, &threads);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, fn, threads, (size_t)smem);
}

template <typename S, bool G>
cudaError_t Step<S, G>::bidir_ctas_per_sm(int W, int* out) {
    *out = 0;
    switch (W) {
        case 64: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_step_bidir<S, 64, G>, 128, 0);
        case 128:
            if constexpr (sizeof(typename Prec<S>::C) == 8) return cudaErrorInvalidValue;
            else return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_step_bidir<S, 128, G>, 256, 0);
        default: return cudaErrorInvalidValue;
    }
}

template <typename S, bool G>
cudaError_t Step<S, G>::step_ring(int D, const RunDesc* d_runs, const Tile* d_tiles, int ntiles, int* queue,
                                  int grid, int parity, uint32_t* err, cudaStream_t s) {
    if (grid <= 0 || ntiles <= 0) return cudaSuccess;
    const void* fn = nullptr;
    int smem = 0, threads = 0;
    cudaError_t e = ring_lookup<S, G>(D, &fn, &smem, &threads);
    if (e != cudaSuccess) return e;
    void* args[] = {(void*)&d_runs, (void*)&d_tiles, (void*)&ntiles, (void*)&queue, (void*)&parity, (void*)&err};
    return cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, (size_t)smem, s);
}

template <typename S, bool G>
cudaError_t Step<S, G>::moments(int W, const RunDesc* d_runs, const Tile* d_tiles, int ntiles, int parity,
                               MomOut out, cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    switch (W) {
        case 64: k_step<S, 64, 1, false, G><<<ntiles, 64, 0, s>>>(d_runs, d_tiles, parity, out); break;
        case 128: k_step<S, 128, 1, false, G><<<ntiles, 128, 0, s>>>(d_runs, d_tiles, parity, out); break;
        case 256: k_step<S, 256, 1, false, G><<<ntiles, 256, 0, s>>>(d_runs, d_tiles, parity, out); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename S>
cudaError_t Launch<S>::densities(const RunDesc* d_runs, int run, int parity, int nodes, double* nA, double* nB,
                                 cudaStream_t s) {
    k_densities<S><<<clamp_grid((nodes + 255) / 256, 4096), 256, 0, s>>>(d_runs, run, parity, nA, nB);
    return cudaGetLastError();
}

template <typename S>
cudaError_t Launch<S>::track(const RunDesc* d_runs, int nruns, int max_cap, int parity, int* first, LogCtl lc,
                             double* zout, cudaStream_t s) {
    if (nruns <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(first, 0x7f, (size_t)4 * nruns * sizeof(int), s);   // kNoFront
    if (e != cudaSuccess) return e;
    if (max_cap > 0) {
        k_track_scan<S><<<dim3((max_cap + kTrackThreads - 1) / kTrackThreads, nruns), kTrackThreads, 0, s>>>(
            d_runs, parity, first);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    k_track_final<S><<<nruns, 32, 0, s>>>(d_runs, parity, first, lc, zout);
    return cudaGetLastError();
}

template <typename S>
cudaError_t Launch<S>::mass(const RunDesc* d_runs, int nruns, const int2* d_rows, int nrows, int parity,
                            double* d_partials, double* d_mass, LogCtl lc, int write_log, uint32_t* d_err,
                            cudaStream_t s) {
    if (nruns <= 0) return cudaSuccess;
    k_mass_rows<S><<<dim3(nrows, kMassChunks), kMassThreads, 0, s>>>(d_runs, d_rows, parity, d_partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_mass_final<<<nruns, kMassThreads, 0, s>>>(d_runs, d_partials, d_mass, lc, write_log, d_err);
    return cudaGetLastError();
}

template <typename S>
cudaError_t Launch<S>::export_pops(const RunDesc* d_runs, int run, int parity, int nx, int ny, void* out,
                                   cudaStream_t s) {
    const long long total = 18LL * nx * ny;
    k_export<S><<<clamp_grid((total + 255) / 256, 8192), 256, 0, s>>>(d_runs, run, parity, static_cast<S*>(out));
    return cudaGetLastError();
}

template <typename S>
cudaError_t Launch<S>::import_pops(const RunDesc* d_runs, int run, int parity, int nx, int ny, const void* in,
                                   cudaStream_t s) {
    const long long total = 18LL * nx * ny;
    k_import<S><<<clamp_grid((total + 255) / 256, 8192), 256, 0, s>>>(d_runs, run, parity,
                                                                      static_cast<const S*>(in));
    return cudaGetLastError();
}

template <typename S>
cudaError_t Launch<S>::get_cols(const RunDesc* d_runs, int run, int parity, int ny, int x0, int ncols, void* out,
                                cudaStream_t s) {
    const long long total = 18LL * ny * ncols;
    k_get_cols<S><<<clamp_grid((total + 255) / 256, 4096), 256, 0, s>>>(d_runs, run, parity, x0, ncols,
                                                                        static_cast<S*>(out));
    return cudaGetLastError();
}

template <typename S>
cudaError_t Launch<S>::set_cols(const RunDesc* d_runs, int run, int parity, int ny, int x0, int ncols,
                                const void* in, cudaStream_t s) {
    const long long total = 18LL * ny * ncols;
    k_set_cols<S><<<clamp_grid((total + 255) / 256, 4096), 256, 0, s>>>(d_runs, run, parity, x0, ncols,
                                                                        static_cast<const S*>(in));
    return cudaGetLastError();
}

}  // namespace sc
