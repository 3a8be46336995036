// FP64 instantiation of the step (standard species) and its reductions.  Built with
// --fmad=false: every product and sum of the canonical order is rounded on
// its own, so the results equal a plain FP64 evaluation of the same order.
#include "lbm_launch.cuh"

namespace sc {

__global__ void __launch_bounds__(kMassThreads) k_mass_final(const RunDesc* __restrict__ runs,
                                                             const double* __restrict__ partials,
                                                             double* __restrict__ mass, LogCtl lc, int write_log,
                                                             uint32_t* __restrict__ err) {
    const RunDesc& rd = runs[blockIdx.x];
    __shared__ double tot[2];
    mass_rows_total(rd.ny * kMassChunks, partials + 2 * (long long)rd.row0 * kMassChunks, tot);
    if (threadIdx.x == 0) {
        const double MA = tot[0], MB = tot[1];
        if (mass) {
            mass[2 * blockIdx.x + 0] = MA;
            mass[2 * blockIdx.x + 1] = MB;
        }
        if (!isfinite(MA) || !isfinite(MB)) atomicOr(err, ERR_NONFINITE);
        if (write_log && rd.log && lc.count) {
            double* rec = rd.log + (*lc.count % lc.cap) * 6;
            rec[4] = MA;
            rec[5] = MB;
        }
    }
}

__global__ void k_log_advance(long long* count) { *count += 1; }

cudaError_t launch_log_advance(LogCtl lc, cudaStream_t s) {
    k_log_advance<<<1, 1, 0, s>>>(lc.count);
    return cudaGetLastError();
}

template struct Launch<double>;
template struct Step<double, false>;

}  // namespace sc
