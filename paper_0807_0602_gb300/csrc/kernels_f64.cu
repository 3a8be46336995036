// FP64 instantiation of the step and its reductions.  Built with
// --fmad=false: every product and sum of the canonical order is rounded on
// its own, so the results equal a plain FP64 evaluation of the same order.
#include "lbm_launch.cuh"

namespace sc {

__global__ void __launch_bounds__(256) k_mass_final(const RunDesc* __restrict__ runs,
                                                    const double* __restrict__ partials, double* __restrict__ mass,
                                                    LogCtl lc, int write_log, uint32_t* __restrict__ err) {
    const RunDesc& rd = runs[blockIdx.x];
    double a = 0.0, b = 0.0;
    for (int y = threadIdx.x; y < rd.ny; y += 256) {
        a = __dadd_rn(a, partials[2 * (rd.row0 + y) + 0]);
        b = __dadd_rn(b, partials[2 * (rd.row0 + y) + 1]);
    }
    __shared__ double s[2][256];
    s[0][threadIdx.x] = a;
    s[1][threadIdx.x] = b;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            s[0][threadIdx.x] = __dadd_rn(s[0][threadIdx.x], s[0][threadIdx.x + h]);
            s[1][threadIdx.x] = __dadd_rn(s[1][threadIdx.x], s[1][threadIdx.x + h]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double MA = s[0][0], MB = s[1][0];
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

}  // namespace sc
