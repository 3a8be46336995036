// Allocation-free variant of the FP64 mass reduction (lbm_mass_noalloc in
// include/lbm.h).
//
// lbm_mass needs per-row partial sums between its two passes and keeps them
// in device memory that lbm_create allocated.  Code that cannot allocate
// device memory at the point where it needs the sums (an allocator callback
// that must not re-enter its allocator, a process whose device memory another
// framework's pool already reserves) gets the same per-row sum and final tree
// here, with the partial sums in one file-scope device array of fixed size,
// shared by every call on a device.
// lbm_mass splits each row into column chunks for parallelism; this variant
// sums a whole row per CTA, so the two agree to rounding, not bit for bit.
#include <mutex>

#include "lbm.h"
#include "lbm_kernels.cuh"

namespace {

constexpr int kMaxRows = LBM_NOALLOC_MAX_ROWS;
constexpr int kMaxDevices = 64;

// Per-row partial sums (species A, B) of the current call.  Every call
// writes all rows it reads before reading them, so nothing needs clearing;
// calls that overlap on the GPU race on this array.
static __device__ __align__(256) double g_row_sums[2 * kMaxRows];

std::mutex g_setup_mutex;
double* g_row_sums_addr[kMaxDevices] = {};   // device address of g_row_sums per device

// Pass 1: one CTA per row (a single column chunk).
template <typename S>
__global__ void __launch_bounds__(sc::kMassThreads) k_rows_noalloc(sc::RunDesc rd, double* __restrict__ part) {
    sc::mass_row_sum<S>(rd, static_cast<const S*>(rd.buf[0]), blockIdx.x, 0, 1, part + 2 * blockIdx.x);
}

// Pass 2: one CTA sums the rows with k_mass_final's tree.
__global__ void __launch_bounds__(sc::kMassThreads) k_final_noalloc(int ny, const double* __restrict__ part,
                                                                    double* __restrict__ mass) {
    sc::mass_rows_total(ny, part, mass);
}

// Device address of g_row_sums for the current device, looked up once per
// device (the name g_row_sums itself is only a host-side handle).
int row_sums_address(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return LBM_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_row_sums_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_row_sums) != cudaSuccess || !p) {
            cudaGetLastError();
            return LBM_ECUDA;
        }
        g_row_sums_addr[dev] = static_cast<double*>(p);
    }
    *out = g_row_sums_addr[dev];
    return LBM_OK;
}

}  // namespace

extern "C" int lbm_mass_noalloc(const lbm_geometry* g, int precision, const void* populations, int pitch,
                                const double rho_ref[2], double* mass, void* stream) {
    if (!g || !populations || !mass) return LBM_EINVAL;
    if (precision < LBM_F64 || precision > LBM_F16S) return LBM_EINVAL;
    if (g->nx < 1 || g->ny < 1 || pitch < g->nx) return LBM_EINVAL;
    if (g->ny > kMaxRows) return LBM_EINVAL;   // more rows than the static partial-sum array holds
    // the row sums index the buffer with 32-bit element offsets ((9 + i) * plane + y * pitch + x)
    if (18LL * g->ny * pitch >= (1LL << 31)) return LBM_EINVAL;
    if (g->solid_mask) return LBM_EINVAL;      // plates only: a mask would have to be copied to the device
    if (g->cap_x0 < 0 || g->cap_x1 < g->cap_x0 || g->cap_x1 > g->nx) return LBM_EINVAL;
    if (g->y_bot < -1 || g->y_bot >= g->ny || g->y_top < -1 || g->y_top >= g->ny) return LBM_EINVAL;
    double* part = nullptr;
    int rc = row_sums_address(&part);
    if (rc) return rc;
    sc::RunDesc rd;
    memset(&rd, 0, sizeof(rd));
    rd.buf[0] = const_cast<void*>(populations);
    rd.nx = g->nx;
    rd.ny = g->ny;
    rd.pitch = pitch;
    rd.nodes = g->nx * g->ny;
    rd.plane = (long long)g->ny * pitch;
    rd.cap_x0 = g->cap_x0;
    rd.cap_x1 = g->cap_x1;
    rd.y_bot = g->y_bot;
    rd.y_top = g->y_top;
    rd.rho_ref[0] = rho_ref ? rho_ref[0] : 0.0;
    rd.rho_ref[1] = rho_ref ? rho_ref[1] : 0.0;
    sc::fill_coef_f32(rd);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    switch (precision) {
        case LBM_F64: k_rows_noalloc<double><<<g->ny, sc::kMassThreads, 0, s>>>(rd, part); break;
        case LBM_F32: k_rows_noalloc<float><<<g->ny, sc::kMassThreads, 0, s>>>(rd, part); break;
        default: k_rows_noalloc<__half><<<g->ny, sc::kMassThreads, 0, s>>>(rd, part); break;
    }
    k_final_noalloc<<<1, sc::kMassThreads, 0, s>>>(g->ny, part, mass);
    if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
    return LBM_OK;
}
