// Internal device-side descriptors and kernel launchers of the Shan-Chen
// D2Q9 library.  Not part of the public ABI (include/lbm.h is).
#pragma once

#include <cuda_fp16.h>

#include "lbm.h"
#ifndef __CUDACC_RTC__
#include <cuda_runtime.h>
#include <stdint.h>
#endif

namespace sc {

// Step coefficients rounded to FP32 on the host: the FP32 and FP16S kernels
// read these, so that no FP64 -> FP32 conversion runs at each CTA's start.
struct CoefF32 {
    float G, Gw[2], taum[2], itau[2], mitau[2], m[2], gx, gy;
    float dA[2][3];
    float sh[2][3];   // FP16S shift w_g rho_ref,k per direction group
};

// One run (one capillary) as the kernels see it.  Populations of buffer b:
//   buf[b] + ((k * 9 + i) * ny + y) * pitch + x     (elements of the storage type)
struct RunDesc {
    void* buf[2];
    long long plane;          // ny * pitch
    int nx, ny, pitch, nodes; // nodes = nx * ny
    int cap_x0, cap_x1, y_bot, y_top;
    const uint8_t* mask;      // device [ny][nx] or nullptr (analytic plates)
    // Eqs. 2, 7-11 parameters; itau = 1 / tau computed on the host in FP64
    double G, GwA, GwB, tauA, tauB, itauA, itauB, gx, gy;
    // molecular masses m_k (rho_k = m_k n_k): the weights m_k / tau_k of U in
    // Eq. 8 and the factors tau_k / m_k of the shift in Eq. 7, in FP64 on the host
    double mA, mB, mitauA, mitauB, taumA, taumB;
    // free rest fraction alpha_k of Eqs. 3-5: dA[k][g] = A_g(alpha_k) - w_g for
    // the groups g = rest, axis, diagonal; gen = 0 when both alpha_k are 4/9
    // and both m_k are 1 (the step kernels of the standard model run then)
    double dA[2][3];
    int gen;
    CoefF32 c32;
    double rho_ref[2];        // FP16S shift per species
    double thr;               // precursor threshold rho_bulk / 3
    // initial layout
    int init_kind, row0;      // row0: first row of this run in the row table
    double x_lo, x_hi, cx, cy, r, rho_major, rho_minor;
    const double* init_nA;    // device [ny][nx] (LBM_INIT_FIELDS)
    const double* init_nB;
    double* log;              // device ring [cap][6] of this run, or nullptr
    uint32_t* err;            // the handle's device error word (ERR_* bits)
};

// Fills rd.c32 from the FP64 fields (round to nearest, as a device conversion
// would).  The FP16S shift stays w_g rho_ref for every alpha_k: it is only the
// offset of the stored values, the same in the step and in the mass sums.
#ifndef __CUDACC_RTC__
inline void fill_coef_f32(RunDesc& rd) {
    CoefF32& c = rd.c32;
    c.G = (float)rd.G;
    c.Gw[0] = (float)rd.GwA;
    c.Gw[1] = (float)rd.GwB;
    c.taum[0] = (float)rd.taumA;
    c.taum[1] = (float)rd.taumB;
    c.itau[0] = (float)rd.itauA;
    c.itau[1] = (float)rd.itauB;
    c.mitau[0] = (float)rd.mitauA;
    c.mitau[1] = (float)rd.mitauB;
    c.m[0] = (float)rd.mA;
    c.m[1] = (float)rd.mB;
    c.gx = (float)rd.gx;
    c.gy = (float)rd.gy;
    const float w[3] = {4.0f / 9.0f, 1.0f / 9.0f, 1.0f / 36.0f};
    for (int k = 0; k < 2; ++k)
        for (int g = 0; g < 3; ++g) {
            c.dA[k][g] = (float)rd.dA[k][g];
            c.sh[k][g] = w[g] * (float)rd.rho_ref[k];
        }
}
#endif

// column chunks (CTAs) per row of the mass reduction
constexpr int kMassChunks = 4;

// collided columns per strip of the persistent ring kernel (LBM_KERNEL_RING)
constexpr int kRingWc = 120;

// opt-in shared memory per CTA on sm_103a (227 KB)
constexpr size_t kMaxSmemPerCta = 232448;

// A CTA's work: run, first collided column x0 (the CTA collides
// min(W - 2, nx - x0) columns, W - 8 for the TMA kernel, 2W - 4 for the pair
// kernel), rows [y0, y1).
struct Tile {
    int run, x0, y0, y1;
};

// Velocity output of the moments pass (whole-fluid velocity, Eq. 12 text).
struct MomOut {
    double* ux;
    double* uy;
    int nx;
};

// Shared state of the logging kernels.
struct LogCtl {
    long long* count;   // records written so far (device)
    int cap;            // ring capacity
    int log_every;
};

enum : uint32_t { ERR_NONFINITE = 1u, ERR_TIMEOUT = 2u, ERR_BOUNDS = 4u };   // ERR_BOUNDS: checked builds

#ifndef __CUDACC_RTC__   // host launchers: not part of a run-time compiled step kernel
// Step kernels (one pass of Eq. 2 over every tile) and the moments pass.
// GEN: the runs have some alpha_k != 4/9 or m_k != 1.
template <typename S, bool GEN>
struct Step {
    static cudaError_t step(int W, const RunDesc* d_runs, const Tile* d_tiles, int ntiles, int parity,
                            cudaStream_t s);
    static cudaError_t step_async(int W, int D, const RunDesc* d_runs, const Tile* d_tiles, int ntiles, int parity,
                                  cudaStream_t s);
    static cudaError_t step_tma(int W, int D, const RunDesc* d_runs, const Tile* d_tiles, int ntiles, int parity,
                                uint32_t* err, cudaStream_t s);
    static cudaError_t step_pf(int W, const RunDesc* d_runs, const Tile* d_tiles, int ntiles, int parity,
                               cudaStream_t s);
    static cudaError_t step_split(int W, const RunDesc* d_runs, const Tile* d_tiles, int ntiles, int parity,
                                  cudaStream_t s);
    static cudaError_t step_l2pf(int W, const RunDesc* d_runs, const Tile* d_tiles, int ntiles, int parity,
                                 cudaStream_t s);
    static cudaError_t step_smem(int W, const RunDesc* d_runs, const Tile* d_tiles, int ntiles, int parity,
                                 cudaStream_t s);
    static cudaError_t step_pair(int W, const RunDesc* d_runs, const Tile* d_tiles, int ntiles, int parity,
                                 cudaStream_t s);
    static cudaError_t step_tile(int W, int R, const RunDesc* d_runs, const Tile* d_tiles, int ntiles, int parity,
                                 cudaStream_t s);
    static cudaError_t step_bidir(int W, const RunDesc* d_runs, const Tile* d_tiles, int ntiles, int parity,
                                  cudaStream_t s);
    static cudaError_t moments(int W, const RunDesc* d_runs, const Tile* d_tiles, int ntiles, int parity,
                               MomOut out, cudaStream_t s);
    // persistent ring kernel (FP32 / FP16S storage, D row slots): `grid` CTAs
    // draw the ntiles segments from the counter pair `queue` (zero before the
    // launch, zero again after it)
    static cudaError_t step_ring(int D, const RunDesc* d_runs, const Tile* d_tiles, int ntiles, int* queue, int grid,
                                 int parity, uint32_t* err, cudaStream_t s);
    // resident CTAs per SM of that kernel (0 if not available)
    static cudaError_t ring_ctas_per_sm(int D, int* out);
    // resident CTAs per SM of the bidirectional march with strips of W threads
    static cudaError_t bidir_ctas_per_sm(int W, int* out);
};

// Initialisation, observables, reductions and population transfers.
template <typename S>
struct Launch {
    static cudaError_t init(const RunDesc* d_runs, int nruns, int max_nodes, cudaStream_t s);
    static cudaError_t densities(const RunDesc* d_runs, int run, int parity, int nodes, double* nA,
                                 double* nB, cudaStream_t s);
    static cudaError_t track(const RunDesc* d_runs, int nruns, int max_cap, int parity, int* first, LogCtl lc,
                             double* zout, cudaStream_t s);
    static cudaError_t mass(const RunDesc* d_runs, int nruns, const int2* d_rows, int nrows, int parity,
                            double* d_partials, double* d_mass, LogCtl lc, int write_log, uint32_t* d_err,
                            cudaStream_t s);
    static cudaError_t export_pops(const RunDesc* d_runs, int run, int parity, int nx, int ny, void* out,
                                   cudaStream_t s);
    static cudaError_t import_pops(const RunDesc* d_runs, int run, int parity, int nx, int ny, const void* in,
                                   cudaStream_t s);
    // column window [x0, x0 + ncols) to / from a packed [18][ny][ncols] buffer
    static cudaError_t get_cols(const RunDesc* d_runs, int run, int parity, int ny, int x0, int ncols, void* out,
                                cudaStream_t s);
    static cudaError_t set_cols(const RunDesc* d_runs, int run, int parity, int ny, int x0, int ncols,
                                const void* in, cudaStream_t s);
};

cudaError_t launch_log_advance(LogCtl lc, cudaStream_t s);

extern template struct Launch<double>;
extern template struct Launch<float>;
extern template struct Launch<__half>;
extern template struct Step<double, false>;
extern template struct Step<double, true>;
extern template struct Step<float, false>;
extern template struct Step<float, true>;
extern template struct Step<__half, false>;
extern template struct Step<__half, true>;
#endif

}  // namespace sc
