// Internal device-side descriptors and kernel launchers of the Shan-Chen
// D2Q9 library.  Not part of the public ABI (include/lbm.h is).
#pragma once

#include <cuda_fp16.h>

#include "lbm.h"
#include <cuda_runtime.h>
#include <stdint.h>

namespace sc {

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
    double rho_ref[2];        // FP16S shift per species
    double thr;               // precursor threshold rho_bulk / 3
    // initial layout
    int init_kind, row0;      // row0: first row of this run in the row table
    double x_lo, x_hi, cx, cy, r, rho_major, rho_minor;
    const double* init_nA;    // device [ny][nx] (LBM_INIT_FIELDS)
    const double* init_nB;
    double* log;              // device ring [cap][6] of this run, or nullptr
};

// column chunks (CTAs) per row of the mass reduction
constexpr int kMassChunks = 4;

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

enum : uint32_t { ERR_NONFINITE = 1u, ERR_TIMEOUT = 2u };

template <typename S>
struct Launch {
    static cudaError_t init(const RunDesc* d_runs, int nruns, int max_nodes, cudaStream_t s);
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
};

cudaError_t launch_log_advance(LogCtl lc, cudaStream_t s);

extern template struct Launch<double>;
extern template struct Launch<float>;
extern template struct Launch<__half>;

}  // namespace sc
