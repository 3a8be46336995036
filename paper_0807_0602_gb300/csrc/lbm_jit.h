// Run-time compilation of the bidirectional march for one grid (internal).
#pragma once

namespace sc {

// The bidirectional march (strips of W threads per group, storage precision
// LBM_F64 / LBM_F32 / LBM_F16S, the density-ratio instantiation if gen)
// compiled for a run of exactly nx x ny nodes with the given pitch and plane
// (elements).  *fn receives a kernel handle for cudaLaunchKernel with the
// arguments of k_step_bidir (runs, tiles, parity) and 2 W threads per CTA.
// Compiled once per key and cached for the life of the process (thread
// safe).  LBM_EINVAL for an unsupported combination, LBM_ECUDA if NVRTC or
// the library load fails (jit_last_log() then holds the compiler's log).
int jit_bidir(int precision, int W, bool gen, int nx, int ny, int pitch, long long plane, const void** fn);
const char* jit_last_log();

}  // namespace sc
