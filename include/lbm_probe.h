/* Streaming probes of the step's memory access pattern (diagnostic).
 *
 * The paper has no counterpart: these kernels reproduce only the memory
 * traffic of one lattice step (18 population planes read and written per
 * node, FP32) without its arithmetic, so that a measured step time can be
 * set against what the access pattern itself reaches on the GPU.
 *
 * Layout: src and dst are device pointers to 18 planes of ny rows of `pitch`
 * FP32 elements each (plane stride ny * pitch), x fastest; only interior
 * nodes 1 <= x < nx - 1, 1 <= y < ny - 1 are touched, so no index wraps.
 * The caller owns both buffers.
 */
#ifndef LBM_PROBE_H
#define LBM_PROBE_H

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_PROBE_PULL 0  /* one thread per node: loads of F_i(x - c_i), store of every plane at x */
#define LBM_PROBE_COPY 1  /* one thread per node: unshifted copy of the 18 planes */
#define LBM_PROBE_MARCH 2 /* one thread per column marching `rows` rows, pull pattern per row */
#define LBM_PROBE_PULL_BLOCKED 3 /* LBM_PROBE_PULL in a blocked layout: blocks of 32 columns holding all
                                    18 planes contiguously, element (q, y, x) at
                                    ((y (pitch / 32) + x / 32) 18 + q) 32 + x % 32; pitch a multiple of
                                    32, nx >= 66, columns 32 .. nx - 33 */
#define LBM_PROBE_COPY_BLOCKED 4 /* LBM_PROBE_COPY in the blocked layout */

/* Launches one probe pass on `stream` (a cudaStream_t, NULL = default) with
 * CTAs of `block` threads (a multiple of 32, at most 1024) and `smem_bytes`
 * of dynamic shared memory that the kernel does not use: it only limits the
 * CTAs resident per SM (0 .. 227 KB).  Returns 0 on success, 1 for invalid
 * arguments (nothing launched), 3 if the launch failed. */
int lbm_probe_stream(int pattern, const float* src, float* dst, int nx, int ny, int pitch, int rows, int block,
                     int smem_bytes, void* stream);

/* Failure-path self-test of the bounded waits (no counterpart in the paper).
 * Launches one CTA that waits, with the same bounded mbarrier wait as the TMA
 * step kernels, on a phase that nothing completes, giving up after `cycles`
 * SM clock cycles (1e3 .. 4e9; the step kernels use 2e9, about 1 s), and
 * reports what the step would: LBM_ETIMEOUT (5) when the wait ran out,
 * LBM_OK if it completed, LBM_EINVAL for a cycle count out of range (nothing
 * launched), LBM_ENOMEM / LBM_ECUDA on CUDA failures.  The kernel faults
 * nothing and leaves the context usable; it synchronises `stream` (a
 * cudaStream_t, NULL = default) and allocates and frees 4 bytes. */
int lbm_selftest_wait_timeout(long long cycles, void* stream);

#ifdef __cplusplus
}
#endif

#endif
