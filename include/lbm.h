/*
 * lbm.h - C ABI of the GB300 binary Shan-Chen D2Q9 capillary library.
 *
 * The library advances the two-component (binary, immiscible) pseudo-
 * potential lattice Boltzmann model of S. Chibbaro, "Capillary filling with
 * pseudo-potential binary Lattice-Boltzmann model":
 *   - per-component BGK equation, Eq. 2 (eq:lbe), Delta t = 1;
 *   - D2Q9 equilibrium, Eqs. 3-5, with rest fraction alpha_k and molecular
 *     mass m_k per species (rho_k = m_k n_k); the defaults alpha_k = 4/9,
 *     m_k = 1 give the standard D2Q9 weights (lbm_options.alpha and
 *     molecular_mass);
 *   - equilibrium-velocity shift rho_k u_k^eq = rho_k U + tau_k F_k, Eq. 7,
 *     with the common velocity U of Eq. 8 (sum over the species);
 *   - bulk force of Eq. 9 with Psi_k = n_k and the coupling written with the
 *     D2Q9 weights w_i (4/9, 1/9, 1/36): F_k = -G n_k sum_i w_i n_kbar(x+c_i) c_i,
 *     i.e. G = 9 g of Eq. 10;
 *   - wall force of Eq. 11 with the same weights:
 *     F_k^w = -G_kw n_k sum_i w_i s(x+c_i) c_i, s = 1 on solid nodes.
 *     Positive couplings repel, negative couplings attract (Numerical
 *     Results section, the two equivalent wetting schemes);
 *   - geometry of Fig. 1: periodic in x and y; two plates of one solid row
 *     each span the capillary; half-way bounce-back fused into the pull;
 *   - interface observables of the Numerical Results section and Figs. 6-8:
 *     the bulk front where phi = (n_A - n_B)/(n_A + n_B) changes sign on the
 *     centre row(s), and the precursor film where n_A falls below
 *     rho_bulk/3 on the fluid rows next to each plate.
 *
 * Species A (index 0) is the invading liquid, species B (index 1) the gas.
 * Lattice units throughout (Delta x = Delta t = 1).
 *
 * Conventions for every call:
 *   - Return value: LBM_OK (0) or a positive LBM_E* code; no exception
 *     crosses the ABI.  Errors raised by kernels (non-finite mass, timeout,
 *     and in checked builds an index outside the buffers) are sticky and
 *     reported by the next synchronising call.
 *   - All work is issued on the stream given in lbm_options at creation
 *     (NULL = the legacy default stream) and is asynchronous unless the
 *     call says it synchronises.
 *   - "host" buffers are ordinary CPU memory; "device" buffers are CUDA
 *     device pointers of the current device.  The caller owns every buffer
 *     it passes; the library owns the device state behind an lbm_t.
 *   - A handle is not thread-safe: one host thread at a time.
 */
#ifndef SHANCHEN_GB300_LBM_H
#define SHANCHEN_GB300_LBM_H

#ifdef __CUDACC_RTC__
/* run-time compilation of the step kernel (NVRTC has no C library headers) */
typedef decltype(sizeof(0)) size_t;
typedef signed char int8_t;
typedef short int16_t;
typedef int int32_t;
typedef long long int64_t;
typedef unsigned char uint8_t;
typedef unsigned short uint16_t;
typedef unsigned int uint32_t;
typedef unsigned long long uint64_t;
#else
#include <stddef.h>
#include <stdint.h>
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define LBM_OK 0
#define LBM_EINVAL 1      /* bad argument: tau <= 1/2, non-finite coupling, bad geometry, bad run index */
#define LBM_ENOMEM 2      /* device allocation failed (library allocator or caller callback) */
#define LBM_ECUDA 3       /* a CUDA runtime call failed (no device, launch error, ...) */
#define LBM_ENONFINITE 4  /* a mass sum came out NaN or infinite: the run has diverged */
#define LBM_ETIMEOUT 5    /* a bounded device wait gave up */
#define LBM_ESTATE 6      /* the call needs state the handle does not have (no log, t = 0, ...) */
#define LBM_EIO 7         /* checkpoint file could not be written or read, or is malformed */
#define LBM_EBOUNDS 8     /* checked builds (-DLBM_CHECKED) only: a kernel found a tile or row outside
                             its run's buffers and skipped every access of it */

/* ---- storage precision of the populations ------------------------------- */
#define LBM_F64 0   /* FP64 populations and FP64 arithmetic */
#define LBM_F32 1   /* FP32 populations and FP32 arithmetic */
#define LBM_F16S 2  /* FP16 storage of f_i - w_i rho_ref,k, FP32 arithmetic */

/* ---- initial layout ------------------------------------------------------ */
#define LBM_INIT_SLAB 0     /* liquid A on columns [x_lo, x_hi), gas B elsewhere */
#define LBM_INIT_DROPLET 1  /* liquid A inside the disc |x - (cx, cy)| < r */
#define LBM_INIT_FIELDS 2   /* caller-given host densities init_nA / init_nB */

typedef struct lbm_s lbm_t;

/* Geometry of one run (Numerical Results section, Fig. 1).
 * nx, ny      lattice size, x fastest; periodic in x and y; nx, ny >= 1.
 * cap_x0/x1   the plates cover columns [cap_x0, cap_x1), 0 <= cap_x0 <= cap_x1 <= nx.
 * y_bot/y_top the two solid plate rows, or -1 for no plate.  The capillary
 *             height is H = y_top - y_bot - 1 fluid rows.
 * solid_mask  optional host uint8 [ny][nx]; non-zero = solid.  Replaces the
 *             plates for the force, the bounce-back and the tracking rows
 *             (the tracking rows still follow y_bot/y_top).  Copied at create.
 * init_*      initial layout; the state starts at rest in equilibrium
 *             (f_i = A_i(alpha_k) n_k, = w_i n_k at alpha_k = 4/9), solid
 *             nodes carry no fluid.  Liquid nodes get
 *             (n_A, n_B) = (rho_major, rho_minor), gas nodes the reverse.
 *             init_nA / init_nB (LBM_INIT_FIELDS) are host [ny][nx] arrays,
 *             copied at create. */
typedef struct lbm_geometry {
    int32_t nx, ny;
    int32_t cap_x0, cap_x1;
    int32_t y_bot, y_top;
    int32_t init_kind;
    int32_t reserved0;
    const uint8_t* solid_mask;
    double x_lo, x_hi;
    double drop_cx, drop_cy, drop_r;
    double rho_major, rho_minor;
    const double* init_nA;
    const double* init_nB;
} lbm_geometry;

/* Device allocator supplied by the caller (for instance a framework's
 * caching allocator).  alloc returns NULL on failure. */
typedef void* (*lbm_alloc_fn)(void* ctx, size_t bytes, void* stream);
typedef void (*lbm_free_fn)(void* ctx, void* ptr, size_t bytes, void* stream);

/* Options shared by all runs of a handle.  Fill with lbm_default_options.
 * precision     LBM_F64 / LBM_F32 / LBM_F16S.
 * log_every     record (t, z_bulk, z_prec_bottom, z_prec_top, M_A, M_B) every
 *               log_every steps, including t = 0; 0 = no log.
 * log_capacity  records kept per run (a ring: the newest log_capacity).
 * autotune      1 = time the candidate tilings during the first lbm_step
 *               call long enough for them (every candidate for 6 steps,
 *               the 4 fastest again in 3 rounds of 32; about 1250 steps
 *               on a large grid) and keep the fastest.  The candidates
 *               include, for the bidirectional march, the tile heights whose
 *               tiles fill one or two waves of resident CTAs, and for a
 *               handle of one run LBM_KERNEL_BIDIR_JIT at those heights
 *               (compiled once per grid and strip width, about 0.5 s each,
 *               where NVRTC is available; left out otherwise).  These are
 *               real steps: tilings change only the schedule, and results
 *               are bit-identical for every tiling.
 * tile_w        CTA width (64, 128 or 256 threads; 0 = default 128);
 * tile_h        rows marched per CTA (0 = default 4, clamped to ny).
 *               The step kernel starts as LBM_KERNEL_SMEM where it takes the
 *               tiling (else LBM_KERNEL_REGISTER); autotune or
 *               lbm_set_schedule change it.
 * graph_chunk   steps captured per CUDA graph when the log is off (0 = 64;
 *               -1 = launch every step directly).
 * rho_ref       FP16S shift per species (ignored otherwise).
 * rho_bulk      base of the precursor threshold rho_bulk / 3 (0 = 2.0).
 * body          constant body force per particle, added to F_k / n_k of
 *               both species (an acceleration when m_k = 1; species k then
 *               accelerates by body / m_k).  Drives the Poiseuille check; 0
 *               for capillary filling.
 * alloc/free    optional device allocator; NULL = cudaMallocAsync on stream.
 * stream        cudaStream_t of all work; NULL = legacy default stream.
 * alpha         rest fraction alpha_k of each species' equilibrium (Model
 *               section, Eqs. 3-5): f_0^eq carries alpha n, the axis and
 *               diagonal directions (1 - alpha)/5 and (1 - alpha)/20 of n,
 *               sound speed c_s^2 = 3 (1 - alpha)/5.  0 <= alpha < 1;
 *               default 4/9 (the standard D2Q9 weights, c_s^2 = 1/3).
 * molecular_mass  m_k > 0 of each species (rho_k = m_k n_k, Model section):
 *               enters the common velocity of Eq. 8 as the weights m_k/tau_k,
 *               the shift of Eq. 7 as tau_k/m_k, and the whole-fluid
 *               velocity of lbm_velocity as sum m_k j_k over sum m_k n_k.
 *               Default 1.  alpha = 4/9 and m = 1 give the same bits as a
 *               handle built without these fields.
 * A zeroed structure is not valid (molecular_mass = 0): start from
 * lbm_default_options. */
typedef struct lbm_options {
    int32_t precision;
    int32_t log_every;
    int32_t log_capacity;
    int32_t autotune;
    int32_t tile_w;
    int32_t tile_h;
    int32_t graph_chunk;
    int32_t reserved0;
    double rho_ref[2];
    double rho_bulk;
    double body[2];
    lbm_alloc_fn alloc;
    lbm_free_fn free;
    void* alloc_ctx;
    void* stream;
    double alpha[2];
    double molecular_mass[2];
} lbm_options;

/* Description of one run's device storage (for callers that read the raw
 * populations).  Populations of buffer b live at
 *   base[b] + ((k * 9 + i) * ny + y) * pitch + x      (elements)
 * for species k (0 = A, 1 = B), direction i of Eq. 6 in the order
 * 0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1) 5:(1,1) 6:(-1,1) 7:(-1,-1) 8:(1,-1),
 * 0 <= x < nx.  Each row also stores the periodic images of columns nx - 1
 * and 0 at x = -1 and x = nx (ghost columns); a row starts LBM_COL0 elements
 * before base + row offset.  current is the buffer holding the
 * post-collision populations of time t. */
#define LBM_COL0 8
typedef struct lbm_run_info {
    int32_t nx, ny, pitch, precision;
    int32_t current;
    int32_t elem_bytes;
    int64_t time;
    void* base[2];
} lbm_run_info;

/* Fills opt with the defaults documented above (FP32, no log, tile 128x4,
 * alpha 4/9, molecular mass 1). */
void lbm_default_options(lbm_options* opt);

/* Creates one run (Model section: Eqs. 2-11 with the given couplings).
 * G_AB    cross-species coupling G (w_i-weighted, = 9 g of Eq. 10), finite.
 * wall    {G_Aw, G_Bw}: wall couplings g_kw rho_w of Eq. 11 in w_i units.
 * tau_A/B relaxation times of Eq. 2, each > 1/2 (nu_k = (tau_k - 1/2)/3).
 * opt     NULL = defaults.  *out receives the handle (NULL on failure).
 * Validates every argument before touching the GPU; returns LBM_EINVAL,
 * LBM_ENOMEM or LBM_ECUDA.  Allocates 2 buffers x 18 populations x ny x pitch
 * elements plus the log and the reduction scratch; runs the init kernel. */
int lbm_create(const lbm_geometry* g, double G_AB, const double wall[2], double tau_A,
               double tau_B, const lbm_options* opt, lbm_t** out);

/* Creates n independent runs advanced together (one launch per step covers
 * every run).  g, G_AB, tau_A, tau_B have n entries, wall has 2n
 * ({G_Aw, G_Bw} per run).  Runs never exchange data. */
int lbm_create_batch(int n, const lbm_geometry* g, const double* G_AB, const double* wall,
                     const double* tau_A, const double* tau_B, const lbm_options* opt,
                     lbm_t** out);

/* Advances every run by n_steps >= 0 steps of Eq. 2 (asynchronous).  The
 * log, when on, is written at every multiple of log_every.  With autotune
 * on, the first call synchronises while it times the candidate tilings. */
int lbm_step(lbm_t* h, int64_t n_steps);

/* Blocks until the handle's stream is idle; returns the sticky status. */
int lbm_sync(lbm_t* h);

/* Time t (steps taken) of the handle.  Host-side counter, no sync. */
int64_t lbm_time(const lbm_t* h);

/* Number of runs in the handle. */
int lbm_num_runs(const lbm_t* h);

/* Storage description of run `run` (see lbm_run_info).  No sync. */
int lbm_run_info_get(const lbm_t* h, int run, lbm_run_info* info);

/* Component densities n_k = sum_i f_i^k at time t (Model section, below
 * Eq. 6; the collision conserves n_k, so this is the density of the streamed
 * state of the last step).  nA, nB: [ny][nx] FP64, solid nodes 0.
 * on_device = 1: device pointers, asynchronous.  on_device = 0: host
 * pointers, the call synchronises. */
int lbm_densities(lbm_t* h, int run, double* nA, double* nB, int on_device);

/* Whole-fluid velocity at time t >= 1 (Model section, below Eq. 12):
 * rho u = sum_k m_k j_k + (1/2) sum_k F_k, rho = sum_k m_k n_k, with the
 * streamed populations and the forces of the last step.  ux, uy: [ny][nx]
 * FP64, solid nodes 0.
 * At t = 0 the fluid is at rest and zeros are written.  on_device as above. */
int lbm_velocity(lbm_t* h, int run, double* ux, double* uy, int on_device);

/* Front positions at time t, measured from cap_x0 (Numerical Results
 * section, Figs. 6-8).  z_bulk: phi = 0 crossing on the centre row (odd H)
 * or the mean over the two centre rows (even H).  z_prec[0], z_prec[1]:
 * first column from the inlet where n_A < rho_bulk/3 on the fluid row next
 * to the bottom / top plate.  Each front is linearly interpolated between
 * the last passing and the first failing column; a row with no failing
 * column reports the capillary length.  Host outputs; synchronises.
 * LBM_ESTATE if the run has no capillary (a plate missing). */
int lbm_interface_positions(lbm_t* h, int run, double* z_bulk, double z_prec[2]);

/* Copies the log ring of run `run` to host rec[capacity][6] (oldest first):
 * (t, z_bulk, z_prec_bottom, z_prec_top, M_A, M_B).  *n_rec receives the
 * number of records copied.  Synchronises.  LBM_ESTATE if the log is off. */
int lbm_get_log(lbm_t* h, int run, double* rec, int capacity, int* n_rec);

/* Per-species mass M_k = sum over fluid nodes and i of f_i^k, summed in
 * FP64 in a fixed order (deterministic).  The collision and the streaming
 * with bounce-back conserve it (Numerical Results section: periodic sides
 * for total mass conservation).  With molecular masses m_k != 1 this is the
 * number of particles of species k; its mass is m_k M_k.  Host output M[2];
 * synchronises.  Sets and returns LBM_ENONFINITE if a sum is NaN or
 * infinite. */
int lbm_mass(lbm_t* h, int run, double M[2]);

/* Copies the populations of time t of run `run` (storage precision, layout
 * [2][9][ny][nx], FP16S values as stored, i.e. f - w_i rho_ref) into out.
 * on_device as in lbm_densities. */
int lbm_populations(lbm_t* h, int run, void* out, int on_device);

/* Column windows of the populations of time t of run `run`, for the x-slab
 * decomposition of one capillary over several lattices (a run too long for
 * one GPU; the paper's Introduction notes that the lattice Boltzmann method
 * parallelises naturally).  lbm_get_columns copies columns
 * [x0, x0 + ncols) of all 18 populations and all rows into buf
 * [2][9][ny][ncols] (storage precision, FP16S values as stored);
 * lbm_set_columns overwrites those columns from buf (and the periodic images
 * of columns 0, 1, nx - 2, nx - 1 that the ring kernels read), so that the
 * next step pulls them.  A slab of width w owned columns is run as a
 * lattice of w + 4 columns whose outer two columns on each side are set,
 * after every step, to the neighbours' edge columns: every owned column then
 * gets exactly the inputs it has in the undivided lattice (the pull reaches
 * one column, the densities of the force one more).  0 <= x0,
 * x0 + ncols <= nx, ncols >= 1 (LBM_EINVAL otherwise).  on_device as in
 * lbm_densities (host buffers: the call synchronises). */
int lbm_get_columns(lbm_t* h, int run, int x0, int ncols, void* buf, int on_device);
int lbm_set_columns(lbm_t* h, int run, int x0, int ncols, const void* buf, int on_device);

/* Tiling in use (CTA width, rows per CTA). */
int lbm_get_tiling(const lbm_t* h, int* tile_w, int* tile_h);

/* Selects a tiling (tile_w in {64,128,256}, tile_h >= 1) for the current step
 * kernel, or with the register kernel (LBM_KERNEL_REGISTER) if the current
 * kernel does not take that tiling.  Results do not depend on it. */
int lbm_set_tiling(lbm_t* h, int tile_w, int tile_h);

/* Full schedule of the step kernel: tiling (tile_w, tile_h) plus the kernel
 * variant and its depth.  Every variant computes the same bits for a given
 * precision; they differ in how the pulled populations reach the collision:
 *   LBM_KERNEL_REGISTER   through registers (tile_w in {64,128,256});
 *   LBM_KERNEL_ASYNC      through a depth-stage cp.async ring in shared memory
 *                         (depth 3 or 4; not for LBM_F16S);
 *   LBM_KERNEL_TMA        through a ring of `depth` row slots (4, 6 or 8)
 *                         filled by bulk copies with mbarrier completion;
 *                         tile_w - 8 columns per CTA; the ring must fit in
 *                         227 KB of shared memory; nx >= 4;
 *   LBM_KERNEL_PIPELINED  parked in shared memory, with the loads of the row
 *                         after next in flight during the collision (tile_w
 *                         <= 128, FP64 <= 64);
 *   LBM_KERNEL_SPLIT      one thread per species and node;
 *   LBM_KERNEL_PREFETCH   through registers, rows prefetched into L2;
 *   LBM_KERNEL_SMEM       parked in shared memory (the default; FP64 tile_w <= 128);
 *   LBM_KERNEL_PAIR       two columns per thread (tile_w <= 128, FP64 64; nx >= 4);
 *   LBM_KERNEL_TILE       one node per thread over tile_w x (tile_h + 2)
 *                         threads (tile_w in {32, 64}, tile_h in {6, 14, 30},
 *                         at most 1024 threads; nx >= 4);
 *   LBM_KERNEL_BIDIR      parked in shared memory, two groups of tile_w
 *                         threads marching away from the tile's middle row,
 *                         each at barriers of its own after the first rows
 *                         (tile_w in {64, 128}, FP64 64);
 *   LBM_KERNEL_RING       a persistent grid of warp-specialised CTAs: one
 *                         producer warp streams the source rows of a strip
 *                         of 120 columns into a ring of `depth` row slots
 *                         (3, 4 or 5) by bulk copies with mbarrier
 *                         completion, two consumer warps collide two columns
 *                         per thread in packed FP32; the CTAs draw row
 *                         segments of the strips from a device counter.
 *                         LBM_F32 and LBM_F16S only; tile_w must be 128 (the
 *                         segment height is chosen by the library, tile_h is
 *                         only recorded); nx >= 4;
 *   LBM_KERNEL_BIDIR_JIT  LBM_KERNEL_BIDIR compiled by NVRTC when the
 *                         schedule is set, with the run's nx, ny, pitch and
 *                         plane as constants, so that every load and store
 *                         addresses its plane and row by an immediate offset
 *                         (same tilings as LBM_KERNEL_BIDIR; handles of one
 *                         run only).  The compiled kernel is cached for the
 *                         process; setting the schedule returns LBM_ECUDA if
 *                         the run-time compiler or the module load fails,
 *                         and the handle then keeps its previous schedule.
 * depth is read by LBM_KERNEL_ASYNC, LBM_KERNEL_TMA and LBM_KERNEL_RING and
 * must be 4 for the others.  lbm_set_schedule returns LBM_EINVAL for an unsupported
 * combination, leaving the schedule unchanged. */
#define LBM_KERNEL_REGISTER 0
#define LBM_KERNEL_ASYNC 1
#define LBM_KERNEL_TMA 2
#define LBM_KERNEL_PIPELINED 3   /* register pull, the next row's loads issued before the collision */
#define LBM_KERNEL_SPLIT 4       /* one thread per species and node (2 tile_w threads per CTA) */
#define LBM_KERNEL_PREFETCH 5    /* register pull, rows streamed into L2 ahead by bulk prefetches */
#define LBM_KERNEL_SMEM 6        /* register pull, pulled rows parked in shared memory: 64 registers */
#define LBM_KERNEL_PAIR 7        /* two columns per thread, vector loads and stores; nx >= 4 */
#define LBM_KERNEL_TILE 8        /* one node per thread, W x (R + 2) tiles: W in {32, 64}, R in {6, 14, 30}
                                    (W = 64: R in {6, 14}); nx >= 4 */
#define LBM_KERNEL_BIDIR 9       /* two thread groups marching away from the tile's middle row */
#define LBM_KERNEL_RING 10       /* persistent producer/consumer ring of bulk-copied row slots (FP32, FP16S) */
#define LBM_KERNEL_BIDIR_JIT 11  /* LBM_KERNEL_BIDIR compiled at run time for the handle's grid (one run) */
int lbm_get_schedule(const lbm_t* h, int* tile_w, int* tile_h, int* kernel, int* depth);
/* The autotuner's finalists (the paper has no counterpart: this reports on the
 * library's own schedule search).  *count = number of finalists (0 before
 * tuning has run); the first min(max, *count) are written: sched[4 j ..
 * 4 j + 3] = (tile_w, tile_h, kernel, depth) of finalist j, ms_per_step[j] =
 * its best per-step time over the final rounds, measured on back-to-back
 * steps.  Host memory, caller-owned; no device work.  LBM_EINVAL for a null
 * handle or count, or max > 0 with a null array. */
int lbm_get_tuning(const lbm_t* h, int max, int* sched, float* ms_per_step, int* count);
int lbm_set_schedule(lbm_t* h, int tile_w, int tile_h, int kernel, int depth);

/* Writes a checkpoint (header, parameters, populations of time t, log) to
 * path; lbm_load re-creates the handle so that stepping on gives results
 * bit-identical to an uninterrupted run.  Both synchronise.  LBM_EIO on
 * file errors.  The file keeps alpha and molecular_mass (format version 2);
 * version 1 files load with the defaults 4/9 and 1. */
int lbm_save(lbm_t* h, const char* path);
int lbm_load(const char* path, const lbm_options* opt, lbm_t** out);

/* Per-species FP64 mass of one population buffer, computed without
 * allocating any memory.  The paper has no counterpart: this is plumbing for
 * callers that cannot allocate device memory at the point where they need
 * the sums, for instance a callback of a caching allocator that must not
 * re-enter that allocator, or a process whose device memory is entirely
 * reserved by another framework's pool (a cudaMalloc there would fail or
 * fragment the pool).  It computes the per-row sums and the final FP64 tree
 * of lbm_mass from a caller-owned buffer instead of a handle; rows are summed
 * by one CTA each instead of lbm_mass's four column chunks, so the two agree
 * to rounding, not bit for bit.
 *
 * g           geometry of the run: nx, ny, the plates (cap_x0, cap_x1, y_bot,
 *             y_top); solid_mask must be NULL (LBM_EINVAL otherwise); the
 *             init fields are ignored.
 * precision   LBM_F64 / LBM_F32 / LBM_F16S: element type of populations.
 * populations device buffer [2][9][ny][pitch] in the layout of lbm_run_info,
 *             pointing at column 0 of row 0 (for a handle:
 *             lbm_run_info.base[current]); pitch >= nx (only columns
 *             0 <= x < nx are read).
 * rho_ref     FP16S shift per species (NULL = 0); ignored otherwise.
 * mass        device double[2] receiving (M_A, M_B); caller-owned.
 * stream      cudaStream_t of the work (NULL = legacy default stream).
 *
 * Limits (LBM_EINVAL beyond them, checked before anything is launched):
 * ny <= LBM_NOALLOC_MAX_ROWS rows, and 18 * ny * pitch < 2^31 elements (the
 * kernels index one buffer with 32-bit element offsets; lbm_create applies
 * the same bound).  The per-row partial sums live in one fixed device array
 * of 2 * LBM_NOALLOC_MAX_ROWS doubles (1 MiB) that every GPU loading the
 * library holds until the process exits.  All calls on a device share that
 * array: calls whose work overlaps on the GPU (different streams, or
 * concurrent host threads) race and must be serialised by the caller; a call
 * writes every row sum it reads before reading it, so nothing carries over
 * from one call to the next.  The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress); make that first call before
 * any stream capture.  No memory is allocated or freed.  Asynchronous;
 * returns LBM_ECUDA if the look-up or a launch fails. */
#define LBM_NOALLOC_MAX_ROWS 65536
int lbm_mass_noalloc(const lbm_geometry* g, int precision, const void* populations, int pitch,
                     const double rho_ref[2], double* mass, void* stream);

/* Failure-path self-test of the bounded device waits (no counterpart in the
 * paper).  Launches one CTA that waits, with the same bounded mbarrier wait as
 * the ring-fed step kernels, on a phase that nothing completes, giving up
 * after `cycles` SM clock cycles (1e3 .. 4e9; the step kernels use 2e9, about
 * 1 s), and reports what a step would: LBM_ETIMEOUT when the wait ran out,
 * LBM_OK if it completed, LBM_EINVAL for a cycle count out of range (nothing
 * launched), LBM_ENOMEM / LBM_ECUDA on CUDA failures.  The kernel faults
 * nothing and leaves the context usable; it synchronises `stream` (a
 * cudaStream_t, NULL = default) and allocates and frees 4 bytes. */
int lbm_selftest_wait_timeout(long long cycles, void* stream);

/* Measured FP64 fused multiply-add rate of the current device (no
 * counterpart in the paper): a kernel of independent DFMA chains on every SM,
 * timed with CUDA events after one warm-up launch; *flops_per_s receives
 * 2 x DFMAs per second.  The denominator of the FP64 step's arithmetic
 * roofline (the FP64 build is bound by GB300's FP64 pipe, not by HBM).
 * Synchronises `stream`; allocates and frees a few bytes; LBM_ECUDA on
 * CUDA failures. */
int lbm_selftest_fp64_rate(double* flops_per_s, void* stream);

/* Sticky device status of the handle (synchronises). */
int lbm_status(lbm_t* h);

/* Static text for a status code. */
const char* lbm_error_string(int code);

/* Frees every device allocation of the handle on its stream.  NULL is a no-op. */
void lbm_destroy(lbm_t* h);

#ifdef __cplusplus
}
#endif
#endif /* SHANCHEN_GB300_LBM_H */
