// Runtime behind the C ABI of include/lbm.h: handles, device allocation,
// tile tables, CUDA-graph chunks of steps, logging, autotuning, checkpoints.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "lbm.h"
#include "lbm_device.h"
#include "lbm_jit.h"

using sc::RunDesc;
using sc::Tile;

namespace {

struct Alloc {
    void* p;
    size_t bytes;
};

struct GraphKey {
    int parity, steps, log;
    bool operator<(const GraphKey& o) const {
        if (parity != o.parity) return parity < o.parity;
        if (steps != o.steps) return steps < o.steps;
        return log < o.log;
    }
};

}  // namespace

struct lbm_s {
    lbm_options opt;
    int precision = LBM_F32;
    int elem = 4;
    int nruns = 0;
    std::vector<RunDesc> runs;    // host copies (device pointers inside)
    RunDesc* d_runs = nullptr;
    std::vector<Tile> tiles;
    Tile* d_tiles = nullptr;
    size_t d_tiles_cap = 0;
    std::vector<int> tile_begin, tile_count;
    int tile_w = 128, tile_h = 4;
    bool gen = false;              // some alpha_k != 4/9 or m_k != 1 (RunDesc::gen)
    int kvar = 6, depth = 4;       // step kernel (LBM_KERNEL_* of lbm.h): 0 register pull, 1 cp.async
                                   // stages of depth D, 2 TMA ring of D row slots, 3 staged pull with the
                                   // loads of row r + 2 in flight, 4 species split over two threads per
                                   // node, 5 register pull with bulk L2 prefetch of rows ahead, 6 register
                                   // pull with the pulled rows parked in shared memory, 7 two columns per
                                   // thread, 8 one node per thread over a W x (R + 2) tile, 9 two thread
                                   // groups marching away from the tile's middle row, 10 persistent
                                   // producer/consumer ring of row slots filled by bulk copies, 11 the
                                   // bidirectional march compiled at run time for the run's grid
    int* d_queue = nullptr;        // ring kernel: segment counter and finished-CTA counter
    int ring_grid = 0;             // ring kernel: CTAs of the persistent grid
    const void* jit_fn = nullptr;  // kvar 11: the bidirectional march compiled for this run's grid
    std::vector<int2> rows;
    int2* d_rows = nullptr;
    double* d_partials = nullptr;
    double* d_mass = nullptr;
    double* d_zout = nullptr;
    int* d_first = nullptr;        // first failing column of each tracked row (4 per run)
    int track_cap = 0;             // longest capillary among the runs (columns the front scan covers)
    double* d_log = nullptr;
    long long* d_logcount = nullptr;
    uint32_t* d_err = nullptr;
    double* d_scratch = nullptr;   // [2][max_nodes] FP64 for host copies
    void* d_popscratch = nullptr;  // [18][max_nodes] storage type
    int max_nodes = 0;
    int64_t t = 0;
    long long nlog = 0;            // host mirror of the log count
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    std::vector<Alloc> allocs;
    std::map<GraphKey, cudaGraphExec_t> graphs;
    bool tuned = false;
    std::vector<int> tune_sched;   // the tuner's finalists, 4 ints each (tile_w, tile_h, kernel, depth)
    std::vector<float> tune_ms;    // and their best ms per step over the final rounds
    int sticky = LBM_OK;
};

namespace {

const char* kErr[] = {"ok", "invalid argument", "out of device memory", "CUDA error",
                      "non-finite mass (the run diverged)", "device wait timed out",
                      "state not available", "checkpoint I/O error",
                      "index outside the run's buffers (checked build)"};

int cuda_fail(lbm_t* h, cudaError_t e) {
    if (e == cudaSuccess) return LBM_OK;
    if (h) h->sticky = LBM_ECUDA;
    fprintf(stderr, "shanchen: CUDA error %s\n", cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
}
#define CK(h, call)                                  \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return cuda_fail(h, e_); \
    } while (0)

void* dalloc(lbm_t* h, size_t bytes) {
    if (bytes == 0) bytes = 256;
    bytes = (bytes + 255) & ~size_t(255);
    void* p = nullptr;
    if (h->opt.alloc) {
        p = h->opt.alloc(h->opt.alloc_ctx, bytes, h->stream);
    } else if (cudaMallocAsync(&p, bytes, h->stream) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) h->allocs.push_back({p, bytes});
    return p;
}

void dfree_all(lbm_t* h) {
    for (auto& a : h->allocs) {
        if (h->opt.free) h->opt.free(h->opt.alloc_ctx, a.p, a.bytes, h->stream);
        else cudaFreeAsync(a.p, h->stream);
    }
    h->allocs.clear();
}

template <typename F>
cudaError_t dispatch(int precision, F&& f) {
    switch (precision) {
        case LBM_F64: return f(sc::Launch<double>());
        case LBM_F32: return f(sc::Launch<float>());
        default: return f(sc::Launch<__half>());
    }
}

// Step launchers of the handle's precision and species model (gen: some
// alpha_k != 4/9 or m_k != 1).
template <typename F>
cudaError_t dispatch_step(const lbm_t* h, F&& f) {
    switch (h->precision) {
        case LBM_F64: return h->gen ? f(sc::Step<double, true>()) : f(sc::Step<double, false>());
        case LBM_F32: return h->gen ? f(sc::Step<float, true>()) : f(sc::Step<float, false>());
        default: return h->gen ? f(sc::Step<__half, true>()) : f(sc::Step<__half, false>());
    }
}

bool finite(double v) { return std::isfinite(v); }

int round_pitch(int nx);

int validate_geometry(const lbm_geometry& g) {
    if (g.nx < 1 || g.ny < 1) return LBM_EINVAL;
    if ((long long)g.nx * g.ny > (1LL << 31) / 2) return LBM_EINVAL;
    // element indices within one buffer are 32-bit in the step kernels
    if (18LL * g.ny * round_pitch(g.nx) >= (1LL << 31)) return LBM_EINVAL;
    if (g.cap_x0 < 0 || g.cap_x1 < g.cap_x0 || g.cap_x1 > g.nx) return LBM_EINVAL;
    if (g.y_bot < -1 || g.y_bot >= g.ny || g.y_top < -1 || g.y_top >= g.ny) return LBM_EINVAL;
    if (g.init_kind < LBM_INIT_SLAB || g.init_kind > LBM_INIT_FIELDS) return LBM_EINVAL;
    if (g.init_kind == LBM_INIT_FIELDS && (!g.init_nA || !g.init_nB)) return LBM_EINVAL;
    if (!finite(g.x_lo) || !finite(g.x_hi) || !finite(g.drop_cx) || !finite(g.drop_cy) || !finite(g.drop_r))
        return LBM_EINVAL;
    if (!finite(g.rho_major) || !finite(g.rho_minor)) return LBM_EINVAL;
    return LBM_OK;
}

int validate_options(const lbm_options& o) {
    if (o.precision < LBM_F64 || o.precision > LBM_F16S) return LBM_EINVAL;
    if (o.log_every < 0 || (o.log_every > 0 && o.log_capacity < 1)) return LBM_EINVAL;
    if (o.tile_w != 0 && o.tile_w != 64 && o.tile_w != 128 && o.tile_w != 256) return LBM_EINVAL;
    if (o.tile_h < 0) return LBM_EINVAL;
    if (!finite(o.rho_ref[0]) || !finite(o.rho_ref[1]) || !finite(o.rho_bulk) || !finite(o.body[0]) ||
        !finite(o.body[1]))
        return LBM_EINVAL;
    if ((o.alloc == nullptr) != (o.free == nullptr)) return LBM_EINVAL;
    for (int k = 0; k < 2; ++k) {
        // Eqs. 3-5 need 0 <= alpha < 1 (positive moving weights); rho_k = m_k n_k needs m_k > 0
        if (!finite(o.alpha[k]) || !(o.alpha[k] >= 0.0) || !(o.alpha[k] < 1.0)) return LBM_EINVAL;
        if (!finite(o.molecular_mass[k]) || !(o.molecular_mass[k] > 0.0)) return LBM_EINVAL;
    }
    return LBM_OK;
}

// Rows hold LBM_COL0 elements before column 0 (ghost image of column nx - 1
// at x = -1) and at least LBM_COL0 after column nx - 1 (image of column 0 at
// x = nx); buffers point at column 0 of row 0.
int round_pitch(int nx) { return (nx + 2 * LBM_COL0 + 63) / 64 * 64; }

// Ring kernel (kvar 10): strips of kRingWc collided columns, cut into
// segments of R rows that the persistent CTAs draw one by one.  R is chosen
// so that the largest number of segments a CTA may have to take, times the
// rows it pulls per segment (R + 2 with the halo rows), is smallest for a
// grid of about G resident CTAs.
void build_ring_tiles(lbm_t* h, int G) {
    h->tiles.clear();
    h->tile_begin.assign(h->nruns, 0);
    h->tile_count.assign(h->nruns, 0);
    int best_R = 1;
    double best = 1e300;
    for (int R : {4, 6, 8, 10, 12, 16, 20, 24, 32, 40, 48, 64, 96, 128, 192, 256, 384, 512}) {
        double items = 0.0, rows = 0.0;
        for (const RunDesc& rd : h->runs) {
            const int strips = (rd.nx + sc::kRingWc - 1) / sc::kRingWc;
            const int chunks = (rd.ny + R - 1) / R;
            items += (double)strips * chunks;
            rows += (double)strips * (rd.ny + 2.0 * chunks);
        }
        const double per_cta = std::max(std::ceil(items / G) * (R + 2), rows / G);
        if (per_cta < best * (1.0 - 1e-9)) {
            best = per_cta;
            best_R = R;
        }
    }
    for (int r = 0; r < h->nruns; ++r) {
        const RunDesc& rd = h->runs[r];
        h->tile_begin[r] = (int)h->tiles.size();
        for (int x0 = 0; x0 < rd.nx; x0 += sc::kRingWc)
            for (int y0 = 0; y0 < rd.ny; y0 += best_R)
                h->tiles.push_back({r, x0, y0, std::min(y0 + best_R, rd.ny)});
        h->tile_count[r] = (int)h->tiles.size() - h->tile_begin[r];
    }
}

void build_tiles(lbm_t* h, int W, int R) {
    h->tiles.clear();
    h->tile_begin.assign(h->nruns, 0);
    h->tile_count.assign(h->nruns, 0);
    // the TMA kernel collides W - 8 columns from x0 multiple of 8, the others W - 2
    // and the pair kernel 2W - 4 from an even x0
    const int Wc = h->kvar == 2 ? W - 8 : (h->kvar == 7 ? 2 * W - 4 : W - 2);
    // (the tile kernel: W - 2 columns and R rows, R fixed by its thread rows)
    for (int r = 0; r < h->nruns; ++r) {
        const RunDesc& rd = h->runs[r];
        const int Rr = std::max(1, std::min(R, rd.ny));
        h->tile_begin[r] = (int)h->tiles.size();
        for (int y0 = 0; y0 < rd.ny; y0 += Rr)
            for (int x0 = 0; x0 < rd.nx; x0 += Wc) h->tiles.push_back({r, x0, y0, std::min(y0 + Rr, rd.ny)});
        h->tile_count[r] = (int)h->tiles.size() - h->tile_begin[r];
    }
}

void drop_graphs(lbm_t* h) {
    for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
    h->graphs.clear();
}

// Resident CTAs of the ring kernel with depth D on this device (all SMs).
int ring_grid_size(lbm_t* h, int D, int* grid) {
    int per_sm = 0, dev = 0, sms = 0;
    CK(h, dispatch_step(h, [&](auto L) { return L.ring_ctas_per_sm(D, &per_sm); }));
    CK(h, cudaGetDevice(&dev));
    CK(h, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (per_sm < 1 || sms < 1) return LBM_EINVAL;
    *grid = per_sm * sms;
    return LBM_OK;
}

int upload_tiles(lbm_t* h, int W, int R) {
    if (h->kvar == 10) {
        int G = 0;
        int rc = ring_grid_size(h, h->depth, &G);
        if (rc) return rc;
        build_ring_tiles(h, G);
        h->ring_grid = G;
        if (!h->d_queue) {
            h->d_queue = static_cast<int*>(dalloc(h, 2 * sizeof(int)));
            if (!h->d_queue) return LBM_ENOMEM;
            CK(h, cudaMemsetAsync(h->d_queue, 0, 2 * sizeof(int), h->stream));
        }
    } else {
        if (h->kvar == 11) {
            const RunDesc& rd = h->runs[0];
            const void* fn = nullptr;
            const int rc = sc::jit_bidir(h->precision, W, h->gen != 0, rd.nx, rd.ny, rd.pitch, rd.plane, &fn);
            if (rc) return rc;
            h->jit_fn = fn;
        }
        build_tiles(h, W, R);
    }
    const size_t need = h->tiles.size() * sizeof(Tile);
    if (need > h->d_tiles_cap) {
        // the old table may still be in use by queued work: keep it until destroy
        Tile* p = static_cast<Tile*>(dalloc(h, need));
        if (!p) return LBM_ENOMEM;
        h->d_tiles = p;
        h->d_tiles_cap = need;
    }
    CK(h, cudaMemcpyAsync(h->d_tiles, h->tiles.data(), need, cudaMemcpyHostToDevice, h->stream));
    // the copy reads pageable host memory: finish it before the vector changes
    CK(h, cudaStreamSynchronize(h->stream));
    h->tile_w = W;
    h->tile_h = R;
    drop_graphs(h);
    return LBM_OK;
}

sc::LogCtl logctl(lbm_t* h) {
    sc::LogCtl lc;
    lc.count = h->d_logcount;
    lc.cap = h->opt.log_capacity;
    lc.log_every = h->opt.log_every;
    return lc;
}

// Issues one time step on stream s (parity = t & 1 of the step).
cudaError_t issue_step(lbm_t* h, int parity, cudaStream_t s) {
    const int W = h->tile_w, nt = (int)h->tiles.size();
    if (h->kvar == 1)
        return dispatch_step(h,
                             [&](auto L) { return L.step_async(W, h->depth, h->d_runs, h->d_tiles, nt, parity, s); });
    if (h->kvar == 2)
        return dispatch_step(h, [&](auto L) {
            return L.step_tma(W, h->depth, h->d_runs, h->d_tiles, nt, parity, h->d_err, s);
        });
    if (h->kvar == 3)
        return dispatch_step(h, [&](auto L) { return L.step_pf(W, h->d_runs, h->d_tiles, nt, parity, s); });
    if (h->kvar == 4)
        return dispatch_step(h, [&](auto L) { return L.step_split(W, h->d_runs, h->d_tiles, nt, parity, s); });
    if (h->kvar == 5)
        return dispatch_step(h, [&](auto L) { return L.step_l2pf(W, h->d_runs, h->d_tiles, nt, parity, s); });
    if (h->kvar == 6)
        return dispatch_step(h, [&](auto L) { return L.step_smem(W, h->d_runs, h->d_tiles, nt, parity, s); });
    if (h->kvar == 7)
        return dispatch_step(h, [&](auto L) { return L.step_pair(W, h->d_runs, h->d_tiles, nt, parity, s); });
    if (h->kvar == 9)
        return dispatch_step(h, [&](auto L) { return L.step_bidir(W, h->d_runs, h->d_tiles, nt, parity, s); });
    if (h->kvar == 8)
        return dispatch_step(h,
                             [&](auto L) { return L.step_tile(W, h->tile_h, h->d_runs, h->d_tiles, nt, parity, s); });
    if (h->kvar == 10)
        return dispatch_step(h, [&](auto L) {
            return L.step_ring(h->depth, h->d_runs, h->d_tiles, nt, h->d_queue, h->ring_grid, parity, h->d_err, s);
        });
    if (h->kvar == 11) {
        if (nt <= 0) return cudaSuccess;
        const RunDesc* runs = h->d_runs;
        const Tile* tiles = h->d_tiles;
        int par = parity;
        void* args[] = {&runs, &tiles, &par};
        return cudaLaunchKernel(h->jit_fn, dim3(nt), dim3(2 * W), args, 0, s);
    }
    return dispatch_step(h, [&](auto L) { return L.step(W, h->d_runs, h->d_tiles, nt, parity, s); });
}

bool schedule_ok(const lbm_t* h, int W, int R, int kvar, int depth) {
    if (R < 1 || kvar < 0 || kvar > 11) return false;
    if (kvar == 11) {   // the bidirectional march compiled for the grid: one run per handle
        if (h->nruns != 1) return false;
        kvar = 9;
    }
    if (kvar == 10) {
        // ring of `depth` row slots (3, 4 or 5) fed by bulk copies: FP32 and
        // FP16S storage; strips of 120 columns (tile_w 128; the segment height
        // is chosen by the library); the windows rely on two ghost columns
        // each side: nx >= 4
        if (h->precision == LBM_F64 || W != 128 || depth < 3 || depth > 5) return false;
        for (const RunDesc& rd : h->runs)
            if (rd.nx < 4) return false;
        return true;
    }
    if (kvar == 9) {
        // two groups of W threads, each staging 2 rows of 18 W populations
        // statically: W in {64, 128} (FP64: 64)
        if (depth != 4 || (W != 64 && W != 128) || (h->precision == LBM_F64 && W != 64)) return false;
        return true;
    }
    if (kvar == 8) {
        // one node per thread: W x (R + 2) threads, pulls read the ghost columns
        if (!((W == 32 && (R == 6 || R == 14 || R == 30)) || (W == 64 && (R == 6 || R == 14)))) return false;
        if (depth != 4) return false;
        for (const RunDesc& rd : h->runs)
            if (rd.nx < 4) return false;
        return true;
    }
    if (W != 64 && W != 128 && W != 256) return false;
    if (kvar == 1 && (h->precision == LBM_F16S || (depth != 3 && depth != 4))) return false;
    if (kvar != 1 && kvar != 2 && depth != 4) return false;   // depth is read by the ring kernels only
    // the shared-memory-staged kernel keeps 18 W populations per row parity in
    // static shared memory: FP64 at W = 256 would exceed the 48 KB static limit
    if (kvar == 6 && h->precision == LBM_F64 && W == 256) return false;
    // the pipelined kernel stages three rows of 18 W populations statically
    if (kvar == 3 && (W > 128 || (h->precision == LBM_F64 && W > 64))) return false;
    if (kvar == 7) {
        // two columns per thread: 2W columns of staged populations per CTA
        // (W <= 128, FP64 W = 64); pulls read the ghost columns: nx >= 4
        if (W > 128 || (h->precision == LBM_F64 && W > 64)) return false;
        for (const RunDesc& rd : h->runs)
            if (rd.nx < 4) return false;
    }
    if (kvar == 2) {
        // ring of `depth` row slots of 18 windows of W - 8 + 32 / elem columns in
        // dynamic shared memory (at most 227 KB), plus the density ring
        if (depth != 4 && depth != 6 && depth != 8) return false;
        if (W == 256 && depth == 8) return false;
        const size_t e = h->elem, ce = h->precision == LBM_F64 ? 8 : 4;
        const size_t win = (size_t)(W - 8) + 2 * (16 / e);
        if ((size_t)depth * 18 * win * e + 8 * W * ce + 8 * (size_t)depth + 16 > sc::kMaxSmemPerCta) return false;
        // the TMA windows rely on two ghost columns each side: nx >= 4
        for (const RunDesc& rd : h->runs)
            if (rd.nx < 4) return false;
    }
    return true;
}

// Issues the log sequence for the state in buffer `parity`.
cudaError_t issue_log(lbm_t* h, int parity, cudaStream_t s) {
    sc::LogCtl lc = logctl(h);
    cudaError_t e = dispatch(h->precision, [&](auto L) {
        return L.track(h->d_runs, h->nruns, h->track_cap, parity, h->d_first, lc, nullptr, s);
    });
    if (e != cudaSuccess) return e;
    e = dispatch(h->precision, [&](auto L) {
        return L.mass(h->d_runs, h->nruns, h->d_rows, (int)h->rows.size(), parity, h->d_partials, nullptr, lc, 1,
                      h->d_err, s);
    });
    if (e != cudaSuccess) return e;
    return sc::launch_log_advance(lc, s);
}

int get_graph(lbm_t* h, int parity, int steps, int with_log, cudaGraphExec_t* out) {
    GraphKey key{parity, steps, with_log};
    auto it = h->graphs.find(key);
    if (it != h->graphs.end()) {
        *out = it->second;
        return LBM_OK;
    }
    cudaGraph_t g = nullptr;
    CK(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int j = 0; j < steps && e == cudaSuccess; ++j) e = issue_step(h, (parity + j) & 1, h->cap_stream);
    if (e == cudaSuccess && with_log) e = issue_log(h, (parity + steps) & 1, h->cap_stream);
    cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(h, e != cudaSuccess ? e : e2);
    }
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(h, e);
    h->graphs[key] = ex;
    *out = ex;
    return LBM_OK;
}

// NVTX range over a scope (header-only NVTX: a no-op unless a profiler is
// attached), so that traces show step chunks, logs and tuning by name.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Advances by n steps without autotuning.
int advance(lbm_t* h, int64_t n) {
    const int le = h->opt.log_every;
    // graph_chunk: 0 = default 64 steps per graph, > 0 = that many, < 0 = no graphs
    const int chunk = le > 0 ? le : (h->opt.graph_chunk <= 0 ? 64 : h->opt.graph_chunk);
    const bool graphs = h->opt.graph_chunk >= 0;
    while (n > 0) {
        int64_t m;
        if (le > 0) m = std::min<int64_t>(n, le - (h->t % le));
        else m = std::min<int64_t>(n, chunk);
        if (graphs && m == chunk && (le == 0 || h->t % le == 0)) {
            NvtxRange range("lbm graph chunk");
            cudaGraphExec_t ex;
            int rc = get_graph(h, (int)(h->t & 1), chunk, le > 0, &ex);
            if (rc) return rc;
            CK(h, cudaGraphLaunch(ex, h->stream));
            h->t += m;
            if (le > 0) h->nlog += 1;
        } else {
            NvtxRange range("lbm steps");
            for (int64_t j = 0; j < m; ++j) {
                CK(h, issue_step(h, (int)(h->t & 1), h->stream));
                h->t += 1;
            }
            if (le > 0 && h->t % le == 0) {
                CK(h, issue_log(h, (int)(h->t & 1), h->stream));
                h->nlog += 1;
            }
        }
        n -= m;
    }
    return LBM_OK;
}

// Tiles of the bidirectional march with strips of W - 2 columns and R rows.
long long bidir_tiles(const lbm_t* h, int W, int R) {
    long long n = 0;
    for (const RunDesc& rd : h->runs) n += (long long)((rd.nx + W - 3) / (W - 2)) * ((rd.ny + R - 1) / R);
    return n;
}

// Smallest tile height whose bidirectional tiles fit in `waves` waves of
// resident CTAs on this device, or 0 (none, or the occupancy is unknown).
int wave_height(lbm_t* h, int W, int waves) {
    int per_sm = 0, dev = 0, sms = 0;
    if (dispatch_step(h, [&](auto L) { return L.bidir_ctas_per_sm(W, &per_sm); }) != cudaSuccess ||
        cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const long long slots = (long long)waves * per_sm * sms;
    int maxny = 1;
    for (const RunDesc& rd : h->runs) maxny = std::max(maxny, rd.ny);
    if (slots < 1 || bidir_tiles(h, W, maxny) > slots) return 0;
    int lo = 1, hi = maxny;   // bidir_tiles falls as R grows: the first R that fits
    while (lo < hi) {
        const int mid = (lo + hi) / 2;
        if (bidir_tiles(h, W, mid) <= slots) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

// Times candidate tilings on the live state: the steps taken are real steps
// (every tiling computes the same bits), only their schedule differs.
int autotune(lbm_t* h, int64_t* n) {
    struct Cand {
        int W, R, kvar, depth;
    };
    int maxny = 1;
    for (auto& rd : h->runs) maxny = std::max(maxny, rd.ny);
    std::vector<int> Rs = {4, 8, 16, 32};
    if (maxny < 32) Rs.push_back(maxny);
    if (maxny >= 96) Rs.push_back(64);   // tall tiles: the TMA ring fills each tile's slots once
    std::sort(Rs.begin(), Rs.end());
    Rs.erase(std::unique(Rs.begin(), Rs.end()), Rs.end());
    // the variants that have been competitive somewhere; the cp.async and
    // species-split kernels stay selectable by lbm_set_schedule
    std::vector<Cand> cands;
    for (int W : {64, 128, 256})
        for (int R : Rs)
            for (int kvar : {6, 9, 0, 5, 3, 7, 2})
                if (schedule_ok(h, W, R, kvar, 4)) cands.push_back({W, R, kvar, 4});
    // the bidirectional march also with the tile heights whose tiles fill one
    // or two waves of resident CTAs exactly (a partial last wave leaves SMs idle)
    for (int W : {64, 128}) {
        for (int waves : {1, 2}) {
            const int R = wave_height(h, W, waves);
            if (R > 0 && std::find(Rs.begin(), Rs.end(), R) == Rs.end() && schedule_ok(h, W, R, 9, 4))
                cands.push_back({W, R, 9, 4});
        }
    }
    // a single run: the bidirectional march compiled for its grid, at the
    // wave-filling heights (only where the run-time compiler is available)
    if (h->nruns == 1) {
        const RunDesc& rd = h->runs[0];
        for (int W : {64, 128}) {
            const void* fn = nullptr;
            if (!schedule_ok(h, W, 4, 11, 4) ||
                sc::jit_bidir(h->precision, W, h->gen, rd.nx, rd.ny, rd.pitch, rd.plane, &fn) != LBM_OK)
                continue;
            for (int waves : {1, 2}) {
                const int R = wave_height(h, W, waves);
                if (R > 0) cands.push_back({W, R, 11, 4});
            }
        }
    }
    for (int W : {32, 64})
        for (int R : {6, 14})
            if (schedule_ok(h, W, R, 8, 4)) cands.push_back({W, R, 8, 4});
    for (int D : {3, 4, 5})
        if (schedule_ok(h, 128, 4, 10, D)) cands.push_back({128, 4, 10, D});
    // pass 1: every candidate for `per` steps; pass 2: the kFinal fastest in
    // `rounds` interleaved rounds of per_final steps each, scored by their
    // best round (candidates within a few per cent of each other are told
    // apart by the longer timing, and a slow drift of the clock hits every
    // finalist alike)
    const int per = 6, kFinal = 4, per_final = 32, rounds = 3;
    const int64_t need =
        (int64_t)cands.size() * (per + 1) + (int64_t)rounds * kFinal * (per_final + 1);
    if (*n < need) return LBM_OK;  // too short to tune now
    cudaEvent_t e0, e1;
    CK(h, cudaEventCreate(&e0));
    CK(h, cudaEventCreate(&e1));
    const int saved_chunk = h->opt.graph_chunk;
    h->opt.graph_chunk = -1;  // direct launches while timing
    int rc = LBM_OK;
    // time candidate c over `steps` steps (after one untimed step); ms < 0 on error
    auto time_cand = [&](const Cand& c, int steps, float& ms) {
        ms = -1.f;
        h->kvar = c.kvar;
        h->depth = c.depth;
        if ((rc = upload_tiles(h, c.W, c.R))) return;
        if ((rc = advance(h, 1))) return;
        cudaError_t e = cudaEventRecord(e0, h->stream);
        if (e == cudaSuccess && (rc = advance(h, steps))) return;
        if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (e != cudaSuccess) {
            rc = cuda_fail(h, e);
            return;
        }
        ms = t / steps;
        *n -= steps + 1;
    };
    std::vector<std::pair<float, int>> pass1;
    for (int i = 0; i < (int)cands.size() && !rc; ++i) {
        float ms = 0.f;
        time_cand(cands[i], per, ms);
        if (!rc) pass1.push_back({ms, i});
    }
    Cand bw = {h->tile_w, h->tile_h, h->kvar, h->depth};
    h->tune_sched.clear();
    h->tune_ms.clear();
    if (!rc) {
        std::sort(pass1.begin(), pass1.end());
        const int nf = std::min(kFinal, (int)pass1.size());
        std::vector<float> fbest(nf, 1e30f);
        for (int round = 0; round < rounds && !rc; ++round)
            for (int j = 0; j < nf && !rc; ++j) {
                float ms = 0.f;
                time_cand(cands[pass1[j].second], per_final, ms);
                if (!rc) fbest[j] = std::min(fbest[j], ms);
            }
        float best = 1e30f;
        for (int j = 0; j < nf && !rc; ++j) {
            const Cand& c = cands[pass1[j].second];
            h->tune_sched.insert(h->tune_sched.end(), {c.W, c.R, c.kvar, c.depth});
            h->tune_ms.push_back(fbest[j]);
            if (fbest[j] < best) {
                best = fbest[j];
                bw = c;
            }
        }
    }
    h->opt.graph_chunk = saved_chunk;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    h->tuned = true;
    h->kvar = bw.kvar;
    h->depth = bw.depth;
    return upload_tiles(h, bw.W, bw.R);
}

int check_run(const lbm_t* h, int run) {
    if (!h || run < 0 || run >= h->nruns) return LBM_EINVAL;
    return LBM_OK;
}

int read_err(lbm_t* h) {
    uint32_t e = 0;
    CK(h, cudaMemcpyAsync(&e, h->d_err, sizeof(e), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (e & sc::ERR_BOUNDS) h->sticky = LBM_EBOUNDS;
    else if (e & sc::ERR_NONFINITE) h->sticky = LBM_ENONFINITE;
    else if (e & sc::ERR_TIMEOUT) h->sticky = LBM_ETIMEOUT;
    return h->sticky;
}

int create_impl(int n, const lbm_geometry* g, const double* G_AB, const double* wall, const double* tau_A,
                const double* tau_B, const lbm_options* opt_in, lbm_t** out) {
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    if (n < 1 || n > 65535 || !g || !G_AB || !wall || !tau_A || !tau_B) return LBM_EINVAL;
    lbm_options opt;
    lbm_default_options(&opt);
    if (opt_in) opt = *opt_in;
    int rc = validate_options(opt);
    if (rc) return rc;
    for (int r = 0; r < n; ++r) {
        if ((rc = validate_geometry(g[r]))) return rc;
        if (!finite(G_AB[r]) || !finite(wall[2 * r]) || !finite(wall[2 * r + 1])) return LBM_EINVAL;
        if (!finite(tau_A[r]) || !finite(tau_B[r]) || !(tau_A[r] > 0.5) || !(tau_B[r] > 0.5)) return LBM_EINVAL;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ECUDA;
    }
    lbm_t* h = new lbm_s();
    h->opt = opt;
    h->precision = opt.precision;
    h->elem = opt.precision == LBM_F64 ? 8 : (opt.precision == LBM_F32 ? 4 : 2);
    h->nruns = n;
    h->stream = static_cast<cudaStream_t>(opt.stream);
    auto fail = [&](int code) {
        lbm_destroy(h);
        return code;
    };
    if (cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) return fail(LBM_ECUDA);

    // sizes and offsets
    std::vector<size_t> off(n);
    size_t total = 0;
    int nrows = 0;
    for (int r = 0; r < n; ++r) {
        const int pitch = round_pitch(g[r].nx);
        const size_t buf = (size_t)18 * g[r].ny * pitch * h->elem;
        const size_t bufa = (buf + 255) & ~size_t(255);
        off[r] = total;
        total += 2 * bufa;
        nrows += g[r].ny;
        h->max_nodes = std::max(h->max_nodes, g[r].nx * g[r].ny);
    }
    char* arena = static_cast<char*>(dalloc(h, total));
    if (!arena) return fail(LBM_ENOMEM);
    // padding columns are read (never used) by the pair kernel's unneeded
    // halo nodes: keep them defined
    if (cudaMemsetAsync(arena, 0, total, h->stream) != cudaSuccess) return fail(LBM_ECUDA);

    // per-run masks and initial fields
    h->runs.resize(n);
    h->rows.clear();
    std::vector<void*> tmp_fields;
    const double rho_bulk = opt.rho_bulk > 0 ? opt.rho_bulk : 2.0;
    for (int r = 0; r < n; ++r) {
        const lbm_geometry& gr = g[r];
        RunDesc& rd = h->runs[r];
        memset(&rd, 0, sizeof(rd));
        rd.nx = gr.nx;
        rd.ny = gr.ny;
        rd.pitch = round_pitch(gr.nx);
        rd.nodes = gr.nx * gr.ny;
        rd.plane = (long long)gr.ny * rd.pitch;
        const size_t buf = (size_t)18 * gr.ny * rd.pitch * h->elem;
        const size_t bufa = (buf + 255) & ~size_t(255);
        rd.buf[0] = arena + off[r] + (size_t)LBM_COL0 * h->elem;
        rd.buf[1] = arena + off[r] + bufa + (size_t)LBM_COL0 * h->elem;
        rd.cap_x0 = gr.cap_x0;
        rd.cap_x1 = gr.cap_x1;
        rd.y_bot = gr.y_bot;
        rd.y_top = gr.y_top;
        rd.G = G_AB[r];
        rd.GwA = wall[2 * r];
        rd.GwB = wall[2 * r + 1];
        rd.tauA = tau_A[r];
        rd.tauB = tau_B[r];
        rd.itauA = 1.0 / tau_A[r];
        rd.itauB = 1.0 / tau_B[r];
        rd.mA = opt.molecular_mass[0];
        rd.mB = opt.molecular_mass[1];
        rd.mitauA = rd.mA * rd.itauA;
        rd.mitauB = rd.mB * rd.itauB;
        rd.taumA = tau_A[r] / rd.mA;
        rd.taumB = tau_B[r] / rd.mB;
        rd.gen = rd.mA != 1.0 || rd.mB != 1.0;
        for (int k = 0; k < 2; ++k) {
            // A_i(alpha) - w_i of Eqs. 3-5: rest alpha - 4/9, axis (1 - alpha)/5 - 1/9,
            // diagonal (1 - alpha)/20 - 1/36
            const double a = opt.alpha[k];
            const bool dflt = a == 4.0 / 9.0;
            rd.dA[k][0] = dflt ? 0.0 : a - 4.0 / 9.0;
            rd.dA[k][1] = dflt ? 0.0 : (1.0 - a) / 5.0 - 1.0 / 9.0;
            rd.dA[k][2] = dflt ? 0.0 : (1.0 - a) / 20.0 - 1.0 / 36.0;
            if (!dflt) rd.gen = 1;
        }
        h->gen = rd.gen != 0;   // alpha and m are options of the handle: the same for every run
        rd.gx = opt.body[0];
        rd.gy = opt.body[1];
        rd.rho_ref[0] = opt.rho_ref[0];
        rd.rho_ref[1] = opt.rho_ref[1];
        rd.thr = rho_bulk / 3.0;
        sc::fill_coef_f32(rd);
        rd.init_kind = gr.init_kind;
        rd.row0 = (int)h->rows.size();
        rd.x_lo = gr.x_lo;
        rd.x_hi = gr.x_hi;
        rd.cx = gr.drop_cx;
        rd.cy = gr.drop_cy;
        rd.r = gr.drop_r;
        rd.rho_major = gr.rho_major;
        rd.rho_minor = gr.rho_minor;
        for (int y = 0; y < gr.ny; ++y) h->rows.push_back(make_int2(r, y));
        const size_t nn = (size_t)gr.nx * gr.ny;
        if (gr.solid_mask) {
            uint8_t* m = static_cast<uint8_t*>(dalloc(h, nn));
            if (!m) return fail(LBM_ENOMEM);
            if (cudaMemcpyAsync(m, gr.solid_mask, nn, cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
                return fail(LBM_ECUDA);
            rd.mask = m;
        }
        if (gr.init_kind == LBM_INIT_FIELDS) {
            double* f = static_cast<double*>(dalloc(h, 2 * nn * sizeof(double)));
            if (!f) return fail(LBM_ENOMEM);
            if (cudaMemcpyAsync(f, gr.init_nA, nn * sizeof(double), cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
                cudaMemcpyAsync(f + nn, gr.init_nB, nn * sizeof(double), cudaMemcpyHostToDevice, h->stream) !=
                    cudaSuccess)
                return fail(LBM_ECUDA);
            rd.init_nA = f;
            rd.init_nB = f + nn;
        }
    }
    // logging and reductions
    if (opt.log_every > 0) {
        h->d_log = static_cast<double*>(dalloc(h, (size_t)n * opt.log_capacity * 6 * sizeof(double)));
        if (!h->d_log) return fail(LBM_ENOMEM);
        if (cudaMemsetAsync(h->d_log, 0, (size_t)n * opt.log_capacity * 6 * sizeof(double), h->stream) != cudaSuccess)
            return fail(LBM_ECUDA);
        for (int r = 0; r < n; ++r) h->runs[r].log = h->d_log + (size_t)r * opt.log_capacity * 6;
    }
    h->d_logcount = static_cast<long long*>(dalloc(h, sizeof(long long)));
    h->d_err = static_cast<uint32_t*>(dalloc(h, sizeof(uint32_t)));
    h->d_partials = static_cast<double*>(dalloc(h, (size_t)2 * sc::kMassChunks * h->rows.size() * sizeof(double)));
    h->d_mass = static_cast<double*>(dalloc(h, (size_t)2 * n * sizeof(double)));
    h->d_zout = static_cast<double*>(dalloc(h, (size_t)3 * n * sizeof(double)));
    h->d_first = static_cast<int*>(dalloc(h, (size_t)4 * n * sizeof(int)));
    for (const RunDesc& rd : h->runs)
        if (rd.y_bot >= 0 && rd.y_top >= 0 && rd.y_top - rd.y_bot >= 2 && rd.cap_x1 > rd.cap_x0)
            h->track_cap = std::max(h->track_cap, rd.cap_x1 - rd.cap_x0);
    h->d_rows = static_cast<int2*>(dalloc(h, h->rows.size() * sizeof(int2)));
    h->d_runs = static_cast<RunDesc*>(dalloc(h, (size_t)n * sizeof(RunDesc)));
    for (RunDesc& rd : h->runs) rd.err = h->d_err;
    if (!h->d_logcount || !h->d_err || !h->d_partials || !h->d_mass || !h->d_zout || !h->d_first || !h->d_rows ||
        !h->d_runs)
        return fail(LBM_ENOMEM);
    if (cudaMemsetAsync(h->d_logcount, 0, sizeof(long long), h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->d_err, 0, sizeof(uint32_t), h->stream) != cudaSuccess ||
        cudaMemcpyAsync(h->d_rows, h->rows.data(), h->rows.size() * sizeof(int2), cudaMemcpyHostToDevice,
                        h->stream) != cudaSuccess ||
        cudaMemcpyAsync(h->d_runs, h->runs.data(), (size_t)n * sizeof(RunDesc), cudaMemcpyHostToDevice, h->stream) !=
            cudaSuccess)
        return fail(LBM_ECUDA);
    cudaError_t e = dispatch(h->precision, [&](auto L) { return L.init(h->d_runs, n, h->max_nodes, h->stream); });
    if (e != cudaSuccess) return fail(cuda_fail(h, e));
    // the host vectors above were read by async copies from pageable memory
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return fail(LBM_ECUDA);
    const int W = opt.tile_w ? opt.tile_w : 128;
    const int R = opt.tile_h ? opt.tile_h : 4;
    // default kernel: the shared-memory-staged march, or the register march
    // for tilings it does not take
    h->kvar = schedule_ok(h, W, R, 6, 4) ? 6 : 0;
    h->depth = 4;
    if ((rc = upload_tiles(h, W, R))) return fail(rc);
    if (opt.log_every > 0) {
        e = issue_log(h, 0, h->stream);
        if (e != cudaSuccess) return fail(cuda_fail(h, e));
        h->nlog = 1;
    }
    h->tuned = !opt.autotune;
    *out = h;
    return LBM_OK;
}

int fetch_fields(lbm_t* h, int run, double* a, double* b, int on_device, bool velocity) {
    const RunDesc& rd = h->runs[run];
    const size_t nn = (size_t)rd.nodes;
    double* da = a;
    double* db = b;
    if (!on_device) {
        if (!h->d_scratch) {
            h->d_scratch = static_cast<double*>(dalloc(h, 2 * (size_t)h->max_nodes * sizeof(double)));
            if (!h->d_scratch) return LBM_ENOMEM;
        }
        da = h->d_scratch;
        db = h->d_scratch + nn;
    }
    cudaError_t e;
    if (!velocity) {
        e = dispatch(h->precision,
                     [&](auto L) { return L.densities(h->d_runs, run, (int)(h->t & 1), rd.nodes, da, db, h->stream); });
    } else if (h->t == 0) {
        e = cudaMemsetAsync(da, 0, nn * sizeof(double), h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(db, 0, nn * sizeof(double), h->stream);
    } else {
        sc::MomOut mo{da, db, rd.nx};
        const int W = h->tile_w;
        e = dispatch_step(h, [&](auto L) {
            return L.moments(W, h->d_runs, h->d_tiles + h->tile_begin[run], h->tile_count[run], (int)((h->t - 1) & 1),
                             mo, h->stream);
        });
    }
    if (e != cudaSuccess) return cuda_fail(h, e);
    if (!on_device) {
        CK(h, cudaMemcpyAsync(a, da, nn * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaMemcpyAsync(b, db, nn * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
    }
    return LBM_OK;
}

}  // namespace

extern "C" {

void lbm_default_options(lbm_options* opt) {
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->precision = LBM_F32;
    opt->log_every = 0;
    opt->log_capacity = 0;
    opt->autotune = 0;
    opt->tile_w = 128;
    opt->tile_h = 4;
    opt->graph_chunk = 0;
    opt->rho_bulk = 2.0;
    opt->alpha[0] = opt->alpha[1] = 4.0 / 9.0;
    opt->molecular_mass[0] = opt->molecular_mass[1] = 1.0;
}

int lbm_create(const lbm_geometry* g, double G_AB, const double wall[2], double tau_A, double tau_B,
               const lbm_options* opt, lbm_t** out) {
    if (!wall) return LBM_EINVAL;
    return create_impl(1, g, &G_AB, wall, &tau_A, &tau_B, opt, out);
}

int lbm_create_batch(int n, const lbm_geometry* g, const double* G_AB, const double* wall, const double* tau_A,
                     const double* tau_B, const lbm_options* opt, lbm_t** out) {
    return create_impl(n, g, G_AB, wall, tau_A, tau_B, opt, out);
}

int lbm_step(lbm_t* h, int64_t n_steps) {
    if (!h || n_steps < 0) return LBM_EINVAL;
    if (h->sticky) return h->sticky;
    NvtxRange range("lbm_step");
    if (!h->tuned) {
        NvtxRange tune("lbm autotune");
        int rc = autotune(h, &n_steps);
        if (rc) return rc;
    }
    return advance(h, n_steps);
}

int lbm_sync(lbm_t* h) {
    if (!h) return LBM_EINVAL;
    CK(h, cudaStreamSynchronize(h->stream));
    return read_err(h);
}

int64_t lbm_time(const lbm_t* h) { return h ? h->t : -1; }

int lbm_num_runs(const lbm_t* h) { return h ? h->nruns : 0; }

int lbm_run_info_get(const lbm_t* h, int run, lbm_run_info* info) {
    if (check_run(h, run) || !info) return LBM_EINVAL;
    const RunDesc& rd = h->runs[run];
    info->nx = rd.nx;
    info->ny = rd.ny;
    info->pitch = rd.pitch;
    info->precision = h->precision;
    info->current = (int)(h->t & 1);
    info->elem_bytes = h->elem;
    info->time = h->t;
    info->base[0] = rd.buf[0];
    info->base[1] = rd.buf[1];
    return LBM_OK;
}

int lbm_densities(lbm_t* h, int run, double* nA, double* nB, int on_device) {
    if (check_run(h, run) || !nA || !nB) return LBM_EINVAL;
    return fetch_fields(h, run, nA, nB, on_device, false);
}

int lbm_velocity(lbm_t* h, int run, double* ux, double* uy, int on_device) {
    if (check_run(h, run) || !ux || !uy) return LBM_EINVAL;
    return fetch_fields(h, run, ux, uy, on_device, true);
}

int lbm_interface_positions(lbm_t* h, int run, double* z_bulk, double z_prec[2]) {
    if (check_run(h, run) || !z_bulk || !z_prec) return LBM_EINVAL;
    const RunDesc& rd = h->runs[run];
    if (rd.y_bot < 0 || rd.y_top < 0 || rd.y_top - rd.y_bot < 2 || rd.cap_x1 <= rd.cap_x0) return LBM_ESTATE;
    sc::LogCtl lc{nullptr, 1, 0};
    cudaError_t e = dispatch(h->precision, [&](auto L) {
        return L.track(h->d_runs, h->nruns, h->track_cap, (int)(h->t & 1), h->d_first, lc, h->d_zout, h->stream);
    });
    if (e != cudaSuccess) return cuda_fail(h, e);
    double z[3];
    CK(h, cudaMemcpyAsync(z, h->d_zout + 3 * run, sizeof(z), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    *z_bulk = z[0];
    z_prec[0] = z[1];
    z_prec[1] = z[2];
    return LBM_OK;
}

int lbm_get_log(lbm_t* h, int run, double* rec, int capacity, int* n_rec) {
    if (check_run(h, run) || !rec || !n_rec || capacity < 0) return LBM_EINVAL;
    if (h->opt.log_every <= 0) return LBM_ESTATE;
    const int cap = h->opt.log_capacity;
    std::vector<double> ring((size_t)cap * 6);
    long long count = 0;
    CK(h, cudaMemcpyAsync(ring.data(), h->runs[run].log, ring.size() * sizeof(double), cudaMemcpyDeviceToHost,
                          h->stream));
    CK(h, cudaMemcpyAsync(&count, h->d_logcount, sizeof(count), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    const long long have = std::min<long long>(count, cap);
    const long long first = count - have;
    const int ncopy = (int)std::min<long long>(have, capacity);
    for (int j = 0; j < ncopy; ++j) {
        const long long idx = (first + j) % cap;
        memcpy(rec + 6 * (size_t)j, ring.data() + 6 * idx, 6 * sizeof(double));
    }
    *n_rec = ncopy;
    return LBM_OK;
}

int lbm_mass(lbm_t* h, int run, double M[2]) {
    if (check_run(h, run) || !M) return LBM_EINVAL;
    sc::LogCtl lc{nullptr, 1, 0};
    cudaError_t e = dispatch(h->precision, [&](auto L) {
        return L.mass(h->d_runs, h->nruns, h->d_rows, (int)h->rows.size(), (int)(h->t & 1), h->d_partials, h->d_mass,
                      lc, 0, h->d_err, h->stream);
    });
    if (e != cudaSuccess) return cuda_fail(h, e);
    CK(h, cudaMemcpyAsync(M, h->d_mass + 2 * run, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (!std::isfinite(M[0]) || !std::isfinite(M[1])) {
        h->sticky = LBM_ENONFINITE;
        return LBM_ENONFINITE;
    }
    return LBM_OK;
}

int lbm_populations(lbm_t* h, int run, void* out, int on_device) {
    if (check_run(h, run) || !out) return LBM_EINVAL;
    const RunDesc& rd = h->runs[run];
    const size_t bytes = (size_t)18 * rd.nodes * h->elem;
    void* d = out;
    if (!on_device) {
        if (!h->d_popscratch) {
            h->d_popscratch = dalloc(h, (size_t)18 * h->max_nodes * h->elem);
            if (!h->d_popscratch) return LBM_ENOMEM;
        }
        d = h->d_popscratch;
    }
    cudaError_t e = dispatch(h->precision, [&](auto L) {
        return L.export_pops(h->d_runs, run, (int)(h->t & 1), rd.nx, rd.ny, d, h->stream);
    });
    if (e != cudaSuccess) return cuda_fail(h, e);
    if (!on_device) {
        CK(h, cudaMemcpyAsync(out, d, bytes, cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
    }
    return LBM_OK;
}

// Column windows of the current populations (x-slab halo exchange).
static int columns_io(lbm_t* h, int run, int x0, int ncols, void* buf, int on_device, bool write) {
    if (check_run(h, run) || !buf) return LBM_EINVAL;
    const RunDesc& rd = h->runs[run];
    if (x0 < 0 || ncols < 1 || x0 > rd.nx - ncols) return LBM_EINVAL;
    const size_t bytes = (size_t)18 * rd.ny * ncols * h->elem;
    void* d = buf;
    if (!on_device) {
        if (!h->d_popscratch) {
            h->d_popscratch = dalloc(h, (size_t)18 * h->max_nodes * h->elem);
            if (!h->d_popscratch) return LBM_ENOMEM;
        }
        d = h->d_popscratch;
        if (write) CK(h, cudaMemcpyAsync(d, buf, bytes, cudaMemcpyHostToDevice, h->stream));
    }
    const int parity = (int)(h->t & 1);
    cudaError_t e = dispatch(h->precision, [&](auto L) {
        return write ? L.set_cols(h->d_runs, run, parity, rd.ny, x0, ncols, d, h->stream)
                     : L.get_cols(h->d_runs, run, parity, rd.ny, x0, ncols, d, h->stream);
    });
    if (e != cudaSuccess) return cuda_fail(h, e);
    if (!on_device) {
        if (!write) CK(h, cudaMemcpyAsync(buf, d, bytes, cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
    }
    return LBM_OK;
}

int lbm_get_columns(lbm_t* h, int run, int x0, int ncols, void* buf, int on_device) {
    return columns_io(h, run, x0, ncols, buf, on_device, false);
}

int lbm_set_columns(lbm_t* h, int run, int x0, int ncols, const void* buf, int on_device) {
    return columns_io(h, run, x0, ncols, const_cast<void*>(buf), on_device, true);
}

int lbm_get_tiling(const lbm_t* h, int* tile_w, int* tile_h) {
    if (!h || !tile_w || !tile_h) return LBM_EINVAL;
    *tile_w = h->tile_w;
    *tile_h = h->tile_h;
    return LBM_OK;
}

int lbm_set_tiling(lbm_t* h, int tile_w, int tile_h) {
    if (!h) return LBM_EINVAL;
    if (!schedule_ok(h, tile_w, tile_h, h->kvar, h->depth)) {
        // the current kernel does not take this tiling: the register march does
        if (!schedule_ok(h, tile_w, tile_h, 0, 4)) return LBM_EINVAL;
        h->kvar = 0;
        h->depth = 4;
    }
    h->tuned = true;
    return upload_tiles(h, tile_w, tile_h);
}

int lbm_get_schedule(const lbm_t* h, int* tile_w, int* tile_h, int* kernel, int* depth) {
    if (!h || !tile_w || !tile_h || !kernel || !depth) return LBM_EINVAL;
    *tile_w = h->tile_w;
    *tile_h = h->tile_h;
    *kernel = h->kvar;
    *depth = h->depth;
    return LBM_OK;
}

int lbm_get_tuning(const lbm_t* h, int max, int* sched, float* ms_per_step, int* count) {
    if (!h || max < 0 || !count || (max > 0 && (!sched || !ms_per_step))) return LBM_EINVAL;
    const int n = (int)h->tune_ms.size();
    *count = n;
    for (int j = 0; j < n && j < max; ++j) {
        for (int q = 0; q < 4; ++q) sched[4 * j + q] = h->tune_sched[4 * j + q];
        ms_per_step[j] = h->tune_ms[j];
    }
    return LBM_OK;
}

int lbm_set_schedule(lbm_t* h, int tile_w, int tile_h, int kernel, int depth) {
    if (!h || !schedule_ok(h, tile_w, tile_h, kernel, depth)) return LBM_EINVAL;
    if (kernel == 11) {   // compile first: if that fails, the handle keeps its schedule
        const RunDesc& rd = h->runs[0];
        const void* fn = nullptr;
        const int rc = sc::jit_bidir(h->precision, tile_w, h->gen, rd.nx, rd.ny, rd.pitch, rd.plane, &fn);
        if (rc) return rc;
    }
    h->tuned = true;
    h->kvar = kernel;
    h->depth = depth;
    return upload_tiles(h, tile_w, tile_h);
}

namespace {
const char kMagic[8] = {'S', 'C', 'L', 'B', 'M', 'C', 'K', '1'};

struct CkHeader {
    char magic[8];
    int32_t version, precision, nruns, log_every, log_capacity, tile_w, tile_h, reserved;
    int64_t t, nlog;
    double rho_ref[2], rho_bulk, body[2];
};
// version 2 appends the species model after the header
struct CkModel {
    double alpha[2], molecular_mass[2];
};
struct CkRun {
    int32_t nx, ny, cap_x0, cap_x1, y_bot, y_top, has_mask, reserved;
    double G, GwA, GwB, tauA, tauB;
};
}  // namespace

int lbm_save(lbm_t* h, const char* path) {
    if (!h || !path) return LBM_EINVAL;
    CK(h, cudaStreamSynchronize(h->stream));
    FILE* fp = fopen(path, "wb");
    if (!fp) return LBM_EIO;
    CkHeader hd;
    memset(&hd, 0, sizeof(hd));
    memcpy(hd.magic, kMagic, 8);
    hd.version = 2;
    hd.precision = h->precision;
    hd.nruns = h->nruns;
    hd.log_every = h->opt.log_every;
    hd.log_capacity = h->opt.log_capacity;
    hd.tile_w = h->tile_w;
    hd.tile_h = h->tile_h;
    hd.t = h->t;
    hd.nlog = h->nlog;
    hd.rho_ref[0] = h->opt.rho_ref[0];
    hd.rho_ref[1] = h->opt.rho_ref[1];
    hd.rho_bulk = h->runs[0].thr * 3.0;
    hd.body[0] = h->opt.body[0];
    hd.body[1] = h->opt.body[1];
    CkModel md;
    for (int k = 0; k < 2; ++k) {
        md.alpha[k] = h->opt.alpha[k];
        md.molecular_mass[k] = h->opt.molecular_mass[k];
    }
    bool ok = fwrite(&hd, sizeof(hd), 1, fp) == 1 && fwrite(&md, sizeof(md), 1, fp) == 1;
    std::vector<char> pops;
    for (int r = 0; r < h->nruns && ok; ++r) {
        const RunDesc& rd = h->runs[r];
        CkRun cr;
        memset(&cr, 0, sizeof(cr));
        cr.nx = rd.nx; cr.ny = rd.ny; cr.cap_x0 = rd.cap_x0; cr.cap_x1 = rd.cap_x1;
        cr.y_bot = rd.y_bot; cr.y_top = rd.y_top; cr.has_mask = rd.mask != nullptr;
        cr.G = rd.G; cr.GwA = rd.GwA; cr.GwB = rd.GwB; cr.tauA = rd.tauA; cr.tauB = rd.tauB;
        ok = fwrite(&cr, sizeof(cr), 1, fp) == 1;
        if (ok && rd.mask) {
            std::vector<uint8_t> m((size_t)rd.nodes);
            if (cudaMemcpy(m.data(), rd.mask, m.size(), cudaMemcpyDeviceToHost) != cudaSuccess) ok = false;
            else ok = fwrite(m.data(), 1, m.size(), fp) == m.size();
        }
        const size_t bytes = (size_t)18 * rd.nodes * h->elem;
        pops.resize(bytes);
        for (int b = 0; b < 2 && ok; ++b) {
            // buffer t & 1 first (the current state), then the previous one
            const int par = (int)((h->t + b) & 1);
            if (!h->d_popscratch) {
                h->d_popscratch = dalloc(h, (size_t)18 * h->max_nodes * h->elem);
                if (!h->d_popscratch) { fclose(fp); return LBM_ENOMEM; }
            }
            cudaError_t e = dispatch(h->precision, [&](auto L) {
                return L.export_pops(h->d_runs, r, par, rd.nx, rd.ny, h->d_popscratch, h->stream);
            });
            if (e == cudaSuccess) e = cudaMemcpyAsync(pops.data(), h->d_popscratch, bytes, cudaMemcpyDeviceToHost, h->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
            if (e != cudaSuccess) { fclose(fp); return cuda_fail(h, e); }
            ok = fwrite(pops.data(), 1, bytes, fp) == bytes;
        }
        if (ok && h->opt.log_every > 0) {
            std::vector<double> ring((size_t)h->opt.log_capacity * 6);
            if (cudaMemcpy(ring.data(), rd.log, ring.size() * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
                ok = false;
            else ok = fwrite(ring.data(), sizeof(double), ring.size(), fp) == ring.size();
        }
    }
    if (fclose(fp) != 0) ok = false;
    return ok ? LBM_OK : LBM_EIO;
}

int lbm_load(const char* path, const lbm_options* opt_in, lbm_t** out) {
    if (!path || !out) return LBM_EINVAL;
    *out = nullptr;
    FILE* fp = fopen(path, "rb");
    if (!fp) return LBM_EIO;
    CkHeader hd;
    if (fread(&hd, sizeof(hd), 1, fp) != 1 || memcmp(hd.magic, kMagic, 8) != 0 ||
        (hd.version != 1 && hd.version != 2) || hd.nruns < 1 || hd.nruns > 65535) {
        fclose(fp);
        return LBM_EIO;
    }
    CkModel md = {{4.0 / 9.0, 4.0 / 9.0}, {1.0, 1.0}};   // version 1: the alpha = 4/9, m = 1 model
    if (hd.version == 2 && fread(&md, sizeof(md), 1, fp) != 1) {
        fclose(fp);
        return LBM_EIO;
    }
    std::vector<CkRun> crs(hd.nruns);
    std::vector<std::vector<uint8_t>> masks(hd.nruns);
    std::vector<std::vector<char>> pops(hd.nruns);
    std::vector<std::vector<double>> rings(hd.nruns);
    const int elem = hd.precision == LBM_F64 ? 8 : (hd.precision == LBM_F32 ? 4 : 2);
    bool ok = true;
    for (int r = 0; r < hd.nruns && ok; ++r) {
        ok = fread(&crs[r], sizeof(CkRun), 1, fp) == 1;
        if (!ok || crs[r].nx < 1 || crs[r].ny < 1 || (long long)crs[r].nx * crs[r].ny > (1LL << 30)) { ok = false; break; }
        const size_t nn = (size_t)crs[r].nx * crs[r].ny;
        if (crs[r].has_mask) {
            masks[r].resize(nn);
            ok = fread(masks[r].data(), 1, nn, fp) == nn;
        }
        pops[r].resize(2 * 18 * nn * elem);
        if (ok) ok = fread(pops[r].data(), 1, pops[r].size(), fp) == pops[r].size();
        if (ok && hd.log_every > 0) {
            rings[r].resize((size_t)hd.log_capacity * 6);
            ok = fread(rings[r].data(), sizeof(double), rings[r].size(), fp) == rings[r].size();
        }
    }
    fclose(fp);
    if (!ok) return LBM_EIO;
    lbm_options opt;
    lbm_default_options(&opt);
    if (opt_in) opt = *opt_in;
    opt.precision = hd.precision;
    opt.log_every = hd.log_every;
    opt.log_capacity = hd.log_capacity;
    opt.rho_ref[0] = hd.rho_ref[0];
    opt.rho_ref[1] = hd.rho_ref[1];
    opt.rho_bulk = hd.rho_bulk;
    opt.body[0] = hd.body[0];
    opt.body[1] = hd.body[1];
    opt.tile_w = hd.tile_w;
    opt.tile_h = hd.tile_h;
    opt.autotune = 0;
    for (int k = 0; k < 2; ++k) {
        opt.alpha[k] = md.alpha[k];
        opt.molecular_mass[k] = md.molecular_mass[k];
    }
    std::vector<lbm_geometry> g(hd.nruns);
    std::vector<double> G(hd.nruns), wall(2 * hd.nruns), tA(hd.nruns), tB(hd.nruns);
    for (int r = 0; r < hd.nruns; ++r) {
        memset(&g[r], 0, sizeof(lbm_geometry));
        g[r].nx = crs[r].nx; g[r].ny = crs[r].ny; g[r].cap_x0 = crs[r].cap_x0; g[r].cap_x1 = crs[r].cap_x1;
        g[r].y_bot = crs[r].y_bot; g[r].y_top = crs[r].y_top;
        g[r].solid_mask = crs[r].has_mask ? masks[r].data() : nullptr;
        g[r].init_kind = LBM_INIT_SLAB;
        G[r] = crs[r].G; wall[2 * r] = crs[r].GwA; wall[2 * r + 1] = crs[r].GwB; tA[r] = crs[r].tauA; tB[r] = crs[r].tauB;
    }
    // the log of a fresh handle starts with a t = 0 record; it is replaced below
    lbm_t* h = nullptr;
    int rc = create_impl(hd.nruns, g.data(), G.data(), wall.data(), tA.data(), tB.data(), &opt, &h);
    if (rc) return rc;
    h->t = hd.t;
    h->nlog = hd.nlog;
    void* d = dalloc(h, (size_t)18 * h->max_nodes * elem);
    if (!d) { lbm_destroy(h); return LBM_ENOMEM; }
    for (int r = 0; r < hd.nruns; ++r) {
        const RunDesc& rd = h->runs[r];
        const size_t bytes = (size_t)18 * rd.nodes * elem;
        for (int b = 0; b < 2; ++b) {
            const int par = (int)((hd.t + b) & 1);
            cudaError_t e = cudaMemcpyAsync(d, pops[r].data() + b * bytes, bytes, cudaMemcpyHostToDevice, h->stream);
            if (e == cudaSuccess)
                e = dispatch(h->precision, [&](auto L) { return L.import_pops(h->d_runs, r, par, rd.nx, rd.ny, d, h->stream); });
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
            if (e != cudaSuccess) { rc = cuda_fail(h, e); lbm_destroy(h); return rc; }
        }
        if (hd.log_every > 0 &&
            cudaMemcpy(rd.log, rings[r].data(), rings[r].size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
            lbm_destroy(h);
            return LBM_ECUDA;
        }
    }
    long long cnt = hd.nlog;
    if (cudaMemcpy(h->d_logcount, &cnt, sizeof(cnt), cudaMemcpyHostToDevice) != cudaSuccess) {
        lbm_destroy(h);
        return LBM_ECUDA;
    }
    *out = h;
    return LBM_OK;
}

int lbm_status(lbm_t* h) {
    if (!h) return LBM_EINVAL;
    CK(h, cudaStreamSynchronize(h->stream));
    return read_err(h);
}

const char* lbm_error_string(int code) {
    if (code < 0 || code > LBM_EBOUNDS) return "unknown status";
    return kErr[code];
}

void lbm_destroy(lbm_t* h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    drop_graphs(h);
    dfree_all(h);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    cudaStreamSynchronize(h->stream);
    cudaGetLastError();
    delete h;
}

}  // extern "C"
