// Warp-specialised, persistent ring kernel of the step (LBM_KERNEL_RING) for
// FP32 and FP16-shifted storage: Eq. 2 with the forces of Eqs. 9-11 and the
// velocities of Eqs. 7-8, in the canonical order of lbm_kernels.cuh, so it
// produces the same bits as every other FP32 / FP16S step kernel.
//
// Design (sm_103a):
//   - one producer warp per CTA streams, with cp.async.bulk (one lane per
//     population plane), the 18 source-row windows that one pulled row needs
//     into a ring of D slots of shared memory; slot completion is an mbarrier
//     transaction count ("full"), slot reuse waits on a second mbarrier that
//     the consumer warps arrive on ("done").  The HBM reads in flight are the
//     ring's slots: they occupy no registers, and the producer keeps fetching
//     across segment boundaries;
//   - two consumer warps collide a strip of kRingWc = 120 columns, two
//     columns per thread in packed FP32: __ffma2_rn / __fadd2_rn / __fmul2_rn
//     round each component exactly as the scalar operation of node_state()
//     and relax() would, so one instruction serves two nodes;
//   - each consumer warp marches its own 60 columns of the strip (plus two
//     halo columns on each side) with its own 4-row density ring in shared
//     memory, so no barrier couples the warps; densities are formed two rows
//     ahead of the collisions, so that while a warp collides row r (reading
//     the densities of rows r - 1, r, r + 1) it also forms those of row r + 2;
//     the pulled populations of the row being collided are read from its slot
//     into registers first, so the slot is released early;
//   - the grid is persistent and its work dynamic: the producer draws
//     segments (a strip's rows [y0, y1)) from a global counter and tags the
//     first slot of each with the segment, so CTAs that start late or run
//     slowly take fewer segments; the last CTA to finish resets the counter.
// Every mbarrier wait is bounded; a consumer that gives up raises a shared
// abort flag, every waiting thread of the CTA then gives up too, each warp
// leaves as a whole, and the producer drains the copies it issued before the
// CTA exits and records ERR_TIMEOUT.
#pragma once

#include "lbm_kernels.cuh"

namespace sc {


template <typename S, int D>
struct RingGeom {
    static constexpr int NCONS = 64;                      // consumer threads (two warps)
    static constexpr int THREADS = NCONS + 32;            // + the producer warp
    static constexpr int OFF = 16 / (int)sizeof(S);      // window starts OFF columns before x0 (16 bytes)
    static constexpr int WIN = kRingWc + 2 * OFF;        // window width in elements (a 16-byte multiple)
    static constexpr int slot_elems = 18 * WIN;
    static constexpr size_t slot_bytes = (size_t)slot_elems * sizeof(S);
    static constexpr int RCW = 2 * 32 + 4;               // density-ring floats per species and consumer warp
    static constexpr size_t ring_bytes = (size_t)D * slot_bytes;
    static constexpr size_t dens_bytes = (size_t)(NCONS / 32) * 4 * 2 * RCW * sizeof(float);
    static constexpr size_t smem_bytes() {
        return ring_bytes + dens_bytes + 2 * D * sizeof(uint64_t) + D * sizeof(int) + 16;
    }
};

// ---- packed FP32 arithmetic of a column pair ------------------------------------
// Each component is rounded as the scalar operation of Ar<float> would round it:
// sub(a, b) = fma(b, -1, a) (an exact product, one rounding) and the negated
// products of the force use -G, which RN rounds symmetrically.
struct P2 {
    static __device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
    static __device__ __forceinline__ float2 sub(float2 a, float2 b) {
        return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
    }
    static __device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
    static __device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
    static __device__ __forceinline__ float2 dup(float a) { return make_float2(a, a); }
};

// Pulled value pairs of the slot: aligned pair (columns e, e + 1 of the
// window) and the pairs shifted by one column.
template <typename S> struct SlotLd;
template <> struct SlotLd<float> {
    static __device__ __forceinline__ float2 al(const float* p, float) { return *reinterpret_cast<const float2*>(p); }
    static __device__ __forceinline__ float2 un(const float* p, float) { return make_float2(p[0], p[1]); }
};
template <> struct SlotLd<__half> {
    static __device__ __forceinline__ float2 al(const __half* p, float sh) {
        return __fadd2_rn(__half22float2(*reinterpret_cast<const __half2*>(p)), make_float2(sh, sh));
    }
    static __device__ __forceinline__ float2 un(const __half* p, float sh) {
        return __fadd2_rn(make_float2(__half2float(p[0]), __half2float(p[1])), make_float2(sh, sh));
    }
};

// Stores of a pair (both components, or one of them) in the storage type.
template <typename S> struct PairSt;
template <> struct PairSt<float> {
    static __device__ __forceinline__ void both(float* p, float2 v, float) { *reinterpret_cast<float2*>(p) = v; }
    static __device__ __forceinline__ void one(float* p, float v, float) { *p = v; }
};
template <> struct PairSt<__half> {
    static __device__ __forceinline__ void both(__half* p, float2 v, float sh) {
        *reinterpret_cast<__half2*>(p) = __float22half2_rn(__fadd2_rn(v, make_float2(-sh, -sh)));
    }
    static __device__ __forceinline__ void one(__half* p, float v, float sh) { *p = __float2half_rn(__fsub_rn(v, sh)); }
};

__device__ __forceinline__ float lane_of(float2 v, int c) { return c ? v.y : v.x; }
__device__ __forceinline__ void set_lane(float2& v, int c, float x) {
    if (c) v.y = x;
    else v.x = x;
}

// Wall sum of Eq. 11 at one node (the same order as node_state).
__device__ __forceinline__ void wall_sum(unsigned m, float& Wx, float& Wy) {
    using A = Ar<float>;
    using Wc = Wt<float>;
    Wx = 0.f;
    Wy = 0.f;
    if (!m) return;
    if (SOL(m, 0, 1)) Wx = A::add(Wx, Wc::w1);
    if (SOL(m, 1, 0)) Wy = A::add(Wy, Wc::w1);
    if (SOL(m, 0, -1)) Wx = A::sub(Wx, Wc::w1);
    if (SOL(m, -1, 0)) Wy = A::sub(Wy, Wc::w1);
    if (SOL(m, 1, 1)) { Wx = A::add(Wx, Wc::w5); Wy = A::add(Wy, Wc::w5); }
    if (SOL(m, 1, -1)) { Wx = A::sub(Wx, Wc::w5); Wy = A::add(Wy, Wc::w5); }
    if (SOL(m, -1, -1)) { Wx = A::sub(Wx, Wc::w5); Wy = A::sub(Wy, Wc::w5); }
    if (SOL(m, -1, 1)) { Wx = A::add(Wx, Wc::w5); Wy = A::sub(Wy, Wc::w5); }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait that also gives up when another thread of the CTA raised the
// abort flag; the first thread to run out of time raises it.
__device__ __forceinline__ bool ring_wait(uint64_t* bar, unsigned parity, volatile int* abort_flag) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long start = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - start > kWaitCycles) {
            *abort_flag = 1;
            return false;
        }
    }
    return true;
}

// The producer's wait for a released slot: the same bounds, with a short
// sleep between polls so that a waiting producer leaves the issue slots to
// the consumer warps of its SM.
__device__ __forceinline__ bool ring_wait_idle(uint64_t* bar, unsigned parity, volatile int* abort_flag) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long start = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - start > kWaitCycles) {
            *abort_flag = 1;
            return false;
        }
        __nanosleep(128);
    }
    return true;
}

// Steps 2-7 of a column pair: momenta, wall and bulk forces from the
// density ring (rows s_m, s_0, s_p; the pair's first column at index rc),
// the velocities of Eqs. 7-8, the shifted equilibria and the BGK update in the
// FP32 order of node_state() and relax(); stores to dst (one or both columns,
// with the ghost images of the edge columns).
template <typename S, int RC, bool G>
__device__ __forceinline__ void collide_pair(const StepCtx<S, G>& cx, const float2 (&f)[2][9], const unsigned (&m)[2],
                                             const float (*dn)[2][RC], int s_m, int s_0, int s_p, int rc,
                                             S* __restrict__ dst, unsigned plane, unsigned orow, const int (&cc)[2],
                                             bool c0, bool c1, int nx, const float (&sh)[2][3]) {
    using Wc = Wt<float>;
    float2 n[2], jx[2], jy[2], ax[2], ay[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        n[k] = *reinterpret_cast<const float2*>(&dn[s_0][k][rc]);
        jx[k] = P2::add(P2::sub(P2::sub(P2::add(P2::sub(f[k][1], f[k][3]), f[k][5]), f[k][6]), f[k][7]), f[k][8]);
        jy[k] = P2::sub(P2::sub(P2::add(P2::add(P2::sub(f[k][2], f[k][4]), f[k][5]), f[k][6]), f[k][7]), f[k][8]);
    }
    float2 Wx = make_float2(0.f, 0.f), Wy = make_float2(0.f, 0.f);
    if (m[0] | m[1]) {
        float a, b;
        wall_sum(m[0], a, b);
        Wx.x = a;
        Wy.x = b;
        wall_sum(m[1], a, b);
        Wx.y = a;
        Wy.y = b;
    }
    const float2 w1 = P2::dup(Wc::w1), w5 = P2::dup(Wc::w5);
    const float2 mw1 = P2::dup(-Wc::w1), mw5 = P2::dup(-Wc::w5);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int kb = 1 - k;
        const float* r0 = &dn[s_0][kb][rc];
        const float* rp = &dn[s_p][kb][rc];
        const float* rm = &dn[s_m][kb][rc];
        const float2 n1 = make_float2(r0[1], r0[2]), n3 = make_float2(r0[-1], r0[0]);
        const float2 n2 = *reinterpret_cast<const float2*>(rp);
        const float2 n5 = make_float2(rp[1], rp[2]), n6 = make_float2(rp[-1], rp[0]);
        const float2 n4 = *reinterpret_cast<const float2*>(rm);
        const float2 n7 = make_float2(rm[-1], rm[0]), n8 = make_float2(rm[1], rm[2]);
        float2 Sx = P2::fma(mw1, n3, P2::mul(w1, n1));
        Sx = P2::fma(w5, n5, Sx);
        Sx = P2::fma(mw5, n6, Sx);
        Sx = P2::fma(mw5, n7, Sx);
        Sx = P2::fma(w5, n8, Sx);
        float2 Sy = P2::fma(mw1, n4, P2::mul(w1, n2));
        Sy = P2::fma(w5, n5, Sy);
        Sy = P2::fma(w5, n6, Sy);
        Sy = P2::fma(mw5, n7, Sy);
        Sy = P2::fma(mw5, n8, Sy);
        const float2 mG = P2::dup(-cx.G), Gw = P2::dup(cx.Gw[k]);
        ax[k] = P2::add(P2::sub(P2::mul(mG, Sx), P2::mul(Gw, Wx)), P2::dup(cx.gx));
        ay[k] = P2::add(P2::sub(P2::mul(mG, Sy), P2::mul(Gw, Wy)), P2::dup(cx.gy));
    }
    const float(&wu)[2] = cx.wU();
    const float2 wu0 = P2::dup(wu[0]), wu1 = P2::dup(wu[1]);
    const float2 den = P2::fma(n[0], wu0, P2::mul(n[1], wu1));
    const float2 numx = P2::fma(jx[0], wu0, P2::mul(jx[1], wu1));
    const float2 numy = P2::fma(jy[0], wu0, P2::mul(jy[1], wu1));
    const float2 rden = make_float2(__frcp_rn(den.x), __frcp_rn(den.y));
    const float2 Ux = P2::mul(numx, rden), Uy = P2::mul(numy, rden);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float2 tm = P2::dup(cx.taum[k]);
        const float2 ux = P2::fma(tm, ax[k], Ux);
        const float2 uy = P2::fma(tm, ay[k], Uy);
        const float2 usq = P2::fma(ux, ux, P2::mul(uy, uy));
        const float2 b = P2::mul(P2::dup(1.5f), usq);
        const float2 nk = n[k];
        const float2 wn1 = P2::mul(P2::dup(Wc::w1), nk), wn5 = P2::mul(P2::dup(Wc::w5), nk);
        const float2 om = P2::dup(1.f - cx.itau[k]), itk = P2::dup(cx.itau[k]);
        const float2 base = make_float2(1.f - b.x, 1.f - b.y);
        const float2 cpv[4] = {ux, uy, P2::add(ux, uy), P2::sub(uy, ux)};
        float2 fn[9];
        float2 moving = make_float2(0.f, 0.f);
        constexpr int ia[4] = {1, 2, 5, 6}, ib[4] = {3, 4, 7, 8};
#pragma unroll
        for (int qd = 0; qd < 4; ++qd) {
            const float2 wn = qd < 2 ? wn1 : wn5;
            const float2 cq = cpv[qd];
            float2 sy = P2::mul(wn, P2::fma(P2::dup(4.5f), P2::mul(cq, cq), base));
            if constexpr (G) sy = P2::fma(P2::dup(cx.dA[k][qd < 2 ? 1 : 2]), nk, sy);
            const float2 an = P2::mul(P2::mul(P2::dup(3.f), wn), cq);
            fn[ia[qd]] = P2::fma(P2::add(sy, an), itk, P2::mul(f[k][ia[qd]], om));
            fn[ib[qd]] = P2::fma(P2::sub(sy, an), itk, P2::mul(f[k][ib[qd]], om));
            moving = P2::add(moving, P2::add(fn[ia[qd]], fn[ib[qd]]));
        }
        fn[0] = P2::sub(nk, moving);
        S* d = dst + ((unsigned)(k * 9) * plane + orow + (unsigned)cc[0]);
        if (c0 && c1) {
#pragma unroll
            for (int i = 0; i < 9; ++i) PairSt<S>::both(d + (unsigned)i * plane, fn[i], sh[k][grp(i)]);
        } else {
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                if (!(c ? c1 : c0)) continue;
                S* dc = dst + ((unsigned)(k * 9) * plane + orow + (unsigned)cc[c]);
#pragma unroll
                for (int i = 0; i < 9; ++i) PairSt<S>::one(dc + (unsigned)i * plane, lane_of(fn[i], c), sh[k][grp(i)]);
            }
        }
        // ghost images of columns 0, 1 (at nx, nx + 1) and nx - 2, nx - 1 (at -2, -1)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            if (!(c ? c1 : c0)) continue;
            const int gr = ghost_r(cc[c], nx), gl = ghost_l(cc[c], nx);
            if (!(gr | gl)) continue;
            S* dc = dst + ((unsigned)(k * 9) * plane + orow + (unsigned)cc[c]);
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                S* pp = dc + (unsigned)i * plane;
                if (gr) PairSt<S>::one(pp + gr, lane_of(fn[i], c), sh[k][grp(i)]);
                if (gl) PairSt<S>::one(pp + gl, lane_of(fn[i], c), sh[k][grp(i)]);
            }
        }
    }
}

template <typename S, int D, bool G>
__global__ void __launch_bounds__(RingGeom<S, D>::THREADS, 5)
    k_step_ring(const RunDesc* __restrict__ runs, const Tile* __restrict__ tiles, int ntiles, int* __restrict__ queue,
                int parity, uint32_t* __restrict__ err) {
    using RG = RingGeom<S, D>;
    using C = typename Prec<S>::C;
    constexpr int OFF = RG::OFF, WIN = RG::WIN, NCONS = RG::NCONS;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    S* ring = reinterpret_cast<S*>(smem_raw);                                           // [D][18][WIN]
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + RG::ring_bytes + RG::dens_bytes);
    uint64_t* done = full + D;
    int* rowitem = reinterpret_cast<int*>(done + D);   // segment of the slot's row (first row only), -1 = end
    volatile int* abort_flag = rowitem + D;

    if (threadIdx.x == 0) {
        for (int d = 0; d < D; ++d) {
            mbar_init(&full[d], 1);
            mbar_init(&done[d], NCONS / 32);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();

    if (threadIdx.x >= NCONS) {
        // ---- producer warp ------------------------------------------------------
        const int lane = threadIdx.x - NCONS;
        int q = 0;   // pulled rows issued so far (all lanes agree)
        bool stop = false;
        auto acquire_slot = [&](int s) {   // slot of sequence s is free (its row s - D released)
            if (s < D) return true;
            int ok = 1;
            if (lane == 0) ok = ring_wait_idle(&done[s % D], (unsigned)((s / D - 1) & 1), abort_flag);
            return __shfl_sync(0xffffffffu, ok, 0) != 0;
        };
        for (;;) {
            int item = 0;
            if (lane == 0) item = atomicAdd(&queue[0], 1);
            item = __shfl_sync(0xffffffffu, item, 0);
            if (item >= ntiles) break;
            const Tile tl = tiles[item];
            const RunDesc& rd = runs[tl.run];
            if (!step_tile_ok(tl, rd)) {   // checked builds: the segment is not touched
                stop = true;
                if (lane == 0) *abort_flag = 1;
                break;
            }
            const int ny = rd.ny, pitch = rd.pitch;
            const unsigned plane = (unsigned)rd.plane;
            const S* __restrict__ src = static_cast<const S*>(rd.buf[parity]);
            const int win_elems = min(WIN, (pitch - LBM_COL0) - (tl.x0 - OFF));
            const unsigned win_bytes = (unsigned)(win_elems * (int)sizeof(S));
            const int npull = tl.y1 - tl.y0 + 2;
            for (int pi = 0; pi < npull; ++pi, ++q) {
                const int d = q % D;
                if (!acquire_slot(q)) {
                    stop = true;
                    break;
                }
                if (lane == 0 && pi == 0) rowitem[d] = item;
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                if (lane == 0) mbar_expect_tx(&full[d], 18u * win_bytes);
                __syncwarp();
                if (lane < 18) {
                    int row = tl.y0 - 1 + pi - cyo(lane % 9);   // in [y0 - 2, y1 + 1]
                    row = row < 0 ? row + ny : (row >= ny ? row - ny : row);
                    row = row < 0 ? row + ny : (row >= ny ? row - ny : row);   // ny = 1
                    const S* g = src + ((unsigned)lane * plane + (unsigned)(row * pitch)) + (tl.x0 - OFF);
                    bulk_g2s(ring + (size_t)d * RG::slot_elems + lane * WIN, g, win_bytes, &full[d]);
                }
            }
            if (stop) break;
        }
        // end marker: the next slot completes with no copy and carries -1
        if (!stop) {
            if (!acquire_slot(q)) stop = true;
            else if (lane == 0) {
                rowitem[q % D] = -1;
                mbar_arrive(&full[q % D]);
            }
        }
        if (lane == 0) {
            // the last CTA to finish resets the segment counter for the next launch
            __threadfence();
            if (atomicAdd(&queue[1], 1) == (int)gridDim.x - 1) {
                atomicExch(&queue[0], 0);
                atomicExch(&queue[1], 0);
            }
            // wait until the consumers released the last rows (every issued copy
            // then has landed); on an abort, drain the copies still in flight
            bool aborted = stop;
            for (int s = max(0, q - D); s < q && !aborted; ++s)
                if (!ring_wait(&done[s % D], (unsigned)((s / D) & 1), abort_flag)) aborted = true;
            if (aborted || *abort_flag) {
                for (int s = max(0, q - D); s < q; ++s) mbar_wait(&full[s % D], (unsigned)((s / D) & 1));
                atomicOr(err, ERR_TIMEOUT);
            }
        }
        return;
    }

    // ---- consumer warps ---------------------------------------------------------
    // Each consumer warp marches on its own: warp w collides columns
    // [x0 + w kRingWc / NCW, x0 + (w + 1) kRingWc / NCW) of the strip with its
    // own density ring, so no barrier couples the warps; they share only the
    // slots (each warp releases a slot once it is done with it).
    constexpr int NCW = NCONS / 32;                      // consumer warps
    constexpr int WCOLS = kRingWc / NCW;                 // collided columns per warp
    constexpr int RCW = RG::RCW;
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    float(*dw)[2][RCW] = reinterpret_cast<float(*)[2][RCW]>(smem_raw + RG::ring_bytes) + 4 * wi;   // [4][2][RCW]
    int q = 0;         // pulled rows consumed so far
    bool to = false;   // this thread gave up waiting
    auto release = [&](int s) {
        __syncwarp();
        if (lane == 0) mbar_arrive(&done[s % D]);
    };
    auto wait_full = [&](int s) {
        if (!to && !ring_wait(&full[s % D], (unsigned)((s / D) & 1), abort_flag)) to = true;
    };

    for (;;) {
        // the slot of the next pulled row carries its segment, or the end marker
        wait_full(q);
        const int item = to ? -1 : rowitem[q % D];
        if (__any_sync(0xffffffffu, to) || item < 0) break;
        const Tile tl = tiles[item];
        const RunDesc& rd = runs[tl.run];
        const int nx = rd.nx, ny = rd.ny, pitch = rd.pitch;
        const unsigned plane = (unsigned)rd.plane;
        const Geo geo{nx, rd.cap_x0, rd.cap_x1, rd.y_bot, rd.y_top, rd.mask};
        const S* __restrict__ src = static_cast<const S*>(rd.buf[parity]);
        S* __restrict__ dst = static_cast<S*>(rd.buf[parity ^ 1]);
        StepCtx<S, G> cx;
        cx.load(rd);
        const int xw0 = tl.x0 + wi * WCOLS, y0 = tl.y0, nrow = tl.y1 - tl.y0;
        const int ncols = min(WCOLS, nx - xw0);   // columns this warp collides (<= 0: none)
        bool abort_all = false;
        // pulled row pi (row y0 - 1 + pi, sequence q + pi) has density-ring row
        // pi & 3; densities run two rows ahead of the collisions, so that a
        // row's collision and the next density pass overlap in each warp

        {
            // lane l holds columns xw0 - 2 + 2l and xw0 - 1 + 2l (lanes 0 and 31
            // only supply halo densities)
            const int e = wi * WCOLS + 2 * lane - 2 + OFF;   // window index of the pair's first column
            const int rc = 2 * lane + 2;                     // density-ring index of the pair's first column
            int cc[2], cm[2], cp[2];
            bool dcol[2], coll[2];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int col = xw0 - 2 + 2 * lane + c;
                dcol[c] = col >= xw0 - 1 && col <= xw0 + ncols;
                coll[c] = col >= xw0 && col < xw0 + ncols;
                int w = col < 0 ? col + nx : (col >= nx ? col - nx : col);
                w = w < 0 ? w + nx : (w >= nx ? w - nx : w);
                if (!dcol[c]) w = 0;
                cc[c] = w;
                cm[c] = w == 0 ? nx - 1 : w - 1;
                cp[c] = w == nx - 1 ? 0 : w + 1;
            }
            const float sh[2][3] = {{cx.sh.v[0][0], cx.sh.v[0][1], cx.sh.v[0][2]},
                                    {cx.sh.v[1][0], cx.sh.v[1][1], cx.sh.v[1][2]}};
            auto masks = [&](const RowIdx& rq, unsigned (&m)[2]) {
#pragma unroll
                for (int c = 0; c < 2; ++c) m[c] = dcol[c] ? nbr_solid(geo, cm[c], cc[c], cp[c], rq.rm, rq.rw, rq.rp) : 0u;
            };
            // pulled population pairs of sequence s (row rw) with half-way
            // bounce-back next to solids (F_opp(i) of the node itself, from src)
            auto pull = [&](int s, int rw, const unsigned (&m)[2], float2 (&f)[2][9]) {
                const S* P = ring + (size_t)(s % D) * RG::slot_elems + e;
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const S* qq = P + k * 9 * WIN;
                    f[k][0] = SlotLd<S>::al(qq, sh[k][0]);
                    f[k][1] = SlotLd<S>::un(qq + 1 * WIN - 1, sh[k][1]);
                    f[k][2] = SlotLd<S>::al(qq + 2 * WIN, sh[k][1]);
                    f[k][3] = SlotLd<S>::un(qq + 3 * WIN + 1, sh[k][1]);
                    f[k][4] = SlotLd<S>::al(qq + 4 * WIN, sh[k][1]);
                    f[k][5] = SlotLd<S>::un(qq + 5 * WIN - 1, sh[k][2]);
                    f[k][6] = SlotLd<S>::un(qq + 6 * WIN + 1, sh[k][2]);
                    f[k][7] = SlotLd<S>::un(qq + 7 * WIN + 1, sh[k][2]);
                    f[k][8] = SlotLd<S>::un(qq + 8 * WIN - 1, sh[k][2]);
                }
                if (m[0] | m[1]) {
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        if (!m[c] || SOL(m[c], 0, 0)) continue;
                        const S* own = src + (unsigned)(rw * pitch + cc[c]);
#pragma unroll
                        for (int k = 0; k < 2; ++k)
#pragma unroll
                            for (int i = 1; i < 9; ++i)
                                if (SOL(m[c], -cyo(i), -cxo(i)))
                                    set_lane(f[k][i], c,
                                             dec(ldg(own + (unsigned)(9 * k + opp(i)) * plane), sh[k][grp(i)]));
                    }
                }
            };
            // densities of sequence s (row r) into density-ring row `slot`
            auto dens_row = [&](int s, int r, int slot) {
                wait_full(s);
                if (to) return;
                const RowIdx rq = rows_of(r, ny);
                unsigned m[2];
                masks(rq, m);
                float2 f[2][9];
                pull(s, rq.rw, m, f);
                float2 n[2];
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    float2 a = P2::add(f[k][0], f[k][1]);
#pragma unroll
                    for (int i = 2; i < 9; ++i) a = P2::add(a, f[k][i]);
                    n[k] = a;
                }
#pragma unroll
                for (int c = 0; c < 2; ++c)
                    if (!dcol[c] || SOL(m[c], 0, 0)) {
                        set_lane(n[0], c, 0.f);
                        set_lane(n[1], c, 0.f);
                    }
                *reinterpret_cast<float2*>(&dw[slot][0][rc]) = n[0];
                *reinterpret_cast<float2*>(&dw[slot][1][rc]) = n[1];
            };
            dens_row(q, y0 - 1, 0);
            release(q);
            dens_row(q + 1, y0, 1);
            dens_row(q + 2, y0 + 1, 2);
            if (nrow == 1) release(q + 2);   // the trailing halo row is not collided
            abort_all = __any_sync(0xffffffffu, to);
            for (int j = 0; j < nrow && !abort_all; ++j) {
                const int s = q + 1 + j;   // sequence of row r
                const int r = y0 + j;
                const RowIdx rq = rows_of(r, ny);
                unsigned m[2] = {0u, 0u};
                float2 f[2][9];
                masks(rq, m);
                pull(s, rq.rw, m, f);
                release(s);
                if (j + 3 <= nrow + 1) {
                    dens_row(s + 2, r + 2, (j + 3) & 3);
                    if (j + 3 == nrow + 1) release(s + 2);
                }
                const bool c0 = !to && coll[0] && !SOL(m[0], 0, 0), c1 = !to && coll[1] && !SOL(m[1], 0, 0);
                if (c0 | c1)
                    collide_pair<S, RCW, G>(cx, f, m, dw, j & 3, (j + 1) & 3, (j + 2) & 3, rc, dst, plane,
                                            (unsigned)(rq.rw * pitch), cc, c0, c1, nx, sh);
                abort_all = __any_sync(0xffffffffu, to);   // (also orders this row's ring reads before reuse)
            }
        }
        if (abort_all) break;
        q += nrow + 2;
    }
}

}  // namespace sc
