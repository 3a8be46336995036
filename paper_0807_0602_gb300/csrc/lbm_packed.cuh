// Species-packed FP32 arithmetic and the species-packed bidirectional march
// (LBM_KERNEL_BIDIR_SP) for FP32 and FP16-shifted storage.
//
// The collision treats species A and B with the same sequence of operations
// (Eqs. 2-7 and 9-11 differ between them only in their coefficients and in
// which species' densities enter the force), so one packed FP32 instruction
// (__ffma2_rn / __fadd2_rn / __fmul2_rn, lane x = A, lane y = B) evaluates
// both.  Each lane is rounded exactly as the scalar operation of Ar<float>,
// in the canonical order of node_state() and relax(), so the populations
// equal those of every other FP32 / FP16S step kernel bit for bit.  Only the
// cross-species sums of Eq. 8 stay scalar.
//
// Shared memory holds the same quantities as k_step_bidir, packed: the
// staged populations as (f_A,i, f_B,i) pairs (one 8-byte store and load per
// direction instead of two 4-byte ones) and the density ring as (n_B, n_A),
// so that each neighbour's pair is already in the lanes of the force sums of
// Eq. 9 (lane k needs the other species' density).
#pragma once

#include "lbm_kernels.cuh"

namespace sc {

// ---- packed FP32 arithmetic -----------------------------------------------------
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

// Wall sum of Eq. 11 (the same for both species), in node_state()'s order.
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

// Per-CTA constants with species A in lane x and B in lane y.
template <bool GEN>
struct Ctx2 {
    float mG, gx, gy;             // -G and the body force
    float2 Gw, taum, itau, om;    // om = 1 - 1/tau_k
    float2 wu;                    // weights of U in Eq. 8 (1/tau_k, or m_k/tau_k with GEN)
    float2 dA[3];                 // GEN: A_g(alpha_k) - w_g per direction group
    float2 sh[3];                 // storage shift w_i rho_ref,k per direction group (FP16S)
    template <typename S>
    __device__ __forceinline__ void load(const StepCtx<S, GEN>& cx) {
        mG = -cx.G;
        gx = cx.gx;
        gy = cx.gy;
        Gw = make_float2(cx.Gw[0], cx.Gw[1]);
        taum = make_float2(cx.taum[0], cx.taum[1]);
        itau = make_float2(cx.itau[0], cx.itau[1]);
        om = make_float2(1.f - cx.itau[0], 1.f - cx.itau[1]);
        const float(&w)[2] = cx.wU();
        wu = make_float2(w[0], w[1]);
#pragma unroll
        for (int g = 0; g < 3; ++g) {
            if constexpr (GEN) dA[g] = make_float2(cx.dA[0][g], cx.dA[1][g]);
            sh[g] = make_float2(cx.sh.v[0][g], cx.sh.v[1][g]);
        }
    }
};

// Loads of (f_A, f_B) at the same offset of planes i and 9 + i, decoded as dec().
template <typename S> struct Ld2;
template <> struct Ld2<float> {
    static __device__ __forceinline__ float2 ld(const float* pa, const float* pb, float2) {
        return make_float2(__ldg(pa), __ldg(pb));
    }
};
template <> struct Ld2<__half> {
    static __device__ __forceinline__ float2 ld(const __half* pa, const __half* pb, float2 sh) {
        return __fadd2_rn(make_float2(__half2float(ldg(pa)), __half2float(ldg(pb))), sh);
    }
};

// Step 1 at one node for both species (pull_node() with the pairs packed).
template <typename S>
__device__ __forceinline__ void pull_node2(const S* __restrict__ src, unsigned plane, unsigned own, unsigned oxm,
                                           unsigned oxp, unsigned orm, unsigned orp, unsigned orm_xm,
                                           unsigned orm_xp, unsigned orp_xm, unsigned orp_xp, unsigned sm,
                                           const float2 (&sh)[3], float2 (&f)[9]) {
    const S* pa = src;
    const S* pb = src + 9u * plane;
    auto L = [&](unsigned o, int g) { return Ld2<S>::ld(pa + o, pb + o, sh[g]); };
    if (sm == 0) {
        f[0] = L(own, 0);
        f[1] = L(1 * plane + oxm, 1);
        f[2] = L(2 * plane + orm, 1);
        f[3] = L(3 * plane + oxp, 1);
        f[4] = L(4 * plane + orp, 1);
        f[5] = L(5 * plane + orm_xm, 2);
        f[6] = L(6 * plane + orm_xp, 2);
        f[7] = L(7 * plane + orp_xp, 2);
        f[8] = L(8 * plane + orp_xm, 2);
        return;
    }
    f[0] = L(own, 0);
    f[1] = L(SOL(sm, 0, -1) ? 3 * plane + own : 1 * plane + oxm, 1);
    f[2] = L(SOL(sm, -1, 0) ? 4 * plane + own : 2 * plane + orm, 1);
    f[3] = L(SOL(sm, 0, 1) ? 1 * plane + own : 3 * plane + oxp, 1);
    f[4] = L(SOL(sm, 1, 0) ? 2 * plane + own : 4 * plane + orp, 1);
    f[5] = L(SOL(sm, -1, -1) ? 7 * plane + own : 5 * plane + orm_xm, 2);
    f[6] = L(SOL(sm, -1, 1) ? 8 * plane + own : 6 * plane + orm_xp, 2);
    f[7] = L(SOL(sm, 1, 1) ? 5 * plane + own : 7 * plane + orp_xp, 2);
    f[8] = L(SOL(sm, 1, -1) ? 6 * plane + own : 8 * plane + orp_xm, 2);
}

// Step 2 for both species: dens9() lane by lane.
__device__ __forceinline__ float2 dens9_2(const float2 (&f)[9]) {
    float2 s = P2::add(f[0], f[1]);
#pragma unroll
    for (int i = 2; i < 9; ++i) s = P2::add(s, f[i]);
    return s;
}

// Steps 2-7 and the store at one fluid node, both species packed: node_state()
// and relax() (the FP32 form) lane by lane.  sdx holds (n_B, n_A) per column.
template <typename S, int W, bool GH, bool G>
__device__ __forceinline__ void collide_node2(const Ctx2<G>& c2, const float2 (&f)[9], unsigned m,
                                              const float2 (*sdx)[W], int s_m, int s_0, int s_p, int t,
                                              S* __restrict__ dst, unsigned plane, unsigned o, int gr, int gl) {
    using Wc = Wt<float>;
    using A = Ar<float>;
    const float2 ownd = sdx[s_0][t];
    const float2 n = make_float2(ownd.y, ownd.x);
    const float2 jx = P2::add(P2::sub(P2::sub(P2::add(P2::sub(f[1], f[3]), f[5]), f[6]), f[7]), f[8]);
    const float2 jy = P2::sub(P2::sub(P2::add(P2::add(P2::sub(f[2], f[4]), f[5]), f[6]), f[7]), f[8]);
    float Wx, Wy;
    wall_sum(m, Wx, Wy);
    // Eq. 9: lane k sums the neighbour densities of species 1 - k
    const float2 n1 = sdx[s_0][t + 1], n2 = sdx[s_p][t], n3 = sdx[s_0][t - 1], n4 = sdx[s_m][t],
                 n5 = sdx[s_p][t + 1], n6 = sdx[s_p][t - 1], n7 = sdx[s_m][t - 1], n8 = sdx[s_m][t + 1];
    const float2 w1 = P2::dup(Wc::w1), w5 = P2::dup(Wc::w5), mw1 = P2::dup(-Wc::w1), mw5 = P2::dup(-Wc::w5);
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
    const float2 mG = P2::dup(c2.mG);
    const float2 ax = P2::add(P2::sub(P2::mul(mG, Sx), P2::mul(c2.Gw, P2::dup(Wx))), P2::dup(c2.gx));
    const float2 ay = P2::add(P2::sub(P2::mul(mG, Sy), P2::mul(c2.Gw, P2::dup(Wy))), P2::dup(c2.gy));
    // Eq. 8 (cross-species sums, scalar) and Eq. 7
    const float den = A::fma(n.x, c2.wu.x, A::mul(n.y, c2.wu.y));
    const float numx = A::fma(jx.x, c2.wu.x, A::mul(jx.y, c2.wu.y));
    const float numy = A::fma(jy.x, c2.wu.x, A::mul(jy.y, c2.wu.y));
    const float rden = __frcp_rn(den);
    const float Ux = A::mul(numx, rden), Uy = A::mul(numy, rden);
    const float2 ux = P2::fma(c2.taum, ax, P2::dup(Ux));
    const float2 uy = P2::fma(c2.taum, ay, P2::dup(Uy));
    const float2 usq = P2::fma(ux, ux, P2::mul(uy, uy));
    const float2 b = P2::mul(P2::dup(1.5f), usq);
    const float2 wn1 = P2::mul(w1, n), wn5 = P2::mul(w5, n);
    const float2 base = make_float2(1.f - b.x, 1.f - b.y);
    const float2 cpv[4] = {ux, uy, P2::add(ux, uy), P2::sub(uy, ux)};
    constexpr int ia[4] = {1, 2, 5, 6}, ib[4] = {3, 4, 7, 8};
    float2 fn[9];
    float2 moving = make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float2 wn = q < 2 ? wn1 : wn5;
        const float2 c = cpv[q];
        float2 sy = P2::mul(wn, P2::fma(P2::dup(4.5f), P2::mul(c, c), base));
        if constexpr (G) sy = P2::fma(c2.dA[q < 2 ? 1 : 2], n, sy);
        const float2 an = P2::mul(P2::mul(P2::dup(3.f), wn), c);
        fn[ia[q]] = P2::fma(P2::add(sy, an), c2.itau, P2::mul(f[ia[q]], c2.om));
        fn[ib[q]] = P2::fma(P2::sub(sy, an), c2.itau, P2::mul(f[ib[q]], c2.om));
        moving = P2::add(moving, P2::add(fn[ia[q]], fn[ib[q]]));
    }
    fn[0] = P2::sub(n, moving);
    S* da = dst + o;
    S* db = dst + (9u * plane + o);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        enc(da + (unsigned)i * plane, fn[i].x, c2.sh[grp(i)].x);
        enc(db + (unsigned)i * plane, fn[i].y, c2.sh[grp(i)].y);
    }
    if (GH) {   // ghost images of the edge columns (rare)
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            S* pa = da + (unsigned)i * plane;
            S* pb = db + (unsigned)i * plane;
            if (gr) {
                enc(pa + gr, fn[i].x, c2.sh[grp(i)].x);
                enc(pb + gr, fn[i].y, c2.sh[grp(i)].y);
            }
            if (gl) {
                enc(pa + gl, fn[i].x, c2.sh[grp(i)].x);
                enc(pb + gl, fn[i].y, c2.sh[grp(i)].y);
            }
        }
    }
}

// ---- species-packed bidirectional march -----------------------------------------
// The march of k_step_bidir (two groups of W threads leaving the tile's middle
// row in opposite directions; step k: pull, barrier, collide) with the
// species packed as above.
template <typename S, int W, bool G>
__global__ void __launch_bounds__(2 * W, (kBidirMinBlocks<S, W>)) k_step_bidir_sp(const RunDesc* __restrict__ runs,
                                                                                 const Tile* __restrict__ tiles,
                                                                                 int parity) {
    static_assert(sizeof(typename Prec<S>::C) == 4, "FP32 arithmetic only");
    __shared__ float2 sdx[8][W];       // [group * 4 + step ring][column]: (n_B, n_A)
    __shared__ float2 psx[2][2][9][W]; // [group][step parity][direction][column]: (f_A, f_B)
    const Tile tl = tiles[blockIdx.x];
    const RunDesc& rd = runs[tl.run];
    if (!step_tile_ok(tl, rd)) return;
    const int nx = rd.nx, ny = rd.ny, pitch = rd.pitch;
    const unsigned plane = (unsigned)rd.plane;
    const Geo geo{nx, rd.cap_x0, rd.cap_x1, rd.y_bot, rd.y_top, rd.mask};
    const S* __restrict__ src = static_cast<const S*>(rd.buf[parity]);
    S* __restrict__ dst = static_cast<S*>(rd.buf[parity ^ 1]);
    Ctx2<G> c2;
    {
        StepCtx<S, G> cx;
        cx.load(rd);
        c2.load(cx);
    }
    const int t = threadIdx.x % W, grp_d = threadIdx.x / W;   // grp_d 0: up (U), 1: down (D)
    const StripCols sc(tl.x0, nx, W, t);
    const int y0 = tl.y0, y1 = tl.y1;
    const int m = y0 + (y1 - y0 + 1) / 2;                     // first row of D
    const int nrows = grp_d == 0 ? m - y0 : y1 - m;
    const int nsteps = (y1 - y0 + 1) / 2 + 1;
    auto row_at = [&](int k) { return grp_d == 0 ? m - 1 - k : m + k; };

    auto pull = [&](int k, unsigned& smask) {
        const RowIdx q = rows_of(row_at(k), ny);
        float2 nd = make_float2(0.f, 0.f);
        smask = 0;
        if (sc.dcol) {
            smask = nbr_solid(geo, sc.xm, sc.xc, sc.xp, q.rm, q.rw, q.rp);
            if (!SOL(smask, 0, 0)) {
                const unsigned bw = (unsigned)(q.rw * pitch), bm = (unsigned)(q.rm * pitch),
                               bp = (unsigned)(q.rp * pitch);
                float2 f[9];
                pull_node2<S>(src, plane, bw + sc.xc, bw + sc.xm, bw + sc.xp, bm + sc.xc, bp + sc.xc, bm + sc.xm,
                              bm + sc.xp, bp + sc.xm, bp + sc.xp, smask, c2.sh, f);
                const float2 n2 = dens9_2(f);
                nd = make_float2(n2.y, n2.x);
                if (sc.coll && k < nrows) {
#pragma unroll
                    for (int i = 0; i < 9; ++i) psx[grp_d][k & 1][i][t] = f[i];
                }
            }
        }
        sdx[grp_d * 4 + (k & 3)][t] = nd;
    };

    unsigned sm_prev = 0, sm_cur = 0;
    for (int k = 0; k < nsteps; ++k) {
        if (k <= nrows) pull(k, sm_cur);
        __syncthreads();
        if (k >= 1 && k <= nrows && sc.coll && !SOL(sm_prev, 0, 0)) {
            const int r = grp_d == 0 ? m - k : m + k - 1;
            const int own = grp_d * 4, other = (1 - grp_d) * 4;
            const int s_new = own + (k & 3), s_row = own + ((k - 1) & 3);
            const int s_old = k >= 2 ? own + ((k - 2) & 3) : other;
            const int s_m = grp_d == 0 ? s_new : s_old, s_p = grp_d == 0 ? s_old : s_new;
            float2 fc[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) fc[i] = psx[grp_d][(k - 1) & 1][i][t];
            const unsigned o = (unsigned)(rows_of(r, ny).rw * pitch + sc.xc);
            const int gr = ghost_r(sc.xc, nx), gl = ghost_l(sc.xc, nx);
            if (gr | gl)
                collide_node2<S, W, true>(c2, fc, sm_prev, sdx, s_m, s_row, s_p, t, dst, plane, o, gr, gl);
            else
                collide_node2<S, W, false>(c2, fc, sm_prev, sdx, s_m, s_row, s_p, t, dst, plane, o, 0, 0);
        }
        sm_prev = sm_cur;
    }
}

}  // namespace sc
