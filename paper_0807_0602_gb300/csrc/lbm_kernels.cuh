// Kernels of the binary Shan-Chen D2Q9 step (S. Chibbaro, "Capillary filling
// with pseudo-potential binary Lattice-Boltzmann model", Model section,
// Eqs. 2-11; Numerical Results section for geometry, bounce-back and fronts).
//
// Included (through lbm_launch.cuh) by one translation unit per storage type
// and species model: kernels_f64.cu / kernels_gen_f64.cu (FP64, built with
// --fmad=false so that every product and sum is rounded separately, in the
// canonical order below), kernels_f32.cu / kernels_gen_f32.cu (FP32) and
// kernels_f16.cu / kernels_gen_f16.cu (FP16-shifted storage); the _gen units
// hold the step kernels of the free-alpha, m_k != 1 species model.
//
// Canonical per-node order (both precisions; FP64 reproduces it bit for bit):
//   1. pull: ft_i(x) = F_i(x - c_i), or F_opp(i)(x) when x - c_i is solid
//      (half-way bounce-back fused into the pull)
//   2. n_k = ((ft_0 + ft_1) + ...) + ft_8; j_k = sum_i c_i ft_i, i ascending
//   3. S_kbar = sum_{i=1..8} (w_i n_kbar(x + c_i)) c_i, i ascending (Eq. 9 with
//      the w_i-weighted G, n = 0 on solids); Wl = sum_i (w_i s(x + c_i)) c_i
//      (Eq. 11); a_k = (-(G S_kbar) - (G_kw Wl)) + g
//   4. U = (j_A mt_A + j_B mt_B) / (n_A mt_A + n_B mt_B), mt_k = m_k / tau_k  (Eq. 8)
//   5. u_k = U + tm_k a_k, tm_k = tau_k / m_k                            (Eq. 7)
//   6. feq_i = (w_i n_k) (((1 + 3 cu) + 4.5 (cu cu)) - 1.5 usq)   (Eqs. 3-5)
//      [+ dA_i n_k with dA_i = A_i(alpha_k) - w_i when alpha_k != 4/9]
//   7. F'_i = ft_i - (ft_i - feq_i) itau_k                               (Eq. 2)
//
// Step kernel design (sm_103a, HBM-bound stencil, no tensor cores):
//   - SoA populations, x fastest, rows padded to `pitch`; every load and store
//     of a warp touches consecutive addresses (the +-1 column shift of the
//     pull only offsets the warp's 128-byte window by one element).
//   - A CTA of W threads owns a strip of W - 2 columns (thread t <-> column
//     x0 - 1 + t; the two edge threads only supply halo densities) and
//     marches down a segment of rows [y0, y1).  Each row is pulled once: its
//     18 populations stay in registers for the collision one iteration later,
//     its two densities go into a 4-row ring in shared memory, so the
//     8-neighbour force reads densities without an HBM round trip.  One
//     __syncthreads per row; the ring depth of 4 makes that sufficient.
//   - Populations are read once and written once per step (72 B/node FP32).
#pragma once

#include "lbm_device.h"

namespace sc {

template <typename S> struct Prec;
template <> struct Prec<double> { using C = double; };
template <> struct Prec<float> { using C = float; };
template <> struct Prec<__half> { using C = float; };

// D2Q9 weights of Eqs. 3-5 at alpha = 4/9 (correctly rounded divisions).
template <typename C> struct Wt;
template <> struct Wt<double> {
    static constexpr double w0 = 4.0 / 9.0, w1 = 1.0 / 9.0, w5 = 1.0 / 36.0;
};
template <> struct Wt<float> {
    static constexpr float w0 = 4.0f / 9.0f, w1 = 1.0f / 9.0f, w5 = 1.0f / 36.0f;
};

// Arithmetic of the collision, spelled out so that no kernel variant can
// contract it differently: FP64 uses separately rounded products and sums in
// the canonical order (fma(a, b, c) = (a b) + c, two roundings); FP32 fuses
// exactly those products into FMAs.  Every step kernel therefore produces the
// same bits for a given precision, whatever its schedule.
template <typename C> struct Ar;
template <> struct Ar<double> {
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
    static __device__ __forceinline__ double fma(double a, double b, double c) { return __dadd_rn(__dmul_rn(a, b), c); }
};
// FP64 evaluates the canonical order; FP32 may use cheaper equivalent forms.
template <typename C> constexpr bool kCanonical = true;
template <> constexpr bool kCanonical<float> = false;

template <> struct Ar<float> {
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
    static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
};

// Storage <-> compute conversion.  FP16S stores f - w_i rho_ref,k.
__device__ __forceinline__ double dec(double v, double) { return v; }
__device__ __forceinline__ float dec(float v, float) { return v; }
__device__ __forceinline__ float dec(__half v, float sh) { return __fadd_rn(__half2float(v), sh); }
__device__ __forceinline__ void enc(double* p, double v, double) { *p = v; }
__device__ __forceinline__ void enc(float* p, float v, float) { *p = v; }
__device__ __forceinline__ void enc(__half* p, float v, float sh) { *p = __float2half_rn(__fsub_rn(v, sh)); }

template <typename S> __device__ __forceinline__ S ldg(const S* p) { return __ldg(p); }
template <> __device__ __forceinline__ __half ldg<__half>(const __half* p) {
    return __ushort_as_half(__ldg(reinterpret_cast<const unsigned short*>(p)));
}

// Shift w_i rho_ref,k of direction group g (0 rest, 1 axis, 2 diagonal).
template <typename S> struct Shift {
    using C = typename Prec<S>::C;
    C v[2][3];
    __device__ __forceinline__ void load(const RunDesc&) {
        for (int k = 0; k < 2; ++k)
            for (int g = 0; g < 3; ++g) v[k][g] = C(0);
    }
};
template <> struct Shift<__half> {
    float v[2][3];
    __device__ __forceinline__ void load(const RunDesc& rd) {
        for (int k = 0; k < 2; ++k)
            for (int g = 0; g < 3; ++g) v[k][g] = rd.c32.sh[k][g];
    }
};
__device__ __forceinline__ constexpr int grp(int i) { return i == 0 ? 0 : (i <= 4 ? 1 : 2); }
// D2Q9 lattice vectors c_i (c_1 = (1, 0), c_2 = (0, 1), c_5 = (1, 1), c_6 = (-1, 1), ...)
// and opposite directions
__device__ __forceinline__ constexpr int cxo(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__device__ __forceinline__ constexpr int cyo(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__device__ __forceinline__ constexpr int opp(int i) { return i == 0 ? 0 : (i <= 4 ? (i + 1) % 4 + 1 : (i - 3) % 4 + 5); }

struct Geo {
    int nx, cx0, cx1, yb, yt;
    const uint8_t* mask;
    __device__ __forceinline__ bool solid(int x, int y) const {
        if (mask) return mask[(long long)y * nx + x] != 0;
        return (y == yb || y == yt) && x >= cx0 && x < cx1;
    }
};

// Solid flags of the 3x3 neighbourhood: bit (dy + 1) * 3 + (dx + 1).
__device__ __forceinline__ unsigned nbr_solid(const Geo& g, int xm, int xc, int xp, int rm, int rw,
                                              int rp) {
    unsigned m = 0;
    if (g.mask) {
        const int xs[3] = {xm, xc, xp};
        const int ys[3] = {rm, rw, rp};
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b)
                if (g.mask[(long long)ys[a] * g.nx + xs[b]]) m |= 1u << (a * 3 + b);
        return m;
    }
    const bool r0 = (rm == g.yb || rm == g.yt), r1 = (rw == g.yb || rw == g.yt),
               r2 = (rp == g.yb || rp == g.yt);
    if (!(r0 | r1 | r2)) return 0;
    const bool c0 = xm >= g.cx0 && xm < g.cx1, c1 = xc >= g.cx0 && xc < g.cx1,
               c2 = xp >= g.cx0 && xp < g.cx1;
    m |= (unsigned)(r0 && c0) << 0 | (unsigned)(r0 && c1) << 1 | (unsigned)(r0 && c2) << 2;
    m |= (unsigned)(r1 && c0) << 3 | (unsigned)(r1 && c1) << 4 | (unsigned)(r1 && c2) << 5;
    m |= (unsigned)(r2 && c0) << 6 | (unsigned)(r2 && c1) << 7 | (unsigned)(r2 && c2) << 8;
    return m;
}
#define SOL(m, dy, dx) (((m) >> (((dy) + 1) * 3 + ((dx) + 1))) & 1u)

// Pull of one node (step 1) and its densities (step 2).
template <typename S>
__device__ __forceinline__ void pull_node(const S* __restrict__ src, unsigned plane, unsigned own,
                                          unsigned oxm, unsigned oxp, unsigned orm, unsigned orp,
                                          unsigned orm_xm, unsigned orm_xp, unsigned orp_xm,
                                          unsigned orp_xp, unsigned sm, const Shift<S>& sh,
                                          typename Prec<S>::C (&f)[2][9]) {
    // source of direction i is x - c_i; offsets: own row/col combos
    if (sm == 0) {   // no solid neighbour (almost every node): no bounce-back selects
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const S* p = src + (unsigned)(k * 9) * plane;
            f[k][0] = dec(ldg(p + own), sh.v[k][0]);
            f[k][1] = dec(ldg(p + (1 * plane + oxm)), sh.v[k][1]);
            f[k][2] = dec(ldg(p + (2 * plane + orm)), sh.v[k][1]);
            f[k][3] = dec(ldg(p + (3 * plane + oxp)), sh.v[k][1]);
            f[k][4] = dec(ldg(p + (4 * plane + orp)), sh.v[k][1]);
            f[k][5] = dec(ldg(p + (5 * plane + orm_xm)), sh.v[k][2]);
            f[k][6] = dec(ldg(p + (6 * plane + orm_xp)), sh.v[k][2]);
            f[k][7] = dec(ldg(p + (7 * plane + orp_xp)), sh.v[k][2]);
            f[k][8] = dec(ldg(p + (8 * plane + orp_xm)), sh.v[k][2]);
        }
        return;
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const S* p = src + (unsigned)(k * 9) * plane;
        f[k][0] = dec(ldg(p + own), sh.v[k][0]);
        f[k][1] = dec(ldg(SOL(sm, 0, -1) ? p + (3 * plane + own) : p + (1 * plane + oxm)), sh.v[k][1]);
        f[k][2] = dec(ldg(SOL(sm, -1, 0) ? p + (4 * plane + own) : p + (2 * plane + orm)), sh.v[k][1]);
        f[k][3] = dec(ldg(SOL(sm, 0, 1) ? p + (1 * plane + own) : p + (3 * plane + oxp)), sh.v[k][1]);
        f[k][4] = dec(ldg(SOL(sm, 1, 0) ? p + (2 * plane + own) : p + (4 * plane + orp)), sh.v[k][1]);
        f[k][5] = dec(ldg(SOL(sm, -1, -1) ? p + (7 * plane + own) : p + (5 * plane + orm_xm)), sh.v[k][2]);
        f[k][6] = dec(ldg(SOL(sm, -1, 1) ? p + (8 * plane + own) : p + (6 * plane + orm_xp)), sh.v[k][2]);
        f[k][7] = dec(ldg(SOL(sm, 1, 1) ? p + (5 * plane + own) : p + (7 * plane + orp_xp)), sh.v[k][2]);
        f[k][8] = dec(ldg(SOL(sm, 1, -1) ? p + (6 * plane + own) : p + (8 * plane + orp_xm)), sh.v[k][2]);
    }
}

template <typename C>
__device__ __forceinline__ C dens9(const C (&f)[9]) {
    using A = Ar<C>;
    return A::add(A::add(A::add(A::add(A::add(A::add(A::add(A::add(f[0], f[1]), f[2]), f[3]), f[4]), f[5]), f[6]),
                         f[7]),
                  f[8]);
}

struct RowIdx {
    int rm, rw, rp;
};
// Rows of a march lie in [-1, ny]: one conditional wrap, no division.
__device__ __forceinline__ RowIdx rows_of(int r, int ny) {
    const int rw = r < 0 ? r + ny : (r >= ny ? r - ny : r);
    RowIdx q;
    q.rw = rw;
    q.rm = rw == 0 ? ny - 1 : rw - 1;
    q.rp = rw == ny - 1 ? 0 : rw + 1;
    return q;
}

// Per-CTA constants of the step.  GEN: the run has some alpha_k != 4/9 or
// m_k != 1 (a separate instantiation of every step kernel, so that the
// standard model carries neither the extra coefficients nor their registers).
template <typename S, bool GEN>
struct StepCtx {
    using C = typename Prec<S>::C;
    C G, Gw[2], taum[2], itau[2], mitau[2], m[2], gx, gy;
    C dA[2][3];   // A_g(alpha_k) - w_g (GEN only; 0 for a species with alpha_k = 4/9)
    Shift<S> sh;
    // With m_k = 1 (not GEN), taum = tau and the weights of U are itau.
    __device__ __forceinline__ const C (&wU() const)[2] {
        if constexpr (GEN) return mitau;
        else return itau;
    }
    __device__ __forceinline__ void load(const RunDesc& rd) {
        sh.load(rd);
        if constexpr (sizeof(C) == 4) {
            const CoefF32& c = rd.c32;
            G = c.G;
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                Gw[k] = c.Gw[k];
                taum[k] = c.taum[k];
                itau[k] = c.itau[k];
                if constexpr (GEN) {
                    mitau[k] = c.mitau[k];
                    m[k] = c.m[k];
#pragma unroll
                    for (int g = 0; g < 3; ++g) dA[k][g] = c.dA[k][g];
                }
            }
            gx = c.gx;
            gy = c.gy;
        } else {
            G = (C)rd.G;
            Gw[0] = (C)rd.GwA;
            Gw[1] = (C)rd.GwB;
            taum[0] = (C)rd.taumA;
            taum[1] = (C)rd.taumB;
            itau[0] = (C)rd.itauA;
            itau[1] = (C)rd.itauB;
            gx = (C)rd.gx;
            gy = (C)rd.gy;
            if constexpr (GEN) {
                mitau[0] = (C)rd.mitauA;
                mitau[1] = (C)rd.mitauB;
                m[0] = (C)rd.mA;
                m[1] = (C)rd.mB;
#pragma unroll
                for (int k = 0; k < 2; ++k)
#pragma unroll
                    for (int g = 0; g < 3; ++g) dA[k][g] = (C)rd.dA[k][g];
            }
        }
    }
};

// Offsets from column x to its ghost images: columns 0 and 1 are mirrored at
// nx and nx + 1, columns nx - 2 and nx - 1 at -2 and -1 (0 = no image).
__device__ __forceinline__ int ghost_r(int x, int nx) { return x < 2 ? nx : 0; }
__device__ __forceinline__ int ghost_l(int x, int nx) { return x >= nx - 2 ? -nx : 0; }

// Steps 2-3 at one fluid node: densities (shared ring), momenta and the
// accelerations a_k of both species.
template <typename S>
struct NodeState {
    using C = typename Prec<S>::C;
    C n[2], jx[2], jy[2], ax[2], ay[2];
};

template <typename S, int W, bool G>
__device__ __forceinline__ void node_state(const StepCtx<S, G>& cx, const typename Prec<S>::C (&fc)[2][9], unsigned m,
                                           const typename Prec<S>::C (*sd)[2][W], int s_m, int s_0, int s_p, int t,
                                           NodeState<S>& ns) {
    using C = typename Prec<S>::C;
    using Wc = Wt<C>;
    using A = Ar<C>;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const C(&f)[9] = fc[k];
        ns.n[k] = sd[s_0][k][t];
        ns.jx[k] = A::add(A::sub(A::sub(A::add(A::sub(f[1], f[3]), f[5]), f[6]), f[7]), f[8]);
        ns.jy[k] = A::sub(A::sub(A::add(A::add(A::sub(f[2], f[4]), f[5]), f[6]), f[7]), f[8]);
    }
    // wall sum of Eq. 11, the same for both species
    C Wx = C(0), Wy = C(0);
    if (m) {
        if (SOL(m, 0, 1)) Wx = A::add(Wx, Wc::w1);                                // i = 1
        if (SOL(m, 1, 0)) Wy = A::add(Wy, Wc::w1);                                // i = 2
        if (SOL(m, 0, -1)) Wx = A::sub(Wx, Wc::w1);                               // i = 3
        if (SOL(m, -1, 0)) Wy = A::sub(Wy, Wc::w1);                               // i = 4
        if (SOL(m, 1, 1)) { Wx = A::add(Wx, Wc::w5); Wy = A::add(Wy, Wc::w5); }   // i = 5
        if (SOL(m, 1, -1)) { Wx = A::sub(Wx, Wc::w5); Wy = A::add(Wy, Wc::w5); }  // i = 6
        if (SOL(m, -1, -1)) { Wx = A::sub(Wx, Wc::w5); Wy = A::sub(Wy, Wc::w5); } // i = 7
        if (SOL(m, -1, 1)) { Wx = A::add(Wx, Wc::w5); Wy = A::sub(Wy, Wc::w5); }  // i = 8
    }
    // bulk force of Eq. 9 from the neighbour densities of the other species:
    // S = ((((w1 n1 - w1 n3) + w5 n5) - w5 n6) - w5 n7) + w5 n8 (and y)
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int kb = 1 - k;
        const C n1 = sd[s_0][kb][t + 1], n2 = sd[s_p][kb][t], n3 = sd[s_0][kb][t - 1], n4 = sd[s_m][kb][t],
                n5 = sd[s_p][kb][t + 1], n6 = sd[s_p][kb][t - 1], n7 = sd[s_m][kb][t - 1], n8 = sd[s_m][kb][t + 1];
        C Sx = A::fma(-Wc::w1, n3, A::mul(Wc::w1, n1));
        Sx = A::fma(Wc::w5, n5, Sx);
        Sx = A::fma(-Wc::w5, n6, Sx);
        Sx = A::fma(-Wc::w5, n7, Sx);
        Sx = A::fma(Wc::w5, n8, Sx);
        C Sy = A::fma(-Wc::w1, n4, A::mul(Wc::w1, n2));
        Sy = A::fma(Wc::w5, n5, Sy);
        Sy = A::fma(Wc::w5, n6, Sy);
        Sy = A::fma(-Wc::w5, n7, Sy);
        Sy = A::fma(-Wc::w5, n8, Sy);
        ns.ax[k] = A::add(A::sub(-A::mul(cx.G, Sx), A::mul(cx.Gw[k], Wx)), cx.gx);
        ns.ay[k] = A::add(A::sub(-A::mul(cx.G, Sy), A::mul(cx.Gw[k], Wy)), cx.gy);
    }
}

// Steps 4-7: common velocity, shifted equilibria and BGK relaxation.
// GEN: the equilibria carry dA_i n_k and U weighs m_k / tau_k.
template <typename S, bool GEN>
__device__ __forceinline__ void relax(const StepCtx<S, GEN>& cx, const typename Prec<S>::C (&fc)[2][9],
                                           const NodeState<S>& ns, typename Prec<S>::C (&fnew)[2][9]) {
    using C = typename Prec<S>::C;
    using Wc = Wt<C>;
    using A = Ar<C>;
    // common velocity (Eq. 8) and shifted equilibrium velocities (Eq. 7)
    const C(&wu)[2] = cx.wU();
    const C den = A::fma(ns.n[0], wu[0], A::mul(ns.n[1], wu[1]));
    const C numx = A::fma(ns.jx[0], wu[0], A::mul(ns.jx[1], wu[1]));
    const C numy = A::fma(ns.jy[0], wu[0], A::mul(ns.jy[1], wu[1]));
    C Ux, Uy;
    if constexpr (kCanonical<C>) {
        Ux = A::div(numx, den);
        Uy = A::div(numy, den);
    } else {
        const C rden = __frcp_rn(den);   // one reciprocal for both components
        Ux = A::mul(numx, rden);
        Uy = A::mul(numy, rden);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const C ux = A::fma(cx.taum[k], ns.ax[k], Ux);
        const C uy = A::fma(cx.taum[k], ns.ay[k], Uy);
        const C usq = A::fma(ux, ux, A::mul(uy, uy));
        const C b = A::mul(C(1.5), usq);
        const C nk = ns.n[k];
        const C wn0 = A::mul(Wc::w0, nk), wn1 = A::mul(Wc::w1, nk), wn5 = A::mul(Wc::w5, nk);
        if constexpr (kCanonical<C>) {
            const C cu[9] = {C(0), ux, uy, -ux, -uy, A::add(ux, uy), A::add(-ux, uy), A::sub(-ux, uy), A::sub(ux, uy)};
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const C wn = i == 0 ? wn0 : (i <= 4 ? wn1 : wn5);
                const C c = cu[i];
                // Eqs. 3-5: wn (((1 + 3 c) + 4.5 (c c)) - b)
                C feq = A::mul(wn, A::sub(A::fma(C(4.5), A::mul(c, c), A::fma(C(3), c, C(1))), b));
                if constexpr (GEN) feq = A::add(feq, A::mul(cx.dA[k][grp(i)], nk));   // free alpha_k
                const C f = fc[k][i];
                fnew[k][i] = A::fma(-A::sub(f, feq), cx.itau[k], f);   // Eq. 2: f - (f - feq) / tau
            }
        } else {
            // Eqs. 3-5 by opposite pairs: feq(+-c) = wn (1 + 4.5 c^2 - b) +- 3 wn c;
            // Eq. 2 as f (1 - 1/tau) + feq / tau
            const C om = C(1) - cx.itau[k], it = cx.itau[k];
            const C base = C(1) - b;
            const C cp[4] = {ux, uy, A::add(ux, uy), A::sub(uy, ux)};
            const int ia[4] = {1, 2, 5, 6}, ib[4] = {3, 4, 7, 8};
            C moving = C(0);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const C wn = q < 2 ? wn1 : wn5;
                const C c = cp[q];
                C sy = A::mul(wn, A::fma(C(4.5), A::mul(c, c), base));
                if constexpr (GEN) sy = A::fma(cx.dA[k][q < 2 ? 1 : 2], nk, sy);   // free alpha_k
                const C an = A::mul(A::mul(C(3), wn), c);
                fnew[k][ia[q]] = A::fma(A::add(sy, an), it, A::mul(fc[k][ia[q]], om));
                fnew[k][ib[q]] = A::fma(A::sub(sy, an), it, A::mul(fc[k][ib[q]], om));
                moving = A::add(moving, A::add(fnew[k][ia[q]], fnew[k][ib[q]]));
            }
            // the collision conserves n_k: the rest population takes what the
            // moving ones leave, so FP32 rounding does not bias the mass
            fnew[k][0] = A::sub(nk, moving);
            (void)wn0;
        }
    }
}

// Steps 2-7 at one fluid node of row `rw`, column `xc` (thread t of the
// strip): densities of this and the neighbouring nodes come from the shared
// ring (slots of rows r-1, r, r+1), the node's pulled populations from fc.
// MODE 0 writes the post-collision populations, MODE 1 the whole-fluid
// velocity rho u = sum_k m_k j_k + (1/2) sum_k n_k a_k, rho = sum_k m_k n_k.
// Populations of columns 0, 1 and nx - 2, nx - 1 are also written to their
// periodic images at x = nx, nx + 1 and x = -2, -1 (ghost columns), so that
// every source row a later step reads is one contiguous window; gr / gl give
// the offsets of those images from the node (0 = none).
template <typename S, int W, int MODE, bool GH, bool G>
__device__ __forceinline__ void collide_node(const StepCtx<S, G>& cx, const typename Prec<S>::C (&fc)[2][9], unsigned m,
                                             const typename Prec<S>::C (*sd)[2][W], int s_m, int s_0, int s_p, int t,
                                             S* __restrict__ dst, unsigned plane, unsigned o, MomOut mo,
                                             long long mo_idx, int gr = 0, int gl = 0) {
    using C = typename Prec<S>::C;
    using A = Ar<C>;
    NodeState<S> ns;
    node_state<S, W>(cx, fc, m, sd, s_m, s_0, s_p, t, ns);
    if (MODE == 1) {
        C rho, px, py;
        if constexpr (G) {
            rho = A::fma(cx.m[0], ns.n[0], A::mul(cx.m[1], ns.n[1]));
            px = A::fma(cx.m[0], ns.jx[0], A::mul(cx.m[1], ns.jx[1]));
            py = A::fma(cx.m[0], ns.jy[0], A::mul(cx.m[1], ns.jy[1]));
        } else {   // m_k = 1
            rho = A::add(ns.n[0], ns.n[1]);
            px = A::add(ns.jx[0], ns.jx[1]);
            py = A::add(ns.jy[0], ns.jy[1]);
        }
        const C fxs = A::fma(ns.n[0], ns.ax[0], A::mul(ns.n[1], ns.ax[1]));
        const C fys = A::fma(ns.n[0], ns.ay[0], A::mul(ns.n[1], ns.ay[1]));
        mo.ux[mo_idx] = (double)A::div(A::fma(C(0.5), fxs, px), rho);
        mo.uy[mo_idx] = (double)A::div(A::fma(C(0.5), fys, py), rho);
        return;
    }
    C fnew[2][9];
    relax<S>(cx, fc, ns, fnew);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        S* d = dst + ((unsigned)(k * 9) * plane + o);
#pragma unroll
        for (int i = 0; i < 9; ++i) enc(d + (unsigned)i * plane, fnew[k][i], cx.sh.v[k][grp(i)]);
        if (GH) {   // ghost images of the edge columns (rare)
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                S* p = d + (unsigned)i * plane;
                if (gr) enc(p + gr, fnew[k][i], cx.sh.v[k][grp(i)]);
                if (gl) enc(p + gl, fnew[k][i], cx.sh.v[k][grp(i)]);
            }
        }
    }
}

// Dispatch: the ghost-writing variant only for the edge columns.
template <typename S, int W, int MODE, bool G>
__device__ __forceinline__ void collide_any(const StepCtx<S, G>& cx, const typename Prec<S>::C (&fc)[2][9], unsigned m,
                                            const typename Prec<S>::C (*sd)[2][W], int s_m, int s_0, int s_p, int t,
                                            S* __restrict__ dst, unsigned plane, unsigned o, MomOut mo,
                                            long long mo_idx, int gr, int gl) {
    if (gr | gl)
        collide_node<S, W, MODE, true>(cx, fc, m, sd, s_m, s_0, s_p, t, dst, plane, o, mo, mo_idx, gr, gl);
    else
        collide_node<S, W, MODE, false>(cx, fc, m, sd, s_m, s_0, s_p, t, dst, plane, o, mo, mo_idx, 0, 0);
}

// Column bookkeeping of a strip: thread t <-> column x0 - 1 + t (wrapped).
struct StripCols {
    int xc, xm, xp, ncols;
    bool dcol, coll;
    __device__ __forceinline__ StripCols(int x0, int nx, int W, int t) {
        ncols = min(W - 2, nx - x0);
        dcol = t < ncols + 2;
        coll = t >= 1 && t <= ncols;
        xc = x0 - 1 + t;
        if (xc < 0) xc += nx;
        else if (xc >= nx) xc -= nx;
        if (!dcol) xc = 0;
        xm = xc == 0 ? nx - 1 : xc - 1;
        xp = xc == nx - 1 ? 0 : xc + 1;
    }
};

// Checked builds (-DLBM_CHECKED): before touching memory, every step kernel
// checks its tile against its run and the run's layout (the invariants all
// row and column indices of the march derive from).  On a violation it sets
// ERR_BOUNDS in the handle's error word and the whole CTA returns without an
// access.  Other builds compile the check away.
__device__ __forceinline__ bool step_tile_ok(const Tile& tl, const RunDesc& rd) {
#ifdef LBM_CHECKED
    const bool ok = tl.x0 >= 0 && tl.x0 < rd.nx && tl.y0 >= 0 && tl.y0 < tl.y1 && tl.y1 <= rd.ny &&
                    rd.nx >= 1 && rd.pitch >= rd.nx + 2 * LBM_COL0 && rd.plane == (long long)rd.ny * rd.pitch;
    if (!ok && threadIdx.x == 0 && rd.err) atomicOr(rd.err, ERR_BOUNDS);
    return ok;
#else
    (void)tl;
    (void)rd;
    return true;
#endif
}

// MODE 0: one time step (read buf[parity], write buf[parity ^ 1]).
// MODE 1: moments of the step from buf[parity] (whole-fluid velocity), no write.
// Pulled populations travel through registers (plain loads).
// Occupancy target of the FP32-arithmetic register kernel: about 640
// threads per SM (96 registers); FP64 keeps the compiler's choice.
template <typename S, int W>
constexpr int kMinBlocks = (sizeof(typename Prec<S>::C) == 8 || W >= 640) ? 1 : 640 / W;

// Bulk prefetch of the strip's source rows from HBM into L2: lane q < 18 of
// warp 0 streams population plane q of a row, columns [x0 - 2, x0 + W - 1]
// rounded out to 16 bytes (contiguous thanks to the ghost columns).
template <typename S, int W>
struct RowPrefetch {
    const S* base = nullptr;   // plane q, row 0, first column of the window
    unsigned bytes = 0;
    __device__ __forceinline__ void init(const S* src, unsigned plane, int pitch, int x0) {
        constexpr int per16 = 16 / (int)sizeof(S);
        const int c0 = (x0 - 2 >= 0 ? x0 - 2 : -per16) & ~(per16 - 1);
        int c1 = min(x0 + W, pitch - LBM_COL0);
        c1 = min((c1 + per16 - 1) & ~(per16 - 1), pitch - LBM_COL0);
        if (threadIdx.x < 18 && c1 > c0) {
            base = src + (unsigned)threadIdx.x * plane + c0;
            bytes = (unsigned)((c1 - c0) * (int)sizeof(S));
        }
    }
    __device__ __forceinline__ void row(int w, int pitch) const {
        if (bytes)
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(base + (unsigned)(w * pitch)),
                         "r"(bytes)
                         : "memory");
    }
};

template <typename S, int W, int MODE, bool L2PF, bool G>
__global__ void __launch_bounds__(W, (kMinBlocks<S, W>)) k_step(const RunDesc* __restrict__ runs,
                                                              const Tile* __restrict__ tiles, int parity, MomOut mo) {
    using C = typename Prec<S>::C;
    __shared__ C sd[4][2][W];

    const Tile tl = tiles[blockIdx.x];
    const RunDesc& rd = runs[tl.run];
    if (!step_tile_ok(tl, rd)) return;
    const int nx = rd.nx, ny = rd.ny, pitch = rd.pitch;
    const long long plane = rd.plane;
    const Geo geo{nx, rd.cap_x0, rd.cap_x1, rd.y_bot, rd.y_top, rd.mask};
    const S* __restrict__ src = static_cast<const S*>(rd.buf[parity]);
    S* __restrict__ dst = static_cast<S*>(rd.buf[parity ^ 1]);
    StepCtx<S, G> cx;
    cx.load(rd);
    const int t = threadIdx.x;
    const StripCols sc(tl.x0, nx, W, t);

    C fc[2][9], fn[2][9];
    unsigned smc = 0, smn = 0;

    auto pull_row = [&](int r, C (&f)[2][9], unsigned& smask, int slot) {
        const RowIdx q = rows_of(r, ny);
        C nA = C(0), nB = C(0);
        smask = 0;
        if (sc.dcol) {
            smask = nbr_solid(geo, sc.xm, sc.xc, sc.xp, q.rm, q.rw, q.rp);
            if (!SOL(smask, 0, 0)) {
                const unsigned bw = (unsigned)(q.rw * pitch), bm = (unsigned)(q.rm * pitch),
                               bp = (unsigned)(q.rp * pitch);
                pull_node<S>(src, plane, bw + sc.xc, bw + sc.xm, bw + sc.xp, bm + sc.xc, bp + sc.xc, bm + sc.xm,
                             bm + sc.xp, bp + sc.xm, bp + sc.xp, smask, cx.sh, f);
                nA = dens9(f[0]);
                nB = dens9(f[1]);
            }
        }
        sd[slot][0][t] = nA;
        sd[slot][1][t] = nB;
    };

    // row r: pull row r + 1 into (fnext, snext), then collide row r from
    // (fcur, scur); the march alternates the two register sets so that no
    // copy is needed between rows
    RowPrefetch<S, W> pf;
    if (L2PF) pf.init(src, (unsigned)plane, pitch, tl.x0);
    auto prefetch = [&](int srow) {   // source row srow in [-2, ny + 5]
        int w = srow < 0 ? srow + ny : srow;
        w = w >= ny ? w - ny : w;
        w = w >= ny ? w % ny : w;     // only for ny < 6
        pf.row(w, pitch);
    };
    auto row = [&](int r, C (&fcur)[2][9], unsigned scur, C (&fnext)[2][9], unsigned& snext) {
        const int s_m = (r - tl.y0) & 3, s_0 = (r - tl.y0 + 1) & 3, s_p = (r - tl.y0 + 2) & 3;
        if (L2PF && r + 4 <= tl.y1 + 1) prefetch(r + 4);   // source row needed three rows later
        pull_row(r + 1, fnext, snext, s_p);
        __syncthreads();
        if (sc.coll) {
            const RowIdx q = rows_of(r, ny);
            if (!SOL(scur, 0, 0))
                collide_any<S, W, MODE>(cx, fcur, scur, sd, s_m, s_0, s_p, t, dst, plane,
                                         (unsigned)(q.rw * pitch + sc.xc), mo, (long long)q.rw * mo.nx + sc.xc,
                                         ghost_r(sc.xc, nx), ghost_l(sc.xc, nx));
            else if (MODE == 1) {
                mo.ux[(long long)q.rw * mo.nx + sc.xc] = 0.0;
                mo.uy[(long long)q.rw * mo.nx + sc.xc] = 0.0;
            }
        }
    };
    const int y0 = tl.y0, y1 = tl.y1;
    if (L2PF)
        for (int sr = y0 - 2; sr <= min(y0 + 3, y1 + 1); ++sr) prefetch(sr);
    pull_row(y0 - 1, fn, smn, 0);
    pull_row(y0, fc, smc, 1);
    int r = y0;
    for (; r + 1 < y1; r += 2) {
        row(r, fc, smc, fn, smn);
        row(r + 1, fn, smn, fc, smc);
    }
    if (r < y1) row(r, fc, smc, fn, smn);
}

// ---- species-split variant -----------------------------------------------------
// A CTA of 2W threads: thread (k, c) = (threadIdx.x / W, threadIdx.x % W)
// owns species k of strip column c (same strip/row march as k_step).  Each
// thread pulls 9 populations instead of 18, so it needs about half the
// registers and twice as many warps fit on an SM.  The species meet through
// shared memory: the density ring (both species, as in k_step) and a
// double-buffered row of momenta j_k for the common velocity.  One
// __syncthreads per row.  The arithmetic per node is that of collide_node,
// done by the thread of each species for its own populations.
template <typename S, int W, bool GH, bool GEN>
__device__ __forceinline__ void collide_species(const StepCtx<S, GEN>& cx, int k, const typename Prec<S>::C (&f)[9],
                                                unsigned m, const typename Prec<S>::C (*sd)[2][W],
                                                const typename Prec<S>::C (*jb)[W], int s_m, int s_0, int s_p, int c,
                                                S* __restrict__ dst, unsigned plane, unsigned o, int gr, int gl) {
    using C = typename Prec<S>::C;
    using Wc = Wt<C>;
    using A = Ar<C>;
    const int kb = 1 - k;
    const C nA = sd[s_0][0][c], nB = sd[s_0][1][c];
    const C jxA = jb[0][c], jyA = jb[1][c], jxB = jb[2][c], jyB = jb[3][c];
    C Wx = C(0), Wy = C(0);
    if (m) {
        if (SOL(m, 0, 1)) Wx = A::add(Wx, Wc::w1);
        if (SOL(m, 1, 0)) Wy = A::add(Wy, Wc::w1);
        if (SOL(m, 0, -1)) Wx = A::sub(Wx, Wc::w1);
        if (SOL(m, -1, 0)) Wy = A::sub(Wy, Wc::w1);
        if (SOL(m, 1, 1)) { Wx = A::add(Wx, Wc::w5); Wy = A::add(Wy, Wc::w5); }
        if (SOL(m, 1, -1)) { Wx = A::sub(Wx, Wc::w5); Wy = A::add(Wy, Wc::w5); }
        if (SOL(m, -1, -1)) { Wx = A::sub(Wx, Wc::w5); Wy = A::sub(Wy, Wc::w5); }
        if (SOL(m, -1, 1)) { Wx = A::add(Wx, Wc::w5); Wy = A::sub(Wy, Wc::w5); }
    }
    const C n1 = sd[s_0][kb][c + 1], n2 = sd[s_p][kb][c], n3 = sd[s_0][kb][c - 1], n4 = sd[s_m][kb][c],
            n5 = sd[s_p][kb][c + 1], n6 = sd[s_p][kb][c - 1], n7 = sd[s_m][kb][c - 1], n8 = sd[s_m][kb][c + 1];
    C Sx = A::fma(-Wc::w1, n3, A::mul(Wc::w1, n1));
    Sx = A::fma(Wc::w5, n5, Sx);
    Sx = A::fma(-Wc::w5, n6, Sx);
    Sx = A::fma(-Wc::w5, n7, Sx);
    Sx = A::fma(Wc::w5, n8, Sx);
    C Sy = A::fma(-Wc::w1, n4, A::mul(Wc::w1, n2));
    Sy = A::fma(Wc::w5, n5, Sy);
    Sy = A::fma(Wc::w5, n6, Sy);
    Sy = A::fma(-Wc::w5, n7, Sy);
    Sy = A::fma(-Wc::w5, n8, Sy);
    const C ax = A::add(A::sub(-A::mul(cx.G, Sx), A::mul(cx.Gw[k], Wx)), cx.gx);
    const C ay = A::add(A::sub(-A::mul(cx.G, Sy), A::mul(cx.Gw[k], Wy)), cx.gy);
    const C(&wu)[2] = cx.wU();
    const C den = A::fma(nA, wu[0], A::mul(nB, wu[1]));
    const C numx = A::fma(jxA, wu[0], A::mul(jxB, wu[1]));
    const C numy = A::fma(jyA, wu[0], A::mul(jyB, wu[1]));
    C Ux, Uy;
    if constexpr (kCanonical<C>) {
        Ux = A::div(numx, den);
        Uy = A::div(numy, den);
    } else {
        const C rden = __frcp_rn(den);
        Ux = A::mul(numx, rden);
        Uy = A::mul(numy, rden);
    }
    const C n = k == 0 ? nA : nB;
    const C ux = A::fma(cx.taum[k], ax, Ux);
    const C uy = A::fma(cx.taum[k], ay, Uy);
    const C usq = A::fma(ux, ux, A::mul(uy, uy));
    const C b = A::mul(C(1.5), usq);
    const C wn0 = A::mul(Wc::w0, n), wn1 = A::mul(Wc::w1, n), wn5 = A::mul(Wc::w5, n);
    C fnew[9];
    if constexpr (kCanonical<C>) {
        const C cu[9] = {C(0), ux, uy, -ux, -uy, A::add(ux, uy), A::add(-ux, uy), A::sub(-ux, uy), A::sub(ux, uy)};
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const C wn = i == 0 ? wn0 : (i <= 4 ? wn1 : wn5);
            const C cc = cu[i];
            C feq = A::mul(wn, A::sub(A::fma(C(4.5), A::mul(cc, cc), A::fma(C(3), cc, C(1))), b));
            if constexpr (GEN) feq = A::add(feq, A::mul(cx.dA[k][grp(i)], n));
            fnew[i] = A::fma(-A::sub(f[i], feq), cx.itau[k], f[i]);
        }
    } else {
        const C om = C(1) - cx.itau[k], it = cx.itau[k];
        const C base = C(1) - b;
        const C cp[4] = {ux, uy, A::add(ux, uy), A::sub(uy, ux)};
        const int ia[4] = {1, 2, 5, 6}, ib[4] = {3, 4, 7, 8};
        C moving = C(0);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const C wn = q < 2 ? wn1 : wn5;
            const C cc = cp[q];
            C sy = A::mul(wn, A::fma(C(4.5), A::mul(cc, cc), base));
            if constexpr (GEN) sy = A::fma(cx.dA[k][q < 2 ? 1 : 2], n, sy);
            const C an = A::mul(A::mul(C(3), wn), cc);
            fnew[ia[q]] = A::fma(A::add(sy, an), it, A::mul(f[ia[q]], om));
            fnew[ib[q]] = A::fma(A::sub(sy, an), it, A::mul(f[ib[q]], om));
            moving = A::add(moving, A::add(fnew[ia[q]], fnew[ib[q]]));
        }
        fnew[0] = A::sub(n, moving);   // exact per-node mass balance
    }
    S* d = dst + ((unsigned)(k * 9) * plane + o);
#pragma unroll
    for (int i = 0; i < 9; ++i) enc(d + (unsigned)i * plane, fnew[i], cx.sh.v[k][grp(i)]);
    if (GH) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            S* p = d + (unsigned)i * plane;
            if (gr) enc(p + gr, fnew[i], cx.sh.v[k][grp(i)]);
            if (gl) enc(p + gl, fnew[i], cx.sh.v[k][grp(i)]);
        }
    }
}

template <typename S>
__device__ __forceinline__ void pull_species(const S* __restrict__ p, unsigned plane, unsigned own, unsigned oxm,
                                             unsigned oxp, unsigned orm, unsigned orp, unsigned orm_xm,
                                             unsigned orm_xp, unsigned orp_xm, unsigned orp_xp, unsigned sm,
                                             typename Prec<S>::C sh0, typename Prec<S>::C sh1,
                                             typename Prec<S>::C sh2, typename Prec<S>::C (&f)[9]) {
    if (sm == 0) {
        f[0] = dec(ldg(p + own), sh0);
        f[1] = dec(ldg(p + (1 * plane + oxm)), sh1);
        f[2] = dec(ldg(p + (2 * plane + orm)), sh1);
        f[3] = dec(ldg(p + (3 * plane + oxp)), sh1);
        f[4] = dec(ldg(p + (4 * plane + orp)), sh1);
        f[5] = dec(ldg(p + (5 * plane + orm_xm)), sh2);
        f[6] = dec(ldg(p + (6 * plane + orm_xp)), sh2);
        f[7] = dec(ldg(p + (7 * plane + orp_xp)), sh2);
        f[8] = dec(ldg(p + (8 * plane + orp_xm)), sh2);
        return;
    }
    f[0] = dec(ldg(p + own), sh0);
    f[1] = dec(ldg(SOL(sm, 0, -1) ? p + (3 * plane + own) : p + (1 * plane + oxm)), sh1);
    f[2] = dec(ldg(SOL(sm, -1, 0) ? p + (4 * plane + own) : p + (2 * plane + orm)), sh1);
    f[3] = dec(ldg(SOL(sm, 0, 1) ? p + (1 * plane + own) : p + (3 * plane + oxp)), sh1);
    f[4] = dec(ldg(SOL(sm, 1, 0) ? p + (2 * plane + own) : p + (4 * plane + orp)), sh1);
    f[5] = dec(ldg(SOL(sm, -1, -1) ? p + (7 * plane + own) : p + (5 * plane + orm_xm)), sh2);
    f[6] = dec(ldg(SOL(sm, -1, 1) ? p + (8 * plane + own) : p + (6 * plane + orm_xp)), sh2);
    f[7] = dec(ldg(SOL(sm, 1, 1) ? p + (5 * plane + own) : p + (7 * plane + orp_xp)), sh2);
    f[8] = dec(ldg(SOL(sm, 1, -1) ? p + (6 * plane + own) : p + (8 * plane + orp_xm)), sh2);
}

template <typename S, int W>
constexpr int kSplitMinBlocks = (sizeof(typename Prec<S>::C) == 8 || 2 * W >= 1024) ? 1 : 1024 / (2 * W);

template <typename S, int W, bool G>
__global__ void __launch_bounds__(2 * W, (kSplitMinBlocks<S, W>)) k_step_split(const RunDesc* __restrict__ runs,
                                                                              const Tile* __restrict__ tiles,
                                                                              int parity) {
    using C = typename Prec<S>::C;
    using A = Ar<C>;
    __shared__ C sd[4][2][W];
    __shared__ C jb[2][4][W];   // [row parity][jxA, jyA, jxB, jyB][column]

    const Tile tl = tiles[blockIdx.x];
    const RunDesc& rd = runs[tl.run];
    if (!step_tile_ok(tl, rd)) return;
    const int nx = rd.nx, ny = rd.ny, pitch = rd.pitch;
    const long long plane = rd.plane;
    const Geo geo{nx, rd.cap_x0, rd.cap_x1, rd.y_bot, rd.y_top, rd.mask};
    const int k = threadIdx.x / W, c = threadIdx.x % W;
    const S* __restrict__ src = static_cast<const S*>(rd.buf[parity]) + (unsigned)(k * 9) * (unsigned)plane;
    S* __restrict__ dst = static_cast<S*>(rd.buf[parity ^ 1]);
    StepCtx<S, G> cx;
    cx.load(rd);
    const C sh0 = cx.sh.v[k][0], sh1 = cx.sh.v[k][1], sh2 = cx.sh.v[k][2];
    const StripCols sc(tl.x0, nx, W, c);

    auto pull_row = [&](int r, C (&f)[9], unsigned& smask, int slot) {
        const RowIdx q = rows_of(r, ny);
        C nk = C(0);
        smask = 0;
        if (sc.dcol) {
            smask = nbr_solid(geo, sc.xm, sc.xc, sc.xp, q.rm, q.rw, q.rp);
            if (!SOL(smask, 0, 0)) {
                const unsigned bw = (unsigned)(q.rw * pitch), bm = (unsigned)(q.rm * pitch),
                               bp = (unsigned)(q.rp * pitch);
                pull_species<S>(src, plane, bw + sc.xc, bw + sc.xm, bw + sc.xp, bm + sc.xc, bp + sc.xc, bm + sc.xm,
                                bm + sc.xp, bp + sc.xm, bp + sc.xp, smask, sh0, sh1, sh2, f);
                nk = dens9(f);
            }
        }
        sd[slot][k][c] = nk;
    };

    const int y0 = tl.y0, y1 = tl.y1;
    C fc[9], fn[9];
    unsigned smc = 0, smn = 0;
    pull_row(y0 - 1, fn, smn, 0);
    pull_row(y0, fc, smc, 1);
    for (int r = y0; r < y1; ++r) {
        const int s_m = (r - y0) & 3, s_0 = (r - y0 + 1) & 3, s_p = (r - y0 + 2) & 3;
        pull_row(r + 1, fn, smn, s_p);
        // momenta of this species at row r for the common velocity
        C (*j)[W] = jb[r & 1];
        if (sc.coll && !SOL(smc, 0, 0)) {
            j[2 * k][c] = A::add(A::sub(A::sub(A::add(A::sub(fc[1], fc[3]), fc[5]), fc[6]), fc[7]), fc[8]);
            j[2 * k + 1][c] = A::sub(A::sub(A::add(A::add(A::sub(fc[2], fc[4]), fc[5]), fc[6]), fc[7]), fc[8]);
        }
        __syncthreads();
        if (sc.coll && !SOL(smc, 0, 0)) {
            const RowIdx q = rows_of(r, ny);
            const int gr = ghost_r(sc.xc, nx), gl = ghost_l(sc.xc, nx);
            const unsigned o = (unsigned)(q.rw * pitch + sc.xc);
            if (gr | gl)
                collide_species<S, W, true>(cx, k, fc, smc, sd, j, s_m, s_0, s_p, c, dst, plane, o, gr, gl);
            else
                collide_species<S, W, false>(cx, k, fc, smc, sd, j, s_m, s_0, s_p, c, dst, plane, o, 0, 0);
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) fc[i] = fn[i];
        smc = smn;
    }
}

// ---- shared-memory-staged register variant -------------------------------------
// k_step's march with the pulled populations of a row parked in shared
// memory (each thread's own slot, double-buffered by row parity) until that
// row is collided, instead of held in registers across the next row's pull.
// Only the row being loaded lives in registers, so the kernel fits in 64
// registers and 1024 threads per SM: twice the nodes in flight of k_step.
template <typename S, int W>
constexpr int kSmemMinBlocks = (sizeof(typename Prec<S>::C) == 8 || W >= 1024) ? 1 : 1024 / W;

template <typename S, int W, bool G>
__global__ void __launch_bounds__(W, (kSmemMinBlocks<S, W>)) k_step_smem(const RunDesc* __restrict__ runs,
                                                                        const Tile* __restrict__ tiles,
                                                                        int parity) {
    using C = typename Prec<S>::C;
    __shared__ C sd[4][2][W];
    __shared__ C ps[2][18][W];   // [row parity][population][thread]

    const Tile tl = tiles[blockIdx.x];
    const RunDesc& rd = runs[tl.run];
    if (!step_tile_ok(tl, rd)) return;
    const int nx = rd.nx, ny = rd.ny, pitch = rd.pitch;
    const long long plane = rd.plane;
    const Geo geo{nx, rd.cap_x0, rd.cap_x1, rd.y_bot, rd.y_top, rd.mask};
    const S* __restrict__ src = static_cast<const S*>(rd.buf[parity]);
    S* __restrict__ dst = static_cast<S*>(rd.buf[parity ^ 1]);
    StepCtx<S, G> cx;
    cx.load(rd);
    const int t = threadIdx.x;
    const StripCols sc(tl.x0, nx, W, t);

    // pull row r into ps[r & 1] (own slot) and its densities into sd[slot]
    auto pull_row = [&](int r, unsigned& smask, int slot) {
        const RowIdx q = rows_of(r, ny);
        C nA = C(0), nB = C(0);
        smask = 0;
        if (sc.dcol) {
            smask = nbr_solid(geo, sc.xm, sc.xc, sc.xp, q.rm, q.rw, q.rp);
            if (!SOL(smask, 0, 0)) {
                const unsigned bw = (unsigned)(q.rw * pitch), bm = (unsigned)(q.rm * pitch),
                               bp = (unsigned)(q.rp * pitch);
                C f[2][9];
                pull_node<S>(src, (unsigned)plane, bw + sc.xc, bw + sc.xm, bw + sc.xp, bm + sc.xc, bp + sc.xc,
                             bm + sc.xm, bm + sc.xp, bp + sc.xm, bp + sc.xp, smask, cx.sh, f);
                nA = dens9(f[0]);
                nB = dens9(f[1]);
                if (sc.coll) {
#pragma unroll
                    for (int k = 0; k < 2; ++k)
#pragma unroll
                        for (int i = 0; i < 9; ++i) ps[r & 1][k * 9 + i][t] = f[k][i];
                }
            }
        }
        sd[slot][0][t] = nA;
        sd[slot][1][t] = nB;
    };

    const int y0 = tl.y0, y1 = tl.y1;
    unsigned smc = 0, smn = 0;
    pull_row(y0 - 1, smn, 0);
    pull_row(y0, smc, 1);
    for (int r = y0; r < y1; ++r) {
        const int s_m = (r - y0) & 3, s_0 = (r - y0 + 1) & 3, s_p = (r - y0 + 2) & 3;
        pull_row(r + 1, smn, s_p);
        __syncthreads();
        if (sc.coll && !SOL(smc, 0, 0)) {
            const RowIdx q = rows_of(r, ny);
            C fc[2][9];
#pragma unroll
            for (int k = 0; k < 2; ++k)
#pragma unroll
                for (int i = 0; i < 9; ++i) fc[k][i] = ps[r & 1][k * 9 + i][t];
            collide_any<S, W, 0>(cx, fc, smc, sd, s_m, s_0, s_p, t, dst, (unsigned)plane,
                                 (unsigned)(q.rw * pitch + sc.xc), MomOut{nullptr, nullptr, 0}, 0,
                                 ghost_r(sc.xc, nx), ghost_l(sc.xc, nx));
        }
        smc = smn;
    }
}

// ---- bidirectional staged variant ---------------------------------------------
// k_step_smem with two groups of W threads per CTA marching away from the
// middle row m of the tile [y0, y1): group U pulls rows m - 1, m - 2, ... up
// to the halo row y0 - 1 and collides m - 1 ... y0; group D pulls m, m + 1,
// ... down to the halo row y1 and collides m ... y1 - 1.  The two groups
// share their first rows through shared memory, so a tile of R rows pulls
// R + 2 rows in R / 2 + 1 steps (k_step_smem: R + 2 steps).  Step k: pull,
// barrier, collide.  After step 0 the groups synchronise separately (named
// barriers of W threads), so that their load and arithmetic phases drift
// apart instead of alternating in lock step (measured on the 8192x160
// capillary, tile 64x18: 41.0 us per step against 43.2 us with one CTA-wide
// barrier per step).  Only the rows of step 0 are read by the other group (at
// its step 1), after the CTA-wide barrier of step 0.  FP64 gives them density
// slots of their own, never reused within the tile (the slots of steps k >= 1
// rotate over 4 per group: group * 5 + 1 + ((k - 1) & 3)); FP32 and FP16S
// rotate all steps over 4 slots per group (group * 4 + (k & 3)) and make the
// barrier of step 2 CTA-wide too, so that no group reuses its step-0 slot (at
// step 4) before the other group has read it.
template <typename S, int W>
constexpr int kBidirMinBlocks = sizeof(typename Prec<S>::C) == 8 ? 1 : 512 / W;   // 64 registers

// bar.sync on barrier 1 or 2 (immediate ids: the kernel reserves three barriers) for N threads
template <int N>
__device__ __forceinline__ void bar_group(int g) {
    if (g == 0) asm volatile("bar.sync 1, %0;\n" ::"n"(N) : "memory");
    else asm volatile("bar.sync 2, %0;\n" ::"n"(N) : "memory");
}

template <typename S, int W, bool G>
__global__ void __launch_bounds__(2 * W, (kBidirMinBlocks<S, W>)) k_step_bidir(const RunDesc* __restrict__ runs,
                                                                              const Tile* __restrict__ tiles,
                                                                              int parity) {
    using C = typename Prec<S>::C;
    // FP32 arithmetic never reads f_0 after the pull (the rest population is
    // n_k minus the moving ones), so it stages 16 populations of the collided
    // columns only, and its density ring has no slots of their own for step 0
    // (a CTA-wide barrier at step 2 keeps them until the other group has read
    // them): 19.5 KB for W = 64, so that 8 CTAs leave L1 a 92 KB share of the
    // SM's 256 KB instead of 60 KB.  FP64 stages all 18 of every column.
    constexpr bool kF = sizeof(C) == 4;
    constexpr int NS = kF ? 4 : 5;      // density slots per group
    constexpr int NP = kF ? 16 : 18;    // staged populations per node
    constexpr int PW = kF ? W - 2 : W;  // staged columns
    __shared__ C sd[2 * NS][2][W];      // [group * NS + step slot][species][column]
    __shared__ C ps[2][2][NP][PW];      // [group][step parity][population][column]

    const Tile tl = tiles[blockIdx.x];
    const RunDesc& rd = runs[tl.run];
    if (!step_tile_ok(tl, rd)) return;
#ifdef LBM_JIT_GRID
    // compiled at run time for one grid (LBM_KERNEL_BIDIR_JIT): its sizes are
    // constants, so the plane and row offsets of the 18 loads and 18 stores
    // fold into the instructions' immediates; a run of another size is refused
    constexpr int nx = LBM_JIT_NX, ny = LBM_JIT_NY, pitch = LBM_JIT_PITCH;
    constexpr unsigned plane = LBM_JIT_PLANE;
    if (rd.nx != nx || rd.ny != ny || rd.pitch != pitch || rd.plane != (long long)plane) {
        if (threadIdx.x == 0 && rd.err) atomicOr(rd.err, ERR_BOUNDS);
        return;
    }
#else
    const int nx = rd.nx, ny = rd.ny, pitch = rd.pitch;
    const unsigned plane = (unsigned)rd.plane;
#endif
    const Geo geo{nx, rd.cap_x0, rd.cap_x1, rd.y_bot, rd.y_top, rd.mask};
    const S* __restrict__ src = static_cast<const S*>(rd.buf[parity]);
    S* __restrict__ dst = static_cast<S*>(rd.buf[parity ^ 1]);
    StepCtx<S, G> cx;
    cx.load(rd);
    const int t = threadIdx.x % W, grp_d = threadIdx.x / W;   // grp_d 0: up (U), 1: down (D)
    const StripCols sc(tl.x0, nx, W, t);
    const int y0 = tl.y0, y1 = tl.y1;
    const int m = y0 + (y1 - y0 + 1) / 2;                     // first row of D
    const int nrows = grp_d == 0 ? m - y0 : y1 - m;          // rows this group collides
    const int nsteps = (y1 - y0 + 1) / 2 + 1;                // same for both groups (U has the larger half)
    // row pulled by this group at step k (the last one is the halo row)
    auto row_at = [&](int k) { return grp_d == 0 ? m - 1 - k : m + k; };
    auto slot = [&](int g, int k) { return kF ? g * NS + (k & 3) : g * NS + (k == 0 ? 0 : 1 + ((k - 1) & 3)); };
    // staged population (kk, i) of this thread's column
    auto pidx = [&](int kk, int i) { return kF ? kk * 8 + i - 1 : kk * 9 + i; };
    const int pc = kF ? t - 1 : t;

    auto pull = [&](int k, unsigned& smask) {
        const int r = row_at(k);
        const RowIdx q = rows_of(r, ny);
        C nA = C(0), nB = C(0);
        smask = 0;
        if (sc.dcol) {
            smask = nbr_solid(geo, sc.xm, sc.xc, sc.xp, q.rm, q.rw, q.rp);
            if (!SOL(smask, 0, 0)) {
                const unsigned bw = (unsigned)(q.rw * pitch), bm = (unsigned)(q.rm * pitch),
                               bp = (unsigned)(q.rp * pitch);
                C f[2][9];
                pull_node<S>(src, plane, bw + sc.xc, bw + sc.xm, bw + sc.xp, bm + sc.xc, bp + sc.xc, bm + sc.xm,
                             bm + sc.xp, bp + sc.xm, bp + sc.xp, smask, cx.sh, f);
                nA = dens9(f[0]);
                nB = dens9(f[1]);
                if (sc.coll && k < nrows) {
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk)
#pragma unroll
                        for (int i = kF ? 1 : 0; i < 9; ++i) ps[grp_d][k & 1][pidx(kk, i)][pc] = f[kk][i];
                }
            }
        }
        sd[slot(grp_d, k)][0][t] = nA;
        sd[slot(grp_d, k)][1][t] = nB;
    };

    unsigned sm_prev = 0, sm_cur = 0;
    for (int k = 0; k < nsteps; ++k) {
        // this group pulls rows 0 .. nrows (the last is its halo row)
        if (k <= nrows) pull(k, sm_cur);
        if (k == 0 || (kF && k == 2))
            __syncthreads();
        else
            bar_group<W>(grp_d);
        // collide the row pulled at step k - 1: U row m - k, D row m + k - 1
        if (k >= 1 && k <= nrows && sc.coll && !SOL(sm_prev, 0, 0)) {
            const int r = grp_d == 0 ? m - k : m + k - 1;
            // rows r - 1, r, r + 1 as density slots: the row beyond the middle at k = 1
            // is the other group's step-0 row
            const int s_new = slot(grp_d, k), s_row = slot(grp_d, k - 1);
            const int s_old = k >= 2 ? slot(grp_d, k - 2) : slot(1 - grp_d, 0);
            const int s_m = grp_d == 0 ? s_new : s_old, s_p = grp_d == 0 ? s_old : s_new;
            C fc[2][9];
#pragma unroll
            for (int kk = 0; kk < 2; ++kk)
#pragma unroll
                for (int i = 0; i < 9; ++i)
                    fc[kk][i] = (kF && i == 0) ? C(0) : ps[grp_d][(k - 1) & 1][pidx(kk, i)][pc];
            const int rw = rows_of(r, ny).rw;
            collide_any<S, W, 0>(cx, fc, sm_prev, sd, s_m, s_row, s_p, t, dst, plane,
                                 (unsigned)(rw * pitch + sc.xc), MomOut{nullptr, nullptr, 0}, 0, ghost_r(sc.xc, nx),
                                 ghost_l(sc.xc, nx));
        }
        sm_prev = sm_cur;
    }
}

// ---- two-columns-per-thread variant ---------------------------------------------
// Thread t of a CTA of W threads owns the column pair (xa, xa + 1),
// xa = x0 - 2 + 2t with x0 even, and marches down the rows of its tile like
// k_step_smem.  Per population plane a pair needs one address: unshifted
// planes are read with one vector load (8 bytes in FP32), x-shifted ones with
// two loads at immediate offsets, and the post-collision populations go out
// as one vector store per plane.  The strip collides the 2W - 4 columns
// [x0, x0 + 2W - 4); column x0 - 1 (thread 0) and x0 + ncols are its halo.
// Pulls read the periodic images of columns -2, -1, nx, nx + 1 from the ghost
// columns (nx >= 4), so the load path never wraps in x.  Nodes next to a
// solid replace the pulled values by bounce-back loads of their own node.
template <typename S> struct Pair;
template <> struct Pair<float> {
    static __device__ __forceinline__ void ld(const float* p, float& a, float& b, float) {
        const float2 v = __ldg(reinterpret_cast<const float2*>(p));
        a = v.x;
        b = v.y;
    }
    static __device__ __forceinline__ void st(float* p, float a, float b, float) {
        *reinterpret_cast<float2*>(p) = make_float2(a, b);
    }
};
template <> struct Pair<double> {
    static __device__ __forceinline__ void ld(const double* p, double& a, double& b, double) {
        const double2 v = __ldg(reinterpret_cast<const double2*>(p));
        a = v.x;
        b = v.y;
    }
    static __device__ __forceinline__ void st(double* p, double a, double b, double) {
        *reinterpret_cast<double2*>(p) = make_double2(a, b);
    }
};
template <> struct Pair<__half> {
    static __device__ __forceinline__ void ld(const __half* p, float& a, float& b, float sh) {
        const unsigned u = __ldg(reinterpret_cast<const unsigned*>(p));
        a = dec(__ushort_as_half((unsigned short)(u & 0xffffu)), sh);
        b = dec(__ushort_as_half((unsigned short)(u >> 16)), sh);
    }
    static __device__ __forceinline__ void st(__half* p, float a, float b, float sh) {
        const unsigned lo = __half_as_ushort(__float2half_rn(__fsub_rn(a, sh)));
        const unsigned hi = __half_as_ushort(__float2half_rn(__fsub_rn(b, sh)));
        *reinterpret_cast<unsigned*>(p) = lo | (hi << 16);
    }
};


// resident CTAs per SM the register allocation aims at: 512 threads (128
// registers) for W = 64, 640 (96 registers) for W = 128; shared memory
// (45 KB per 128 threads) allows at most 640
template <typename S, int W>
constexpr int kPairMinBlocks = sizeof(typename Prec<S>::C) == 8 ? 1 : (W >= 128 ? 5 : 8);

template <typename S, int W, bool G>
__global__ void __launch_bounds__(W, (kPairMinBlocks<S, W>)) k_step_pair(const RunDesc* __restrict__ runs,
                                                                        const Tile* __restrict__ tiles, int parity) {
    using C = typename Prec<S>::C;
    constexpr int NC = 2 * W;                       // ring columns: strip column c <-> x = x0 - 2 + c
    __shared__ __align__(16) C sd[4][2][NC];
    __shared__ __align__(16) C ps[2][18][NC];       // [row parity][population][strip column]

    const Tile tl = tiles[blockIdx.x];
    const RunDesc& rd = runs[tl.run];
    if (!step_tile_ok(tl, rd)) return;
    const int nx = rd.nx, ny = rd.ny, pitch = rd.pitch;
    const unsigned plane = (unsigned)rd.plane;
    const Geo geo{nx, rd.cap_x0, rd.cap_x1, rd.y_bot, rd.y_top, rd.mask};
    const S* __restrict__ src = static_cast<const S*>(rd.buf[parity]);
    S* __restrict__ dst = static_cast<S*>(rd.buf[parity ^ 1]);
    StepCtx<S, G> cx;
    cx.load(rd);
    const int t = threadIdx.x;
    const int x0 = tl.x0;
    const int ncols = min(NC - 4, nx - x0);
    const int c0 = 2 * t;                           // strip column of node 0
    const int xa = x0 - 2 + c0;                     // unwrapped column of node 0, in [-2, nx + 1] when active
    const bool act = c0 <= ncols + 2;
    bool need[2], coll[2];
    int xw[2], xmw[2], xpw[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int c = c0 + j;
        need[j] = act && c >= 1 && c <= ncols + 2;
        coll[j] = act && c >= 2 && c < ncols + 2;
        int x = xa + j;
        x = x < 0 ? x + nx : (x >= nx ? x - nx : x);
        if (!act) x = 0;
        xw[j] = x;
        xmw[j] = x == 0 ? nx - 1 : x - 1;
        xpw[j] = x == nx - 1 ? 0 : x + 1;
    }

    // pull row r for both nodes, densities into ring slot `slot`, populations
    // into ps[r & 1] when `stage`
    auto pull_row = [&](int r, unsigned (&sm)[2], int slot, bool stage) {
        C n[2][2] = {{C(0), C(0)}, {C(0), C(0)}};   // [node][species]
        sm[0] = sm[1] = 0;
        if (act) {
            const RowIdx q = rows_of(r, ny);
            sm[0] = nbr_solid(geo, xmw[0], xw[0], xpw[0], q.rm, q.rw, q.rp);
            sm[1] = nbr_solid(geo, xmw[1], xw[1], xpw[1], q.rm, q.rw, q.rp);
            const S* Pw = src + (q.rw * pitch + xa);
            const S* Pm = src + (q.rm * pitch + xa);
            const S* Pp = src + (q.rp * pitch + xa);
            C f[2][2][9];   // [node][species][direction]
#pragma unroll
            for (int k = 0; k < 2; ++k)
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const S* P = (cyo(i) == 0 ? Pw : (cyo(i) > 0 ? Pm : Pp)) + (unsigned)(9 * k + i) * plane;
                    const C sh = cx.sh.v[k][grp(i)];
                    if (cxo(i) == 0) {
                        Pair<S>::ld(P, f[0][k][i], f[1][k][i], sh);
                    } else if (cxo(i) > 0) {   // source column x - 1
                        f[0][k][i] = dec(ldg(P - 1), sh);
                        f[1][k][i] = dec(ldg(P), sh);
                    } else {                   // source column x + 1
                        f[0][k][i] = dec(ldg(P + 1), sh);
                        f[1][k][i] = dec(ldg(P + 2), sh);
                    }
                }
            if (sm[0] | sm[1]) {   // half-way bounce-back next to a solid (step 1)
#pragma unroll
                for (int j = 0; j < 2; ++j)
                    if (sm[j] && !SOL(sm[j], 0, 0)) {
#pragma unroll
                        for (int k = 0; k < 2; ++k)
#pragma unroll
                            for (int i = 1; i < 9; ++i)
                                if (SOL(sm[j], -cyo(i), -cxo(i)))
                                    f[j][k][i] = dec(ldg(Pw + (unsigned)(9 * k + opp(i)) * plane + j),
                                                     cx.sh.v[k][grp(i)]);
                    }
            }
#pragma unroll
            for (int j = 0; j < 2; ++j)
                if (need[j] && !SOL(sm[j], 0, 0)) {
                    n[j][0] = dens9(f[j][0]);
                    n[j][1] = dens9(f[j][1]);
                }
            if (stage) {
#pragma unroll
                for (int k = 0; k < 2; ++k)
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        ps[r & 1][9 * k + i][c0] = f[0][k][i];
                        ps[r & 1][9 * k + i][c0 + 1] = f[1][k][i];
                    }
            }
        }
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            sd[slot][k][c0] = n[0][k];
            sd[slot][k][c0 + 1] = n[1][k];
        }
    };

    const int y0 = tl.y0, y1 = tl.y1;
    unsigned smc[2] = {0, 0}, smn[2] = {0, 0};
    pull_row(y0 - 1, smn, 0, false);
    pull_row(y0, smc, 1, true);
    for (int r = y0; r < y1; ++r) {
        const int s_m = (r - y0) & 3, s_0 = (r - y0 + 1) & 3, s_p = (r - y0 + 2) & 3;
        pull_row(r + 1, smn, s_p, r + 1 < y1);
        __syncthreads();
        const bool f0 = coll[0] && !SOL(smc[0], 0, 0), f1 = coll[1] && !SOL(smc[1], 0, 0);
        if (f0 | f1) {
            const int rw = rows_of(r, ny).rw;
            S* Q = dst + (rw * pitch + xa);
            C fn0[2][9], fn1[2][9];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                if (!(j == 0 ? f0 : f1)) continue;
                C fc[2][9];
#pragma unroll
                for (int k = 0; k < 2; ++k)
#pragma unroll
                    for (int i = 0; i < 9; ++i) fc[k][i] = ps[r & 1][9 * k + i][c0 + j];
                NodeState<S> ns;
                node_state<S, NC>(cx, fc, smc[j], sd, s_m, s_0, s_p, c0 + j, ns);
                relax<S>(cx, fc, ns, j == 0 ? fn0 : fn1);
            }
            if (f0 & f1) {
#pragma unroll
                for (int k = 0; k < 2; ++k)
#pragma unroll
                    for (int i = 0; i < 9; ++i)
                        Pair<S>::st(Q + (unsigned)(9 * k + i) * plane, fn0[k][i], fn1[k][i], cx.sh.v[k][grp(i)]);
            } else {
#pragma unroll
                for (int k = 0; k < 2; ++k)
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        S* d = Q + (unsigned)(9 * k + i) * plane;
                        if (f0) enc(d, fn0[k][i], cx.sh.v[k][grp(i)]);
                        if (f1) enc(d + 1, fn1[k][i], cx.sh.v[k][grp(i)]);
                    }
            }
            // ghost images of the edge columns (rare)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int gr = ghost_r(xw[j], nx), gl = ghost_l(xw[j], nx);
                if ((j == 0 ? f0 : f1) && (gr | gl)) {
#pragma unroll
                    for (int k = 0; k < 2; ++k)
#pragma unroll
                        for (int i = 0; i < 9; ++i) {
                            S* d = Q + (unsigned)(9 * k + i) * plane + j;
                            const C v = j == 0 ? fn0[k][i] : fn1[k][i];
                            if (gr) enc(d + gr, v, cx.sh.v[k][grp(i)]);
                            if (gl) enc(d + gl, v, cx.sh.v[k][grp(i)]);
                        }
                }
            }
        }
        smc[0] = smn[0];
        smc[1] = smn[1];
    }
}

// ---- one-node-per-thread tile variant ----------------------------------------------
// A CTA of W x TY threads pulls the W x TY nodes of columns x0 - 1 .. x0 + W - 2
// and rows y0 - 1 .. y0 + TY - 2 at once (every thread's 18 loads in flight
// together, no march), puts their densities in shared memory, and after one
// __syncthreads collides the (W - 2) x (TY - 2) interior.  The halo nodes cost
// redundant pulls (L2 hits) instead of serial row latency.  Pulls read the
// ghost columns, so no x index wraps on the load path (nx >= 4).
template <typename S, int W, int TY>
constexpr int kTileMinBlocks = sizeof(typename Prec<S>::C) == 8 ? 1 : 1024 / (W * TY);   // 64 registers

template <typename S, int W, int TY, bool G>
__global__ void __launch_bounds__(W * TY, (kTileMinBlocks<S, W, TY>)) k_step_tile(const RunDesc* __restrict__ runs,
                                                                                const Tile* __restrict__ tiles,
                                                                                int parity) {
    using C = typename Prec<S>::C;
    __shared__ C sd[TY][2][W];   // [tile row][species][tile column]

    const Tile tl = tiles[blockIdx.x];
    const RunDesc& rd = runs[tl.run];
    if (!step_tile_ok(tl, rd)) return;
    const int nx = rd.nx, ny = rd.ny, pitch = rd.pitch;
    const unsigned plane = (unsigned)rd.plane;
    const S* __restrict__ src = static_cast<const S*>(rd.buf[parity]);
    const int tx = threadIdx.x % W, ty = threadIdx.x / W;
    const int x = tl.x0 - 1 + tx;                          // unwrapped column, in [-1, nx] when active
    const int r = tl.y0 - 1 + ty;                          // unwrapped row, in [-1, ny] when active
    const bool act = x <= min(tl.x0 + W - 2, nx) && r <= tl.y1;
    StepCtx<S, G> cx;
    cx.load(rd);
    const RowIdx q = rows_of(act ? r : 0, ny);
    const int xw = x < 0 ? x + nx : (x >= nx ? x - nx : x);
    unsigned m = 0;
    C f[2][9];
    C nA = C(0), nB = C(0);
    if (act) {
        const Geo geo{nx, rd.cap_x0, rd.cap_x1, rd.y_bot, rd.y_top, rd.mask};
        m = nbr_solid(geo, xw == 0 ? nx - 1 : xw - 1, xw, xw == nx - 1 ? 0 : xw + 1, q.rm, q.rw, q.rp);
        if (!SOL(m, 0, 0)) {
            // offsets from column -2, so that every offset is non-negative
            const unsigned bw = (unsigned)(q.rw * pitch), bm = (unsigned)(q.rm * pitch), bp = (unsigned)(q.rp * pitch);
            const unsigned xo = (unsigned)(x + 2);
            pull_node<S>(src - 2, plane, bw + xo, bw + (xo - 1), bw + (xo + 1), bm + xo, bp + xo, bm + (xo - 1),
                         bm + (xo + 1), bp + (xo - 1), bp + (xo + 1), m, cx.sh, f);
            nA = dens9(f[0]);
            nB = dens9(f[1]);
        }
    }
    sd[ty][0][tx] = nA;
    sd[ty][1][tx] = nB;
    __syncthreads();
    const bool coll = act && tx >= 1 && tx < W - 1 && x < nx && ty >= 1 && ty < TY - 1 && r < tl.y1;
    if (coll && !SOL(m, 0, 0))
        collide_any<S, W, 0>(cx, f, m, sd, ty - 1, ty, ty + 1, tx, static_cast<S*>(rd.buf[parity ^ 1]), plane,
                             (unsigned)(q.rw * pitch + xw), MomOut{nullptr, nullptr, 0}, 0, ghost_r(xw, nx),
                             ghost_l(xw, nx));
}

// ---- software-pipelined staged variant ---------------------------------------
// k_step_smem's march with the loads of row r + 2 issued (into raw
// registers) before row r is collided, and decoded (densities into the ring,
// populations into a 3-row shared-memory stage) only after the collision:
// every thread keeps a row of HBM reads in flight through the arithmetic of
// the previous one.  Same column/row march, same collision, same bits.
template <typename S>
__device__ __forceinline__ void issue_pull(const S* __restrict__ src, unsigned plane, unsigned own, unsigned oxm,
                                           unsigned oxp, unsigned orm, unsigned orp, unsigned orm_xm,
                                           unsigned orm_xp, unsigned orp_xm, unsigned orp_xp, unsigned sm,
                                           S (&raw)[18]) {
    if (sm == 0) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const S* p = src + (unsigned)(k * 9) * plane;
            S* r = raw + k * 9;
            r[0] = ldg(p + own);
            r[1] = ldg(p + (1 * plane + oxm));
            r[2] = ldg(p + (2 * plane + orm));
            r[3] = ldg(p + (3 * plane + oxp));
            r[4] = ldg(p + (4 * plane + orp));
            r[5] = ldg(p + (5 * plane + orm_xm));
            r[6] = ldg(p + (6 * plane + orm_xp));
            r[7] = ldg(p + (7 * plane + orp_xp));
            r[8] = ldg(p + (8 * plane + orp_xm));
        }
        return;
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const S* p = src + (unsigned)(k * 9) * plane;
        S* r = raw + k * 9;
        r[0] = ldg(p + own);
        r[1] = ldg(SOL(sm, 0, -1) ? p + (3 * plane + own) : p + (1 * plane + oxm));
        r[2] = ldg(SOL(sm, -1, 0) ? p + (4 * plane + own) : p + (2 * plane + orm));
        r[3] = ldg(SOL(sm, 0, 1) ? p + (1 * plane + own) : p + (3 * plane + oxp));
        r[4] = ldg(SOL(sm, 1, 0) ? p + (2 * plane + own) : p + (4 * plane + orp));
        r[5] = ldg(SOL(sm, -1, -1) ? p + (7 * plane + own) : p + (5 * plane + orm_xm));
        r[6] = ldg(SOL(sm, -1, 1) ? p + (8 * plane + own) : p + (6 * plane + orm_xp));
        r[7] = ldg(SOL(sm, 1, 1) ? p + (5 * plane + own) : p + (7 * plane + orp_xp));
        r[8] = ldg(SOL(sm, 1, -1) ? p + (6 * plane + own) : p + (8 * plane + orp_xm));
    }
}

template <typename S, int W>
constexpr int kPipeMinBlocks = (sizeof(typename Prec<S>::C) == 8 || W >= 768) ? 1 : 768 / W;   // <= 85 registers

template <typename S, int W, bool G>
__global__ void __launch_bounds__(W, (kPipeMinBlocks<S, W>)) k_step_pf(const RunDesc* __restrict__ runs,
                                                                      const Tile* __restrict__ tiles, int parity) {
    using C = typename Prec<S>::C;
    __shared__ C sd[4][2][W];
    __shared__ C ps[3][18][W];   // pulled populations of rows y0 + 3m + {0, 1, 2}: [row][population][thread]

    const Tile tl = tiles[blockIdx.x];
    const RunDesc& rd = runs[tl.run];
    if (!step_tile_ok(tl, rd)) return;
    const int nx = rd.nx, ny = rd.ny, pitch = rd.pitch;
    const unsigned plane = (unsigned)rd.plane;
    const Geo geo{nx, rd.cap_x0, rd.cap_x1, rd.y_bot, rd.y_top, rd.mask};
    const S* __restrict__ src = static_cast<const S*>(rd.buf[parity]);
    S* __restrict__ dst = static_cast<S*>(rd.buf[parity ^ 1]);
    StepCtx<S, G> cx;
    cx.load(rd);
    const int t = threadIdx.x;
    const StripCols sc(tl.x0, nx, W, t);
    const int y0 = tl.y0, y1 = tl.y1;

    // issue the loads of row p into raw; smask = solid flags around (x, p)
    auto issue = [&](int p, S (&raw)[18], unsigned& smask) {
        const RowIdx q = rows_of(p, ny);
        smask = 0;
        if (sc.dcol) {
            smask = nbr_solid(geo, sc.xm, sc.xc, sc.xp, q.rm, q.rw, q.rp);
            if (!SOL(smask, 0, 0)) {
                const unsigned bw = (unsigned)(q.rw * pitch), bm = (unsigned)(q.rm * pitch),
                               bp = (unsigned)(q.rp * pitch);
                issue_pull<S>(src, plane, bw + sc.xc, bw + sc.xm, bw + sc.xp, bm + sc.xc, bp + sc.xc, bm + sc.xm,
                              bm + sc.xp, bp + sc.xm, bp + sc.xp, smask, raw);
            }
        }
    };
    // decode pulled row p: densities into ring slot `slot`, populations into
    // ps when p is a collided row of the tile
    auto finish = [&](int p, const S (&raw)[18], unsigned smask, int slot) {
        C nA = C(0), nB = C(0);
        if (sc.dcol && !SOL(smask, 0, 0)) {
            C f[2][9];
#pragma unroll
            for (int k = 0; k < 2; ++k)
#pragma unroll
                for (int i = 0; i < 9; ++i) f[k][i] = dec(raw[k * 9 + i], cx.sh.v[k][grp(i)]);
            nA = dens9(f[0]);
            nB = dens9(f[1]);
            if (sc.coll && p >= y0 && p < y1) {
                const int b = (p - y0) % 3;
#pragma unroll
                for (int k = 0; k < 2; ++k)
#pragma unroll
                    for (int i = 0; i < 9; ++i) ps[b][k * 9 + i][t] = f[k][i];
            }
        }
        sd[slot][0][t] = nA;
        sd[slot][1][t] = nB;
    };

    S rn[18];
    unsigned smc = 0, smn = 0, smq = 0;
    issue(y0 - 1, rn, smq);
    finish(y0 - 1, rn, smq, 0);        // halo row: densities only
    issue(y0, rn, smc);
    finish(y0, rn, smc, 1);
    issue(y0 + 1, rn, smn);
    finish(y0 + 1, rn, smn, 2);
    __syncthreads();
    for (int r = y0; r < y1; ++r) {
        const int s_m = (r - y0) & 3, s_0 = (r - y0 + 1) & 3, s_p = (r - y0 + 2) & 3, s_n = (r - y0 + 3) & 3;
        // the loads of row r + 2 stay in flight while row r is collided
        const bool ahead = r + 2 <= y1;
        if (ahead) issue(r + 2, rn, smq);
        if (sc.coll && !SOL(smc, 0, 0)) {
            const int b = (r - y0) % 3;
            C fc[2][9];
#pragma unroll
            for (int k = 0; k < 2; ++k)
#pragma unroll
                for (int i = 0; i < 9; ++i) fc[k][i] = ps[b][k * 9 + i][t];
            const int rw = rows_of(r, ny).rw;
            collide_any<S, W, 0>(cx, fc, smc, sd, s_m, s_0, s_p, t, dst, plane, (unsigned)(rw * pitch + sc.xc),
                                  MomOut{nullptr, nullptr, 0}, 0, ghost_r(sc.xc, nx), ghost_l(sc.xc, nx));
        }
        // slot s_n held row r - 2, last read by the collision of row r - 1
        if (ahead) finish(r + 2, rn, smq, s_n);
        __syncthreads();
        smc = smn;
        smn = smq;
    }
}

// ---- asynchronous-copy variant ---------------------------------------------
// Same arithmetic and the same strip/row march as k_step, but each thread's
// 18 pulled values of a row are fetched with cp.async into a D-deep ring of
// shared-memory stages, D - 1 rows ahead of the row being consumed.  The
// loads in flight then live in shared memory instead of registers, so every
// CTA keeps several rows of HBM reads outstanding.  Each thread reads back
// only the values it copied itself, so the stage ring needs no barrier; only
// the density ring does (one __syncthreads per row, as in k_step).
__device__ __forceinline__ void cp_async(void* smem, const void* gmem, int bytes_is_8) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    if (bytes_is_8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <typename S, int W, int D, bool G>
__global__ void __launch_bounds__(W) k_step_async(const RunDesc* __restrict__ runs, const Tile* __restrict__ tiles,
                                                  int parity) {
    static_assert(sizeof(S) == 4 || sizeof(S) == 8, "cp.async needs 4- or 8-byte elements");
    using C = typename Prec<S>::C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S* stage = reinterpret_cast<S*>(smem_raw);                        // [D][18][W]
    C(*sd)[2][W] = reinterpret_cast<C(*)[2][W]>(smem_raw + (size_t)D * 18 * W * sizeof(S));   // [4][2][W]

    const Tile tl = tiles[blockIdx.x];
    const RunDesc& rd = runs[tl.run];
    if (!step_tile_ok(tl, rd)) return;
    const int nx = rd.nx, ny = rd.ny, pitch = rd.pitch;
    const long long plane = rd.plane;
    const Geo geo{nx, rd.cap_x0, rd.cap_x1, rd.y_bot, rd.y_top, rd.mask};
    const S* __restrict__ src = static_cast<const S*>(rd.buf[parity]);
    S* __restrict__ dst = static_cast<S*>(rd.buf[parity ^ 1]);
    StepCtx<S, G> cx;
    cx.load(rd);
    const int t = threadIdx.x;
    const StripCols sc(tl.x0, nx, W, t);
    const int y0 = tl.y0, y1 = tl.y1;

    // issue the pulls of row p into stage slot p % D; returns nothing, the
    // solid mask of row p is recomputed when the row is consumed
    auto issue = [&](int p) {
        if (p <= y1 && sc.dcol) {
            const RowIdx q = rows_of(p, ny);
            const unsigned m = nbr_solid(geo, sc.xm, sc.xc, sc.xp, q.rm, q.rw, q.rp);
            if (!SOL(m, 0, 0)) {
                const unsigned bw = (unsigned)(q.rw * pitch), bm = (unsigned)(q.rm * pitch),
                               bp = (unsigned)(q.rp * pitch);
                const long long own = bw + sc.xc;
                S* st = stage + (size_t)(((p - y0 + 1) % D) * 18) * W + t;
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const S* pk = src + (long long)k * 9 * plane;
                    S* sk = st + k * 9 * W;
                    const int b8 = sizeof(S) == 8;
                    cp_async(sk + 0 * W, pk + own, b8);
                    cp_async(sk + 1 * W, SOL(m, 0, -1) ? pk + 3 * plane + own : pk + 1 * plane + bw + sc.xm, b8);
                    cp_async(sk + 2 * W, SOL(m, -1, 0) ? pk + 4 * plane + own : pk + 2 * plane + bm + sc.xc, b8);
                    cp_async(sk + 3 * W, SOL(m, 0, 1) ? pk + 1 * plane + own : pk + 3 * plane + bw + sc.xp, b8);
                    cp_async(sk + 4 * W, SOL(m, 1, 0) ? pk + 2 * plane + own : pk + 4 * plane + bp + sc.xc, b8);
                    cp_async(sk + 5 * W, SOL(m, -1, -1) ? pk + 7 * plane + own : pk + 5 * plane + bm + sc.xm, b8);
                    cp_async(sk + 6 * W, SOL(m, -1, 1) ? pk + 8 * plane + own : pk + 6 * plane + bm + sc.xp, b8);
                    cp_async(sk + 7 * W, SOL(m, 1, 1) ? pk + 5 * plane + own : pk + 7 * plane + bp + sc.xp, b8);
                    cp_async(sk + 8 * W, SOL(m, 1, -1) ? pk + 6 * plane + own : pk + 8 * plane + bp + sc.xm, b8);
                }
            }
        }
        cp_commit();
    };
    // consume row p: copy this thread's staged values out, densities to the ring
    auto consume = [&](int p, C (&f)[2][9], unsigned& smask, int slot) {
        const RowIdx q = rows_of(p, ny);
        C nA = C(0), nB = C(0);
        smask = 0;
        if (sc.dcol) {
            smask = nbr_solid(geo, sc.xm, sc.xc, sc.xp, q.rm, q.rw, q.rp);
            if (!SOL(smask, 0, 0)) {
                const S* st = stage + (size_t)(((p - y0 + 1) % D) * 18) * W + t;
#pragma unroll
                for (int k = 0; k < 2; ++k)
#pragma unroll
                    for (int i = 0; i < 9; ++i) f[k][i] = dec(st[(k * 9 + i) * W], cx.sh.v[k][grp(i)]);
                nA = dens9(f[0]);
                nB = dens9(f[1]);
            }
        }
        sd[slot][0][t] = nA;
        sd[slot][1][t] = nB;
    };

    C fc[2][9], fn[2][9];
    unsigned smc = 0, smn = 0;
#pragma unroll
    for (int j = 0; j < D; ++j) issue(y0 - 1 + j);
    cp_wait<D - 1>();
    consume(y0 - 1, fn, smn, 0);
    issue(y0 - 1 + D);
    cp_wait<D - 1>();
    consume(y0, fc, smc, 1);
    issue(y0 + D);
    for (int r = y0; r < y1; ++r) {
        const int s_m = (r - y0) & 3, s_0 = (r - y0 + 1) & 3, s_p = (r - y0 + 2) & 3;
        cp_wait<D - 1>();
        consume(r + 1, fn, smn, s_p);
        issue(r + 1 + D);
        __syncthreads();
        if (sc.coll && !SOL(smc, 0, 0)) {
            const RowIdx q = rows_of(r, ny);
            collide_any<S, W, 0>(cx, fc, smc, sd, s_m, s_0, s_p, t, dst, plane, (unsigned)(q.rw * pitch + sc.xc),
                                  MomOut{nullptr, nullptr, 0}, 0, ghost_r(sc.xc, nx), ghost_l(sc.xc, nx));
        }
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
            for (int i = 0; i < 9; ++i) fc[k][i] = fn[k][i];
        smc = smn;
    }
    cp_wait<0>();
}

// ---- TMA-staged variant ------------------------------------------------------
// Bulk copies (cp.async.bulk, issued by 18 lanes of warp 0, one population
// plane each) stream the source data of every row the CTA pulls into a ring
// of D slots of shared memory, one slot per pulled row: slot p holds plane i
// of source row p - c_iy (a contiguous window of that row, thanks to the
// ghost columns), completing on the slot's mbarrier.  Row p's slot is read
// twice: by the pull that feeds the density ring (iteration p - 1) and by the
// collision of row p (iteration p), which re-reads its populations from the
// slot instead of holding them in registers.  A slot is refilled with row
// p + D once the barrier of iteration p + 1 has passed, so D - 2 rows are in
// flight beyond the one being pulled and the HBM reads need no registers.
// All shared-memory reads of a row use compile-time offsets from one base.
//
// Column mapping: a CTA collides the Wc = W - 8 columns [x0, x0 + Wc)
// (x0 a multiple of 8, so global stores of a warp start on a 32-byte
// sector); thread t < Wc owns column x0 + t, threads Wc and Wc + 1 supply the
// densities of the halo columns x0 - 1 and x0 + Wc.  The density ring is
// indexed by column offset j + 1 (j in [-1, Wc]).
//
// Every mbarrier wait is bounded: a thread that gives up sets a flag, the
// per-row __syncthreads_or makes the exit block-uniform, the CTA drains the
// copies it issued (bounded again) and records ERR_TIMEOUT.
constexpr long long kWaitCycles = 2000000000LL;   // ~1 s of SM clock per wait

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait (by elapsed SM cycles, whatever each try_wait suspends for);
// returns false if the phase did not complete in time.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, long long limit = kWaitCycles) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long start = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - start > limit) return false;
    return true;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

template <typename S, int W, int D>
struct TmaGeom {
    static constexpr int Wc = W - 8;                      // collided columns per CTA
    static constexpr int OFF = 16 / (int)sizeof(S);       // window starts OFF columns before x0
    static constexpr int WIN = Wc + 2 * OFF;              // window width (elements), 16-byte multiple
    static constexpr size_t slot_elems = (size_t)18 * WIN;
    static constexpr size_t ring_bytes = (size_t)D * slot_elems * sizeof(S);
    static constexpr size_t smem_bytes() {
        return ring_bytes + 4 * 2 * W * sizeof(typename Prec<S>::C) + D * sizeof(uint64_t) + 16;
    }
};

// Pulled populations of one node from a ring slot: P points at the node's
// column in plane 0 of the slot (row offsets c_iy were applied by the copy).
template <typename S, int WIN>
__device__ __forceinline__ void pull_slot(const S* P, unsigned m, const Shift<S>& sh, typename Prec<S>::C (&f)[2][9]) {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const S* q = P + k * 9 * WIN;
        f[k][0] = dec(q[0], sh.v[k][0]);
        f[k][1] = dec(q[1 * WIN - 1], sh.v[k][1]);
        f[k][2] = dec(q[2 * WIN], sh.v[k][1]);
        f[k][3] = dec(q[3 * WIN + 1], sh.v[k][1]);
        f[k][4] = dec(q[4 * WIN], sh.v[k][1]);
        f[k][5] = dec(q[5 * WIN - 1], sh.v[k][2]);
        f[k][6] = dec(q[6 * WIN + 1], sh.v[k][2]);
        f[k][7] = dec(q[7 * WIN + 1], sh.v[k][2]);
        f[k][8] = dec(q[8 * WIN - 1], sh.v[k][2]);
    }
}

// pull_slot next to a solid: bounce-back takes the node's own opposite
// population F_opp(i)(x), read from the source buffer (gown: the node in
// plane 0), since the slot holds the planes of other rows for c_iy != 0.
template <typename S, int WIN>
__device__ __forceinline__ void pull_slot_bb(const S* P, unsigned m, const Shift<S>& sh, const S* __restrict__ gown,
                                             unsigned plane, typename Prec<S>::C (&f)[2][9]) {
    pull_slot<S, WIN>(P, m, sh, f);
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int i = 1; i < 9; ++i)
            if (SOL(m, -cyo(i), -cxo(i))) f[k][i] = dec(ldg(gown + (unsigned)(9 * k + opp(i)) * plane), sh.v[k][grp(i)]);
}

template <typename S, int W, int D, bool G>
__global__ void __launch_bounds__(W) k_step_tma(const RunDesc* __restrict__ runs, const Tile* __restrict__ tiles,
                                                int parity, uint32_t* __restrict__ err) {
    using C = typename Prec<S>::C;
    using TG = TmaGeom<S, W, D>;
    constexpr int Wc = TG::Wc, OFF = TG::OFF, WIN = TG::WIN;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    S* ring = reinterpret_cast<S*>(smem_raw);                                              // [D][18][WIN]
    C(*sd)[2][W] = reinterpret_cast<C(*)[2][W]>(smem_raw + TG::ring_bytes);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + TG::ring_bytes + 4 * 2 * W * sizeof(C));

    const Tile tl = tiles[blockIdx.x];
    const RunDesc& rd = runs[tl.run];
    if (!step_tile_ok(tl, rd)) return;
    const int nx = rd.nx, ny = rd.ny, pitch = rd.pitch;
    const unsigned plane = (unsigned)rd.plane;
    const Geo geo{nx, rd.cap_x0, rd.cap_x1, rd.y_bot, rd.y_top, rd.mask};
    const S* __restrict__ src = static_cast<const S*>(rd.buf[parity]);
    S* __restrict__ dst = static_cast<S*>(rd.buf[parity ^ 1]);
    StepCtx<S, G> cx;
    cx.load(rd);
    const int t = threadIdx.x;
    const int x0 = tl.x0, y0 = tl.y0, y1 = tl.y1;
    const int ncols = min(Wc, nx - x0);
    // column of this thread: j in [-1, ncols] (density), -2 = idle
    int j = -2;
    if (t < ncols) j = t;
    else if (t == Wc) j = -1;
    else if (t == Wc + 1) j = ncols;
    const bool dcol = j >= -1;
    const bool coll = j >= 0 && j < ncols;
    int xc = x0 + j;
    if (xc < 0) xc += nx;
    else if (xc >= nx) xc -= nx;
    if (!dcol) xc = 0;
    const int xm = xc == 0 ? nx - 1 : xc - 1;
    const int xp = xc == nx - 1 ? 0 : xc + 1;
    const int sdc = j + 1;                 // density ring column
    const int wc = (dcol ? j : 0) + OFF;   // column of this node inside a window
    // window bytes of one plane row, clipped to the allocated row
    const int win_elems = min(WIN, (pitch - LBM_COL0) - (x0 - OFF));
    const unsigned win_bytes = (unsigned)(win_elems * (int)sizeof(S));
    const int npull = (y1 - y0) + 2;       // pulled rows y0 - 1 .. y1: sequence numbers 0 .. npull - 1

    if (t == 0) {
        for (int q = 0; q < D; ++q) mbar_init(&bars[q], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();

    // warp 0 issues the pulled rows sq = issued .. last; lane q < 18 copies
    // plane q of source row (y0 - 1 + sq) - c_qy into slot sq % D
    int issued = 0;   // meaningful in warp 0 only (all its lanes agree)
    auto issue_upto = [&](int last) {
        for (; issued <= last && issued < npull; ++issued) {
            const int sq = issued, slot = sq % D;
            if (t == 0) mbar_expect_tx(&bars[slot], 18u * win_bytes);
            if (t < 18) {
                int row = y0 - 1 + sq - cyo(t % 9);                            // in [-2, ny + 1]
                row = row < 0 ? row + ny : (row >= ny ? row - ny : row);
                row = row < 0 ? row + ny : (row >= ny ? row - ny : row);       // ny = 1
                const S* g = src + ((unsigned)t * plane + (unsigned)(row * pitch)) + (x0 - OFF);
                bulk_g2s(ring + (size_t)slot * TG::slot_elems + t * WIN, g, win_bytes, &bars[slot]);
            }
        }
    };
    bool timed_out = false;
    auto wait_row = [&](int sq) {
        if (!timed_out && !mbar_wait(&bars[sq % D], (unsigned)((sq / D) & 1))) timed_out = true;
    };
    // pulled populations of this node in row sequence sq (row y0 - 1 + sq)
    auto pull = [&](int sq, int rw, unsigned m, C (&f)[2][9]) {
        const S* P = ring + (size_t)(sq % D) * TG::slot_elems + wc;
        if (m == 0) pull_slot<S, WIN>(P, 0, cx.sh, f);
        else pull_slot_bb<S, WIN>(P, m, cx.sh, src + (rw * pitch + xc), plane, f);
    };
    // densities of row sequence sq into density-ring slot `slot_d`
    auto pull_dens = [&](int sq, unsigned& smask, int slot_d) {
        const RowIdx q = rows_of(y0 - 1 + sq, ny);
        C nA = C(0), nB = C(0);
        smask = 0;
        if (dcol) {
            smask = nbr_solid(geo, xm, xc, xp, q.rm, q.rw, q.rp);
            if (!SOL(smask, 0, 0)) {
                C f[2][9];
                pull(sq, q.rw, smask, f);
                nA = dens9(f[0]);
                nB = dens9(f[1]);
            }
            sd[slot_d][0][sdc] = nA;
            sd[slot_d][1][sdc] = nB;
        }
    };

    unsigned smc = 0, smn = 0;
    bool abort_cta = false;
    // prologue: fill the ring, then the densities of rows y0 - 1 and y0
    if (t < 32) issue_upto(D - 1);
    wait_row(0);
    wait_row(1);
    if (!timed_out) {
        pull_dens(0, smn, 0);
        pull_dens(1, smc, 1);
    }
    for (int r = y0; r < y1; ++r) {
        const int sq = r - y0 + 1;   // sequence number of row r
        const int s_m = (r - y0) & 3, s_0 = (r - y0 + 1) & 3, s_p = (r - y0 + 2) & 3;
        wait_row(sq + 1);
        if (!timed_out) pull_dens(sq + 1, smn, s_p);
        // past this barrier every thread is done with the collision of row
        // r - 1 (slot of sq - 1) and with the densities of rows up to r + 1
        if (__syncthreads_or(timed_out)) {
            abort_cta = true;
            break;
        }
        if (t < 32) {
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            issue_upto(sq - 1 + D);
        }
        if (coll && !SOL(smc, 0, 0)) {
            const int rw = rows_of(r, ny).rw;
            C fc[2][9];
            pull(sq, rw, smc, fc);
            collide_any<S, W, 0>(cx, fc, smc, sd, s_m, s_0, s_p, sdc, dst, plane, (unsigned)(rw * pitch + xc),
                                  MomOut{nullptr, nullptr, 0}, 0, ghost_r(xc, nx), ghost_l(xc, nx));
        }
        smc = smn;
    }
    // a timeout in the prologue, or in a row after the last barrier, still
    // reaches every thread here
    if (!abort_cta && __syncthreads_or(timed_out)) abort_cta = true;
    if (abort_cta && t == 0) {
        // drain the copies this CTA issued before it exits (bounded): the last
        // fill of each slot completes after every earlier one
        for (int sq = max(0, issued - D); sq < issued; ++sq) mbar_wait(&bars[sq % D], (unsigned)((sq / D) & 1));
        atomicOr(err, ERR_TIMEOUT);
    }
    // without a timeout every issued row (sq < npull) was waited on above
}

template <typename S, int W, int D>
constexpr size_t async_smem_bytes() {
    return (size_t)D * 18 * W * sizeof(S) + 4 * 2 * W * sizeof(typename Prec<S>::C);
}

// ---- initial state: f_i = f_i^eq(n^0, u = 0) = A_i n^0 on fluid nodes -----
template <typename S>
__global__ void k_init(const RunDesc* __restrict__ runs) {
    using C = typename Prec<S>::C;
    using Wc = Wt<C>;
    const RunDesc& rd = runs[blockIdx.y];
    Shift<S> sh;
    sh.load(rd);
    const Geo geo{rd.nx, rd.cap_x0, rd.cap_x1, rd.y_bot, rd.y_top, rd.mask};
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < rd.nodes; q += gridDim.x * blockDim.x) {
        const int y = q / rd.nx, x = q - y * rd.nx;
        const bool sol = geo.solid(x, y);
        double n0[2] = {0.0, 0.0};
        if (!sol) {
            bool liquid;
            if (rd.init_kind == 0) {
                liquid = (double)x >= rd.x_lo && (double)x < rd.x_hi;
            } else if (rd.init_kind == 1) {
                const double dx = __dsub_rn((double)x, rd.cx), dy = __dsub_rn((double)y, rd.cy);
                liquid = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)) < __dmul_rn(rd.r, rd.r);
            } else {
                liquid = false;
            }
            if (rd.init_kind == 2) {
                n0[0] = rd.init_nA[q];
                n0[1] = rd.init_nB[q];
            } else {
                n0[0] = liquid ? rd.rho_major : rd.rho_minor;
                n0[1] = liquid ? rd.rho_minor : rd.rho_major;
            }
        }
        const long long o = (long long)y * rd.pitch + x;
        for (int b = 0; b < 2; ++b) {
            S* base = static_cast<S*>(rd.buf[b]);
            for (int k = 0; k < 2; ++k) {
                const C n = (C)n0[k];
                for (int i = 0; i < 9; ++i) {
                    const C w = i == 0 ? Wc::w0 : (i <= 4 ? Wc::w1 : Wc::w5);
                    C feq = Ar<C>::mul(w, n);
                    if (rd.gen) feq = Ar<C>::add(feq, Ar<C>::mul((C)rd.dA[k][grp(i)], n));
                    S* p = base + ((long long)k * 9 + i) * rd.plane + o;
                    const int gr = ghost_r(x, rd.nx), gl = ghost_l(x, rd.nx);
                    if (sol) {
                        *p = S(0.0f);
                        if (gr) p[gr] = S(0.0f);
                        if (gl) p[gl] = S(0.0f);
                    } else {
                        enc(p, feq, sh.v[k][grp(i)]);
                        if (gr) enc(p + gr, feq, sh.v[k][grp(i)]);
                        if (gl) enc(p + gl, feq, sh.v[k][grp(i)]);
                    }
                }
            }
        }
    }
}

// FP64 density of species k at node (x, y): sum of the decoded populations
// in i order, accumulated in FP64.
template <typename S>
__device__ __forceinline__ double node_density(const RunDesc& rd, const S* base, const Shift<S>& sh, int k,
                                               long long o) {
    double acc = 0.0;
#pragma unroll
    for (int i = 0; i < 9; ++i)
        acc = __dadd_rn(acc, (double)dec(ldg(base + ((long long)k * 9 + i) * rd.plane + o), sh.v[k][grp(i)]));
    return acc;
}

template <typename S>
__global__ void k_densities(const RunDesc* __restrict__ runs, int run, int parity, double* __restrict__ nA,
                            double* __restrict__ nB) {
    const RunDesc& rd = runs[run];
    Shift<S> sh;
    sh.load(rd);
    const Geo geo{rd.nx, rd.cap_x0, rd.cap_x1, rd.y_bot, rd.y_top, rd.mask};
    const S* base = static_cast<const S*>(rd.buf[parity]);
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < rd.nodes; q += gridDim.x * blockDim.x) {
        const int y = q / rd.nx, x = q - y * rd.nx;
        if (geo.solid(x, y)) {
            nA[q] = 0.0;
            nB[q] = 0.0;
            continue;
        }
        const long long o = (long long)y * rd.pitch + x;
        nA[q] = node_density<S>(rd, base, sh, 0, o);
        nB[q] = node_density<S>(rd, base, sh, 1, o);
    }
}

template <typename S>
__global__ void k_export(const RunDesc* __restrict__ runs, int run, int parity, S* __restrict__ out) {
    const RunDesc& rd = runs[run];
    const S* base = static_cast<const S*>(rd.buf[parity]);
    const long long total = 18LL * rd.nodes;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const long long ki = q / rd.nodes;
        const int rem = (int)(q - ki * rd.nodes);
        const int y = rem / rd.nx, x = rem - y * rd.nx;
        out[q] = base[ki * rd.plane + (long long)y * rd.pitch + x];
    }
}

template <typename S>
__global__ void k_import(const RunDesc* __restrict__ runs, int run, int parity, const S* __restrict__ in) {
    const RunDesc& rd = runs[run];
    S* base = static_cast<S*>(rd.buf[parity]);
    const long long total = 18LL * rd.nodes;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const long long ki = q / rd.nodes;
        const int rem = (int)(q - ki * rd.nodes);
        const int y = rem / rd.nx, x = rem - y * rd.nx;
        S* p = base + ki * rd.plane + (long long)y * rd.pitch + x;
        *p = in[q];
        const int gr = ghost_r(x, rd.nx), gl = ghost_l(x, rd.nx);
        if (gr) p[gr] = in[q];
        if (gl) p[gl] = in[q];
    }
}

// Populations of the column window [x0, x0 + ncols) (0 <= x0, x0 + ncols <= nx)
// to / from a packed buffer [18][ny][ncols]; writes also refresh the ghost
// images of columns 0, 1 and nx - 2, nx - 1 (the x-slab halo exchange).
template <typename S>
__global__ void k_get_cols(const RunDesc* __restrict__ runs, int run, int parity, int x0, int ncols,
                           S* __restrict__ out) {
    const RunDesc& rd = runs[run];
    const S* base = static_cast<const S*>(rd.buf[parity]);
    const long long per = (long long)rd.ny * ncols, total = 18 * per;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const long long ki = q / per;
        const int rem = (int)(q - ki * per);
        const int y = rem / ncols, x = x0 + (rem - y * ncols);
        out[q] = base[ki * rd.plane + (long long)y * rd.pitch + x];
    }
}

template <typename S>
__global__ void k_set_cols(const RunDesc* __restrict__ runs, int run, int parity, int x0, int ncols,
                           const S* __restrict__ in) {
    const RunDesc& rd = runs[run];
    S* base = static_cast<S*>(rd.buf[parity]);
    const long long per = (long long)rd.ny * ncols, total = 18 * per;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const long long ki = q / per;
        const int rem = (int)(q - ki * per);
        const int y = rem / ncols, x = x0 + (rem - y * ncols);
        S* p = base + ki * rd.plane + (long long)y * rd.pitch + x;
        *p = in[q];
        const int gr = ghost_r(x, rd.nx), gl = ghost_l(x, rd.nx);
        if (gr) p[gr] = in[q];
        if (gl) p[gl] = in[q];
    }
}

// ---- fronts (Numerical Results section, Figs. 6-8) -------------------------
// Four tracked rows per run, scanned from cap_x0:
//   g = 0, 1: the centre row(s) with v = phi = (n_A - n_B)/(n_A + n_B);
//   g = 2, 3: the fluid rows next to the bottom / top plate with
//             v = n_A - rho_bulk / 3.
// The scan gives every capillary column of every tracked row its own
// thread; a thread whose column fails (v < 0) takes part in an atomicMin, so
// first[4 run + g] ends as the first failing column x* whatever the order
// (deterministic).  The finishing kernel then interpolates
// z = (x* - 1 - cap_x0) + v(x* - 1) / (v(x* - 1) - v(x*)) in FP64.
template <typename S>
__device__ __forceinline__ double front_value(const RunDesc& rd, const S* base, const Shift<S>& sh, int x,
                                              int y, bool prec) {
    const long long o = (long long)y * rd.pitch + x;
    const double a = node_density<S>(rd, base, sh, 0, o);
    if (prec) return __dsub_rn(a, rd.thr);
    const double b = node_density<S>(rd, base, sh, 1, o);
    return __ddiv_rn(__dsub_rn(a, b), __dadd_rn(a, b));
}

// Whether the run has a channel to track, and tracked row g of it.
__device__ __forceinline__ bool track_has(const RunDesc& rd) {
    return rd.y_bot >= 0 && rd.y_top >= 0 && rd.y_top - rd.y_bot >= 2 && rd.cap_x1 > rd.cap_x0;
}
__device__ __forceinline__ int track_row(const RunDesc& rd, int g) {
    const int H = rd.y_top - rd.y_bot - 1;
    if (g == 0) return (H % 2 == 0) ? rd.y_bot + H / 2 : rd.y_bot + (H + 1) / 2;
    if (g == 1) return (H % 2 == 0) ? rd.y_bot + H / 2 + 1 : rd.y_bot + (H + 1) / 2;
    return g == 2 ? rd.y_bot + 1 : rd.y_top - 1;
}

constexpr int kTrackThreads = 256;
constexpr int kNoFront = 0x7f7f7f7f;   // "no failing column" (the byte pattern first[] is reset to)

// grid (column chunks of kTrackThreads, runs); first[] preset to kNoFront
template <typename S>
__global__ void __launch_bounds__(kTrackThreads) k_track_scan(const RunDesc* __restrict__ runs, int parity,
                                                             int* __restrict__ first) {
    const RunDesc& rd = runs[blockIdx.y];
    if (!track_has(rd)) return;
    const int x = rd.cap_x0 + blockIdx.x * kTrackThreads + threadIdx.x;
    if (x >= rd.cap_x1) return;
    Shift<S> sh;
    sh.load(rd);
    const S* base = static_cast<const S*>(rd.buf[parity]);
#pragma unroll
    for (int g = 0; g < 4; ++g)
        if (front_value<S>(rd, base, sh, x, track_row(rd, g), g >= 2) < 0.0) atomicMin(&first[4 * blockIdx.y + g], x);
}

// one warp per run: lanes 0-3 interpolate their row's front, lane 0 writes
template <typename S>
__global__ void __launch_bounds__(32) k_track_final(const RunDesc* __restrict__ runs, int parity,
                                                   const int* __restrict__ first, LogCtl lc,
                                                   double* __restrict__ zout) {
    const RunDesc& rd = runs[blockIdx.x];
    const int g = threadIdx.x;
    const bool has = track_has(rd);
    double z = __longlong_as_double(0x7ff8000000000000LL);   // NaN: no channel
    if (g < 4 && has) {
        Shift<S> sh;
        sh.load(rd);
        const S* base = static_cast<const S*>(rd.buf[parity]);
        const int y = track_row(rd, g);
        const bool prec = g >= 2;
        const int found = first[4 * blockIdx.x + g];
        if (found == kNoFront) {
            z = (double)(rd.cap_x1 - rd.cap_x0);
        } else {
            const int xp = found == 0 ? rd.nx - 1 : found - 1;
            const double v = front_value<S>(rd, base, sh, found, y, prec);
            const double vp = front_value<S>(rd, base, sh, xp, y, prec);
            if (!(vp >= 0.0)) z = (double)(found - rd.cap_x0);
            else z = __dadd_rn((double)(found - 1 - rd.cap_x0), __ddiv_rn(vp, __dsub_rn(vp, v)));
        }
    }
    const double z0 = __shfl_sync(0xffffffffu, z, 0), z1 = __shfl_sync(0xffffffffu, z, 1);
    const double z2 = __shfl_sync(0xffffffffu, z, 2), z3 = __shfl_sync(0xffffffffu, z, 3);
    if (g == 0) {
        double zb = z0;
        if (has) {
            const int H = rd.y_top - rd.y_bot - 1;
            if (H % 2 == 0) zb = __dmul_rn(0.5, __dadd_rn(z0, z1));
        }
        if (zout) {
            zout[blockIdx.x * 3 + 0] = zb;
            zout[blockIdx.x * 3 + 1] = z2;
            zout[blockIdx.x * 3 + 2] = z3;
        }
        if (rd.log && lc.count) {
            const long long c = *lc.count;
            double* rec = rd.log + (c % lc.cap) * 6;
            rec[0] = (double)(c * (long long)lc.log_every);
            rec[1] = zb;
            rec[2] = z2;
            rec[3] = z3;
        }
    }
}

// ---- deterministic FP64 mass sums -----------------------------------------
// Pass 1: kMassChunks CTAs of kMassThreads per (run, row): thread t of chunk
// c sums columns c kMassThreads + t, then every kMassChunks kMassThreads
// further, in order, then a fixed shared-memory tree.  Pass 2: one CTA per
// run sums its (row, chunk) partials the same way.  The order never depends
// on timing, so repeated runs give identical bits.
//
// FP64 storage sums the populations in FP64.  FP32 and FP16 storage hold
// FP32 values: a thread accumulates them in a compensated FP32 pair (Knuth's
// TwoSum keeps every rounding error, so hi + lo carries about 48 significant
// bits) and enters FP64 once, at the tree; the FP64 pipe of sm_103a, a small
// fraction of its FP32 rate, then does a few operations per thread instead
// of two per population.
constexpr int kMassThreads = 256;   // kMassChunks (column chunks per row) is in lbm_device.h

// Knuth's TwoSum: s + e == a + b exactly (round-to-nearest FP32).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
struct Sum2f {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float v) {
        float s, e;
        two_sum(hi, v, s, e);
        hi = s;
        lo = __fadd_rn(lo, e);
    }
    __device__ __forceinline__ double value() const { return __dadd_rn((double)hi, (double)lo); }
};

// Sum over columns chunk * kMassThreads + t + j * nchunks * kMassThreads
// of row y (thread t, j = 0, 1, ...), then the CTA's tree.
template <typename S>
__device__ __forceinline__ void mass_row_sum(const RunDesc& rd, const S* base, int y, int chunk, int nchunks,
                                             double* out2) {
    const int x_first = chunk * kMassThreads + (int)threadIdx.x, x_step = nchunks * kMassThreads;
    Shift<S> sh;
    sh.load(rd);
    const Geo geo{rd.nx, rd.cap_x0, rd.cap_x1, rd.y_bot, rd.y_top, rd.mask};
    const unsigned plane = (unsigned)rd.plane;
    double a = 0.0, b = 0.0;
    if constexpr (sizeof(typename Prec<S>::C) == 8) {
        for (int x = x_first; x < rd.nx; x += x_step) {
            if (geo.solid(x, y)) continue;
            const long long o = (long long)y * rd.pitch + x;
            a = __dadd_rn(a, node_density<S>(rd, base, sh, 0, o));
            b = __dadd_rn(b, node_density<S>(rd, base, sh, 1, o));
        }
    } else {
        Sum2f sa, sb;
        const S* row = base + (long long)y * rd.pitch;
        for (int x = x_first; x < rd.nx; x += x_step) {
            if (geo.solid(x, y)) continue;
            const S* p = row + x;
#pragma unroll
            for (int i = 0; i < 9; ++i) sa.add(dec(ldg(p + (unsigned)i * plane), sh.v[0][grp(i)]));
#pragma unroll
            for (int i = 0; i < 9; ++i) sb.add(dec(ldg(p + (unsigned)(9 + i) * plane), sh.v[1][grp(i)]));
        }
        a = sa.value();
        b = sb.value();
    }
    __shared__ double s[2][kMassThreads];
    s[0][threadIdx.x] = a;
    s[1][threadIdx.x] = b;
    __syncthreads();
    for (int h = kMassThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            s[0][threadIdx.x] = __dadd_rn(s[0][threadIdx.x], s[0][threadIdx.x + h]);
            s[1][threadIdx.x] = __dadd_rn(s[1][threadIdx.x], s[1][threadIdx.x + h]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out2[0] = s[0][0];
        out2[1] = s[1][0];
    }
}

template <typename S>
__global__ void __launch_bounds__(kMassThreads) k_mass_rows(const RunDesc* __restrict__ runs,
                                                            const int2* __restrict__ rows, int parity,
                                                            double* __restrict__ partials) {
    const int2 ry = rows[blockIdx.x];
    const RunDesc& rd = runs[ry.x];
#ifdef LBM_CHECKED
    if (ry.y < 0 || ry.y >= rd.ny) {
        if (threadIdx.x == 0 && rd.err) atomicOr(rd.err, ERR_BOUNDS);
        return;
    }
#endif
    mass_row_sum<S>(rd, static_cast<const S*>(rd.buf[parity]), ry.y, blockIdx.y, kMassChunks,
                    partials + 2 * ((long long)blockIdx.x * kMassChunks + blockIdx.y));
}

// Pass 2 over the rows of one run (shared with the allocation-free variant).
__device__ __forceinline__ void mass_rows_total(int ny, const double* part, double* out2) {
    double a = 0.0, b = 0.0;
    for (int y = threadIdx.x; y < ny; y += kMassThreads) {
        a = __dadd_rn(a, part[2 * y + 0]);
        b = __dadd_rn(b, part[2 * y + 1]);
    }
    __shared__ double s[2][kMassThreads];
    s[0][threadIdx.x] = a;
    s[1][threadIdx.x] = b;
    __syncthreads();
    for (int h = kMassThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            s[0][threadIdx.x] = __dadd_rn(s[0][threadIdx.x], s[0][threadIdx.x + h]);
            s[1][threadIdx.x] = __dadd_rn(s[1][threadIdx.x], s[1][threadIdx.x + h]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out2[0] = s[0][0];
        out2[1] = s[1][0];
    }
}

__global__ void __launch_bounds__(kMassThreads) k_mass_final(const RunDesc* __restrict__ runs,
                                                    const double* __restrict__ partials, double* __restrict__ mass,
                                                    LogCtl lc, int write_log, uint32_t* __restrict__ err);

}  // namespace sc
