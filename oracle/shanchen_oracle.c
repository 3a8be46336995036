/*
 * Plain FP64 CPU oracle of the binary (two-component, immiscible) Shan-Chen
 * D2Q9 lattice Boltzmann step in a 2-D capillary.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * statement of what the GPU path must compute.  Only the tests, the smoke
 * check and the CPU-baseline / reference leg of the benchmark may build,
 * load or call it; the product library never does.  It shares no code,
 * header, table or constant with the CUDA path.
 *
 * Paper: S. Chibbaro, "Capillary filling with pseudo-potential binary
 * Lattice-Boltzmann model" (Model section and Numerical Results section).
 * Equation numbers follow the order of the paper's numbered equations:
 *   Eq. 2  (eq:lbe)      BGK lattice Boltzmann equation per component
 *   Eqs. 3-5 (eq:feq1-3) D2Q9 equilibrium with free alpha_k
 *   Eq. 6                discrete velocities c_i
 *   Eq. 7                equilibrium-velocity shift rho_k u^eq = rho_k U + tau_k F_k
 *   Eq. 8                common velocity U
 *   Eq. 9  (forcing)     bulk pseudo-potential force, Psi_k = n_k
 *   Eq. 10               interaction matrix (g at distance 1, g/4 at sqrt 2)
 *   Eq. 11 (forcingw)    wall-fluid force
 *
 * Readings taken where the paper is silent or ambiguous (all are part of the
 * canonical step this oracle defines):
 *   - Eqs. 3-5 are written as the usual w_i n (1 + 3 c.u + 9/2 (c.u)^2 -
 *     3/2 u.u), w = 4/9, 1/9, 1/36, which they are at alpha_k = 4/9, plus
 *     (A_i(alpha_k) - w_i) n with A_0 = alpha, A_1..4 = (1 - alpha)/5,
 *     A_5..8 = (1 - alpha)/20 when alpha_k != 4/9 (only the isotropic part of
 *     the equilibrium depends on alpha).  m_k weights the common velocity of
 *     Eq. 8 (rho_k = m_k n_k, rho_k u_k = m_k j_k) and divides the velocity
 *     shift of Eq. 7; defaults alpha_k = 4/9, m_k = 1.
 *   - The coupling is written with the w_i weights: G = 9 g, so the bulk
 *     acceleration is a_k = -G sum_i w_i n_kbar(x+c_i) c_i and F_k = n_k a_k.
 *     The wall force uses the same weights: a_k^w = -G_kw sum_i w_i s(x+c_i) c_i
 *     with s = 1 on solid nodes.  Positive couplings repel.
 *   - The sum in Eq. 8 runs over the species k.
 *   - Psi_k = n_k = 0 on solid nodes; the wall acts only through G_kw.
 *   - Bounce-back (Numerical Results section) is the half-way rule fused into
 *     the pull: a population whose source node is solid is replaced by the
 *     opposite population of the same node.
 *   - Delta t = 1; every operation below is done in the stated order so that
 *     a second implementation doing the same order agrees to the last bit.
 *
 * Canonical order of one step (F holds post-collision populations):
 *   1. pull: ft_i(x) = F_i(x - c_i) if that node is fluid, else F_opp(i)(x)
 *   2. n_k = ((ft_0 + ft_1) + ...) + ft_8; j_k = sum_i ft_i c_i, i ascending
 *   3. S_kbar = sum_{i=1..8} (w_i n_kbar(x+c_i)) c_i, i ascending;
 *      Wl = sum_{i=1..8} (w_i s(x+c_i)) c_i; a_k = (-(G S_kbar) - (G_kw Wl)) + g
 *   4. U = (j_A mt_A + j_B mt_B) / (n_A mt_A + n_B mt_B), mt_k = m_k (1/tau_k)
 *      precomputed (1/tau_k itself for m_k = 1)
 *   5. u_k = U + tm_k a_k, tm_k = tau_k / m_k precomputed (tau_k for m_k = 1)
 *   6. feq_i = (w_i n_k) (((1 + 3 cu) + 4.5 (cu cu)) - 1.5 usq), then
 *      feq_i + (dA_i n_k) with dA_i = A_i(alpha_k) - w_i when alpha_k != 4/9
 *   7. F'_i = ft_i - (ft_i - feq_i) (1/tau_k)
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no FMA contraction).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Eq. 6: c_0 = 0; c_1..4 = (cos((i-1)pi/2), sin((i-1)pi/2));
 * c_5..8 = sqrt2 (cos((i-5)pi/2 + pi/4), sin(...)). */
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
/* opposite direction: c_opp(i) = -c_i */
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};

/* Eqs. 3-5 at alpha = 4/9: rest weight 4/9, axis 1/9, diagonal 1/36. */
static double weight(int i) {
    if (i == 0) return 4.0 / 9.0;
    if (i <= 4) return 1.0 / 9.0;
    return 1.0 / 36.0;
}

typedef struct {
    int32_t nx, ny;          /* periodic grid, x fastest */
    int32_t cap_x0, cap_x1;  /* plates cover columns [cap_x0, cap_x1) */
    int32_t y_bot, y_top;    /* solid plate rows; -1 = no such plate */
    double G;                /* cross-species coupling (w_i-weighted) */
    double Gw[2];            /* wall couplings of species A and B */
    double tau[2];           /* relaxation times */
    double body[2];          /* body acceleration (test-only drive) */
    double rho_bulk;         /* precursor threshold base: n_A < rho_bulk / 3 */
    double alpha[2];         /* Eqs. 3-5 free parameter per species (4/9: standard D2Q9) */
    double mass[2];          /* molecular masses m_k (rho_k = m_k n_k) */
} oc_params;

typedef struct {
    oc_params p;
    uint8_t* solid;  /* [ny][nx] */
    double* F;       /* [2][9][ny][nx] post-collision populations */
    double* Fprev;   /* populations before the last step (for the velocity) */
    double* ft;      /* scratch: streamed populations */
    double* n;       /* scratch: [2][ny][nx] densities */
    long step;
} oc_state;

static size_t NODES(const oc_params* p) { return (size_t)p->nx * (size_t)p->ny; }
static size_t IDX(const oc_params* p, int k, int i, int x, int y) {
    return (((size_t)k * 9 + (size_t)i) * (size_t)p->ny + (size_t)y) * (size_t)p->nx + (size_t)x;
}
static int wrap(int v, int n) { return ((v % n) + n) % n; }

/* Capillary geometry (Numerical Results section, Fig. 1): two plates made of
 * one solid row each, spanning [cap_x0, cap_x1); everything else is fluid and
 * periodic.  A caller-given mask replaces the plates. */
static void build_solid(oc_state* s, const uint8_t* mask) {
    const oc_params* p = &s->p;
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            int sol;
            if (mask) sol = mask[(size_t)y * p->nx + x] != 0;
            else sol = (y == p->y_bot || y == p->y_top) && x >= p->cap_x0 && x < p->cap_x1;
            s->solid[(size_t)y * p->nx + x] = (uint8_t)sol;
        }
}

static int is_solid(const oc_state* s, int x, int y) {
    return s->solid[(size_t)wrap(y, s->p.ny) * s->p.nx + wrap(x, s->p.nx)];
}

/* Isotropic part of Eqs. 3-5 minus its alpha = 4/9 value, dA_i = A_i(alpha) -
 * w_i (A_0 = alpha, A_1..4 = (1 - alpha)/5, A_5..8 = (1 - alpha)/20); zero
 * for alpha = 4/9. */
static void alpha_shift(double alpha, double dA[3]) {
    if (alpha == 4.0 / 9.0) {
        dA[0] = dA[1] = dA[2] = 0.0;
        return;
    }
    dA[0] = alpha - 4.0 / 9.0;
    dA[1] = (1.0 - alpha) / 5.0 - 1.0 / 9.0;
    dA[2] = (1.0 - alpha) / 20.0 - 1.0 / 36.0;
}

/* Eqs. 3-5 for free alpha (canonical order, see header). */
void oc_feq_alpha(double n, double ux, double uy, double alpha, double* feq) {
    double dA[3];
    alpha_shift(alpha, dA);
    double usq = ux * ux + uy * uy;
    for (int i = 0; i < 9; ++i) {
        double cu = CX[i] * ux + CY[i] * uy;
        feq[i] = (weight(i) * n) * (((1.0 + 3.0 * cu) + 4.5 * (cu * cu)) - 1.5 * usq);
        if (alpha != 4.0 / 9.0) feq[i] = feq[i] + dA[i == 0 ? 0 : (i <= 4 ? 1 : 2)] * n;
    }
}

/* Eqs. 3-5 with alpha = 4/9. */
void oc_feq(double n, double ux, double uy, double* feq) { oc_feq_alpha(n, ux, uy, 4.0 / 9.0, feq); }

/* Left-hand side of Eq. 2 with half-way bounce-back at solid nodes:
 * the population moving along c_i arrives at x from x - c_i. */
static void stream(const oc_state* s, const double* F, double* ft) {
    const oc_params* p = &s->p;
    for (int k = 0; k < 2; ++k)
        for (int i = 0; i < 9; ++i)
            for (int y = 0; y < p->ny; ++y)
                for (int x = 0; x < p->nx; ++x) {
                    size_t o = IDX(p, k, i, x, y);
                    if (is_solid(s, x, y)) { ft[o] = 0.0; continue; }
                    int xs = wrap(x - CX[i], p->nx), ys = wrap(y - CY[i], p->ny);
                    if (is_solid(s, xs, ys)) ft[o] = F[IDX(p, k, OPP[i], x, y)];
                    else ft[o] = F[IDX(p, k, i, xs, ys)];
                }
}

/* n_k = sum_i f_i (Model section, below Eq. 6), i ascending; 0 on solids. */
static void densities_of(const oc_state* s, const double* f, double* n) {
    const oc_params* p = &s->p;
    for (int k = 0; k < 2; ++k)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                double acc = 0.0;
                if (!is_solid(s, x, y))
                    for (int i = 0; i < 9; ++i) acc = acc + f[IDX(p, k, i, x, y)];
                n[((size_t)k * p->ny + y) * p->nx + x] = acc;
            }
}

/* Acceleration a_k = F_k / n_k at node (x, y) from Eq. 9 (bulk, Psi = n),
 * Eq. 10 (weights) and Eq. 11 (wall) plus the optional body acceleration. */
static void accel_at(const oc_state* s, const double* n, int x, int y, double a[2][2]) {
    const oc_params* p = &s->p;
    double S[2][2], Wl[2] = {0.0, 0.0};
    for (int k = 0; k < 2; ++k) { S[k][0] = 0.0; S[k][1] = 0.0; }
    for (int i = 1; i < 9; ++i) {
        int xn = wrap(x + CX[i], p->nx), yn = wrap(y + CY[i], p->ny);
        double sflag = is_solid(s, xn, yn) ? 1.0 : 0.0;
        for (int k = 0; k < 2; ++k) {
            double nn = n[((size_t)k * p->ny + yn) * p->nx + xn];
            S[k][0] = S[k][0] + (weight(i) * nn) * CX[i];
            S[k][1] = S[k][1] + (weight(i) * nn) * CY[i];
        }
        Wl[0] = Wl[0] + (weight(i) * sflag) * CX[i];
        Wl[1] = Wl[1] + (weight(i) * sflag) * CY[i];
    }
    for (int k = 0; k < 2; ++k) {
        int kb = 1 - k;
        for (int d = 0; d < 2; ++d)
            a[k][d] = (-(p->G * S[kb][d]) - (p->Gw[k] * Wl[d])) + p->body[d];
    }
}

/* Number-density momentum j_k = sum_i c_i f_i, i ascending (rho_k u_k = m_k j_k). */
static void momentum_at(const oc_state* s, const double* f, int k, int x, int y, double j[2]) {
    const oc_params* p = &s->p;
    double jx = 0.0, jy = 0.0;
    for (int i = 0; i < 9; ++i) {
        double v = f[IDX(p, k, i, x, y)];
        jx = jx + v * CX[i];
        jy = jy + v * CY[i];
    }
    j[0] = jx;
    j[1] = jy;
}

/* Right-hand side of Eq. 2 at every fluid node, with u^eq from Eqs. 7-8. */
static void collide(oc_state* s, const double* ft, const double* n, double* Fout) {
    const oc_params* p = &s->p;
    double itau[2] = {1.0 / p->tau[0], 1.0 / p->tau[1]};
    double mt[2] = {p->mass[0] * itau[0], p->mass[1] * itau[1]};
    double tm[2] = {p->tau[0] / p->mass[0], p->tau[1] / p->mass[1]};
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            if (is_solid(s, x, y)) {
                for (int k = 0; k < 2; ++k)
                    for (int i = 0; i < 9; ++i) Fout[IDX(p, k, i, x, y)] = 0.0;
                continue;
            }
            double nk[2], j[2][2], a[2][2];
            for (int k = 0; k < 2; ++k) {
                nk[k] = n[((size_t)k * p->ny + y) * p->nx + x];
                momentum_at(s, ft, k, x, y, j[k]);
            }
            accel_at(s, n, x, y, a);
            double U[2];
            double den = nk[0] * mt[0] + nk[1] * mt[1];
            for (int d = 0; d < 2; ++d) U[d] = (j[0][d] * mt[0] + j[1][d] * mt[1]) / den;
            for (int k = 0; k < 2; ++k) {
                double ueq[2];
                for (int d = 0; d < 2; ++d) ueq[d] = U[d] + tm[k] * a[k][d];
                double feq[9];
                oc_feq_alpha(nk[k], ueq[0], ueq[1], p->alpha[k], feq);
                for (int i = 0; i < 9; ++i) {
                    double f = ft[IDX(p, k, i, x, y)];
                    Fout[IDX(p, k, i, x, y)] = f - (f - feq[i]) * itau[k];
                }
            }
        }
}

/* ---- public API (ctypes) ---------------------------------------------- */

oc_state* oc_create(const oc_params* prm, const uint8_t* mask, const double* nA0, const double* nB0) {
    if (!prm || prm->nx < 1 || prm->ny < 1 || !nA0 || !nB0) return NULL;
    if (!(prm->tau[0] > 0.5) || !(prm->tau[1] > 0.5)) return NULL;
    if (!(prm->mass[0] > 0.0) || !(prm->mass[1] > 0.0)) return NULL;
    if (!(prm->alpha[0] < 1.0) || !(prm->alpha[1] < 1.0)) return NULL;
    oc_state* s = (oc_state*)calloc(1, sizeof(oc_state));
    s->p = *prm;
    size_t N = NODES(prm);
    s->solid = (uint8_t*)calloc(N, 1);
    s->F = (double*)calloc(18 * N, sizeof(double));
    s->Fprev = (double*)calloc(18 * N, sizeof(double));
    s->ft = (double*)calloc(18 * N, sizeof(double));
    s->n = (double*)calloc(2 * N, sizeof(double));
    build_solid(s, mask);
    /* Initial state: equilibrium at rest, f_i = f_i^eq(n^0, u = 0). */
    for (int y = 0; y < prm->ny; ++y)
        for (int x = 0; x < prm->nx; ++x) {
            if (is_solid(s, x, y)) continue;
            for (int k = 0; k < 2; ++k) {
                double n0 = (k == 0 ? nA0 : nB0)[(size_t)y * prm->nx + x];
                double feq[9];
                oc_feq_alpha(n0, 0.0, 0.0, prm->alpha[k], feq);
                for (int i = 0; i < 9; ++i) s->F[IDX(prm, k, i, x, y)] = feq[i];
            }
        }
    s->step = 0;
    return s;
}

void oc_destroy(oc_state* s) {
    if (!s) return;
    free(s->solid); free(s->F); free(s->Fprev); free(s->ft); free(s->n);
    free(s);
}

/* One or more full steps of Eq. 2 in the canonical order. */
void oc_step(oc_state* s, int nsteps) {
    size_t N = NODES(&s->p);
    for (int t = 0; t < nsteps; ++t) {
        memcpy(s->Fprev, s->F, 18 * N * sizeof(double));
        stream(s, s->Fprev, s->ft);
        densities_of(s, s->ft, s->n);
        collide(s, s->ft, s->n, s->F);
        s->step += 1;
    }
}

long oc_time(const oc_state* s) { return s->step; }

/* Streaming alone (for the permutation check): Fout = pull(Fin). */
void oc_stream(const oc_state* s, const double* Fin, double* Fout) { stream(s, Fin, Fout); }

/* Collision alone on given streamed populations (densities recomputed). */
void oc_collide(oc_state* s, const double* ft, double* Fout) {
    densities_of(s, ft, s->n);
    collide(s, ft, s->n, Fout);
}

void oc_get_populations(const oc_state* s, double* F) {
    memcpy(F, s->F, 18 * NODES(&s->p) * sizeof(double));
}
void oc_set_populations(oc_state* s, const double* F) {
    memcpy(s->F, F, 18 * NODES(&s->p) * sizeof(double));
}
void oc_get_solid(const oc_state* s, uint8_t* out) { memcpy(out, s->solid, NODES(&s->p)); }

/* n_k at the current time: collision conserves n_k, so the sum of the
 * post-collision populations equals the density of the streamed state. */
void oc_densities(const oc_state* s, double* nA, double* nB) {
    size_t N = NODES(&s->p);
    double* n = (double*)malloc(2 * N * sizeof(double));
    densities_of(s, s->F, n);
    memcpy(nA, n, N * sizeof(double));
    memcpy(nB, n + N, N * sizeof(double));
    free(n);
}

/* Accelerations of both species for given density fields (Eqs. 9-11):
 * out = [aAx, aAy, aBx, aBy] planes of nx*ny. */
void oc_accel(const oc_state* s, const double* nA, const double* nB, double* out) {
    const oc_params* p = &s->p;
    size_t N = NODES(p);
    double* n = (double*)malloc(2 * N * sizeof(double));
    for (size_t q = 0; q < N; ++q) {
        n[q] = s->solid[q] ? 0.0 : nA[q];
        n[N + q] = s->solid[q] ? 0.0 : nB[q];
    }
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            double a[2][2];
            size_t q = (size_t)y * p->nx + x;
            accel_at(s, n, x, y, a);
            out[q] = a[0][0]; out[N + q] = a[0][1];
            out[2 * N + q] = a[1][0]; out[3 * N + q] = a[1][1];
        }
    free(n);
}

/* Whole-fluid velocity at the current time (Model section, below Eq. 12):
 * rho u = sum_k rho_k u_k + (1/2) sum_k F_k with rho = sum_k m_k n_k and
 * rho_k u_k = m_k j_k, computed from the streamed populations of the last
 * step.  Returns 0 at t = 0 (the fluid is at rest). */
int oc_velocity(const oc_state* s, double* ux, double* uy) {
    const oc_params* p = &s->p;
    size_t N = NODES(p);
    if (s->step == 0) {
        memset(ux, 0, N * sizeof(double));
        memset(uy, 0, N * sizeof(double));
        return 0;
    }
    double* ft = (double*)malloc(18 * N * sizeof(double));
    double* n = (double*)malloc(2 * N * sizeof(double));
    stream(s, s->Fprev, ft);
    densities_of(s, ft, n);
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            size_t q = (size_t)y * p->nx + x;
            if (is_solid(s, x, y)) { ux[q] = 0.0; uy[q] = 0.0; continue; }
            double jA[2], jB[2], a[2][2];
            momentum_at(s, ft, 0, x, y, jA);
            momentum_at(s, ft, 1, x, y, jB);
            accel_at(s, n, x, y, a);
            double nA = n[q], nB = n[N + q];
            const double mA = p->mass[0], mB = p->mass[1];
            const double rho = (mA * nA) + (mB * nB);
            ux[q] = (((mA * jA[0]) + (mB * jB[0])) + 0.5 * ((nA * a[0][0]) + (nB * a[1][0]))) / rho;
            uy[q] = (((mA * jA[1]) + (mB * jB[1])) + 0.5 * ((nA * a[0][1]) + (nB * a[1][1]))) / rho;
        }
    free(ft);
    free(n);
    return 1;
}

/* Per-species mass: sum over fluid nodes and i of F (plain sequential sum). */
void oc_mass(const oc_state* s, double* M) {
    const oc_params* p = &s->p;
    for (int k = 0; k < 2; ++k) {
        double acc = 0.0;
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                if (is_solid(s, x, y)) continue;
                for (int i = 0; i < 9; ++i) acc = acc + s->F[IDX(p, k, i, x, y)];
            }
        M[k] = acc;
    }
}

/* Total post-collision momentum sum_x sum_k m_k sum_i c_i F_i (rho_k u_k = m_k j_k). */
void oc_momentum(const oc_state* s, double* P) {
    const oc_params* p = &s->p;
    double px = 0.0, py = 0.0;
    for (int k = 0; k < 2; ++k)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                if (is_solid(s, x, y)) continue;
                double j[2];
                momentum_at(s, s->F, k, x, y, j);
                px = px + p->mass[k] * j[0];
                py = py + p->mass[k] * j[1];
            }
    P[0] = px;
    P[1] = py;
}

/* ---- interface tracking (Numerical Results section, Figs. 6-8) --------- */

/* First column x* in [cap_x0, cap_x1) of row y where v(x) < 0, with
 * v = phi = (n_A - n_B)/(n_A + n_B) for the bulk front ("front at the
 * centre of the interface") and v = n_A - rho_bulk/3 for the precursor
 * film ("liquid density 1/3 of the bulk").  z is measured from cap_x0 and
 * linearly interpolated between x*-1 and x*; a row with no such x gives
 * the capillary length. */
static double front_row(const oc_state* s, const double* n, int y, int precursor) {
    const oc_params* p = &s->p;
    size_t N = NODES(p);
    double thr = p->rho_bulk / 3.0;
    double vprev = 0.0, v = 0.0;
    int found = -1;
    for (int x = p->cap_x0; x < p->cap_x1; ++x) {
        size_t q = (size_t)y * p->nx + x;
        double nA = n[q], nB = n[N + q];
        v = precursor ? (nA - thr) : ((nA - nB) / (nA + nB));
        if (v < 0.0) { found = x; break; }
    }
    if (found < 0) return (double)(p->cap_x1 - p->cap_x0);
    {
        int xp = wrap(found - 1, p->nx);
        size_t q = (size_t)y * p->nx + xp;
        double nA = n[q], nB = n[N + q];
        vprev = precursor ? (nA - thr) : ((nA - nB) / (nA + nB));
    }
    if (!(vprev >= 0.0)) return (double)(found - p->cap_x0);
    return (double)(found - 1 - p->cap_x0) + vprev / (vprev - v);
}

/* out[0] = bulk front (mean of the two centre rows for even H, the centre
 * row for odd H), out[1], out[2] = precursor fronts on the fluid rows next
 * to the bottom and top plates.  Returns -1 if the geometry has no channel. */
int oc_interface(const oc_state* s, double* out) {
    const oc_params* p = &s->p;
    if (p->y_bot < 0 || p->y_top < 0 || p->y_top - p->y_bot < 2 || p->cap_x1 <= p->cap_x0) {
        out[0] = out[1] = out[2] = NAN;
        return -1;
    }
    size_t N = NODES(p);
    double* n = (double*)malloc(2 * N * sizeof(double));
    densities_of(s, s->F, n);
    int H = p->y_top - p->y_bot - 1;
    if (H % 2 == 0) {
        double z1 = front_row(s, n, p->y_bot + H / 2, 0);
        double z2 = front_row(s, n, p->y_bot + H / 2 + 1, 0);
        out[0] = 0.5 * (z1 + z2);
    } else {
        out[0] = front_row(s, n, p->y_bot + (H + 1) / 2, 0);
    }
    out[1] = front_row(s, n, p->y_bot + 1, 1);
    out[2] = front_row(s, n, p->y_top - 1, 1);
    free(n);
    return 0;
}

/* Mixture pressure (Model section, the non-ideal gas law below Eq. 11),
 * with c_0^2 = 1/3 and the w_i-weighted coupling: p = (n_A + n_B)/3 +
 * G n_A n_B / 3. */
double oc_pressure(double nA, double nB, double G) {
    return (nA + nB) / 3.0 + G * nA * nB / 3.0;
}

/* The same for free alpha_k and m_k: the momentum flux of species k carries
 * m_k n_k (c_s^k)^2 with (c_s^k)^2 = 3 (1 - alpha_k) / 5 (Model section):
 * p = m_A cA n_A + m_B cB n_B + G n_A n_B / 3. */
double oc_pressure_general(double nA, double nB, double G, double alphaA, double alphaB, double mA, double mB) {
    double cA = 3.0 * (1.0 - alphaA) / 5.0, cB = 3.0 * (1.0 - alphaB) / 5.0;
    return (mA * cA * nA + mB * cB * nB) + G * nA * nB / 3.0;
}
