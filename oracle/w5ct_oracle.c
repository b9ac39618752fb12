/*
 * w5ct_oracle.c -- plain FP64 CPU oracle of the fifth-order finite-difference
 * WENO + constrained-transport (CT) ideal-MHD scheme of Donnert et al.,
 * "WENO-Wombat" (arXiv:1812.04278).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference that the CUDA library is checked against.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it.  It
 * shares no code, header, table or constant with the CUDA path.
 *
 * Everything is IEEE double, compiled without FMA contraction.  Loops run
 * over cells and interfaces in the order the paper describes; there is no
 * tiling, fusion or vectorisation.  OpenMP only distributes independent
 * cells/interfaces over threads (no reduction is parallel, so results do
 * not depend on the thread count).
 *
 * What the paper fixes and where (section / equation of the paper):
 *   conservation law, flux F_x ............ Sec. 2, Eqs. (mhdA)-(fluxes)
 *   total pressure, energy ................ Sec. 2, Eq. (P)
 *   wave speeds ........................... Sec. 2, Eqs. (slow),(fast),(ca)
 *   eigenvectors, degeneracy handling ..... Appendix A
 *   conservative update ................... Sec. 2, Eq. (num)
 *   CFL time step ......................... Sec. 2.1, Eq. (cfl)
 *   RK4 in q / q_save form ................ Sec. 2.1
 *   characteristic WENO5 / WENO5-Z ........ Sec. 2.2, Eq. (FWENO)
 *   CT transport fluxes, corner EMFs ...... Sec. 2.3, Eqs. (fct1)-(ox3)
 *   face-field update, 4th-order B_cell ... Sec. 2.3
 *   1-D and 3-D program flow .............. Sec. 3.1.1, Sec. 3.1.3
 *
 * Readings of passages that are garbled or ambiguous (each one is applied
 * identically here and in the CUDA path; the list is in the design notes):
 *   R1  P* = P + B^2/2 (the printed B_y^2 + B_z^2 lacks the 1/2).
 *   R2  c_f^2, c_slow^2 = (c_s^2 + B^2/rho +- sqrt(d))/2 with
 *       d = (c_s^2 - c_A^2)^2 + b_t^2 (b_t^2 + 2 c_A^2 + 2 c_s^2),
 *       c_f^2 - c_s^2 and c_s^2 - c_slow^2 obtained without cancellation,
 *       c_slow^2 = c_s^2 c_A^2 / c_f^2 (the same root, without cancellation).
 *   R3  m = 2,6 are the Alfven and m = 3,5 the slow waves (the appendix
 *       swaps the two labels); upper sign for m <= 3.
 *   R4  characteristic 7-vector (rho, m_n, m_t1, m_t2, B_t1, B_t2, E).
 *   R5  beta normalised by |B_t|.
 *   R6  sgn(B_n) = +1 iff B_n >= eps_B (so sgn(0) = -1).
 *   R7  fast-mode left eigenvector corrected (1/(2 c_s^2) on all seven
 *       components, gamma_1 alpha_f v^2 +- Gamma_f, -+ alpha_f c_f,
 *       + sqrt(rho) c_s alpha_s beta in the B rows).
 *   R7b entropy right eigenvector energy row = v^2/2 (printed as 1/2).
 *   R8  interface state = arithmetic mean of the two cells' primitives.
 *   R9  alpha(m) = max(|lambda_m(i)|, |lambda_m(i+1)|), cell eigenvalues.
 *   R10 WENO-Z alpha_k = d_k (1 + (tau_5/(eps_Z + IS_k))^2).
 *   R12 sweep frames are cyclic: x:(x,y,z), y:(y,z,x), z:(z,x,y).
 *   R13 CT corrections: g*_x = g_x + <B_y v_x>_j, g*_z = g_z + <B_y v_z>_j.
 *   R14 b_k = b0 - c_k dt curl Omega(q_{k-1}); cell B of q_k = interp(b_k);
 *       final b = b0 - dt curl(sum_k w'_k Omega_k), w' = (1,2,2,1)/6;
 *       E is not changed when cell B is re-interpolated.
 *   R15 dt = CFL / sum_d (S_d / dx_d), S_d = max(|v_d| + c_f^d).
 *   R17 optional floors act only inside primitive recovery.
 *   R19 the 1/12 central term uses the unsplit projected flux.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* configuration and context                                          */
/* ------------------------------------------------------------------ */

typedef struct {
    double gamma;      /* adiabatic index */
    double cfl;        /* Courant number, Sec. 2.1 (0.8 in the paper) */
    int weno_variant;  /* 0 = Jiang-Shu, 1 = WENO-Z (R10), 2 = WENO-Z as printed */
    double eps_js;     /* 1e-6, Sec. 2.2 */
    double eps_z;      /* 1e-40, Sec. 2.2 */
    double eps_b;      /* 1e-30, Appendix A */
    int floors;        /* 0 = off (paper default), 1 = on (R17) */
    double rho_min, p_min;
} ora_config;

typedef struct {
    ora_config c;
    int nx, ny, nz;
    long n;
    double dx, dy, dz;
    double *q[5];      /* rho, m_x, m_y, m_z, E at cell centres */
    double *b[3];      /* b_x at (i+1/2,j,k), b_y at (i,j+1/2,k), b_z at (i,j,k+1/2) */
    long floor_hits;
    int nonphysical;
    int have_state;
} ora_ctx;

enum { ORA_OK = 0, ORA_ERR_ARG = -1, ORA_ERR_STATE = -3, ORA_ERR_NONPHYSICAL = -4 };

static inline int wrap(int i, int n) { int r = i % n; return r < 0 ? r + n : r; }
static inline long idx3(const ora_ctx *c, int i, int j, int k) {
    return (long)wrap(i, c->nx) + (long)c->nx * ((long)wrap(j, c->ny) + (long)c->ny * (long)wrap(k, c->nz));
}
static double sq(double x) { return x * x; }
static double dmax(double a, double b) { return a > b ? a : b; }

int ora_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Host threads of the following calls (n >= 1); used to time the oracle on
 * one core and on all cores. */
int ora_set_num_threads(int n) {
    if (n < 1) return -1;
#ifdef _OPENMP
    omp_set_num_threads(n);
#endif
    return 0;
}

int ora_create(const ora_config *cfg, ora_ctx **out) {
    if (!cfg || !out) return ORA_ERR_ARG;
    if (!(cfg->gamma > 1.0) || !(cfg->cfl > 0.0)) return ORA_ERR_ARG;
    if (cfg->weno_variant < 0 || cfg->weno_variant > 2) return ORA_ERR_ARG;
    ora_ctx *c = (ora_ctx *)calloc(1, sizeof(ora_ctx));
    if (!c) return ORA_ERR_ARG;
    c->c = *cfg;
    *out = c;
    return ORA_OK;
}

static void free_fields(ora_ctx *c) {
    for (int f = 0; f < 5; f++) { free(c->q[f]); c->q[f] = NULL; }
    for (int f = 0; f < 3; f++) { free(c->b[f]); c->b[f] = NULL; }
}

int ora_destroy(ora_ctx *c) {
    if (!c) return ORA_ERR_ARG;
    free_fields(c);
    free(c);
    return ORA_OK;
}

int ora_init_grid(ora_ctx *c, int nx, int ny, int nz, double dx, double dy, double dz) {
    if (!c || nx < 1 || ny < 1 || nz < 1 || !(dx > 0) || !(dy > 0) || !(dz > 0)) return ORA_ERR_ARG;
    free_fields(c);
    c->nx = nx; c->ny = ny; c->nz = nz;
    c->n = (long)nx * ny * nz;
    c->dx = dx; c->dy = dy; c->dz = dz;
    for (int f = 0; f < 5; f++) c->q[f] = (double *)calloc((size_t)c->n, sizeof(double));
    for (int f = 0; f < 3; f++) c->b[f] = (double *)calloc((size_t)c->n, sizeof(double));
    c->have_state = 0;
    c->floor_hits = 0;
    c->nonphysical = 0;
    return ORA_OK;
}

/* cons: 5 planes of n doubles (rho, mx, my, mz, E); bface: 3 planes (bx, by, bz) */
int ora_set_state(ora_ctx *c, const double *cons, const double *bface) {
    if (!c || !cons || !bface || c->n == 0) return ORA_ERR_ARG;
    for (int f = 0; f < 5; f++) memcpy(c->q[f], cons + (size_t)f * c->n, (size_t)c->n * sizeof(double));
    for (int f = 0; f < 3; f++) memcpy(c->b[f], bface + (size_t)f * c->n, (size_t)c->n * sizeof(double));
    c->have_state = 1;
    c->nonphysical = 0;
    return ORA_OK;
}

/* ------------------------------------------------------------------ */
/* Sec. 2.3: fourth-order face -> cell interpolation of b             */
/* ------------------------------------------------------------------ */

/* B_x(i) = (-b_x(i-2) + 9 b_x(i-1) + 9 b_x(i) - b_x(i+1)) / 16, where the
 * face array index i stores the face at i+1/2. */
static void cell_B(const ora_ctx *c, double *const b[3], double *Bc[3]) {
#pragma omp parallel for schedule(static)
    for (int k = 0; k < c->nz; k++)
        for (int j = 0; j < c->ny; j++)
            for (int i = 0; i < c->nx; i++) {
                long p = idx3(c, i, j, k);
                Bc[0][p] = (-b[0][idx3(c, i - 2, j, k)] + 9.0 * b[0][idx3(c, i - 1, j, k)]
                            + 9.0 * b[0][idx3(c, i, j, k)] - b[0][idx3(c, i + 1, j, k)]) / 16.0;
                Bc[1][p] = (-b[1][idx3(c, i, j - 2, k)] + 9.0 * b[1][idx3(c, i, j - 1, k)]
                            + 9.0 * b[1][idx3(c, i, j, k)] - b[1][idx3(c, i, j + 1, k)]) / 16.0;
                Bc[2][p] = (-b[2][idx3(c, i, j, k - 2)] + 9.0 * b[2][idx3(c, i, j, k - 1)]
                            + 9.0 * b[2][idx3(c, i, j, k)] - b[2][idx3(c, i, j, k + 1)]) / 16.0;
            }
}

/* ------------------------------------------------------------------ */
/* Sec. 2, Eqs. (P), (fluxes): primitives and the flux in a sweep frame */
/* ------------------------------------------------------------------ */

/* Primitive state of one cell in the frame (n, t1, t2):
 * w = (rho, v_n, v_t1, v_t2, B_n, B_t1, B_t2, P).  Returns 1 if a floor
 * was applied (R17), sets *bad if the state is not physical. */
static int primitives(const ora_config *cfg, double rho, const double m[3], double E,
                      const double B[3], const int ax[3], double w[8], int *bad) {
    int hit = 0;
    double r = rho;
    if (cfg->floors && r < cfg->rho_min) { r = cfg->rho_min; hit = 1; }
    double v[3] = { m[0] / r, m[1] / r, m[2] / r };
    double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    double B2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    double P = (cfg->gamma - 1.0) * (E - 0.5 * r * v2 - 0.5 * B2);
    if (cfg->floors && P < cfg->p_min) { P = cfg->p_min; hit = 1; }
    if (!(r > 0.0) || !(P > 0.0) || !isfinite(P)) *bad = 1;
    w[0] = r;
    w[1] = v[ax[0]]; w[2] = v[ax[1]]; w[3] = v[ax[2]];
    w[4] = B[ax[0]]; w[5] = B[ax[1]]; w[6] = B[ax[2]];
    w[7] = P;
    return hit;
}

/* Flux along n of the 7-vector (rho, m_n, m_t1, m_t2, B_t1, B_t2, E),
 * Eq. (fluxes) with R1 for P*; the B_n component (zero) is dropped (R4). */
static void frame_flux(const double w[8], double E, double F[7]) {
    double rho = w[0], vn = w[1], vt1 = w[2], vt2 = w[3];
    double Bn = w[4], Bt1 = w[5], Bt2 = w[6], P = w[7];
    double Ps = P + 0.5 * (Bn * Bn + Bt1 * Bt1 + Bt2 * Bt2);
    double vB = vn * Bn + vt1 * Bt1 + vt2 * Bt2;
    F[0] = rho * vn;
    F[1] = rho * vn * vn + Ps - Bn * Bn;
    F[2] = rho * vn * vt1 - Bn * Bt1;
    F[3] = rho * vn * vt2 - Bn * Bt2;
    F[4] = Bt1 * vn - Bn * vt1;
    F[5] = Bt2 * vn - Bn * vt2;
    F[6] = (E + Ps) * vn - Bn * vB;
}

/* ------------------------------------------------------------------ */
/* Sec. 2, Eqs. (slow),(fast),(ca) with R2                            */
/* ------------------------------------------------------------------ */

typedef struct {
    double cs2, cs, ca, cf2, cf, cslow2, cslow;
    double fmc;  /* c_f^2 - c_s^2 */
    double cms;  /* c_s^2 - c_slow^2 */
} speeds;

static void wave_speeds(double gamma, double rho, double P, double Bn, double Bt1, double Bt2, speeds *s) {
    double cs2 = gamma * P / rho;
    double ca2 = Bn * Bn / rho;
    double bt2 = (Bt1 * Bt1 + Bt2 * Bt2) / rho;
    double d = sq(cs2 - ca2) + bt2 * (bt2 + 2.0 * ca2 + 2.0 * cs2);
    double sd = sqrt(d);
    double a = ca2 + bt2 - cs2;            /* B^2/rho - c_s^2 */
    double fmc, cms;
    if (a >= 0.0) {
        fmc = 0.5 * (a + sd);
        cms = fmc > 0.0 ? cs2 * bt2 / fmc : 0.0;   /* (c_f^2-c_s^2)(c_s^2-c_slow^2) = c_s^2 b_t^2 */
    } else {
        cms = 0.5 * (sd - a);
        fmc = cms > 0.0 ? cs2 * bt2 / cms : 0.0;
    }
    s->cs2 = cs2;
    s->cs = sqrt(cs2);
    s->ca = fabs(Bn) / sqrt(rho);
    s->fmc = fmc;
    s->cms = cms;
    s->cf2 = cs2 + fmc;
    /* c_slow^2 c_f^2 = c_s^2 c_A^2 gives c_slow^2 without cancellation */
    s->cslow2 = s->cf2 > 0.0 ? cs2 * ca2 / s->cf2 : 0.0;
    s->cf = sqrt(s->cf2);
    s->cslow = sqrt(s->cslow2);
}

/* ------------------------------------------------------------------ */
/* Appendix A: left / right eigenvectors (rows m = 1..7 -> 0..6)       */
/* ------------------------------------------------------------------ */

/* L[m][c] is component c of the m-th left eigenvector, R[m][c] component c
 * of the m-th right eigenvector, lam[m] the m-th eigenvalue, ordered
 * (v-c_f, v-c_A, v-c_slow, v, v+c_slow, v+c_A, v+c_f) (Sec. 2, R3). */
static void eigensystem(const double w[8], double gamma, double eps_b,
                        double L[7][7], double R[7][7], double lam[7]) {
    double rho = w[0], vn = w[1], vt1 = w[2], vt2 = w[3];
    double Bn = w[4], Bt1 = w[5], Bt2 = w[6], P = w[7];
    speeds s;
    wave_speeds(gamma, rho, P, Bn, Bt1, Bt2, &s);
    double cs = s.cs, cs2 = s.cs2, cf = s.cf, cslow = s.cslow, ca = s.ca;

    /* alpha_f, alpha_s (Eq. alpha): c_f^2 - c_slow^2 = fmc + cms */
    double dfs = s.fmc + s.cms;
    double af, as;
    if (sqrt(dfs) >= eps_b) {
        af = sqrt(dmax(s.cms / dfs, 0.0));
        as = sqrt(dmax(s.fmc / dfs, 0.0));
    } else {
        af = 1.0;
        as = 1.0;
    }
    /* beta (R5) and sgn(B_n) (R6) */
    double bt = Bt1 * Bt1 + Bt2 * Bt2;
    double b1, b2;
    if (bt > eps_b) {
        double m = sqrt(bt);
        b1 = Bt1 / m;
        b2 = Bt2 / m;
    } else {
        b1 = 1.0 / sqrt(2.0);
        b2 = 1.0 / sqrt(2.0);
    }
    double sg = (Bn >= eps_b) ? 1.0 : -1.0;

    double g1 = 0.5 * (gamma - 1.0);
    double g2 = (gamma - 2.0) / (gamma - 1.0);
    double tau = (gamma - 1.0) / cs2;
    double v2 = vn * vn + vt1 * vt1 + vt2 * vt2;
    double sr = sqrt(rho);
    double bv = b1 * vt1 + b2 * vt2;
    double Gf = af * cf * vn - as * cslow * sg * bv;
    double Ga = sg * (b2 * vt1 - b1 * vt2);
    double Gs = as * cslow * vn + af * cf * sg * bv;
    double pre = 1.0 / (2.0 * cs2);

    for (int pass = 0; pass < 2; pass++) {
        double sgn = pass == 0 ? 1.0 : -1.0;   /* upper sign for m <= 3 */
        int mf = pass == 0 ? 0 : 6;            /* fast */
        int ma = pass == 0 ? 1 : 5;            /* Alfven */
        int ms = pass == 0 ? 2 : 4;            /* slow */

        /* fast mode, R7 */
        L[mf][0] = pre * (g1 * af * v2 + sgn * Gf);
        L[mf][1] = pre * ((1.0 - gamma) * af * vn - sgn * af * cf);
        L[mf][2] = pre * ((1.0 - gamma) * af * vt1 + sgn * cslow * as * b1 * sg);
        L[mf][3] = pre * ((1.0 - gamma) * af * vt2 + sgn * cslow * as * b2 * sg);
        L[mf][4] = pre * ((1.0 - gamma) * af * Bt1 + sr * cs * as * b1);
        L[mf][5] = pre * ((1.0 - gamma) * af * Bt2 + sr * cs * as * b2);
        L[mf][6] = pre * ((gamma - 1.0) * af);
        R[mf][0] = af;
        R[mf][1] = af * (vn - sgn * cf);
        R[mf][2] = af * vt1 + sgn * cslow * as * b1 * sg;
        R[mf][3] = af * vt2 + sgn * cslow * as * b2 * sg;
        R[mf][4] = cs * as * b1 / sr;
        R[mf][5] = cs * as * b2 / sr;
        R[mf][6] = af * (0.5 * v2 + s.cf2 - g2 * cs2) - sgn * Gf;

        /* Alfven mode (printed under "slow", R3) */
        L[ma][0] = 0.5 * Ga;
        L[ma][1] = 0.0;
        L[ma][2] = -0.5 * b2 * sg;
        L[ma][3] = 0.5 * b1 * sg;
        L[ma][4] = -sgn * 0.5 * sr * b2;
        L[ma][5] = sgn * 0.5 * sr * b1;
        L[ma][6] = 0.0;
        R[ma][0] = 0.0;
        R[ma][1] = 0.0;
        R[ma][2] = -b2 * sg;
        R[ma][3] = b1 * sg;
        R[ma][4] = -sgn * b2 / sr;
        R[ma][5] = sgn * b1 / sr;
        R[ma][6] = -Ga;

        /* slow mode (printed under "Alfven", R3) */
        L[ms][0] = pre * (g1 * as * v2 + sgn * Gs);
        L[ms][1] = pre * ((1.0 - gamma) * as * vn - sgn * as * cslow);
        L[ms][2] = pre * ((1.0 - gamma) * as * vt1 - sgn * cf * af * b1 * sg);
        L[ms][3] = pre * ((1.0 - gamma) * as * vt2 - sgn * cf * af * b2 * sg);
        L[ms][4] = pre * ((1.0 - gamma) * as * Bt1 - sr * cs * af * b1);
        L[ms][5] = pre * ((1.0 - gamma) * as * Bt2 - sr * cs * af * b2);
        L[ms][6] = pre * ((gamma - 1.0) * as);
        R[ms][0] = as;
        R[ms][1] = as * (vn - sgn * cslow);
        R[ms][2] = as * vt1 - sgn * cf * af * b1 * sg;
        R[ms][3] = as * vt2 - sgn * cf * af * b2 * sg;
        R[ms][4] = -cs * af * b1 / sr;
        R[ms][5] = -cs * af * b2 / sr;
        R[ms][6] = as * (0.5 * v2 + s.cslow2 - g2 * cs2) - sgn * Gs;
    }
    /* entropy mode, R7b */
    L[3][0] = 1.0 - 0.5 * tau * v2;
    L[3][1] = tau * vn;
    L[3][2] = tau * vt1;
    L[3][3] = tau * vt2;
    L[3][4] = tau * Bt1;
    L[3][5] = tau * Bt2;
    L[3][6] = -tau;
    R[3][0] = 1.0;
    R[3][1] = vn;
    R[3][2] = vt1;
    R[3][3] = vt2;
    R[3][4] = 0.0;
    R[3][5] = 0.0;
    R[3][6] = 0.5 * v2;

    lam[0] = vn - cf;
    lam[1] = vn - ca;
    lam[2] = vn - cslow;
    lam[3] = vn;
    lam[4] = vn + cslow;
    lam[5] = vn + ca;
    lam[6] = vn + cf;
}

/* ------------------------------------------------------------------ */
/* Sec. 2.2: WENO interpolant phi_N and the characteristic face flux   */
/* ------------------------------------------------------------------ */

static double phi_n(double a, double b, double c, double d, const ora_config *cfg) {
    double IS0 = 13.0 * sq(a - b) + 3.0 * sq(a - 3.0 * b);
    double IS1 = 13.0 * sq(b - c) + 3.0 * sq(b + c);
    double IS2 = 13.0 * sq(c - d) + 3.0 * sq(3.0 * c - d);
    double a0, a1, a2;
    if (cfg->weno_variant == 0) {
        a0 = 1.0 / sq(cfg->eps_js + IS0);
        a1 = 6.0 / sq(cfg->eps_js + IS1);
        a2 = 3.0 / sq(cfg->eps_js + IS2);
    } else if (cfg->weno_variant == 1) {
        double t5 = fabs(IS0 - IS2);
        a0 = 1.0 * (1.0 + sq(t5 / (cfg->eps_z + IS0)));
        a1 = 6.0 * (1.0 + sq(t5 / (cfg->eps_z + IS1)));
        a2 = 3.0 * (1.0 + sq(t5 / (cfg->eps_z + IS2)));
    } else {
        double t5 = fabs(IS0 - IS2);
        a0 = 1.0 * (1.0 + t5 / sq(cfg->eps_z + IS0));
        a1 = 6.0 * (1.0 + t5 / sq(cfg->eps_z + IS1));
        a2 = 3.0 * (1.0 + t5 / sq(cfg->eps_z + IS2));
    }
    double w0 = a0 / (a0 + a1 + a2);
    double w2 = a2 / (a0 + a1 + a2);
    return w0 / 3.0 * (a - 2.0 * b + c) + (w2 - 0.5) / 6.0 * (b - 2.0 * c + d);
}

/* Eq. (FWENO) for one characteristic field: Fs[k], qs[k] are the projected
 * flux and state at k = i-2 .. i+3 (array index 0..5), alpha the LF speed. */
static double weno_char_flux(const double Fs[6], const double qs[6], double alpha, const ora_config *cfg) {
    double dFp[5], dFm[5];
    for (int j = 0; j < 5; j++) {       /* differences at i-3/2 .. i+5/2 */
        double dF = Fs[j + 1] - Fs[j];
        double dq = qs[j + 1] - qs[j];
        dFp[j] = 0.5 * (dF + alpha * dq);
        dFm[j] = 0.5 * (dF - alpha * dq);
    }
    double central = (-Fs[1] + 7.0 * Fs[2] + 7.0 * Fs[3] - Fs[4]) / 12.0;
    return central - phi_n(dFp[0], dFp[1], dFp[2], dFp[3], cfg)
                   + phi_n(dFm[4], dFm[3], dFm[2], dFm[1], cfg);
}

/* per-cell data of one sweep */
typedef struct {
    double w[8];    /* primitives in the frame */
    double u[7];    /* characteristic-system state (rho, m_n, m_t1, m_t2, B_t1, B_t2, E) */
    double F[7];    /* flux along n */
    double lam[7];  /* cell eigenvalues (R9) */
} cellq;

/* Face flux at i+1/2 from the six cells i-2 .. i+3 (Sec. 2.2, Appendix A). */
static void face_flux(const cellq *st[6], const ora_config *cfg, double Fface[7]) {
    double wa[8];
    for (int v = 0; v < 8; v++) wa[v] = 0.5 * (st[2]->w[v] + st[3]->w[v]);   /* R8 */
    double L[7][7], R[7][7], lam[7];
    eigensystem(wa, cfg->gamma, cfg->eps_b, L, R, lam);
    double Fsf[7];
    for (int m = 0; m < 7; m++) {
        double alpha = dmax(fabs(st[2]->lam[m]), fabs(st[3]->lam[m]));   /* R9 */
        double Fs[6], qs[6];
        for (int k = 0; k < 6; k++) {
            double f = 0.0, q = 0.0;
            for (int c = 0; c < 7; c++) {
                f += L[m][c] * st[k]->F[c];
                q += L[m][c] * st[k]->u[c];
            }
            Fs[k] = f;
            qs[k] = q;
        }
        Fsf[m] = weno_char_flux(Fs, qs, alpha, cfg);
    }
    for (int c = 0; c < 7; c++) {
        double f = 0.0;
        for (int m = 0; m < 7; m++) f += Fsf[m] * R[m][c];
        Fface[c] = f;
    }
}

static void fill_cellq(const ora_config *cfg, double rho, const double m[3], double E, const double B[3],
                       const int ax[3], cellq *cq, long *hits, int *bad) {
    if (primitives(cfg, rho, m, E, B, ax, cq->w, bad)) (*hits)++;
    frame_flux(cq->w, E, cq->F);
    cq->u[0] = rho;
    cq->u[1] = m[ax[0]];
    cq->u[2] = m[ax[1]];
    cq->u[3] = m[ax[2]];
    cq->u[4] = B[ax[1]];
    cq->u[5] = B[ax[2]];
    cq->u[6] = E;
    speeds s;
    wave_speeds(cfg->gamma, cq->w[0], cq->w[7], cq->w[4], cq->w[5], cq->w[6], &s);
    double vn = cq->w[1];
    cq->lam[0] = vn - s.cf;
    cq->lam[1] = vn - s.ca;
    cq->lam[2] = vn - s.cslow;
    cq->lam[3] = vn;
    cq->lam[4] = vn + s.cslow;
    cq->lam[5] = vn + s.ca;
    cq->lam[6] = vn + s.cf;
}

/* ------------------------------------------------------------------ */
/* Sec. 3.1.3: one directional sweep                                  */
/* ------------------------------------------------------------------ */

/* Sweep along axis a (0,1,2).  Adds -(F_{+} - F_{-})/dx_a of the five
 * non-magnetic fields to D and stores the two CT transport fluxes of the
 * tangential field components on the faces (Eqs. fct1-fct6, R13):
 * s1 for component t1, s2 for component t2 of the frame (R12). */
static void sweep(ora_ctx *c, int a, double *const qs[5], double *const Bc[3],
                  double *D[5], double *s1, double *s2) {
    int ax[3] = { a, (a + 1) % 3, (a + 2) % 3 };
    int nn[3] = { c->nx, c->ny, c->nz };
    double h = a == 0 ? c->dx : (a == 1 ? c->dy : c->dz);
    cellq *cq = (cellq *)malloc((size_t)c->n * sizeof(cellq));
    long hits = 0;
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : hits) reduction(| : bad)
    for (long p = 0; p < c->n; p++) {
        double m[3] = { qs[1][p], qs[2][p], qs[3][p] };
        double B[3] = { Bc[0][p], Bc[1][p], Bc[2][p] };
        long lh = 0;
        int lb = 0;
        fill_cellq(&c->c, qs[0][p], m, qs[4][p], B, ax, &cq[p], &lh, &lb);
        hits += lh;
        bad |= lb;
    }
    c->floor_hits += hits;
    if (bad) c->nonphysical = 1;

    double *Ff = (double *)malloc((size_t)c->n * 7 * sizeof(double));   /* face fluxes */
#pragma omp parallel for schedule(static)
    for (int k = 0; k < c->nz; k++)
        for (int j = 0; j < c->ny; j++)
            for (int i = 0; i < c->nx; i++) {
                int ijk[3] = { i, j, k };
                const cellq *st[6];
                for (int s = 0; s < 6; s++) {
                    int q3[3] = { ijk[0], ijk[1], ijk[2] };
                    q3[a] = wrap(ijk[a] - 2 + s, nn[a]);
                    st[s] = &cq[idx3(c, q3[0], q3[1], q3[2])];
                }
                long p = idx3(c, i, j, k);
                double F[7];
                face_flux(st, &c->c, F);
                for (int v = 0; v < 7; v++) Ff[p * 7 + v] = F[v];
                /* CT transport fluxes on this face: F_{B_t} + <B_n v_t> */
                s1[p] = F[4] + 0.5 * (st[2]->w[4] * st[2]->w[2] + st[3]->w[4] * st[3]->w[2]);
                s2[p] = F[5] + 0.5 * (st[2]->w[4] * st[2]->w[3] + st[3]->w[4] * st[3]->w[3]);
            }
    /* flux divergence of the non-magnetic components, Eq. (num) */
    static const int lab_of_frame_m[3][3] = { { 1, 2, 3 }, { 2, 3, 1 }, { 3, 1, 2 } };
#pragma omp parallel for schedule(static)
    for (int k = 0; k < c->nz; k++)
        for (int j = 0; j < c->ny; j++)
            for (int i = 0; i < c->nx; i++) {
                int q3[3] = { i, j, k };
                q3[a] -= 1;
                long p = idx3(c, i, j, k);
                long pm = idx3(c, q3[0], q3[1], q3[2]);
                D[0][p] -= (Ff[p * 7 + 0] - Ff[pm * 7 + 0]) / h;
                for (int t = 0; t < 3; t++) {
                    int lab = lab_of_frame_m[a][t];
                    D[lab][p] -= (Ff[p * 7 + 1 + t] - Ff[pm * 7 + 1 + t]) / h;
                }
                D[4][p] -= (Ff[p * 7 + 6] - Ff[pm * 7 + 6]) / h;
            }
    free(Ff);
    free(cq);
}

/* Eqs. (ox1)-(ox3): corner EMFs from the starred fluxes.
 *   x-faces: fy = f*_y, fz = f*_z;  y-faces: gz = g*_z, gx = g*_x;
 *   z-faces: hx = h*_x, hy = h*_y.
 * Om[0] = Omega_x at (i+1/2, j+1/2, k), Om[1] = Omega_y at (i, j+1/2, k+1/2),
 * Om[2] = Omega_z at (i+1/2, j, k+1/2). */
static void corner_emf(const ora_ctx *c, const double *fy, const double *fz, const double *gz,
                       const double *gx, const double *hx, const double *hy, double *Om[3]) {
#pragma omp parallel for schedule(static)
    for (int k = 0; k < c->nz; k++)
        for (int j = 0; j < c->ny; j++)
            for (int i = 0; i < c->nx; i++) {
                long p = idx3(c, i, j, k);
                Om[0][p] = 0.5 * (gx[p] + gx[idx3(c, i + 1, j, k)]) - 0.5 * (fy[p] + fy[idx3(c, i, j + 1, k)]);
                Om[1][p] = 0.5 * (hy[p] + hy[idx3(c, i, j + 1, k)]) - 0.5 * (gz[p] + gz[idx3(c, i, j, k + 1)]);
                Om[2][p] = 0.5 * (fz[p] + fz[idx3(c, i, j, k + 1)]) - 0.5 * (hx[p] + hx[idx3(c, i + 1, j, k)]);
            }
}

/* Sec. 2.3: b_out = b_in + fac * db/dt, with db/dt on the faces taken from
 * the face equations of the paper (dbx/dt = -(Om_x(j)-Om_x(j-1))/dy
 * + (Om_z(k)-Om_z(k-1))/dz and cyclic). */
static void ct_update(const ora_ctx *c, double *const b_in[3], double *const Om[3], double fac, double *b_out[3]) {
#pragma omp parallel for schedule(static)
    for (int k = 0; k < c->nz; k++)
        for (int j = 0; j < c->ny; j++)
            for (int i = 0; i < c->nx; i++) {
                long p = idx3(c, i, j, k);
                double dbx = -(Om[0][p] - Om[0][idx3(c, i, j - 1, k)]) / c->dy
                             + (Om[2][p] - Om[2][idx3(c, i, j, k - 1)]) / c->dz;
                double dby = -(Om[1][p] - Om[1][idx3(c, i, j, k - 1)]) / c->dz
                             + (Om[0][p] - Om[0][idx3(c, i - 1, j, k)]) / c->dx;
                double dbz = -(Om[2][p] - Om[2][idx3(c, i - 1, j, k)]) / c->dx
                             + (Om[1][p] - Om[1][idx3(c, i, j - 1, k)]) / c->dy;
                b_out[0][p] = b_in[0][p] + fac * dbx;
                b_out[1][p] = b_in[1][p] + fac * dby;
                b_out[2][p] = b_in[2][p] + fac * dbz;
            }
}

/* ------------------------------------------------------------------ */
/* Sec. 2.1 + Sec. 3.1.3 (R14): the RK4 / CT driver                    */
/* ------------------------------------------------------------------ */

/* Right-hand side of one stage: from the stage state (qs, bs) it returns
 * dq/dt of the five non-magnetic fields in D and the corner EMFs in Om. */
typedef void (*ora_rhs_fn)(ora_ctx *c, void *user, double *const qs[5], double *const bs[3],
                           double *D[5], double *Om[3]);

static double **alloc_planes(int nf, long n) {
    double **a = (double **)malloc((size_t)nf * sizeof(double *));
    for (int f = 0; f < nf; f++) a[f] = (double *)calloc((size_t)n, sizeof(double));
    return a;
}
static void free_planes(double **a, int nf) {
    for (int f = 0; f < nf; f++) free(a[f]);
    free(a);
}

static void rk4_ct_drive(ora_ctx *c, double dt, ora_rhs_fn rhs, void *user) {
    static const double ck[4] = { 0.5, 0.5, 1.0, 1.0 / 6.0 };           /* stage factors */
    static const double wk[4] = { 1.0 / 3.0, 2.0 / 3.0, 1.0 / 3.0, 1.0 };  /* q_save weights */
    static const double wo[4] = { 1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0 };  /* EMF weights, R14 */
    long n = c->n;
    double **q0 = alloc_planes(5, n), **qsave = alloc_planes(5, n), **qs = alloc_planes(5, n);
    double **b0 = alloc_planes(3, n), **bs = alloc_planes(3, n), **Oacc = alloc_planes(3, n);
    double **D = alloc_planes(5, n), **Om = alloc_planes(3, n);
    for (int f = 0; f < 5; f++)
        for (long p = 0; p < n; p++) {
            q0[f][p] = c->q[f][p];
            qs[f][p] = c->q[f][p];
            qsave[f][p] = -4.0 / 3.0 * q0[f][p];
        }
    for (int f = 0; f < 3; f++)
        for (long p = 0; p < n; p++) {
            b0[f][p] = c->b[f][p];
            bs[f][p] = c->b[f][p];
        }
    for (int s = 0; s < 4; s++) {
        for (int f = 0; f < 5; f++) memset(D[f], 0, (size_t)n * sizeof(double));
        rhs(c, user, qs, bs, D, Om);
        for (int f = 0; f < 5; f++)
            for (long p = 0; p < n; p++) {
                qs[f][p] = q0[f][p] + ck[s] * dt * D[f][p];
                qsave[f][p] = qsave[f][p] + wk[s] * qs[f][p];
            }
        for (int f = 0; f < 3; f++)
            for (long p = 0; p < n; p++) Oacc[f][p] = Oacc[f][p] + wo[s] * Om[f][p];
        if (s < 3) ct_update(c, b0, Om, ck[s] * dt, bs);
    }
    for (int f = 0; f < 5; f++) memcpy(c->q[f], qsave[f], (size_t)n * sizeof(double));
    ct_update(c, b0, Oacc, dt, c->b);   /* the final CT update of q_save */
    free_planes(q0, 5); free_planes(qsave, 5); free_planes(qs, 5);
    free_planes(b0, 3); free_planes(bs, 3); free_planes(Oacc, 3);
    free_planes(D, 5); free_planes(Om, 3);
}

static void mhd_rhs(ora_ctx *c, void *user, double *const qs[5], double *const bs[3],
                    double *D[5], double *Om[3]) {
    (void)user;
    long n = c->n;
    double **Bc = alloc_planes(3, n);
    double **st = alloc_planes(6, n);   /* fy, fz, gz, gx, hx, hy */
    cell_B(c, bs, Bc);
    sweep(c, 0, qs, Bc, D, st[0], st[1]);   /* x: t1 = y, t2 = z */
    sweep(c, 1, qs, Bc, D, st[2], st[3]);   /* y: t1 = z, t2 = x */
    sweep(c, 2, qs, Bc, D, st[4], st[5]);   /* z: t1 = x, t2 = y */
    corner_emf(c, st[0], st[1], st[2], st[3], st[4], st[5], Om);
    free_planes(Bc, 3);
    free_planes(st, 6);
}

int ora_step(ora_ctx *c, double dt) {
    if (!c || !(dt > 0.0) || !isfinite(dt)) return ORA_ERR_ARG;
    if (!c->have_state) return ORA_ERR_STATE;
    rk4_ct_drive(c, dt, mhd_rhs, NULL);
    return c->nonphysical ? ORA_ERR_NONPHYSICAL : ORA_OK;
}

/* The same driver with a linear right-hand side dq/dt = M q acting on the
 * field pair (rho, m_x) and Omega = 0: a check of the stage coefficients. */
static void linear_rhs(ora_ctx *c, void *user, double *const qs[5], double *const bs[3],
                       double *D[5], double *Om[3]) {
    (void)bs;
    const double *M = (const double *)user;
    for (long p = 0; p < c->n; p++) {
        D[0][p] = M[0] * qs[0][p] + M[1] * qs[1][p];
        D[1][p] = M[2] * qs[0][p] + M[3] * qs[1][p];
        D[2][p] = D[3][p] = D[4][p] = 0.0;
        Om[0][p] = Om[1][p] = Om[2][p] = 0.0;
    }
}

int ora_step_linear(ora_ctx *c, double dt, const double M[4]) {
    if (!c || !M || !c->have_state) return ORA_ERR_ARG;
    rk4_ct_drive(c, dt, linear_rhs, (void *)M);
    return ORA_OK;
}

/* ------------------------------------------------------------------ */
/* state readback, Eq. (cfl) speeds, diagnostics                      */
/* ------------------------------------------------------------------ */

int ora_get_state(ora_ctx *c, double *cons, double *bface, double *bcell) {
    if (!c || !c->have_state) return ORA_ERR_STATE;
    long n = c->n;
    if (cons)
        for (int f = 0; f < 5; f++) memcpy(cons + (size_t)f * n, c->q[f], (size_t)n * sizeof(double));
    if (bface)
        for (int f = 0; f < 3; f++) memcpy(bface + (size_t)f * n, c->b[f], (size_t)n * sizeof(double));
    if (bcell) {
        double *Bc[3] = { bcell, bcell + n, bcell + 2 * n };
        cell_B(c, c->b, Bc);
    }
    return ORA_OK;
}

/* S_d = max over cells of |v_d| + c_f^d (Eq. cfl), c_f^d with B_n = B_d. */
int ora_max_signal_speed(ora_ctx *c, double out[3]) {
    if (!c || !out) return ORA_ERR_ARG;
    if (!c->have_state) return ORA_ERR_STATE;
    double **Bc = alloc_planes(3, c->n);
    cell_B(c, c->b, Bc);
    double S[3] = { 0.0, 0.0, 0.0 };
    int bad = 0;
    for (long p = 0; p < c->n; p++) {
        double m[3] = { c->q[1][p], c->q[2][p], c->q[3][p] };
        double B[3] = { Bc[0][p], Bc[1][p], Bc[2][p] };
        for (int a = 0; a < 3; a++) {
            int ax[3] = { a, (a + 1) % 3, (a + 2) % 3 };
            double w[8];
            primitives(&c->c, c->q[0][p], m, c->q[4][p], B, ax, w, &bad);
            speeds s;
            wave_speeds(c->c.gamma, w[0], w[7], w[4], w[5], w[6], &s);
            S[a] = dmax(S[a], fabs(w[1]) + s.cf);
        }
    }
    free_planes(Bc, 3);
    out[0] = S[0]; out[1] = S[1]; out[2] = S[2];
    return bad ? ORA_ERR_NONPHYSICAL : ORA_OK;
}

/* dt = CFL / sum_d (S_d / dx_d), Eq. (cfl) with R15 */
int ora_cfl_dt(ora_ctx *c, double *dt) {
    double S[3];
    int rc = ora_max_signal_speed(c, S);
    if (rc) return rc;
    *dt = c->c.cfl / (S[0] / c->dx + S[1] / c->dy + S[2] / c->dz);
    return ORA_OK;
}

/* discrete div b at cell centres: L_inf and RMS */
int ora_div_b_norm(ora_ctx *c, double *linf, double *l2) {
    if (!c || !linf || !l2) return ORA_ERR_ARG;
    if (!c->have_state) return ORA_ERR_STATE;
    double mx = 0.0, s2 = 0.0;
    for (int k = 0; k < c->nz; k++)
        for (int j = 0; j < c->ny; j++)
            for (int i = 0; i < c->nx; i++) {
                long p = idx3(c, i, j, k);
                double d = (c->b[0][p] - c->b[0][idx3(c, i - 1, j, k)]) / c->dx
                         + (c->b[1][p] - c->b[1][idx3(c, i, j - 1, k)]) / c->dy
                         + (c->b[2][p] - c->b[2][idx3(c, i, j, k - 1)]) / c->dz;
                mx = dmax(mx, fabs(d));
                s2 += d * d;
            }
    *linf = mx;
    *l2 = sqrt(s2 / (double)c->n);
    return ORA_OK;
}

/* volume integrals of rho, m_x, m_y, m_z, E, b_x, b_y, b_z */
int ora_conserved_totals(ora_ctx *c, double out[8]) {
    if (!c || !out) return ORA_ERR_ARG;
    if (!c->have_state) return ORA_ERR_STATE;
    double dv = c->dx * c->dy * c->dz;
    for (int f = 0; f < 8; f++) {
        const double *a = f < 5 ? c->q[f] : c->b[f - 5];
        double s = 0.0;
        for (long p = 0; p < c->n; p++) s += a[p];
        out[f] = s * dv;
    }
    return ORA_OK;
}

int ora_status(ora_ctx *c, long long *floor_hits, int *nonphysical) {
    if (!c) return ORA_ERR_ARG;
    if (floor_hits) *floor_hits = c->floor_hits;
    if (nonphysical) *nonphysical = c->nonphysical;
    return ORA_OK;
}

/* ------------------------------------------------------------------ */
/* Sec. 3.1.1: the one-dimensional program (no CT; B_n constant)       */
/* ------------------------------------------------------------------ */

/* u: 7 planes of nx doubles (rho, m_x, m_y, m_z, B_y, B_z, E), advanced
 * in place by one RK4 step along x with the paper's q / q_save form. */
int ora1d_step(const ora_config *cfg, int nx, double dx, double Bx, double *u, double dt) {
    if (!cfg || !u || nx < 1 || !(dx > 0) || !(dt > 0)) return ORA_ERR_ARG;
    static const double ck[4] = { 0.5, 0.5, 1.0, 1.0 / 6.0 };
    static const double wk[4] = { 1.0 / 3.0, 2.0 / 3.0, 1.0 / 3.0, 1.0 };
    int ax[3] = { 0, 1, 2 };
    double *q0 = (double *)malloc((size_t)7 * nx * sizeof(double));
    double *qsave = (double *)malloc((size_t)7 * nx * sizeof(double));
    double *qs = (double *)malloc((size_t)7 * nx * sizeof(double));
    double *Ff = (double *)malloc((size_t)7 * nx * sizeof(double));
    cellq *cq = (cellq *)malloc((size_t)nx * sizeof(cellq));
    int bad = 0;
    long hits = 0;
    for (int v = 0; v < 7; v++)
        for (int i = 0; i < nx; i++) {
            q0[v * nx + i] = u[v * nx + i];
            qs[v * nx + i] = u[v * nx + i];
            qsave[v * nx + i] = -4.0 / 3.0 * u[v * nx + i];
        }
    for (int s = 0; s < 4; s++) {
        for (int i = 0; i < nx; i++) {
            double m[3] = { qs[1 * nx + i], qs[2 * nx + i], qs[3 * nx + i] };
            double B[3] = { Bx, qs[4 * nx + i], qs[5 * nx + i] };
            fill_cellq(cfg, qs[i], m, qs[6 * nx + i], B, ax, &cq[i], &hits, &bad);
        }
        for (int i = 0; i < nx; i++) {
            const cellq *st[6];
            for (int k = 0; k < 6; k++) st[k] = &cq[wrap(i - 2 + k, nx)];
            double F[7];
            face_flux(st, cfg, F);
            for (int v = 0; v < 7; v++) Ff[v * nx + i] = F[v];
        }
        for (int v = 0; v < 7; v++)
            for (int i = 0; i < nx; i++) {
                double d = -(Ff[v * nx + i] - Ff[v * nx + wrap(i - 1, nx)]) / dx;
                qs[v * nx + i] = q0[v * nx + i] + ck[s] * dt * d;
                qsave[v * nx + i] = qsave[v * nx + i] + wk[s] * qs[v * nx + i];
            }
    }
    /* the 7-vector is (rho, m_n, m_t1, m_t2, B_t1, B_t2, E) = (rho, mx, my, mz, By, Bz, E) */
    memcpy(u, qsave, (size_t)7 * nx * sizeof(double));
    free(q0); free(qsave); free(qs); free(Ff); free(cq);
    return bad ? ORA_ERR_NONPHYSICAL : ORA_OK;
}

/* ------------------------------------------------------------------ */
/* entry points used by the unit tests of the pieces                   */
/* ------------------------------------------------------------------ */

/* w = (rho, v_n, v_t1, v_t2, B_n, B_t1, B_t2, P); L, R row-major 7x7 */
void ora_eigensystem(const double w[8], double gamma, double eps_b, double *L, double *R, double *lam) {
    double l[7][7], r[7][7];
    eigensystem(w, gamma, eps_b, l, r, lam);
    for (int m = 0; m < 7; m++)
        for (int c = 0; c < 7; c++) {
            L[m * 7 + c] = l[m][c];
            R[m * 7 + c] = r[m][c];
        }
}

void ora_frame_flux(const double w[8], double E, double *F) { frame_flux(w, E, F); }

void ora_wave_speeds(double gamma, const double w[8], double out[4]) {
    speeds s;
    wave_speeds(gamma, w[0], w[7], w[4], w[5], w[6], &s);
    out[0] = s.cs; out[1] = s.ca; out[2] = s.cslow; out[3] = s.cf;
}

double ora_phi_n(double a, double b, double c, double d, const ora_config *cfg) { return phi_n(a, b, c, d, cfg); }

double ora_weno_char_flux(const double Fs[6], const double qs[6], double alpha, const ora_config *cfg) {
    return weno_char_flux(Fs, qs, alpha, cfg);
}
