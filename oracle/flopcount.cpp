// flopcount.cpp -- algorithmic operation counts of the scheme, obtained by
// compiling the oracle's own source (w5ct_oracle.c) with a counting scalar
// type in place of double.
//
// TEST INFRASTRUCTURE ONLY, like the oracle it includes.  The benchmark's
// roofline divides these counts by measured kernel times; the test suite
// builds and runs this program and checks the constants the benchmark uses.
//
// What counts: every +, -, *, / and sqrt on a floating-point value counts 1
// (compound assignments too); negation, comparisons, max and |x| count 0.
// No contraction: a multiply followed by an add counts 2.
//
// Printed (one line of JSON), for the WENO variant given on the command
// line (0 = JS, 1 = Z):
//   cell   operations of one cell's recovery in one sweep (primitives,
//          Eq. P; the frame flux; the three wave speeds), fill_cellq;
//   face   operations of one interface in one sweep: the interface state,
//          the Appendix A eigensystem, the projections of the six-point
//          stencil, LF split, phi_N and back-projection (face_flux), plus
//          the two CT transport fluxes of Eqs. (fct1)-(fct6);
//   div    operations of one cell's flux divergence in one sweep;
//   step   operations per zone of one whole RK4 + CT step (ora_step), and
//   sweep  the per-zone total of one sweep (cell + face + div),
//   step_reverse  operations per zone of the reverse sweep of one step in
//          reverse-mode differentiation with respect to the step's input
//          state (q^n, b^n), dt held fixed, and
//   adjoint_step  step + step_reverse: the vector-Jacobian product of one
//          step, its forward stages recomputed once,
// measured on a generic smooth state of 12 x 10 x 8 cells (every field
// varies, no degenerate branch is taken).
//
// Reverse-mode counts (Griewank's operation-by-operation rule, with an
// activity analysis: a value is active when it depends on the input state;
// operations on passive values cost nothing in reverse).  For c = f(a, b),
// each active operand's adjoint receives one contribution, and every
// contribution costs its multiplications and divisions plus the one
// addition that accumulates it:
//   c = a +- b     1 per active operand
//   c = a * b      2 per active operand (c_bar * b, accumulate)
//   c = a / b      t = c_bar / b once, a_bar += t (1), b_bar -= t c (2):
//                  4 with both active, 2 with a only, 3 with b only
//   c = sqrt(a)    3 (c_bar / c, times 1/2, accumulate)
//   c = -a, |a|    1 (signed accumulation)
// Selections (max, branches) copy a value and cost 0 either way.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cmath>

static long long g_ops = 0;   // forward operations
static long long g_rev = 0;   // reverse-mode operations (see above)

static inline long long rev_div(bool a, bool b) { return (a && b) ? 4 : a ? 2 : b ? 3 : 0; }

struct Flop {
    double v;
    bool act;   // depends on the input state
    Flop() = default;
    constexpr Flop(double x) : v(x), act(false) {}
    constexpr Flop(double x, bool a) : v(x), act(a) {}
    explicit operator int() const { return (int)v; }
    explicit operator long() const { return (long)v; }
    Flop &operator+=(Flop o) { ++g_ops; g_rev += act + o.act; v += o.v; act = act || o.act; return *this; }
    Flop &operator-=(Flop o) { ++g_ops; g_rev += act + o.act; v -= o.v; act = act || o.act; return *this; }
    Flop &operator*=(Flop o) { ++g_ops; g_rev += 2 * (act + o.act); v *= o.v; act = act || o.act; return *this; }
    Flop &operator/=(Flop o) { ++g_ops; g_rev += rev_div(act, o.act); v /= o.v; act = act || o.act; return *this; }
};
static inline Flop operator+(Flop a, Flop b) { ++g_ops; g_rev += a.act + b.act; return Flop(a.v + b.v, a.act || b.act); }
static inline Flop operator-(Flop a, Flop b) { ++g_ops; g_rev += a.act + b.act; return Flop(a.v - b.v, a.act || b.act); }
static inline Flop operator*(Flop a, Flop b) {
    ++g_ops;
    g_rev += 2 * (a.act + b.act);
    return Flop(a.v * b.v, a.act || b.act);
}
static inline Flop operator/(Flop a, Flop b) {
    ++g_ops;
    g_rev += rev_div(a.act, b.act);
    return Flop(a.v / b.v, a.act || b.act);
}
static inline Flop operator-(Flop a) { g_rev += a.act; return Flop(-a.v, a.act); }
static inline bool operator<(Flop a, Flop b) { return a.v < b.v; }
static inline bool operator>(Flop a, Flop b) { return a.v > b.v; }
static inline bool operator<=(Flop a, Flop b) { return a.v <= b.v; }
static inline bool operator>=(Flop a, Flop b) { return a.v >= b.v; }
static inline bool operator==(Flop a, Flop b) { return a.v == b.v; }
static inline bool operator!=(Flop a, Flop b) { return a.v != b.v; }
static inline Flop sqrt(Flop a) { ++g_ops; g_rev += a.act ? 3 : 0; return Flop(std::sqrt(a.v), a.act); }
static inline Flop fabs(Flop a) { g_rev += a.act; return Flop(std::fabs(a.v), a.act); }
static inline bool isfinite(Flop a) { return std::isfinite(a.v); }

#define double Flop
#include "w5ct_oracle.c"
#undef double

// a smooth, generic periodic state: rho ~ 1, P ~ 0.6, |v| ~ 0.5, an oblique
// mean field with a 20% perturbation (no branch of Appendix A degenerates)
static void generic_state(int nx, int ny, int nz, double *cons, double *bface) {
    const double tp = 6.283185307179586, g = 5.0 / 3.0;
    const long n = (long)nx * ny * nz;
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                const long p = i + (long)nx * (j + (long)ny * k);
                const double x = (i + 0.5) / nx, y = (j + 0.5) / ny, z = (k + 0.5) / nz;
                const double rho = 1.0 + 0.1 * std::sin(tp * (x + 2 * y) + 0.3);
                const double P = 0.6 + 0.05 * std::cos(tp * (y - z) + 1.1);
                const double v[3] = {0.5 * std::sin(tp * z + 0.7), 0.4 * std::cos(tp * (x + z)), 0.3 * std::sin(tp * (y + 0.2))};
                const double b[3] = {0.8 + 0.2 * std::sin(tp * (y + z)), -0.5 + 0.2 * std::cos(tp * (x + 0.4)),
                                     0.6 + 0.2 * std::sin(tp * (x - y) + 0.9)};
                double B2 = 0.0, v2 = 0.0;
                for (int c = 0; c < 3; c++) {
                    bface[c * n + p] = b[c];
                    B2 += b[c] * b[c];
                    v2 += v[c] * v[c];
                    cons[(1 + c) * n + p] = rho * v[c];
                }
                cons[p] = rho;
                cons[4 * n + p] = P / (g - 1.0) + 0.5 * rho * v2 + 0.5 * B2;
            }
}

int main(int argc, char **argv) {
    const int variant = argc > 1 ? atoi(argv[1]) : 1;
    const int nx = 12, ny = 10, nz = 8;
    const long n = (long)nx * ny * nz;
    ora_config cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.gamma = 5.0 / 3.0;
    cfg.cfl = 0.8;
    cfg.weno_variant = variant;
    cfg.eps_js = 1e-6;
    cfg.eps_z = 1e-40;
    cfg.eps_b = 1e-30;
    ora_ctx *c = nullptr;
    if (ora_create(&cfg, &c) != ORA_OK || ora_init_grid(c, nx, ny, nz, 1.0 / nx, 1.0 / ny, 1.0 / nz) != ORA_OK) return 1;
    double *cons = (double *)malloc(sizeof(double) * 5 * n), *bface = (double *)malloc(sizeof(double) * 3 * n);
    generic_state(nx, ny, nz, cons, bface);
    Flop *cf = (Flop *)malloc(sizeof(Flop) * 5 * n), *bf = (Flop *)malloc(sizeof(Flop) * 3 * n);
    for (long p = 0; p < 5 * n; p++) cf[p] = Flop(cons[p], true);
    for (long p = 0; p < 3 * n; p++) bf[p] = Flop(bface[p], true);
    if (ora_set_state(c, cf, bf) != ORA_OK) return 1;

    // per-cell recovery and per-face flux along x, counted call by call
    Flop **Bc = alloc_planes(3, n);
    cell_B(c, c->b, Bc);
    const int ax[3] = {0, 1, 2};
    cellq *cq = (cellq *)malloc(sizeof(cellq) * n);
    long hits = 0;
    int bad = 0;
    long long t0 = g_ops;
    for (long p = 0; p < n; p++) {
        Flop m[3] = {c->q[1][p], c->q[2][p], c->q[3][p]};
        Flop B[3] = {Bc[0][p], Bc[1][p], Bc[2][p]};
        fill_cellq(&c->c, c->q[0][p], m, c->q[4][p], B, ax, &cq[p], &hits, &bad);
    }
    const long long cell_ops = g_ops - t0;
    t0 = g_ops;
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                const cellq *st[6];
                for (int s = 0; s < 6; s++) st[s] = &cq[idx3(c, i - 2 + s, j, k)];
                Flop F[7];
                face_flux(st, &c->c, F);
            }
    const long long face_core_ops = g_ops - t0;

    // one whole sweep (recovery, faces, transport fluxes, divergence)
    Flop **D = alloc_planes(5, n), **S = alloc_planes(2, n);
    t0 = g_ops;
    sweep(c, 0, c->q, Bc, D, S[0], S[1]);
    const long long sweep_ops = g_ops - t0;

    // one whole RK4 + CT step, from the active input state (dt passive)
    if (ora_set_state(c, cf, bf) != ORA_OK) return 1;
    t0 = g_ops;
    const long long r0 = g_rev;
    if (ora_step(c, Flop(1e-3)) != ORA_OK) return 1;
    const long long step_ops = g_ops - t0, step_rev = g_rev - r0;
    if (bad || hits) return 1;

    const double per_cell = (double)cell_ops / n, per_face_core = (double)face_core_ops / n;
    const double per_sweep = (double)sweep_ops / n, per_step = (double)step_ops / n;
    const double per_step_rev = (double)step_rev / n;
    // the divergence: three operations per conserved field (difference,
    // division by the spacing, accumulation)
    const double per_div = 15.0;
    const double per_face = per_sweep - per_cell - per_div;
    printf("{\"variant\": %d, \"cell\": %.4f, \"face_core\": %.4f, \"face\": %.4f, \"div\": %.4f, "
           "\"sweep\": %.4f, \"step\": %.4f, \"step_reverse\": %.4f, \"adjoint_step\": %.4f}\n",
           variant, per_cell, per_face_core, per_face, per_div, per_sweep, per_step, per_step_rev,
           per_step + per_step_rev);
    free_planes(Bc, 3);
    free_planes(D, 5);
    free_planes(S, 2);
    free(cq);
    free(cons);
    free(bface);
    free(cf);
    free(bf);
    ora_destroy(c);
    return 0;
}
