// w5ct_adjoint.cuh -- adjoint (vector-Jacobian product) of one RK4 + CT step
// of fixed dt, and of the initial-condition map from primitive fields and an
// edge vector potential.
//
// One step is linear in its stage results: with D_s the flux divergence and
// Omega_s the corner EMFs of stage s (Sec. 2.1, Eq. num, Eqs. ox1-ox3),
//   q_{s+1} = q^n + c_s dt D_s,   b_{s+1} = b^n + c_s dt curl Omega_s  (s < 3),
//   q^{n+1} = q^n + dt sum_s w_s D_s,   b^{n+1} = b^n + dt curl sum_s w_s Omega_s,
// c = (1/2, 1/2, 1), w = (1, 2, 2, 1)/6.  (D_s, Omega_s) depend on the stage
// state through the sweeps (nonlinear, per face) and the divergence, EMF
// average and cell-field interpolation (linear).  The adjoint runs the
// stages backwards: the linear maps by their transposes (the kernels below),
// the sweeps by adj_sweep_kernel, which contracts the incoming flux adjoints
// with the 7 x 48 Jacobian of each face obtained with dual numbers.
#pragma once
#include <cuda_runtime.h>

#include "w5ct_dual.cuh"
#include "w5ct_kernels.cuh"

namespace w5ct {

// ---------------------------------------------------------------- sweep adjoint

template <typename B>
struct AdjSweepArgs {
    int nx, ny, nz;
    const B *q[5];          // stage state (rho, m, E), arithmetic type
    const B *bc[3];         // the stage's cell-centred field
    const double *lamF[5];  // dL/dF of this axis' face fluxes (lab order)
    const double *lamS[2];  // dL/dS of this axis' transport fluxes
    double *cb;             // 48 planes: cb[(s * 8 + v) * n + p] = d(lam . out_p)/d(input v of stencil cell s)
    Phys<B> K;
};

// Face p (the interface between cell p and its successor along AX) reads
// stencil cells p-2 .. p+3; its outputs are the five lab-order face fluxes
// and the two transport fluxes.  The face function is evaluated exactly as in
// the sweep (cell_fill + face_flux) with dual numbers of ND directions: pass
// (s, c) seeds inputs c*ND .. c*ND+ND-1 of stencil cell s (inputs rho, m_x,
// m_y, m_z, E, B_x, B_y, B_z), and the tangents of the outputs are
// contracted with lam.  48/ND passes give the whole 7 x 48 Jacobian; a small
// ND keeps the dual state in registers and the code small.
constexpr int kAdjND = 2;

template <int AX, typename B, int VAR>
__global__ void __launch_bounds__(128) adj_sweep_kernel(AdjSweepArgs<B> a) {
    constexpr int ND = kAdjND;
    using D = Dual<B, ND>;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const long long n = (long long)nx * ny * nz;
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int i = (int)(p % nx);
    const long long r = p / nx;
    const int j = (int)(r % ny), k = (int)(r / ny);
    B in[6][8];
#pragma unroll
    for (int s = 0; s < 6; ++s) {
        const int ii = AX == 0 ? wrapi(i - 2 + s, nx) : i;
        const int jj = AX == 1 ? wrapi(j - 2 + s, ny) : j;
        const int kk = AX == 2 ? wrapi(k - 2 + s, nz) : k;
        const size_t g = (size_t)ii + (size_t)nx * ((size_t)jj + (size_t)ny * (size_t)kk);
#pragma unroll
        for (int f = 0; f < 5; ++f) in[s][f] = a.q[f][g];
#pragma unroll
        for (int f = 0; f < 3; ++f) in[s][5 + f] = a.bc[f][g];
    }
    // adjoints of the outputs in the frame order of face_flux
    double lam[7];
    lam[0] = a.lamF[0][p];
    lam[1] = a.lamF[1 + AX][p];
    lam[2] = a.lamF[1 + (AX + 1) % 3][p];
    lam[3] = a.lamF[1 + (AX + 2) % 3][p];
    lam[4] = a.lamF[4][p];
    lam[5] = a.lamS[0][p];
    lam[6] = a.lamS[1][p];
    const Phys<D> K = promote<B, ND>(a.K);
    bool bad = false, hit = false;
    // the six cells' quantities without tangents; a pass seeds one cell
    D cq[NCQ * 6];
    auto fill = [&](int c, int seed0) {
        D x[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            x[v] = D((double)in[c][v]);
            if (v >= seed0 && v < seed0 + ND) x[v].d[v - seed0] = B(1);
        }
        cell_fill<D, AX>(cq + c, 6, x[0], x[1], x[2], x[3], x[4], x[5], x[6], x[7], K, bad, hit);
    };
#pragma unroll 1
    for (int c = 0; c < 6; ++c) fill(c, -ND);
#pragma unroll 1
    for (int pass = 0; pass < 6 * (8 / ND); ++pass) {
        const int s = pass / (8 / ND), v0 = (pass % (8 / ND)) * ND;
        fill(s, v0);
        D Ff[7], s1, s2;
        face_flux<D, VAR>(cq, 6, 1, K, Ff, s1, s2);
#pragma unroll
        for (int t = 0; t < ND; ++t) {
            const double g = lam[0] * (double)Ff[0].d[t] + lam[1] * (double)Ff[1].d[t] + lam[2] * (double)Ff[2].d[t] +
                             lam[3] * (double)Ff[3].d[t] + lam[4] * (double)Ff[6].d[t] + lam[5] * (double)s1.d[t] +
                             lam[6] * (double)s2.d[t];
            a.cb[(size_t)(s * 8 + v0 + t) * (size_t)n + (size_t)p] = g;
        }
        fill(s, -ND);       // back to no tangents
    }
}

// Cell p collects, in a fixed order, the contributions of the six faces whose
// stencils hold it (face p - s + 2 holds it as stencil cell s):
// lamq[v] += ... (v < 5), lambc[v - 5] += ... (v >= 5).
template <int AX>
__global__ void __launch_bounds__(256) adj_gather_kernel(int nx, int ny, int nz, const double *__restrict__ cb,
                                                         double *lq0, double *lq1, double *lq2, double *lq3,
                                                         double *lq4, double *lb0, double *lb1, double *lb2) {
    const long long n = (long long)nx * ny * nz;
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int i = (int)(p % nx);
    const long long r = p / nx;
    const int j = (int)(r % ny), k = (int)(r / ny);
    size_t face[6];
#pragma unroll
    for (int s = 0; s < 6; ++s) {
        const int ii = AX == 0 ? wrapi(i + 2 - s, nx) : i;
        const int jj = AX == 1 ? wrapi(j + 2 - s, ny) : j;
        const int kk = AX == 2 ? wrapi(k + 2 - s, nz) : k;
        face[s] = (size_t)ii + (size_t)nx * ((size_t)jj + (size_t)ny * (size_t)kk);
    }
    double *out[8] = {lq0, lq1, lq2, lq3, lq4, lb0, lb1, lb2};
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        double acc = 0.0;
#pragma unroll
        for (int s = 0; s < 6; ++s) acc += cb[(size_t)(s * 8 + v) * (size_t)n + face[s]];
        out[v][p] += acc;
    }
}

// ---------------------------------------------------------------- linear parts

struct AdjGrid {
    int nx, ny, nz;
    double rdx, rdy, rdz;
    __device__ __forceinline__ size_t at(int i, int j, int k) const {
        return (size_t)wrapi(i, nx) + (size_t)nx * ((size_t)wrapi(j, ny) + (size_t)ny * (size_t)wrapi(k, nz));
    }
};

__device__ __forceinline__ bool adj_cell(const AdjGrid &g, int &i, int &j, int &k, size_t &p) {
    const long long n = (long long)g.nx * g.ny * g.nz;
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= n) return false;
    i = (int)(q % g.nx);
    const long long r = q / g.nx;
    j = (int)(r % g.ny);
    k = (int)(r / g.ny);
    p = (size_t)q;
    return true;
}

// stage sources: lamD = cf lamq_fin + cn lamq_next, mu = cf lamb_fin + cn lamb_next
// (mu is the adjoint of the stage's face-field increment dt-scaled curl Omega)
static __global__ void __launch_bounds__(256) adj_sources_kernel(long long n, double cf, double cn,
                                                                 const double *__restrict__ lq_fin,
                                                                 const double *__restrict__ lb_fin,
                                                                 const double *__restrict__ lq_next,
                                                                 const double *__restrict__ lb_next, double *lamD,
                                                                 double *mu) {
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= n) return;
#pragma unroll
    for (int f = 0; f < 5; ++f) {
        const size_t o = (size_t)f * (size_t)n + (size_t)p;
        lamD[o] = cf * lq_fin[o] + (lq_next ? cn * lq_next[o] : 0.0);
    }
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        const size_t o = (size_t)f * (size_t)n + (size_t)p;
        mu[o] = cf * lb_fin[o] + (lb_next ? cn * lb_next[o] : 0.0);
    }
}

// lamO = curl^T mu for the face update of Sec. 2.3:
//   db_x = -(O_x - O_x(j-1)) rdy + (O_z - O_z(k-1)) rdz
//   db_y = -(O_y - O_y(k-1)) rdz + (O_x - O_x(i-1)) rdx
//   db_z = -(O_z - O_z(i-1)) rdx + (O_y - O_y(j-1)) rdy
static __global__ void __launch_bounds__(256) adj_curl_kernel(AdjGrid g, const double *__restrict__ mu, double *lamO) {
    int i, j, k;
    size_t p;
    if (!adj_cell(g, i, j, k, p)) return;
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    const double *mx = mu, *my = mu + n, *mz = mu + 2 * n;
    lamO[p] = g.rdy * (mx[g.at(i, j + 1, k)] - mx[p]) + g.rdx * (my[p] - my[g.at(i + 1, j, k)]);
    lamO[n + p] = g.rdz * (my[g.at(i, j, k + 1)] - my[p]) + g.rdy * (mz[p] - mz[g.at(i, j + 1, k)]);
    lamO[2 * n + p] = g.rdz * (mx[p] - mx[g.at(i, j, k + 1)]) + g.rdx * (mz[g.at(i + 1, j, k)] - mz[p]);
}

// Flux adjoints from lamD (transpose of Eq. num) and lamO (transpose of the
// EMF averages of Eqs. ox1-ox3):
//   O_x = (g*_x + g*_x(i+1))/2 - (f*_y + f*_y(j+1))/2
//   O_y = (h*_y + h*_y(j+1))/2 - (g*_z + g*_z(k+1))/2
//   O_z = (f*_z + f*_z(k+1))/2 - (h*_x + h*_x(i+1))/2
// lamF: 15 planes (axis-major: x fields 0..4, y, z); lamS: 6 planes
// (f*_y, f*_z, g*_z, g*_x, h*_x, h*_y, the storage order of the sweeps).
static __global__ void __launch_bounds__(256) adj_flux_kernel(AdjGrid g, const double *__restrict__ lamD,
                                                              const double *__restrict__ lamO, double *lamF,
                                                              double *lamS) {
    int i, j, k;
    size_t p;
    if (!adj_cell(g, i, j, k, p)) return;
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    const size_t px = g.at(i + 1, j, k), py = g.at(i, j + 1, k), pz = g.at(i, j, k + 1);
#pragma unroll
    for (int f = 0; f < 5; ++f) {
        const double *L = lamD + (size_t)f * n;
        const double c = L[p];
        lamF[(size_t)f * n + p] = g.rdx * (L[px] - c);
        lamF[(size_t)(5 + f) * n + p] = g.rdy * (L[py] - c);
        lamF[(size_t)(10 + f) * n + p] = g.rdz * (L[pz] - c);
    }
    const double *Ox = lamO, *Oy = lamO + n, *Oz = lamO + 2 * n;
    const double ox = Ox[p], oy = Oy[p], oz = Oz[p];
    lamS[p] = -0.5 * (ox + Ox[g.at(i, j - 1, k)]);              // f*_y
    lamS[n + p] = 0.5 * (oz + Oz[g.at(i, j, k - 1)]);           // f*_z
    lamS[2 * n + p] = -0.5 * (oy + Oy[g.at(i, j, k - 1)]);      // g*_z
    lamS[3 * n + p] = 0.5 * (ox + Ox[g.at(i - 1, j, k)]);       // g*_x
    lamS[4 * n + p] = -0.5 * (oz + Oz[g.at(i - 1, j, k)]);      // h*_x
    lamS[5 * n + p] = 0.5 * (oy + Oy[g.at(i, j - 1, k)]);       // h*_y
}

// Transpose of the fourth-order face -> centre interpolation of Sec. 2.3,
// B_d(i) = (9 (b_d(i-1) + b_d(i)) - (b_d(i-2) + b_d(i+1))) / 16 along d:
// lamb_d(m) = (9 (lamB(m+1) + lamB(m)) - (lamB(m+2) + lamB(m-1))) / 16.
// Writes lamb (3 planes) and adds lamq, lamb into the step's outputs.
static __global__ void __launch_bounds__(256) adj_interp_kernel(AdjGrid g, const double *__restrict__ lamBc,
                                                                const double *__restrict__ lamq, double *lamb,
                                                                double *out_q, double *out_b) {
    int i, j, k;
    size_t p;
    if (!adj_cell(g, i, j, k, p)) return;
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    const double s = 1.0 / 16.0;
    const double *Lx = lamBc, *Ly = lamBc + n, *Lz = lamBc + 2 * n;
    const double bx = (9.0 * (Lx[g.at(i + 1, j, k)] + Lx[p]) - (Lx[g.at(i + 2, j, k)] + Lx[g.at(i - 1, j, k)])) * s;
    const double by = (9.0 * (Ly[g.at(i, j + 1, k)] + Ly[p]) - (Ly[g.at(i, j + 2, k)] + Ly[g.at(i, j - 1, k)])) * s;
    const double bz = (9.0 * (Lz[g.at(i, j, k + 1)] + Lz[p]) - (Lz[g.at(i, j, k + 2)] + Lz[g.at(i, j, k - 1)])) * s;
    const double bb[3] = {bx, by, bz};
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        lamb[(size_t)f * n + p] = bb[f];
        out_b[(size_t)f * n + p] += bb[f];
    }
#pragma unroll
    for (int f = 0; f < 5; ++f) out_q[(size_t)f * n + p] += lamq[(size_t)f * n + p];
}

// ---------------------------------------------------------------- misfit

// L = 1/2 dV sum over cells of |q - q*|^2 + |b - b*|^2 (five conserved and
// three face fields); lam = dV (q - q*), dV (b - b*).  Per-block partial sums.
static __global__ void __launch_bounds__(kRedThreads) misfit_partial_kernel(long long n, double dV, const double *q,
                                                                            const double *b, const double *tq,
                                                                            const double *tb, double *lq, double *lb,
                                                                            double *part) {
    __shared__ double red[32];
    double v[1] = {0.0};
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int f = 0; f < 5; ++f) {
            const size_t o = (size_t)f * (size_t)n + (size_t)p;
            const double d = q[o] - tq[o];
            v[0] += d * d;
            lq[o] = dV * d;
        }
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            const size_t o = (size_t)f * (size_t)n + (size_t)p;
            const double d = b[o] - tb[o];
            v[0] += d * d;
            lb[o] = dV * d;
        }
    }
    bool ismax[1] = {false};
    block_reduce<double, 1>(v, ismax, red);
    if (threadIdx.x == 0) part[blockIdx.x] = 0.5 * dV * v[0];
}

// ---------------------------------------------------------------- initial state

// Face field b = curl A + B0 of an edge vector potential (A_x at (i, j+1/2,
// k+1/2), A_y at (i+1/2, j, k+1/2), A_z at (i+1/2, j+1/2, k) in cell units
// from the centre of cell (i, j, k)), first-order discrete curl (Sec. 4.1).
static __global__ void __launch_bounds__(256) ic_curl_kernel(AdjGrid g, const double *__restrict__ A, double B0x,
                                                             double B0y, double B0z, double *bface) {
    int i, j, k;
    size_t p;
    if (!adj_cell(g, i, j, k, p)) return;
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    const double *Ax = A, *Ay = A + n, *Az = A + 2 * n;
    bface[p] = (Az[p] - Az[g.at(i, j - 1, k)]) * g.rdy - (Ay[p] - Ay[g.at(i, j, k - 1)]) * g.rdz + B0x;
    bface[n + p] = (Ax[p] - Ax[g.at(i, j, k - 1)]) * g.rdz - (Az[p] - Az[g.at(i - 1, j, k)]) * g.rdx + B0y;
    bface[2 * n + p] = (Ay[p] - Ay[g.at(i - 1, j, k)]) * g.rdx - (Ax[p] - Ax[g.at(i, j - 1, k)]) * g.rdy + B0z;
}

// sixth-order face -> centre weights of the initial conditions (Sec. 4.14),
// faces i-5/2 .. i+5/2 = face indices i-3 .. i+2, divided by 256
__device__ __forceinline__ double ic_w6(int o) {
    return o == 0 || o == 5 ? 3.0 / 256.0 : o == 1 || o == 4 ? -25.0 / 256.0 : 150.0 / 256.0;
}

__device__ __forceinline__ void ic_cell_field(const AdjGrid &g, const double *bface, int i, int j, int k,
                                              double (&Bc)[3]) {
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    Bc[0] = Bc[1] = Bc[2] = 0.0;
#pragma unroll
    for (int o = 0; o < 6; ++o) {
        const double w = ic_w6(o);
        Bc[0] += w * bface[g.at(i - 3 + o, j, k)];
        Bc[1] += w * bface[n + g.at(i, j - 3 + o, k)];
        Bc[2] += w * bface[2 * n + g.at(i, j, k - 3 + o)];
    }
}

// conserved state (rho, rho v, E) with E from Eq. P, the cell field from the
// sixth-order interpolation of the faces
static __global__ void __launch_bounds__(256) ic_cons_kernel(AdjGrid g, double gm1, const double *__restrict__ rho,
                                                             const double *__restrict__ v, const double *__restrict__ P,
                                                             const double *__restrict__ bface, double *cons) {
    int i, j, k;
    size_t p;
    if (!adj_cell(g, i, j, k, p)) return;
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    double Bc[3];
    ic_cell_field(g, bface, i, j, k, Bc);
    const double r = rho[p], vx = v[p], vy = v[n + p], vz = v[2 * n + p];
    cons[p] = r;
    cons[n + p] = r * vx;
    cons[2 * n + p] = r * vy;
    cons[3 * n + p] = r * vz;
    cons[4 * n + p] = P[p] / gm1 + 0.5 * r * (vx * vx + vy * vy + vz * vz) + 0.5 * (Bc[0] * Bc[0] + Bc[1] * Bc[1] + Bc[2] * Bc[2]);
}

// adjoint of ic_cons_kernel in rho and v; lamBc = Bc lamE (3 planes, scratch)
static __global__ void __launch_bounds__(256) ic_cons_adjoint_kernel(AdjGrid g, const double *__restrict__ rho,
                                                                     const double *__restrict__ v,
                                                                     const double *__restrict__ bface,
                                                                     const double *__restrict__ lcons, double *lrho,
                                                                     double *lv, double *lBc) {
    int i, j, k;
    size_t p;
    if (!adj_cell(g, i, j, k, p)) return;
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    double Bc[3];
    ic_cell_field(g, bface, i, j, k, Bc);
    const double r = rho[p], vv[3] = {v[p], v[n + p], v[2 * n + p]};
    const double lE = lcons[4 * n + p];
    double lr = lcons[p] + 0.5 * lE * (vv[0] * vv[0] + vv[1] * vv[1] + vv[2] * vv[2]);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double lm = lcons[(size_t)(1 + d) * n + p];
        lr += vv[d] * lm;
        lv[(size_t)d * n + p] = r * lm + r * vv[d] * lE;
        lBc[(size_t)d * n + p] = Bc[d] * lE;
    }
    lrho[p] = lr;
}

// lamb = lam_bface + (sixth-order interpolation)^T lamBc
static __global__ void __launch_bounds__(256) ic_interp_adjoint_kernel(AdjGrid g, const double *__restrict__ lbface,
                                                                       const double *__restrict__ lBc, double *lb) {
    int i, j, k;
    size_t p;
    if (!adj_cell(g, i, j, k, p)) return;
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    double s[3] = {lbface[p], lbface[n + p], lbface[2 * n + p]};
    // face m feeds cell m + 3 - o with weight w_o
#pragma unroll
    for (int o = 0; o < 6; ++o) {
        const double w = ic_w6(o);
        s[0] += w * lBc[g.at(i + 3 - o, j, k)];
        s[1] += w * lBc[n + g.at(i, j + 3 - o, k)];
        s[2] += w * lBc[2 * n + g.at(i, j, k + 3 - o)];
    }
    lb[p] = s[0];
    lb[n + p] = s[1];
    lb[2 * n + p] = s[2];
}

// lamA = curl^T lamb (transpose of ic_curl_kernel)
static __global__ void __launch_bounds__(256) ic_curl_adjoint_kernel(AdjGrid g, const double *__restrict__ lb,
                                                                     double *lA) {
    int i, j, k;
    size_t p;
    if (!adj_cell(g, i, j, k, p)) return;
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    const double *bx = lb, *by = lb + n, *bz = lb + 2 * n;
    // b_y(i,j,k) has +A_x/dz, b_y(i,j,k+1) -A_x/dz; b_z(i,j,k) -A_x/dy, b_z(i,j+1,k) +A_x/dy
    lA[p] = (by[p] - by[g.at(i, j, k + 1)]) * g.rdz - (bz[p] - bz[g.at(i, j + 1, k)]) * g.rdy;
    // b_z: +A_y/dx at (i), -A_y/dx at (i+1); b_x: -A_y/dz at (k), +A_y/dz at (k+1)
    lA[n + p] = (bz[p] - bz[g.at(i + 1, j, k)]) * g.rdx - (bx[p] - bx[g.at(i, j, k + 1)]) * g.rdz;
    // b_x: +A_z/dy at (j), -A_z/dy at (j+1); b_y: -A_z/dx at (i), +A_z/dx at (i+1)
    lA[2 * n + p] = (bx[p] - bx[g.at(i, j + 1, k)]) * g.rdy - (by[p] - by[g.at(i + 1, j, k)]) * g.rdx;
}

// Defined in w5ct_adjoint{32,64}{js,z}.cu (one translation unit per
// arithmetic type and WENO variant, compiled in parallel).
template <typename B, int VAR>
cudaError_t launch_adj_sweep(int axis, const AdjSweepArgs<B> &a, cudaStream_t s);

template <typename B, int VAR>
cudaError_t launch_adj_sweep_impl(int axis, const AdjSweepArgs<B> &a, cudaStream_t s) {
    const long long n = (long long)a.nx * a.ny * a.nz;
    const unsigned nb = (unsigned)((n + 127) / 128);
    if (axis == 0)
        adj_sweep_kernel<0, B, VAR><<<nb, 128, 0, s>>>(a);
    else if (axis == 1)
        adj_sweep_kernel<1, B, VAR><<<nb, 128, 0, s>>>(a);
    else
        adj_sweep_kernel<2, B, VAR><<<nb, 128, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace w5ct
