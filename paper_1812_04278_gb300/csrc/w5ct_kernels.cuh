// w5ct_kernels.cuh -- CUDA kernels of one RK4 + CT step (sm_103a).
//
// Data layout in HBM (one periodic patch, x fastest, one plane per field):
//   FP64 state   q0[5] (rho, m, E), b0[3] (forward faces)   -- q^n, b^n
//   FP64 accum.  acc[5] = sum_k w_k c_k D_k, oacc[3] = sum_k w'_k Omega_k
//   Real stage   qs[5], bs[3] (stage state), bc[3] (cell-centred B)
//   Real faces   F{x,y,z}[5] lab-ordered face fluxes, S{x,y,z}[2] CT
//                transport fluxes (x: f*_y, f*_z; y: g*_z, g*_x; z: h*_x, h*_y)
// Real is double (FP64 path) or float (FP32-bulk path).
//
// Per stage:  cellb -> sweep<x> -> sweep<y> -> sweep<z> -> update<stage>.
#pragma once
#include <cstdint>

#include "w5ct_physics.cuh"

namespace w5ct {

__device__ __forceinline__ int wrapi(int g, int n) {
    if ((unsigned)g < (unsigned)n) return g;
    const int r = g % n;
    return r < 0 ? r + n : r;
}

// ======================================================================
// characteristic sweep (Sec. 2.2 + Appendix A + Eqs. fct1-fct6)
// ======================================================================

template <typename Real>
struct SweepArgs {
    int nx, ny, nz;
    const Real *q[5];
    const Real *bc[3];
    Real *F[5];
    Real *S[2];
    Phys<Real> K;
    int *flag;
    unsigned long long *hits;
    int dw = 0;   // host-side choice: FP64 single-patch sweeps with the double-word WENO
};

// Cells whose loads a thread of a single-axis sweep kernel issues together
// when it stages a cell box (kernels that inline several sweeps stage one
// cell at a time: their larger code measured slower with the batch).
constexpr int kStageBatch = 3;

// Tile of one block: BX lanes along x (coalesced loads and stores; every
// tile has x fastest), T2 faces or pencils in the second direction, each
// thread computing FPT of them (the block is BX x T2/FPT threads).
//  x-sweep: BX faces along x  x  T2 pencils along y
//  y-sweep: BX pencils along x  x  T2 faces along y
//  z-sweep: BX pencils along x  x  T2 faces along z
// The cell box adds the 2 + 3 stencil cells along the sweep axis.
template <int AX, int T2, int BX_ = 32, int FPT_ = T2 / 8>
struct SweepTile {
    static_assert(T2 % FPT_ == 0, "faces per thread must divide the tile height");
    static constexpr int BX = BX_;
    static constexpr int FPT = FPT_;                 // faces per thread
    static constexpr int ROWS = T2 / FPT_;           // thread rows of the block
    static constexpr int NT = BX * ROWS;
    static_assert(NT % 32 == 0 && NT <= 1024, "whole warps per block");
    static constexpr int BY = (AX == 2) ? 1 : T2;
    static constexpr int BZ = (AX == 2) ? T2 : 1;
    static constexpr int CX = BX + (AX == 0 ? 5 : 0);
    static constexpr int CY = BY + (AX == 1 ? 5 : 0);
    static constexpr int CZ = BZ + (AX == 2 ? 5 : 0);
    static constexpr int NC = CX * CY * CZ;
    static constexpr int ST = (AX == 0) ? 1 : (AX == 1) ? CX : CX * CY;
};

// Patch geometry: cell counts, the patch's first cell in every plane (several
// patches share the planes back to back) and the inverse spacings.
struct PatchGeom {
    int nx, ny, nz, pad;
    long long off;
    double rdx, rdy, rdz;     // 1/dx, 1/dy, 1/dz
    double dx, dy, dz;
};

// One sweep tile (tile indices tbx, tby, tbz) of the patch described by g,
// computed by the block's NT threads, numbered (tx, ty) in [0, BX) x
// [0, ROWS).  sm: shared memory of box_quantities<Real>() * NC elements.  SB: cells whose loads
// a thread issues together when it stages the cell box.
template <int AX, typename Real, int VAR, int T2, int BX, int FPT, int SB = kStageBatch, bool DWW = false>
__device__ __forceinline__ void sweep_tile_at(const SweepArgs<Real> &a, const PatchGeom &pg, int tbx, int tby, int tbz,
                                              Real *sm, int tx, int ty) {
    using TT = SweepTile<AX, T2, BX, FPT>;
    const int nx = pg.nx, ny = pg.ny, nz = pg.nz;
    const size_t off = (size_t)pg.off;
    const int x0 = tbx * TT::BX, y0 = tby * TT::BY, z0 = tbz * TT::BZ;
    const int ox = x0 - (AX == 0 ? 2 : 0), oy = y0 - (AX == 1 ? 2 : 0), oz = z0 - (AX == 2 ? 2 : 0);
    const int tid = tx + TT::BX * ty;

    // phase 1: per-cell primitives, flux and speeds of the cell box.  A
    // thread issues the loads of up to SB of its cells before it fills any
    // of them, so that the box costs one memory latency per batch rather
    // than one per cell.
    bool bad = false, hit = false;
    constexpr int NIT = (TT::NC + TT::NT - 1) / TT::NT;
    constexpr int B = NIT < SB ? NIT : SB;
#pragma unroll
    for (int it0 = 0; it0 < NIT; it0 += B) {
        Real v[B][8];
#pragma unroll
        for (int j = 0; j < B; ++j) {
            const int c = tid + (it0 + j) * TT::NT;
            if (it0 + j < NIT && c < TT::NC) {
                const int cx = c % TT::CX;
                const int cy = (c / TT::CX) % TT::CY;
                const int cz = c / (TT::CX * TT::CY);
                const int gx = wrapi(ox + cx, nx), gy = wrapi(oy + cy, ny), gz = wrapi(oz + cz, nz);
                const size_t g = off + (size_t)gx + (size_t)nx * ((size_t)gy + (size_t)ny * (size_t)gz);
#pragma unroll
                for (int f = 0; f < 5; ++f) v[j][f] = a.q[f][g];
#pragma unroll
                for (int f = 0; f < 3; ++f) v[j][5 + f] = a.bc[f][g];
            }
        }
#pragma unroll
        for (int j = 0; j < B; ++j) {
            const int c = tid + (it0 + j) * TT::NT;
            if (it0 + j < NIT && c < TT::NC)
                cell_fill<Real, AX>(sm + c, TT::NC, v[j][0], v[j][1], v[j][2], v[j][3], v[j][4], v[j][5], v[j][6],
                                    v[j][7], a.K, bad, hit);
        }
    }
    if (bad) atomicOr(a.flag, 1);
    if (a.K.floors) {
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        if ((tid & 31) == 0 && m) atomicAdd(a.hits, (unsigned long long)__popc(m));
    }
    __syncthreads();

    // difference pass (FP64): the forward differences of F and u of every
    // cell that has a successor along the sweep axis (the last one has none
    // and no stencil needs it)
    if constexpr (box_diff<Real>()) {
        constexpr int NIT = (TT::NC + TT::NT - 1) / TT::NT;
        constexpr int LAST = (AX == 0 ? TT::CX : AX == 1 ? TT::CY : TT::CZ) - 1;
        CellDiff<Real> d[NIT];
        bool has[NIT];
#pragma unroll
        for (int it = 0; it < NIT; ++it) {
            const int c = tid + it * TT::NT;
            const int ca = AX == 0 ? c % TT::CX : AX == 1 ? (c / TT::CX) % TT::CY : c / (TT::CX * TT::CY);
            has[it] = c < TT::NC && ca < LAST;
            if (has[it]) box_diff_load<Real>(sm, TT::NC, c, TT::ST, d[it]);
        }
        __syncthreads();
#pragma unroll
        for (int it = 0; it < NIT; ++it)
            if (has[it]) box_diff_store<Real>(sm, TT::NC, tid + it * TT::NT, d[it]);
        __syncthreads();
    }

    // phase 2: FPT interfaces per thread
#pragma unroll 1
    for (int r = 0; r < TT::FPT; ++r) {
        const int t2 = ty + TT::ROWS * r;
        const int bx = tx;
        const int by = (AX == 2) ? 0 : t2;
        const int bz = (AX == 2) ? t2 : 0;
        const int gx = x0 + bx, gy = y0 + by, gz = z0 + bz;
        if (gx < nx && gy < ny && gz < nz) {
            const int c0 = bx + TT::CX * (by + TT::CY * bz);   // stencil cell i-2
            Real Ff[7], s1, s2;
            face_flux<Real, VAR, box_diff<Real>(), DWW>(sm + c0, TT::NC, TT::ST, a.K, Ff, s1, s2);
            const size_t g = off + (size_t)gx + (size_t)nx * ((size_t)gy + (size_t)ny * (size_t)gz);
            a.F[0][g] = Ff[0];
            a.F[1 + AX][g] = Ff[1];
            a.F[1 + (AX + 1) % 3][g] = Ff[2];
            a.F[1 + (AX + 2) % 3][g] = Ff[3];
            a.F[4][g] = Ff[6];
            a.S[0][g] = s1;
            a.S[1][g] = s2;
        }
    }
}

// sweep_tile_at with the axis and the tile shape (BX lanes, T2 faces or
// pencils, FPT faces per thread) known only at run time: one copy of the
// face arithmetic serves every shape, for a kernel that runs all of them
// (the fused step, whose instruction cache would not hold nine inlined
// copies).  The cell box is stored sweep-axis-major -- cell (s, p) at
// s + CS p, s along the sweep axis (CS = faces along the axis + 5), p the
// pencil -- and quantity q of a cell NQS elements after quantity q - 1: the
// stencil stride is 1 and the quantity stride the compile-time NQS (at
// least the largest box, CS x pencils), so the face arithmetic's shared
// loads take constant offsets whatever the shape.  Outputs go to the flux
// planes of `a` (the sweep's arguments for axis ax).  Same arithmetic per
// face as sweep_tile_at.
template <typename Real, int VAR, int NQS>
__device__ __forceinline__ void sweep_tile_rt(const SweepArgs<Real> &a, const PatchGeom &pg, int ax, int BX, int T2,
                                              int FPT, int tbx, int tby, int tbz, Real *sm, int tx, int ty) {
    const int nx = pg.nx, ny = pg.ny, nz = pg.nz;
    const size_t off = (size_t)pg.off;
    const int ROWS = T2 / FPT, NT = BX * ROWS;
    const int BY = ax == 2 ? 1 : T2, BZ = ax == 2 ? T2 : 1;
    const int x0 = tbx * BX, y0 = tby * BY, z0 = tbz * BZ;
    const int CS = (ax == 0 ? BX : T2) + 5;          // cells along the sweep axis
    const int NPC = ax == 0 ? T2 : BX;              // pencils
    const int NCELL = CS * NPC;
    const int tid = tx + BX * ty;

    // phase 1: per-cell quantities of the cell box, traversed x fastest
    // (coalesced loads): the x-sweep's fastest box index is s, the y- and
    // z-sweeps' is p; stepped by NT with a carry (no division per cell)
    bool bad = false, hit = false;
    {
        const int F = ax == 0 ? CS : NPC;
        int fi = tid % F, si = tid / F;
        const int df = NT % F, ds = NT / F;
        for (int c = tid; c < NCELL; c += NT) {
            const int sa = ax == 0 ? fi : si, p = ax == 0 ? si : fi;
            const int gx = wrapi(ax == 0 ? x0 - 2 + sa : x0 + p, nx);
            const int gy = wrapi(ax == 1 ? y0 - 2 + sa : (ax == 0 ? y0 + p : y0), ny);
            const int gz = wrapi(ax == 2 ? z0 - 2 + sa : z0, nz);
            const size_t g = off + (size_t)gx + (size_t)nx * ((size_t)gy + (size_t)ny * (size_t)gz);
            cell_fill_axis<Real>(sm + sa + CS * p, NQS, a.q[0][g], a.q[1][g], a.q[2][g], a.q[3][g], a.q[4][g],
                                 a.bc[0][g], a.bc[1][g], a.bc[2][g], ax, a.K, bad, hit);
            fi += df;
            const int carry = fi >= F;
            fi -= carry ? F : 0;
            si += ds + carry;
        }
    }
    if (bad) atomicOr(a.flag, 1);
    if (a.K.floors) {
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        if ((tid & 31) == 0 && m) atomicAdd(a.hits, (unsigned long long)__popc(m));
    }
    __syncthreads();

    // phase 2: FPT interfaces per thread
#pragma unroll 1
    for (int r = 0; r < FPT; ++r) {
        const int t2 = ty + ROWS * r;
        const int gx = x0 + tx, gy = y0 + (ax == 2 ? 0 : t2), gz = z0 + (ax == 2 ? t2 : 0);
        if (gx < nx && gy < ny && gz < nz) {
            // stencil cell i-2 of the face: s = the face's position along the axis
            const int c0 = ax == 0 ? tx + CS * t2 : t2 + CS * tx;
            Real Ff[7], s1, s2;
            face_flux<Real, VAR>(sm + c0, NQS, 1, a.K, Ff, s1, s2);
            const size_t g = off + (size_t)gx + (size_t)nx * ((size_t)gy + (size_t)ny * (size_t)gz);
            // lab components of the frame momentum flux (n, t1, t2)
            Real *const fn = ax == 0 ? a.F[1] : (ax == 1 ? a.F[2] : a.F[3]);
            Real *const f1 = ax == 0 ? a.F[2] : (ax == 1 ? a.F[3] : a.F[1]);
            Real *const f2 = ax == 0 ? a.F[3] : (ax == 1 ? a.F[1] : a.F[2]);
            a.F[0][g] = Ff[0];
            fn[g] = Ff[1];
            f1[g] = Ff[2];
            f2[g] = Ff[3];
            a.F[4][g] = Ff[6];
            a.S[0][g] = s1;
            a.S[1][g] = s2;
        }
    }
}

// One tile computed by the whole block, blockDim = (BX, ROWS).
template <int AX, typename Real, int VAR, int T2, int BX = 32, int FPT = T2 / 8, int SB = kStageBatch,
          bool DWW = false>
__device__ __forceinline__ void sweep_tile(const SweepArgs<Real> &a, const PatchGeom &pg, int tbx, int tby, int tbz,
                                           Real *sm) {
    sweep_tile_at<AX, Real, VAR, T2, BX, FPT, SB, DWW>(a, pg, tbx, tby, tbz, sm, (int)threadIdx.x, (int)threadIdx.y);
}

// One tile per block over a single patch: BX x T2 / FPT threads (at most
// 256), FPT faces per thread.  DW (double only): the WENO part of every
// field's flux in double-word arithmetic (weno_field).
template <int AX, typename Real, int VAR, int T2, int MINB, int FPT = T2 / 8, int BX = 32, bool DW = false>
__global__ void __launch_bounds__(SweepTile<AX, T2, BX, FPT>::NT, MINB) sweep_kernel(SweepArgs<Real> a) {
    extern __shared__ __align__(16) unsigned char w5ct_smem[];
    PatchGeom pg;
    pg.nx = a.nx;
    pg.ny = a.ny;
    pg.nz = a.nz;
    pg.off = 0;
    sweep_tile<AX, Real, VAR, T2, BX, FPT, kStageBatch, DW>(a, pg, blockIdx.x, blockIdx.y, blockIdx.z,
                                                            reinterpret_cast<Real *>(w5ct_smem));
}

// Tile tables hold int4 (patch | axis << 28, tile x, tile y, tile z).
constexpr int kItemAxisShift = 28;
constexpr int kItemPatchMask = (1 << kItemAxisShift) - 1;

// Several patches: block b computes tile tiles[b] = (patch, tbx, tby, tbz)
// of shape SweepTile<AX, T2, BX, FPT>.
template <int AX, typename Real, int VAR, int T2, int MINB, int BX, int FPT>
__global__ void __launch_bounds__(SweepTile<AX, T2, BX, FPT>::NT, MINB)
    sweep_batched_kernel(SweepArgs<Real> a, const PatchGeom *__restrict__ pgs, const int4 *__restrict__ tiles) {
    extern __shared__ __align__(16) unsigned char w5ct_smem[];
    const int4 t = tiles[blockIdx.x];
    const PatchGeom pg = pgs[t.x & kItemPatchMask];
    sweep_tile<AX, Real, VAR, T2, BX, FPT>(a, pg, t.y, t.z, t.w, reinterpret_cast<Real *>(w5ct_smem));
}

// ======================================================================
// cell-centred field: fourth-order interpolation of the faces (Sec. 2.3)
// ======================================================================

template <typename Real>
__device__ __forceinline__ void cellb_cell(int nx, int ny, int nz, size_t off, int i, int j, int k,
                                           const Real *__restrict__ bx, const Real *__restrict__ by,
                                           const Real *__restrict__ bz, Real *__restrict__ Bx, Real *__restrict__ By,
                                           Real *__restrict__ Bz) {
    // the cell and its periodic neighbours as offsets from it (one 64-bit
    // index, small integer offsets)
    const long long sy = nx, sz = (long long)nx * ny;
    const long long p = (long long)off + i + sy * j + sz * k;
    const long long xm2 = wrapi(i - 2, nx) - i, xm1 = wrapi(i - 1, nx) - i, xp1 = wrapi(i + 1, nx) - i;
    const long long ym2 = (wrapi(j - 2, ny) - j) * sy, ym1 = (wrapi(j - 1, ny) - j) * sy, yp1 = (wrapi(j + 1, ny) - j) * sy;
    const long long zm2 = (wrapi(k - 2, nz) - k) * sz, zm1 = (wrapi(k - 1, nz) - k) * sz, zp1 = (wrapi(k + 1, nz) - k) * sz;
    const Real s = Real(1.0 / 16.0);
    Bx[p] = (Real(9) * (bx[p + xm1] + bx[p]) - (bx[p + xm2] + bx[p + xp1])) * s;
    By[p] = (Real(9) * (by[p + ym1] + by[p]) - (by[p + ym2] + by[p + yp1])) * s;
    Bz[p] = (Real(9) * (bz[p + zm1] + bz[p]) - (bz[p + zm2] + bz[p + zp1])) * s;
}

// The cell field of one patch: a block of 32 x 8 (x, y) columns marches
// along z over `chunk` planes, keeping the z-stencil's four b_z values in
// registers (one new b_z load per cell; same arithmetic as cellb_cell).
// The chunk is 16 planes, halved while the grid would have fewer than
// kCellbMinBlocks blocks (small patches keep one block per 32 x 8 x 1 cells).
constexpr int kCellbChunk = 16, kCellbMinBlocks = 1024;

inline int cellb_chunk(int nx, int ny, int nz) {
    const long long cols = (long long)((nx + 31) / 32) * ((ny + 7) / 8);
    int chunk = kCellbChunk;
    while (chunk > 1 && cols * ((nz + chunk - 1) / chunk) < kCellbMinBlocks) chunk /= 2;
    return chunk;
}

inline dim3 cellb_grid(int nx, int ny, int nz) {
    const int chunk = cellb_chunk(nx, ny, nz);
    return dim3((nx + 31) / 32, (ny + 7) / 8, (nz + chunk - 1) / chunk);
}

template <typename Real>
__global__ void __launch_bounds__(256) cellb_kernel(int nx, int ny, int nz, int chunk, const Real *__restrict__ bx,
                                                    const Real *__restrict__ by, const Real *__restrict__ bz,
                                                    Real *__restrict__ Bx, Real *__restrict__ By, Real *__restrict__ Bz) {
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y;
    const int k0 = blockIdx.z * chunk, k1 = min(k0 + chunk, nz);
    if (i >= nx || j >= ny) return;
    const long long sy = nx, sz = (long long)nx * ny;
    const long long xm2 = wrapi(i - 2, nx) - i, xm1 = wrapi(i - 1, nx) - i, xp1 = wrapi(i + 1, nx) - i;
    const long long ym2 = (wrapi(j - 2, ny) - j) * sy, ym1 = (wrapi(j - 1, ny) - j) * sy, yp1 = (wrapi(j + 1, ny) - j) * sy;
    const long long col = i + sy * j;
    const Real s = Real(1.0 / 16.0);
    Real z0 = bz[col + sz * wrapi(k0 - 2, nz)], z1 = bz[col + sz * wrapi(k0 - 1, nz)], z2 = bz[col + sz * k0];
#pragma unroll 4
    for (int k = k0; k < k1; ++k) {
        const long long p = col + sz * k;
        const Real z3 = bz[col + sz * (k + 1 < nz ? k + 1 : 0)];
        Bx[p] = (Real(9) * (bx[p + xm1] + bx[p]) - (bx[p + xm2] + bx[p + xp1])) * s;
        By[p] = (Real(9) * (by[p + ym1] + by[p]) - (by[p + ym2] + by[p + yp1])) * s;
        Bz[p] = (Real(9) * (z1 + z2) - (z0 + z3)) * s;
        z0 = z1;
        z1 = z2;
        z2 = z3;
    }
}

// Cell blocks of the batched cell-wise kernels: block b of 256 threads takes
// the cells cells[b].y .. cells[b].y + 255 of patch cells[b].x, counted in
// storage order (x fastest) and clipped to the patch, so that every block
// but the last of a patch is full whatever the patch's sizes.
constexpr int kCellBlock = 256;

struct CellIdx {
    int i, j, k;
    bool ok;
};

__device__ __forceinline__ CellIdx cell_of_block(const int4 &t, const PatchGeom &pg) {
    const int idx = t.y + (int)threadIdx.x;
    CellIdx c;
    c.ok = idx < pg.nx * pg.ny * pg.nz;
    const int row = idx / pg.nx;
    c.i = idx - row * pg.nx;
    c.k = row / pg.ny;
    c.j = row - c.k * pg.ny;
    return c;
}

template <typename Real>
__global__ void __launch_bounds__(kCellBlock) cellb_batched_kernel(const PatchGeom *__restrict__ pgs,
                                                                   const int4 *__restrict__ cells,
                                                                   const Real *__restrict__ bx,
                                                                   const Real *__restrict__ by,
                                                                   const Real *__restrict__ bz, Real *__restrict__ Bx,
                                                                   Real *__restrict__ By, Real *__restrict__ Bz) {
    const int4 t = cells[blockIdx.x];
    const PatchGeom pg = pgs[t.x];
    const CellIdx c = cell_of_block(t, pg);
    if (!c.ok) return;
    cellb_cell<Real>(pg.nx, pg.ny, pg.nz, (size_t)pg.off, c.i, c.j, c.k, bx, by, bz, Bx, By, Bz);
}

// ======================================================================
// stage update: flux divergence (Eq. num), RK4 stage (Sec. 2.1), corner
// EMFs (Eqs. ox1-ox3), face-field update (Sec. 2.3) and the final CT
// update from the accumulated EMFs (Sec. 3.1.3)
// ======================================================================

template <typename Real>
struct UpdateArgs {
    int nx, ny, nz;
    Real rdx, rdy, rdz;          // 1/dx etc. (stage arithmetic)
    double drdx, drdy, drdz;     // 1/dx etc. (final FP64 curl)
    const Real *Fx[5], *Fy[5], *Fz[5];
    const Real *Sx[2], *Sy[2], *Sz[2];
    double *q0[5], *acc[5], *b0[3], *oacc[3];
    Real *qs[5], *bs[3];
    // q^n, b^n in the arithmetic type: the double arrays themselves when
    // Real = double, a float copy written at the last stage when Real = float
    Real *q0r[5], *b0r[3];
    const double *dt;
};

// stage factors c_k of Sec. 2.1 (1/2, 1/2, 1, 1/6) and the products w_k c_k
// of the q_save weights (1/3, 2/3, 1/3, 1) with them, (1, 2, 2, 1)/6, which
// are also the weights of the accumulated EMFs
template <int S>
struct StageW {
    static constexpr double c = S == 0 ? 0.5 : S == 1 ? 0.5 : S == 2 ? 1.0 : 1.0 / 6.0;
    static constexpr double wc = (S == 0 || S == 3) ? 1.0 / 6.0 : 1.0 / 3.0;
};

#ifndef W5CT_UPD_MINB
#define W5CT_UPD_MINB 1
#endif
// Minimum resident blocks per SM of the single-patch stage update.  The float
// form streams float fluxes and double accumulators (HBM-bound): 4 blocks/SM
// (64 registers) hide more memory latency than 2 (at 96-115 registers), 2.2%
// on the 256^3 FP32-bulk step.  The double form is FP64-pipe bound: 1.
#ifndef W5CT_F32_UPD_MINB
#define W5CT_F32_UPD_MINB 4
#endif
template <typename Real>
struct UpdTuning {
    static constexpr int MINB = sizeof(Real) == 4 ? W5CT_F32_UPD_MINB : W5CT_UPD_MINB;
};

// geometry of the patch an update thread works on
template <typename Real>
struct UpdGeom {
    int nx, ny, nz;
    size_t off;                  // first cell of the patch in every plane
    Real rdx, rdy, rdz;          // 1/dx etc. (stage arithmetic)
    double drdx, drdy, drdz;     // 1/dx etc. (final FP64 curl)
};

// float <-> double conversions done on the integer pipes for finite normal
// values, from the IEEE 754 binary32 / binary64 layouts (exponent bias 127 /
// 1023, 23 / 52 fraction bits); double -> float rounds to nearest, ties to
// even, so both equal the hardware conversions bit for bit.  Zeros,
// subnormals, infinities and NaNs take the hardware conversion.  A
// conversion that involves double issues to the FP64 pipe, which the
// FP32-bulk stage update keeps busy with its accumulations.
// The hardware conversions of the rare cases sit in functions that are not
// inlined, so that the compiler branches around them instead of issuing
// them, predicated off, on the FP64 pipe for every value.
static __device__ __noinline__ double f2d_special(float x) { return (double)x; }
static __device__ __noinline__ float d2f_special(double x) { return (float)x; }

__device__ __forceinline__ double f2d_exact(float x) {
    const unsigned u = __float_as_uint(x);
    const unsigned e = (u >> 23) & 0xffu;
    if (e == 0u || e == 0xffu) return f2d_special(x);
    const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3);
    return __hiloint2double((int)hi, (int)(u << 29));
}

__device__ __forceinline__ float d2f_rn(double x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const int fe = (int)((u >> 52) & 0x7ffu) - 896;          // binary32 exponent field
    if (fe < 1 || fe > 254) return d2f_special(x);
    const unsigned long long m = u & 0xfffffffffffffULL;
    const unsigned mant = (unsigned)(m >> 29);
    const unsigned long long rem = m & 0x1fffffffULL, half = 1ULL << 28;
    unsigned r = ((unsigned)(u >> 32) & 0x80000000u) | ((unsigned)fe << 23) | mant;
    if (rem > half || (rem == half && (mant & 1u))) ++r;     // a carry moves into the exponent (or to inf)
    return __uint_as_float(r);
}

template <typename Real>
__device__ __forceinline__ double to_double(Real x) {
    if constexpr (std::is_same<Real, float>::value)
        return f2d_exact(x);
    else
        return (double)x;
}

template <typename Real>
__device__ __forceinline__ Real from_double(double x) {
    if constexpr (std::is_same<Real, float>::value)
        return d2f_rn(x);
    else
        return (Real)x;
}

// One cell's update at RK stage STAGE (0..3, a run-time value here);
// update_cell<Real, STAGE> below is the same with the stage fixed at compile
// time.
template <typename Real>
__device__ __forceinline__ void update_cell_rt(const UpdateArgs<Real> &a, const UpdGeom<Real> &ug, int i, int j, int k,
                                               double dt, int STAGE) {
    const int nx = ug.nx, ny = ug.ny, nz = ug.nz;
    const int im = i > 0 ? i - 1 : nx - 1, ip = i + 1 < nx ? i + 1 : 0;
    const int jm = j > 0 ? j - 1 : ny - 1, jp = j + 1 < ny ? j + 1 : 0;
    const int km = k > 0 ? k - 1 : nz - 1, kp = k + 1 < nz ? k + 1 : 0;
    // the cell and its periodic neighbours as offsets from it (one 64-bit
    // index, offsets per axis that add independently)
    const long long sy = nx, sz = (long long)nx * ny;
    const long long p = (long long)ug.off + i + sy * j + sz * k;
    const long long xm = im - i, xp = ip - i, ym = (jm - j) * sy, yp = (jp - j) * sy, zm = (km - k) * sz,
                    zp = (kp - k) * sz;
    const double c = STAGE == 0 ? StageW<0>::c : STAGE == 1 ? StageW<1>::c : STAGE == 2 ? StageW<2>::c : StageW<3>::c;
    const double wc = STAGE == 0 ? StageW<0>::wc : STAGE == 1 ? StageW<1>::wc : STAGE == 2 ? StageW<2>::wc
                                                                                          : StageW<3>::wc;

    // Every load of this thread is issued before its first store, so that
    // they can all be in flight together (the compiler cannot move a load
    // above a store to a buffer that might alias it).

    // ---- flux divergence (Eq. num) of the five conserved fields
    Real D[5];
    {
        const long long pxm = p + xm, pym = p + ym, pzm = p + zm;
#pragma unroll
        for (int f = 0; f < 5; ++f)
            D[f] = (a.Fx[f][pxm] - a.Fx[f][p]) * ug.rdx + (a.Fy[f][pym] - a.Fy[f][p]) * ug.rdy +
                   (a.Fz[f][pzm] - a.Fz[f][p]) * ug.rdz;
    }

    // ---- corner EMFs (Eqs. ox1-ox3) from the transport fluxes
    const Real *fy = a.Sx[0], *fz = a.Sx[1], *gz = a.Sy[0], *gx = a.Sy[1], *hx = a.Sz[0], *hy = a.Sz[1];
    const Real h = Real(0.5);
    // Omega_x at the edge of cell q: g*_x averaged over x (q, q + dx), f*_y
    // over y (q, q + dy)
    auto Ox = [&](long long q, long long dx, long long dy) -> Real {
        return h * (gx[q] + gx[q + dx]) - h * (fy[q] + fy[q + dy]);
    };
    // Omega_y: h*_y averaged over y, g*_z over z
    auto Oy = [&](long long q, long long dy, long long dz) -> Real {
        return h * (hy[q] + hy[q + dy]) - h * (gz[q] + gz[q + dz]);
    };
    // Omega_z: f*_z averaged over z, h*_x over x
    auto Oz = [&](long long q, long long dz, long long dx) -> Real {
        return h * (fz[q] + fz[q + dz]) - h * (hx[q] + hx[q + dx]);
    };
    const Real ox_c = Ox(p, xp, yp);                // Omega_x(i, j, k)
    const Real ox_jm = Ox(p + ym, xp, -ym);         // Omega_x(i, j-1, k)
    const Real ox_im = Ox(p + xm, -xm, yp);         // Omega_x(i-1, j, k)
    const Real oy_c = Oy(p, yp, zp);                // Omega_y(i, j, k)
    const Real oy_km = Oy(p + zm, yp, -zm);         // Omega_y(i, j, k-1)
    const Real oy_jm = Oy(p + ym, -ym, zp);         // Omega_y(i, j-1, k)
    const Real oz_c = Oz(p, zp, xp);                // Omega_z(i, j, k)
    const Real oz_km = Oz(p + zm, -zm, xp);         // Omega_z(i, j, k-1)
    const Real oz_im = Oz(p + xm, zp, -xm);         // Omega_z(i-1, j, k)

    // ---- accumulators of this cell
    double accv[5];
#pragma unroll
    for (int f = 0; f < 5; ++f) accv[f] = STAGE == 0 ? 0.0 : a.acc[f][p];

    if (STAGE < 3) {
        // The stage state is of the arithmetic type, so it is formed in that
        // type from q^n, b^n (identical to the double expression when Real is
        // double); the accumulators stay in double.
        Real q0v[5], b0v[3];
        double oav[3];
#pragma unroll
        for (int f = 0; f < 5; ++f) q0v[f] = a.q0r[f][p];
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            b0v[f] = a.b0r[f][p];
            oav[f] = STAGE == 0 ? 0.0 : a.oacc[f][p];
        }
        // RK stage (Sec. 2.1) and face equations of Sec. 2.3 with this stage's EMFs
        const Real dbx = -(ox_c - ox_jm) * ug.rdy + (oz_c - oz_km) * ug.rdz;
        const Real dby = -(oy_c - oy_km) * ug.rdz + (ox_c - ox_im) * ug.rdx;
        const Real dbz = -(oz_c - oz_im) * ug.rdx + (oy_c - oy_jm) * ug.rdy;
        const Real cdt = from_double<Real>(c * dt);
#pragma unroll
        for (int f = 0; f < 5; ++f) {
            a.qs[f][p] = q0v[f] + cdt * D[f];
            a.acc[f][p] = accv[f] + wc * to_double(D[f]);
        }
        a.bs[0][p] = b0v[0] + cdt * dbx;
        a.bs[1][p] = b0v[1] + cdt * dby;
        a.bs[2][p] = b0v[2] + cdt * dbz;
        a.oacc[0][p] = oav[0] + wc * to_double(ox_c);
        a.oacc[1][p] = oav[1] + wc * to_double(oy_c);
        a.oacc[2][p] = oav[2] + wc * to_double(oz_c);
    } else {
        double q0v[5], b0v[3];
#pragma unroll
        for (int f = 0; f < 5; ++f) q0v[f] = a.q0[f][p];
#pragma unroll
        for (int f = 0; f < 3; ++f) b0v[f] = a.b0[f][p];
        // accumulated EMFs sum_k w'_k Omega_k, in double, at the nine edges
        const double *Ax = a.oacc[0], *Ay = a.oacc[1], *Az = a.oacc[2];
        const double ax_c = Ax[p] + wc * to_double(ox_c);
        const double ax_jm = Ax[p + ym] + wc * to_double(ox_jm);
        const double ax_im = Ax[p + xm] + wc * to_double(ox_im);
        const double ay_c = Ay[p] + wc * to_double(oy_c);
        const double ay_km = Ay[p + zm] + wc * to_double(oy_km);
        const double ay_jm = Ay[p + ym] + wc * to_double(oy_jm);
        const double az_c = Az[p] + wc * to_double(oz_c);
        const double az_km = Az[p + zm] + wc * to_double(oz_km);
        const double az_im = Az[p + xm] + wc * to_double(oz_im);
        const double dbx = -(ax_c - ax_jm) * ug.drdy + (az_c - az_km) * ug.drdz;
        const double dby = -(ay_c - ay_km) * ug.drdz + (ax_c - ax_im) * ug.drdx;
        const double dbz = -(az_c - az_im) * ug.drdx + (ay_c - ay_jm) * ug.drdy;
        // last stage: q^{n+1} = q0 + dt sum_k w_k c_k D_k and the final CT update
        constexpr bool kCopy = !std::is_same<Real, double>::value;   // float copy of q^{n+1}, b^{n+1}
#pragma unroll
        for (int f = 0; f < 5; ++f) {
            const double qn = q0v[f] + dt * (accv[f] + wc * to_double(D[f]));
            const Real qr = from_double<Real>(qn);
            a.q0[f][p] = qn;
            a.qs[f][p] = qr;
            if (kCopy) a.q0r[f][p] = qr;
        }
        const double bn[3] = {b0v[0] + dt * dbx, b0v[1] + dt * dby, b0v[2] + dt * dbz};
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            const Real br = from_double<Real>(bn[f]);
            a.b0[f][p] = bn[f];
            a.bs[f][p] = br;
            if (kCopy) a.b0r[f][p] = br;
        }
    }
}

template <typename Real, int STAGE>
__device__ __forceinline__ void update_cell(const UpdateArgs<Real> &a, const UpdGeom<Real> &ug, int i, int j, int k,
                                            double dt) {
    update_cell_rt<Real>(a, ug, i, j, k, dt, STAGE);
}

template <typename Real, int STAGE>
__global__ void __launch_bounds__(256, UpdTuning<Real>::MINB) update_kernel(UpdateArgs<Real> a) {
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
    if (i >= a.nx || j >= a.ny) return;
    const UpdGeom<Real> ug = {a.nx, a.ny, a.nz, 0, a.rdx, a.rdy, a.rdz, a.drdx, a.drdy, a.drdz};
    update_cell<Real, STAGE>(a, ug, i, j, k, *a.dt);
}

// Several patches: block b updates the cells of cell block cells[b] (see
// cell_of_block) with that patch's dt, dts[patch].
template <typename Real, int STAGE>
__global__ void __launch_bounds__(kCellBlock, W5CT_UPD_MINB) update_batched_kernel(UpdateArgs<Real> a,
                                                                                   const PatchGeom *__restrict__ pgs,
                                                                                   const int4 *__restrict__ cells,
                                                                                   const double *__restrict__ dts) {
    const int4 t = cells[blockIdx.x];
    const PatchGeom pg = pgs[t.x];
    const CellIdx c = cell_of_block(t, pg);
    if (!c.ok) return;
    const UpdGeom<Real> ug = {pg.nx, pg.ny, pg.nz, (size_t)pg.off, (Real)pg.rdx, (Real)pg.rdy, (Real)pg.rdz,
                              pg.rdx, pg.rdy, pg.rdz};
    update_cell<Real, STAGE>(a, ug, c.i, c.j, c.k, dts[t.x]);
}

// ======================================================================
// reductions
// ======================================================================

constexpr int kRedThreads = 256;

template <typename T, int N>
__device__ __forceinline__ void block_reduce(T (&v)[N], bool is_max[N], T *red /* N*32 */) {
    // warp level
#pragma unroll
    for (int q = 0; q < N; ++q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const T other = __shfl_xor_sync(0xffffffffu, v[q], o);
            v[q] = is_max[q] ? (other > v[q] ? other : v[q]) : v[q] + other;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < N; ++q) red[q * 32 + warp] = v[q];
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int q = 0; q < N; ++q) {
            T x = lane < nw ? red[q * 32 + lane] : (is_max[q] ? T(0) : T(0));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const T other = __shfl_xor_sync(0xffffffffu, x, o);
                x = is_max[q] ? (other > x ? other : x) : x + other;
            }
            v[q] = x;
        }
    }
}

// |v_d| + c_f^d of one cell for d = x, y, z folded into v (Eq. cfl)
template <typename Real>
__device__ __forceinline__ void cell_speeds(Real r, Real m0, Real m1, Real m2, Real E, Real bx, Real by, Real bz,
                                            const Phys<Real> &K, double (&v)[3], bool &bad) {
    if (K.floors && r < K.rho_min) r = K.rho_min;
    const Real ir = M<Real>::rcp_(r);
    const Real vx = m0 * ir, vy = m1 * ir, vz = m2 * ir;
    Real P = K.gm1 * (E - Real(0.5) * r * (vx * vx + vy * vy + vz * vz) - Real(0.5) * (bx * bx + by * by + bz * bz));
    if (K.floors && P < K.p_min) P = K.p_min;
    if (!(r > Real(0)) || !M<Real>::finite_pos(P)) bad = true;
    v[0] = fmax(v[0], (double)signal_speed<Real>(r, vx, P, bx, by, bz, K));
    v[1] = fmax(v[1], (double)signal_speed<Real>(r, vy, P, by, bz, bx, K));
    v[2] = fmax(v[2], (double)signal_speed<Real>(r, vz, P, bz, bx, by, K));
}

// |v_d| + c_f^d maxima of the stage state (Eq. cfl)
template <typename Real>
__global__ void __launch_bounds__(kRedThreads) speed_kernel(long long n, int nx, int ny, const Real *q0, const Real *q1,
                                                            const Real *q2, const Real *q3, const Real *q4,
                                                            const Real *B0, const Real *B1, const Real *B2,
                                                            Phys<Real> K, unsigned long long *smax, int *flag) {
    __shared__ double red[3 * 32];
    double v[3] = {0.0, 0.0, 0.0};
    bool bad = false;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x)
        cell_speeds<Real>(q0[p], q1[p], q2[p], q3[p], q4[p], B0[p], B1[p], B2[p], K, v, bad);
    if (bad) atomicOr(flag, 1);
    bool ismax[3] = {true, true, true};
    block_reduce<double, 3>(v, ismax, red);
    if (threadIdx.x == 0) {
        // non-negative doubles order like their bit patterns
        atomicMax(&smax[0], (unsigned long long)__double_as_longlong(v[0]));
        atomicMax(&smax[1], (unsigned long long)__double_as_longlong(v[1]));
        atomicMax(&smax[2], (unsigned long long)__double_as_longlong(v[2]));
    }
}

// Several patches: block b covers the cells of cell block cells[b] (see
// cell_of_block); the maxima of patch p go to smax[3 p .. 3 p + 2] (zeroed
// before).
template <typename Real>
__global__ void __launch_bounds__(kCellBlock) speed_batched_kernel(const PatchGeom *__restrict__ pgs,
                                                                   const int4 *__restrict__ cells, const Real *q0,
                                                                   const Real *q1, const Real *q2, const Real *q3,
                                                                   const Real *q4, const Real *B0, const Real *B1,
                                                                   const Real *B2, Phys<Real> K,
                                                                   unsigned long long *smax, int *flag) {
    const int4 t = cells[blockIdx.x];
    const PatchGeom pg = pgs[t.x];
    const int tid = threadIdx.x;
    double v[3] = {0.0, 0.0, 0.0};
    bool bad = false;
    if (t.y + tid < pg.nx * pg.ny * pg.nz) {
        // storage order: the block's cells are consecutive in the patch
        const size_t p = (size_t)pg.off + (size_t)t.y + (size_t)tid;
        cell_speeds<Real>(q0[p], q1[p], q2[p], q3[p], q4[p], B0[p], B1[p], B2[p], K, v, bad);
    }
    if (bad) atomicOr(flag, 1);
    // block maxima over the 8 warps of the 256-thread block
    __shared__ double red2[3 * 32];
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] = fmax(v[q], __shfl_xor_sync(0xffffffffu, v[q], o));
    if ((tid & 31) == 0)
        for (int q = 0; q < 3; ++q) red2[q * 32 + (tid >> 5)] = v[q];
    __syncthreads();
    if (tid < 32) {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            double x = tid < 8 ? red2[q * 32 + tid] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
            if (tid == 0) atomicMax(&smax[3 * t.x + q], (unsigned long long)__double_as_longlong(x));
        }
    }
}

// dt of every patch, as dt_kernel: dts[p] = CFL / sum_d (S_d / dx_d)
static __global__ void dt_batched_kernel(const PatchGeom *__restrict__ pgs, int npatch,
                                         const unsigned long long *smax, double cfl, double *dts, double *dts_copy) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npatch) return;
    const double s0 = __longlong_as_double((long long)smax[3 * p + 0]);
    const double s1 = __longlong_as_double((long long)smax[3 * p + 1]);
    const double s2 = __longlong_as_double((long long)smax[3 * p + 2]);
    const PatchGeom pg = pgs[p];
    const double sum = __dadd_rn(__dadd_rn(__ddiv_rn(s0, pg.dx), __ddiv_rn(s1, pg.dy)), __ddiv_rn(s2, pg.dz));
    const double v = __ddiv_rn(cfl, sum);
    dts[p] = v;
    if (dts_copy) dts_copy[p] = v;
}

static __global__ void fill_kernel(double *dst, int n, double v) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) dst[p] = v;
}

// dt = CFL / sum_d (S_d / dx_d), with the same rounded operations as the
// host-side w5ct_cfl_dt (no contraction), so both give the same dt
static __global__ void dt_kernel(const unsigned long long *smax, double cfl, double dx, double dy, double dz,
                                 double *dt, double *dt_copy) {
    const double s0 = __longlong_as_double((long long)smax[0]);
    const double s1 = __longlong_as_double((long long)smax[1]);
    const double s2 = __longlong_as_double((long long)smax[2]);
    const double sum = __dadd_rn(__dadd_rn(__ddiv_rn(s0, dx), __ddiv_rn(s1, dy)), __ddiv_rn(s2, dz));
    const double v = __ddiv_rn(cfl, sum);
    *dt = v;
    if (dt_copy) *dt_copy = v;
}

static __global__ void set_scalar_kernel(double *dst, double v) { *dst = v; }

// discrete div b: per-block max |div| and sum div^2
static __global__ void __launch_bounds__(kRedThreads) divb_partial_kernel(int nx, int ny, int nz, const double *bx, const double *by,
                                                                   const double *bz, double rdx, double rdy, double rdz,
                                                                   double *part) {
    __shared__ double red[2 * 32];
    const long long n = (long long)nx * ny * nz;
    double v[2] = {0.0, 0.0};
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(p % nx);
        const long long r = p / nx;
        const int j = (int)(r % ny), k = (int)(r / ny);
        const long long pxm = p - i + (i > 0 ? i - 1 : nx - 1);
        const long long pym = p + (long long)nx * ((j > 0 ? j - 1 : ny - 1) - j);
        const long long pzm = p + (long long)nx * ny * ((k > 0 ? k - 1 : nz - 1) - k);
        const double d = (bx[p] - bx[pxm]) * rdx + (by[p] - by[pym]) * rdy + (bz[p] - bz[pzm]) * rdz;
        v[0] = fmax(v[0], fabs(d));
        v[1] += d * d;
    }
    bool ismax[2] = {true, false};
    block_reduce<double, 2>(v, ismax, red);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x + 0] = v[0];
        part[2 * blockIdx.x + 1] = v[1];
    }
}

// per-block sums of up to 8 planes
static __global__ void __launch_bounds__(kRedThreads) sums_partial_kernel(long long n, int nplanes, const double *const *planes,
                                                                   double *part) {
    __shared__ double red[8 * 32];
    double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int f = 0; f < 8; ++f)
            if (f < nplanes) v[f] += planes[f][p];
    }
    bool ismax[8] = {false, false, false, false, false, false, false, false};
    block_reduce<double, 8>(v, ismax, red);
    if (threadIdx.x == 0)
        for (int f = 0; f < nplanes; ++f) part[8 * blockIdx.x + f] = v[f];
}

// one block: combine nblk partial records of `stride` values in a fixed order;
// value q is a max if (maxmask >> q) & 1, else a sum.
static __global__ void __launch_bounds__(kRedThreads) finalize_kernel(const double *part, int nblk, int stride, int nval,
                                                               unsigned maxmask, double *out) {
    __shared__ double red[8 * 32];
    double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    bool ismax[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) ismax[q] = (maxmask >> q) & 1u;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (q < nval) {
                const double x = part[(size_t)b * stride + q];
                v[q] = ismax[q] ? fmax(v[q], x) : v[q] + x;
            }
        }
    }
    block_reduce<double, 8>(v, ismax, red);
    if (threadIdx.x == 0)
        for (int q = 0; q < nval; ++q) out[q] = v[q];
}

// double -> Real copy of a plane
template <typename Real>
__global__ void __launch_bounds__(256) to_real_kernel(long long n, const double *src, Real *dst) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x)
        dst[p] = (Real)src[p];
}

}  // namespace w5ct
