// w5ct_fused.cuh -- one RK4 + CT step of every patch of a batch in a single
// persistent launch (the fused schedule of the batched path).
//
// The step is a list of work items, built on the host: per stage s and patch
// p, the blocks of kFusedCells cells of p's cell field (Sec. 2.3), at s = 0
// the blocks of p's CFL reduction (Eq. cfl) and p's dt, the sweep tiles of p
// along x, y and z (Sec. 2.2), and the blocks of p's stage update (Eq. num,
// Sec. 2.1, Eqs. ox1-ox3), ordered phase by phase within a stage (every
// patch's cell fields, then the CFL items, then the sweeps, then the
// updates).  Each block of the persistent grid takes the next item from a
// device counter and first waits until the items it depends on -- all of
// them earlier in the list and all of the same patch -- are done:
//
//   cell field (p, s > 0)  after the update (p, s - 1)
//   CFL blocks (p)         after the cell field (p, 0)
//   dt (p)                 after the CFL blocks (p)
//   sweep tiles (p, s)     after the cell field (p, s)
//   update (p, s)          after the sweep tiles (p, s) and, at s = 0, dt (p)
//
// A dependency is always dequeued before the item that waits on it, by a
// block that is running, and waits only point backwards in the list, so the
// chain of waits ends at an item that can finish: the launch completes
// without any assumption on how many blocks are resident.  A block fetches
// its next item index while it works on the current one, and skips the
// check of a dependency it has already seen complete (counters only grow
// within a step).  Every wait is
// bounded (an iteration limit with a short sleep): on expiry the block sets
// bit 2 of the context's flag and an abort word that makes every other block
// stop, and the step reports W5CT_ERR_TIMEOUT.
//
// Memory ordering: a block publishes an item with __syncthreads, a fence and
// an atomicAdd on the item's counter (a release pattern of the PTX memory
// model); a waiter reads the counter, fences (an acquire pattern) and
// releases its threads with __syncthreads, which orders their loads after
// the producer's stores (the grid-synchronisation pattern).  No load of the
// kernel goes through the non-coherent read-only path.
#pragma once
#include <cuda_runtime.h>

#include "w5ct_internal.h"

namespace w5ct {

enum FusedItem { FI_CELLB = 0, FI_SPEED = 1, FI_DT = 2, FI_SWEEP = 3, FI_UPDATE = 4 };

// cells of one cell-wise item (eight per thread of a float block, four of a
// double block): the per-item bookkeeping (queue, dependency check, fence,
// counter) is then shared by 1024 cells
constexpr int kFusedCells = 1024;

// item: x = patch, y = type | stage << 3 | axis << 5 | v << 8; for a sweep
// item z = the first of its w tiles, tile index i + nbx (j + nb1 k) among the
// patch's tiles of variant v along the axis; for a cell-wise item z = its
// first cell and w = 0
__host__ __device__ inline int fused_tag(int type, int stage, int axis, int v) {
    return type | (stage << 3) | (axis << 5) | (v << 8);
}

// Block of the fused kernel: in float 128 threads, four blocks per SM (the
// register budget of the float sweep, 128 per thread), so that the 8-lane
// tiles that suit patches 16, 24 or 48 cells wide need no sub-tiles; in
// double 256 threads, one block per SM (255 registers).
template <typename Real>
struct FusedBlock {
    static constexpr int NT = sizeof(Real) == 4 ? 128 : 256;
    static constexpr int MINB = sizeof(Real) == 4 ? 4 : 1;
};

// Sweep tiles of the fused kernel (lanes along x BX, faces or pencils T2 in
// the second direction, FPT per thread; BX x T2 / FPT = the block):
//   float   0: 32 x 8 (2 per thread)   1: 16 x 16 (2)   2: 8 x 16 (1)
//   double  0: 32 x 16 (2)
template <typename Real, int V>
struct FusedShape;
template <>
struct FusedShape<float, 0> {
    static constexpr int BX = 32, T2 = 8, FPT = 2;
};
template <>
struct FusedShape<float, 1> {
    static constexpr int BX = 16, T2 = 16, FPT = 2;
};
template <>
struct FusedShape<float, 2> {
    static constexpr int BX = 8, T2 = 16, FPT = 1;
};
template <>
struct FusedShape<double, 0> {
    static constexpr int BX = 32, T2 = 16, FPT = 2;
};

template <typename Real>
constexpr int fused_variants() {
    return sizeof(Real) == 4 ? 3 : 1;
}

// (BX, T2) of fused tile variant v (host side, for the work list)
template <typename Real>
inline void fused_tile_shape(int v, int &bx, int &t2) {
    if (sizeof(Real) == 8 || v == 0) {
        bx = 32;
        t2 = sizeof(Real) == 8 ? 16 : 8;
    } else {
        bx = v == 1 ? 16 : 8;
        t2 = 16;
    }
}

// (BX, T2, FPT) of fused tile variant v (device side)
template <typename Real>
__device__ __forceinline__ void fused_shape_rt(int v, int &bx, int &t2, int &fpt) {
    if constexpr (sizeof(Real) == 4) {
        bx = v == 0 ? FusedShape<float, 0>::BX : v == 1 ? FusedShape<float, 1>::BX : FusedShape<float, 2>::BX;
        t2 = v == 0 ? FusedShape<float, 0>::T2 : v == 1 ? FusedShape<float, 1>::T2 : FusedShape<float, 2>::T2;
        fpt = v == 0 ? FusedShape<float, 0>::FPT : v == 1 ? FusedShape<float, 1>::FPT : FusedShape<float, 2>::FPT;
    } else {
        bx = FusedShape<double, 0>::BX;
        t2 = FusedShape<double, 0>::T2;
        fpt = FusedShape<double, 0>::FPT;
    }
}

// Tile variant V of the sweep along AX: its cell box (cells along the axis x
// pencils, sweep_tile_rt's layout)
template <typename Real, int AX, int V>
struct FusedTile {
    using S = FusedShape<Real, V>;
    static_assert(S::BX * (S::T2 / S::FPT) == FusedBlock<Real>::NT, "one tile per block");
    static constexpr int cells = ((AX == 0 ? S::BX : S::T2) + 5) * (AX == 0 ? S::T2 : S::BX);
};

template <typename Real, int V>
__host__ __device__ constexpr int fused_cells_v() {
    constexpr int a = FusedTile<Real, 0, V>::cells, b = FusedTile<Real, 1, V>::cells, c = FusedTile<Real, 2, V>::cells;
    return a > b ? (a > c ? a : c) : (b > c ? b : c);
}

// the quantity stride of the fused kernel's cell box: the largest box of its
// tile variants (float 416 cells, double 672)
template <typename Real>
__host__ __device__ constexpr int fused_nqs() {
    if constexpr (sizeof(Real) == 4) {
        constexpr int a = fused_cells_v<float, 0>(), b = fused_cells_v<float, 1>(), c = fused_cells_v<float, 2>();
        return a > b ? (a > c ? a : c) : (b > c ? b : c);
    } else {
        return fused_cells_v<double, 0>();
    }
}

// Per-patch completion counters, zeroed at the start of every step:
// cellb[s][p], sweep[s][p], update[s][p], speed[p], dt[p].
struct FusedCounters {
    int *queue;      // next item
    int *abort;      // set when a wait expires
    int *done;       // 14 * npatch counters
    int npatch;
    __device__ int *cellb(int s, int p) const { return done + s * npatch + p; }
    __device__ int *sweep(int s, int p) const { return done + (4 + s) * npatch + p; }
    __device__ int *update(int s, int p) const { return done + (8 + s) * npatch + p; }
    __device__ int *speed(int p) const { return done + 12 * npatch + p; }
    __device__ int *dtc(int p) const { return done + 13 * npatch + p; }
};

template <typename Real>
struct FusedArgs {
    SweepArgs<Real> a[3];        // sweeps along x, y, z (flux outputs per axis)
    UpdateArgs<Real> u;          // stage update (u.dt unused: dts below)
    const Real *bs[3];           // stage face field -> cell field a[*].bc
    Real *bc[3];
    const PatchGeom *pgs;
    const int4 *items;
    int nitems;
    const int *ncb;              // cell-wise items per patch
    const int *ntile;            // sweep tiles (three axes) per patch
    FusedCounters ctr;
    int cfl;                     // 1: dt of each patch from its state; 0: dts given
    double cfl_number;
    double *dts;                 // per-patch dt (written when cfl, read by the updates)
    double *dts_out;             // optional copy of the dts
    unsigned long long *smax;    // 3 per patch, zeroed before the launch
    long long spin_limit;
};

// thread 0 of a block: wait until *ctr >= target; false if aborted or
// expired.  seen[0..1]: the last two counters this block saw complete.
__device__ __forceinline__ bool fused_wait(const FusedCounters &C, const int *ctr, int target, long long limit,
                                           int *flag, const int *(&seen)[2]) {
    if (ctr == seen[0] || ctr == seen[1]) return true;
    long long it = 0;
    for (;;) {
        const int v = *(volatile const int *)ctr;
        if (v >= target) {
            __threadfence();
            seen[1] = seen[0];
            seen[0] = ctr;
            return true;
        }
        if (*(volatile const int *)C.abort) return false;
        if (++it > limit) {
            atomicExch(C.abort, 1);
            atomicOr(flag, 2);
            return false;
        }
        __nanosleep(256);
    }
}

// the cell-centred field of one cell (Sec. 2.3), plain loads
template <typename Real>
__device__ __forceinline__ void fused_cellb(const PatchGeom &g, int i, int j, int k, const Real *bx, const Real *by,
                                            const Real *bz, Real *Bx, Real *By, Real *Bz) {
    const long long sy = g.nx, sz = (long long)g.nx * g.ny;
    const long long p = g.off + i + sy * j + sz * k;
    const long long xm2 = wrapi(i - 2, g.nx) - i, xm1 = wrapi(i - 1, g.nx) - i, xp1 = wrapi(i + 1, g.nx) - i;
    const long long ym2 = (wrapi(j - 2, g.ny) - j) * sy, ym1 = (wrapi(j - 1, g.ny) - j) * sy,
                    yp1 = (wrapi(j + 1, g.ny) - j) * sy;
    const long long zm2 = (wrapi(k - 2, g.nz) - k) * sz, zm1 = (wrapi(k - 1, g.nz) - k) * sz,
                    zp1 = (wrapi(k + 1, g.nz) - k) * sz;
    const Real s = Real(1.0 / 16.0);
    Bx[p] = (Real(9) * (bx[p + xm1] + bx[p]) - (bx[p + xm2] + bx[p + xp1])) * s;
    By[p] = (Real(9) * (by[p + ym1] + by[p]) - (by[p + ym2] + by[p + yp1])) * s;
    Bz[p] = (Real(9) * (bz[p + zm1] + bz[p]) - (bz[p + zm2] + bz[p + zp1])) * s;
}

template <typename Real, int VAR>
__global__ void __launch_bounds__(FusedBlock<Real>::NT, FusedBlock<Real>::MINB) fused_step_kernel(FusedArgs<Real> A) {
    constexpr int NT = FusedBlock<Real>::NT;
    extern __shared__ __align__(16) unsigned char w5ct_smem[];
    __shared__ int s_item, s_ok, s_next;
    __shared__ const int *s_seen[2];              // thread 0: counters seen complete
    __shared__ double s_red[3 * 32];
    Real *sm = reinterpret_cast<Real *>(w5ct_smem);
    const int tid = threadIdx.x + 32 * threadIdx.y;
    const FusedCounters &C = A.ctr;
    // thread 0's queue state lives in shared memory, not in registers that
    // every thread would carry through the sweep arithmetic
    if (tid == 0) {
        s_seen[0] = nullptr;
        s_seen[1] = nullptr;
        s_next = atomicAdd(C.queue, 1);
    }
    for (;;) {
        if (tid == 0) s_item = s_next;
        __syncthreads();
        const int it = s_item;
        if (it >= A.nitems) break;
        // the following item, fetched while this one runs
        if (tid == 0) s_next = atomicAdd(C.queue, 1);
        const int4 t = A.items[it];
        const int p = t.x;
        const int type = t.y & 7, stage = (t.y >> 3) & 3, axis = (t.y >> 5) & 3, v = t.y >> 8;
        const PatchGeom pg = A.pgs[p];
        // ---- wait for this item's dependencies (thread 0), then release the block
        if (tid == 0) {
            bool ok = true;
            switch (type) {
                case FI_CELLB:
                    if (stage > 0) ok = fused_wait(C, C.update(stage - 1, p), A.ncb[p], A.spin_limit, A.a[0].flag, s_seen);
                    break;
                case FI_SPEED: ok = fused_wait(C, C.cellb(0, p), A.ncb[p], A.spin_limit, A.a[0].flag, s_seen); break;
                case FI_DT: ok = fused_wait(C, C.speed(p), A.ncb[p], A.spin_limit, A.a[0].flag, s_seen); break;
                case FI_SWEEP:
                    ok = fused_wait(C, C.cellb(stage, p), A.ncb[p], A.spin_limit, A.a[0].flag, s_seen);
                    break;
                default:
                    ok = fused_wait(C, C.sweep(stage, p), A.ntile[p], A.spin_limit, A.a[0].flag, s_seen);
                    if (ok && stage == 0) ok = fused_wait(C, C.dtc(p), 1, A.spin_limit, A.a[0].flag, s_seen);
                    break;
            }
            s_ok = ok ? 1 : 0;
        }
        __syncthreads();
        if (!s_ok) break;
        // ---- the item's work
        int *done = nullptr;
        if (type == FI_SWEEP) {
            // t.w consecutive tiles from t.z (one item's bookkeeping for all);
            // one copy of the sweep code for every axis and tile shape
            int bx, t2, fpt;
            fused_shape_rt<Real>(v, bx, t2, fpt);
            const SweepArgs<Real> &a = A.a[axis];
            const int nbx = (pg.nx + bx - 1) / bx;
            const int nb1 = axis == 2 ? pg.ny : (pg.ny + t2 - 1) / t2;
#pragma unroll 1
            for (int q = 0; q < t.w; ++q) {
                if (q > 0) __syncthreads();          // the tile box in shared memory is reused
                const int L = t.z + q;
                const int r = L / nbx;
                const int i = L - r * nbx, k = r / nb1, j = r - k * nb1;
                sweep_tile_rt<Real, VAR, fused_nqs<Real>()>(a, pg, axis, bx, t2, fpt, i, j, k, sm, tid % bx, tid / bx);
            }
            done = C.sweep(stage, p);
        } else if (type == FI_DT) {
            if (tid == 0 && A.cfl) {
                const double s0 = __longlong_as_double((long long)A.smax[3 * p + 0]);
                const double s1 = __longlong_as_double((long long)A.smax[3 * p + 1]);
                const double s2 = __longlong_as_double((long long)A.smax[3 * p + 2]);
                const double sum = __dadd_rn(__dadd_rn(__ddiv_rn(s0, pg.dx), __ddiv_rn(s1, pg.dy)), __ddiv_rn(s2, pg.dz));
                const double v = __ddiv_rn(A.cfl_number, sum);
                A.dts[p] = v;
                if (A.dts_out) A.dts_out[p] = v;
            }
            done = C.dtc(p);
        } else {
            // kFusedCells consecutive cells of the patch (storage order),
            // cells t.z + tid + NT r
            const int ncell = pg.nx * pg.ny * pg.nz;
            if (type == FI_CELLB) {
#pragma unroll 1
                for (int r = 0; r < kFusedCells / NT; ++r) {
                    const int idx = t.z + tid + NT * r;
                    if (idx < ncell) {
                        const int row = idx / pg.nx;
                        const int i = idx - row * pg.nx, k = row / pg.ny, j = row - k * pg.ny;
                        fused_cellb<Real>(pg, i, j, k, A.bs[0], A.bs[1], A.bs[2], A.bc[0], A.bc[1], A.bc[2]);
                    }
                }
                done = C.cellb(stage, p);
            } else if (type == FI_SPEED) {
                if (A.cfl) {
                    double v[3] = {0.0, 0.0, 0.0};
                    bool bad = false;
#pragma unroll 1
                    for (int r = 0; r < kFusedCells / NT; ++r) {
                        const int idx = t.z + tid + NT * r;
                        if (idx < ncell) {
                            const size_t q = (size_t)pg.off + (size_t)idx;
                            const SweepArgs<Real> &a = A.a[0];
                            cell_speeds<Real>(a.q[0][q], a.q[1][q], a.q[2][q], a.q[3][q], a.q[4][q], a.bc[0][q],
                                              a.bc[1][q], a.bc[2][q], a.K, v, bad);
                        }
                    }
                    if (bad) atomicOr(A.a[0].flag, 1);
                    // maxima over the block's NT / 32 warps
#pragma unroll
                    for (int d = 0; d < 3; ++d)
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) v[d] = fmax(v[d], __shfl_xor_sync(0xffffffffu, v[d], o));
                    if ((tid & 31) == 0)
                        for (int d = 0; d < 3; ++d) s_red[d * 32 + (tid >> 5)] = v[d];
                    __syncthreads();
                    if (tid < 32) {
                        for (int d = 0; d < 3; ++d) {
                            double x = tid < NT / 32 ? s_red[d * 32 + tid] : 0.0;
#pragma unroll
                            for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
                            if (tid == 0) atomicMax(&A.smax[3 * p + d], (unsigned long long)__double_as_longlong(x));
                        }
                    }
                }
                done = C.speed(p);
            } else {
                const UpdGeom<Real> ug = {pg.nx, pg.ny, pg.nz, (size_t)pg.off, (Real)pg.rdx, (Real)pg.rdy,
                                          (Real)pg.rdz, pg.rdx, pg.rdy, pg.rdz};
                const double dt = A.dts[p];
#pragma unroll 1
                for (int r = 0; r < kFusedCells / NT; ++r) {
                    const int idx = t.z + tid + NT * r;
                    if (idx >= ncell) break;
                    const int row = idx / pg.nx;
                    const int i = idx - row * pg.nx, k = row / pg.ny, j = row - k * pg.ny;
                    update_cell_rt<Real>(A.u, ug, i, j, k, dt, stage);
                }
                done = C.update(stage, p);
            }
        }
        // ---- publish: every thread's writes, then the counter
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            atomicAdd(done, 1);
        }
    }
}

// Defined in w5ct_fused32.cu / w5ct_fused64.cu.
template <typename Real>
cudaError_t launch_fused_step(int variant, const FusedArgs<Real> &A, int blocks, cudaStream_t s);
template <typename Real>
cudaError_t fused_grid(int variant, int &blocks, size_t &smem);

// shared memory of the fused kernel: the cell box of its largest sweep tile
template <typename Real, int VAR>
size_t fused_smem() {
    return (size_t)fused_nqs<Real>() * NCQ * sizeof(Real);
}

template <typename Real, int VAR>
cudaError_t fused_grid_impl(int &blocks, size_t &smem) {
    smem = fused_smem<Real, VAR>();
    cudaError_t e = cudaFuncSetAttribute(fused_step_kernel<Real, VAR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    int dev = 0, sms = 0, per = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fused_step_kernel<Real, VAR>, FusedBlock<Real>::NT, smem);
    blocks = sms * (per > 0 ? per : 1);
    return e;
}

template <typename Real, int VAR>
cudaError_t launch_fused_impl(const FusedArgs<Real> &A, int blocks, cudaStream_t s) {
    fused_step_kernel<Real, VAR><<<blocks, dim3(32, FusedBlock<Real>::NT / 32), fused_smem<Real, VAR>(), s>>>(A);
    return cudaGetLastError();
}

}  // namespace w5ct
