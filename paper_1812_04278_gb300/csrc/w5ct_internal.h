// w5ct_internal.h -- declarations shared by the translation units of libw5ct.
#pragma once
#include <cuda_runtime.h>

#include "w5ct_kernels.cuh"

namespace w5ct {

// Record the text that w5ct_last_error(NULL) returns (calls without a context).
void set_global_error(const char *text);

// Launch the characteristic sweep along `axis` (0, 1, 2) with WENO variant
// `variant` (0 = JS, 1 = Z) over one patch, in tiles `t2` faces or pencils
// high (0: the type's default, SweepTuning; the FP64 sweep also takes the
// shorter tiles of small_tile_heights).  Defined in w5ct_sweep32.cu /
// w5ct_sweep64.cu.
template <typename Real>
cudaError_t launch_sweep(int axis, int variant, int t2, const SweepArgs<Real> &a, cudaStream_t s);

// The FP64 single-patch sweeps of the default tiles with the WENO part of
// every flux in double-word arithmetic (launch_sweep takes them when a.dw is
// set and the tile is the default one), and the shared-memory allowance of
// their kernels.  Defined in w5ct_sweep64dw.cu.
cudaError_t launch_sweep_f64dw(int axis, int variant, const SweepArgs<double> &a, cudaStream_t s);
cudaError_t prepare_sweeps_f64dw();

// Sweep tiling per arithmetic type: faces per block in the second tile
// direction (x-sweep: pencils along y; y- and z-sweeps: faces along the
// axis) and the minimum resident blocks per SM the register budget targets.
template <typename Real>
struct SweepTuning;

// Defaults measured on GB300 (FP32 at 256^3: 2 blocks/SM of 16-high tiles,
// 1.6x faster than 1 block of 8-high tiles; 3 blocks/SM or 32-high y/z tiles
// are slower.  FP64 at 256^3: FP64-pipe bound, one 256-thread block of
// 16-high tiles per SM; its cell box with the forward differences (NBQ
// planes) leaves no room for 32-high tiles, which without the differences
// were 1% faster; 384- or 512-thread blocks measured within 0.5%).
#ifndef W5CT_F32_T2X
#define W5CT_F32_T2X 16
#endif
#ifndef W5CT_F32_T2YZ
#define W5CT_F32_T2YZ 16
#endif
#ifndef W5CT_F32_MINB
#define W5CT_F32_MINB 2
#endif
#ifndef W5CT_F64_T2X
#define W5CT_F64_T2X 16
#endif
#ifndef W5CT_F64_T2YZ
#define W5CT_F64_T2YZ 16
#endif
#ifndef W5CT_F64_MINB
#define W5CT_F64_MINB 1
#endif
// FP64 y- and z-sweeps: tiles of 16 pencils x 32 faces, whose cell box (37 x
// 16 cells) stages 1.16 cells per face instead of the 1.31 of 32 x 16 (21 x
// 32 cells); the x-sweep's 32 x 16 tile already stages 37 x 16.
#ifndef W5CT_F64_BXYZ
#define W5CT_F64_BXYZ 16
#endif
#ifndef W5CT_F64_T2YZ_NARROW
#define W5CT_F64_T2YZ_NARROW 32
#endif

#ifndef W5CT_F32_FPT
#define W5CT_F32_FPT 2
#endif
template <>
struct SweepTuning<float> {
    static constexpr int T2X = W5CT_F32_T2X, T2YZ = W5CT_F32_T2YZ, MINB = W5CT_F32_MINB, FPT = W5CT_F32_FPT;
};
template <>
struct SweepTuning<double> {
    static constexpr int T2X = W5CT_F64_T2X, T2YZ = W5CT_F64_T2YZ, MINB = W5CT_F64_MINB, FPT = W5CT_F64_T2X / 8,
                         BXYZ = W5CT_F64_BXYZ;
};

template <int AX, typename Real>
struct SweepCfg {
    static constexpr bool kNarrow = sizeof(Real) == 8 && AX != 0;   // FP64 y/z: 16 x 32
    static constexpr int T2 = AX == 0 ? SweepTuning<Real>::T2X : kNarrow ? W5CT_F64_T2YZ_NARROW : SweepTuning<Real>::T2YZ;
    static constexpr int BX = kNarrow ? W5CT_F64_BXYZ : 32;
    static constexpr int MINB = SweepTuning<Real>::MINB;
    static constexpr int FPT = SweepTuning<Real>::FPT;
    using TT = SweepTile<AX, T2, BX, FPT>;
    static constexpr size_t smem = (size_t)TT::NC * box_quantities<Real>() * sizeof(Real);
};

// Single-patch sweep in tiles of BX x T2 faces, FPT per thread (the block
// is BX x T2 / FPT threads).
template <int AX, typename Real, int VAR, int T2, int MINB, int FPT, int BX = 32, bool DW = false>
struct SinglePatchSweep {
    using TT = SweepTile<AX, T2, BX, FPT>;
    static constexpr size_t smem = (size_t)TT::NC * box_quantities<Real>() * sizeof(Real);
    static cudaError_t prepare() {
        return cudaFuncSetAttribute(sweep_kernel<AX, Real, VAR, T2, MINB, FPT, BX, DW>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    static dim3 grid(int nx, int ny, int nz) {
        if (AX == 0 || AX == 1) return dim3((nx + BX - 1) / BX, (ny + TT::BY - 1) / TT::BY, nz);
        return dim3((nx + BX - 1) / BX, ny, (nz + TT::BZ - 1) / TT::BZ);
    }
    static cudaError_t launch(const SweepArgs<Real> &a, cudaStream_t s) {
        sweep_kernel<AX, Real, VAR, T2, MINB, FPT, BX, DW><<<grid(a.nx, a.ny, a.nz), dim3(BX, TT::ROWS), smem, s>>>(a);
        return cudaGetLastError();
    }
};

// Tile shapes of the batched sweeps (chosen per patch and axis by the
// autotuner).  Variant 0 is SweepCfg's tile (32 lanes) in float and 32 x 16
// in double (patches are 16 to 64 cells across); the float path also
// has narrower tiles that waste fewer lanes on patches whose sizes are not
// multiples of 32 or of 16: (BX, T2, faces per thread) = (16, 16, 1),
// (8, 16, 1), (8, 8, 1).  Every variant keeps 128 registers per thread: min
// blocks per SM = 512 / threads per block.
constexpr int kMaxTileVariants = 4;

template <int AX, typename Real, int V>
struct TileV;
constexpr int kBatchedF64T2 = 16;
template <int AX, typename Real>
struct TileV<AX, Real, 0> {
    static constexpr int T2 = sizeof(Real) == 8 ? kBatchedF64T2 : SweepCfg<AX, Real>::T2, BX = 32, FPT = T2 / 8,
                         MINB = SweepCfg<AX, Real>::MINB;
};
template <int AX, typename Real>
struct TileV<AX, Real, 1> {
    static constexpr int T2 = 16, BX = 16, FPT = 1, MINB = 2;
};
template <int AX, typename Real>
struct TileV<AX, Real, 2> {
    static constexpr int T2 = 16, BX = 8, FPT = 1, MINB = 4;
};
template <int AX, typename Real>
struct TileV<AX, Real, 3> {
    static constexpr int T2 = 8, BX = 8, FPT = 1, MINB = 8;
};

template <typename Real>
inline int num_tile_variants() {
    return sizeof(Real) == 4 ? kMaxTileVariants : 1;
}

// (BX, T2) of variant v along axis `axis` (host side, for the tile tables)
template <typename Real>
inline void tile_shape(int axis, int v, int &bx, int &t2) {
    if (v == 0) {
        bx = 32;
        t2 = sizeof(Real) == 8 ? kBatchedF64T2 : axis == 0 ? SweepTuning<Real>::T2X : SweepTuning<Real>::T2YZ;
    } else {
        bx = v == 1 ? 16 : 8;
        t2 = v == 3 ? 8 : 16;
    }
}

template <int AX, typename Real, int VAR, int V>
struct BatchedSweep {
    using C = TileV<AX, Real, V>;
    using TT = SweepTile<AX, C::T2, C::BX, C::FPT>;
    static constexpr size_t smem = (size_t)TT::NC * box_quantities<Real>() * sizeof(Real);
    static cudaError_t prepare() {
        return cudaFuncSetAttribute(sweep_batched_kernel<AX, Real, VAR, C::T2, C::MINB, C::BX, C::FPT>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    static cudaError_t launch(const SweepArgs<Real> &a, const PatchGeom *pgs, const int4 *tiles, int ntiles,
                              cudaStream_t s) {
        sweep_batched_kernel<AX, Real, VAR, C::T2, C::MINB, C::BX, C::FPT>
            <<<ntiles, dim3(C::BX, TT::ROWS), smem, s>>>(a, pgs, tiles);
        return cudaGetLastError();
    }
};

// Persistent sweep of one tile variant over the three axes: a grid of
// resident blocks takes work items (tiles of any axis, the axis in bits 28-29
// of item.x, the patch in bits 0-27) from a device counter with atomicAdd
// until the list is exhausted.  Nothing waits on another block, so the
// queue needs no spin; the counter is zeroed before the launch.  The three
// axes' sweeps of a stage are independent (all read the stage state), so one
// queue covers them and their tails overlap.
template <typename Real, int VAR, int V>
struct PersistentSweep {
    using C0 = TileV<0, Real, V>;
    using C1 = TileV<1, Real, V>;
    using C2 = TileV<2, Real, V>;
    using T0 = SweepTile<0, C0::T2, C0::BX, C0::FPT>;
    using T1 = SweepTile<1, C1::T2, C1::BX, C1::FPT>;
    using T2_ = SweepTile<2, C2::T2, C2::BX, C2::FPT>;
    static_assert(T0::NT == T1::NT && T1::NT == T2_::NT && C0::BX == C1::BX && C1::BX == C2::BX,
                  "one block shape for the three axes");
    static constexpr int NT = T0::NT, BX = C0::BX, ROWS = T0::ROWS, MINB = C0::MINB;
    static constexpr size_t smem0 = (size_t)T0::NC * box_quantities<Real>() * sizeof(Real);
    static constexpr size_t smem1 = (size_t)T1::NC * box_quantities<Real>() * sizeof(Real);
    static constexpr size_t smem2 = (size_t)T2_::NC * box_quantities<Real>() * sizeof(Real);
    static constexpr size_t smem = smem0 > smem1 ? (smem0 > smem2 ? smem0 : smem2) : (smem1 > smem2 ? smem1 : smem2);
};

template <typename Real, int VAR, int V>
__global__ void __launch_bounds__(PersistentSweep<Real, VAR, V>::NT, PersistentSweep<Real, VAR, V>::MINB)
    sweep_persistent_kernel(SweepArgs<Real> a0, SweepArgs<Real> a1, SweepArgs<Real> a2,
                            const PatchGeom *__restrict__ pgs, const int4 *__restrict__ items, int nitems,
                            int *counter) {
    using P = PersistentSweep<Real, VAR, V>;
    extern __shared__ __align__(16) unsigned char w5ct_smem[];
    __shared__ int s_item;
    Real *sm = reinterpret_cast<Real *>(w5ct_smem);
    for (;;) {
        if (threadIdx.x == 0 && threadIdx.y == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= nitems) break;           // the same value in every thread of the block
        const int4 t = items[it];
        const int ax = t.x >> kItemAxisShift;
        const PatchGeom pg = pgs[t.x & kItemPatchMask];
        if (ax == 0)
            sweep_tile<0, Real, VAR, P::C0::T2, P::BX, P::C0::FPT, 1>(a0, pg, t.y, t.z, t.w, sm);
        else if (ax == 1)
            sweep_tile<1, Real, VAR, P::C1::T2, P::BX, P::C1::FPT, 1>(a1, pg, t.y, t.z, t.w, sm);
        else
            sweep_tile<2, Real, VAR, P::C2::T2, P::BX, P::C2::FPT, 1>(a2, pg, t.y, t.z, t.w, sm);
        __syncthreads();                   // shared memory and s_item are reused
    }
}

template <typename Real, int VAR, int V>
struct PersistentLaunch {
    using P = PersistentSweep<Real, VAR, V>;
    static cudaError_t prepare() {
        return cudaFuncSetAttribute(sweep_persistent_kernel<Real, VAR, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)P::smem);
    }
    // resident blocks of this kernel on the whole device
    static cudaError_t grid(int &blocks) {
        int dev = 0, sms = 0, per = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, sweep_persistent_kernel<Real, VAR, V>, P::NT, P::smem);
        blocks = sms * (per > 0 ? per : 1);
        return e;
    }
    static cudaError_t launch(const SweepArgs<Real> (&a)[3], const PatchGeom *pgs, const int4 *items, int nitems,
                              int *counter, int blocks, cudaStream_t s) {
        sweep_persistent_kernel<Real, VAR, V><<<blocks, dim3(P::BX, P::ROWS), P::smem, s>>>(a[0], a[1], a[2], pgs, items,
                                                                                         nitems, counter);
        return cudaGetLastError();
    }
};

// allow the dynamic shared memory of every sweep kernel of this type
template <int AX, typename Real, int VAR>
cudaError_t prepare_sweep_axis() {
    using C = SweepCfg<AX, Real>;
    cudaError_t e = cudaFuncSetAttribute(sweep_kernel<AX, Real, VAR, C::T2, C::MINB, C::FPT, C::BX>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem);
    if (e != cudaSuccess) return e;
    if constexpr (std::is_same<Real, double>::value) {
        if ((e = SinglePatchSweep<AX, Real, VAR, 8, C::MINB, 1>::prepare()) != cudaSuccess) return e;
        if ((e = SinglePatchSweep<AX, Real, VAR, 4, C::MINB, 1>::prepare()) != cudaSuccess) return e;
    }
    if ((e = BatchedSweep<AX, Real, VAR, 0>::prepare()) != cudaSuccess) return e;
    if constexpr (sizeof(Real) == 4) {
        if ((e = BatchedSweep<AX, Real, VAR, 1>::prepare()) != cudaSuccess) return e;
        if ((e = BatchedSweep<AX, Real, VAR, 2>::prepare()) != cudaSuccess) return e;
        if ((e = BatchedSweep<AX, Real, VAR, 3>::prepare()) != cudaSuccess) return e;
    }
    if constexpr (AX == 0) {
        if ((e = PersistentLaunch<Real, VAR, 0>::prepare()) != cudaSuccess) return e;
        if constexpr (sizeof(Real) == 4) {
            if ((e = PersistentLaunch<Real, VAR, 1>::prepare()) != cudaSuccess) return e;
            if ((e = PersistentLaunch<Real, VAR, 2>::prepare()) != cudaSuccess) return e;
            if ((e = PersistentLaunch<Real, VAR, 3>::prepare()) != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

template <typename Real>
cudaError_t prepare_sweeps_impl() {
    cudaError_t e;
    if constexpr (std::is_same<Real, double>::value)
        if ((e = prepare_sweeps_f64dw()) != cudaSuccess) return e;
    if ((e = prepare_sweep_axis<0, Real, 0>()) != cudaSuccess) return e;
    if ((e = prepare_sweep_axis<1, Real, 0>()) != cudaSuccess) return e;
    if ((e = prepare_sweep_axis<2, Real, 0>()) != cudaSuccess) return e;
    if ((e = prepare_sweep_axis<0, Real, 1>()) != cudaSuccess) return e;
    if ((e = prepare_sweep_axis<1, Real, 1>()) != cudaSuccess) return e;
    return prepare_sweep_axis<2, Real, 1>();
}

// Defined in w5ct_sweep32.cu / w5ct_sweep64.cu.
template <typename Real>
cudaError_t prepare_sweeps();
// Tiles `tiles` (all of tile variant tv) of the batched sweep along `axis`.
template <typename Real>
cudaError_t launch_sweep_batched(int axis, int variant, int tv, const SweepArgs<Real> &a, const PatchGeom *pgs,
                                 const int4 *tiles, int ntiles, cudaStream_t s);

// The persistent sweep of tile variant tv over items (three axes, see
// sweep_persistent_kernel) with `blocks` resident blocks; and that block count.
template <typename Real>
cudaError_t launch_sweep_persistent(int variant, int tv, const SweepArgs<Real> (&a)[3], const PatchGeom *pgs,
                                    const int4 *items, int nitems, int *counter, int blocks, cudaStream_t s);
template <typename Real>
cudaError_t persistent_grid(int variant, int tv, int &blocks);

template <typename Real, int VAR>
cudaError_t launch_sweep_persistent_v(int tv, const SweepArgs<Real> (&a)[3], const PatchGeom *pgs, const int4 *items,
                                      int nitems, int *counter, int blocks, cudaStream_t s) {
    if constexpr (sizeof(Real) == 4) {
        if (tv == 1) return PersistentLaunch<Real, VAR, 1>::launch(a, pgs, items, nitems, counter, blocks, s);
        if (tv == 2) return PersistentLaunch<Real, VAR, 2>::launch(a, pgs, items, nitems, counter, blocks, s);
        if (tv == 3) return PersistentLaunch<Real, VAR, 3>::launch(a, pgs, items, nitems, counter, blocks, s);
    }
    if (tv != 0) return cudaErrorInvalidValue;
    return PersistentLaunch<Real, VAR, 0>::launch(a, pgs, items, nitems, counter, blocks, s);
}

template <typename Real, int VAR>
cudaError_t persistent_grid_v(int tv, int &blocks) {
    if constexpr (sizeof(Real) == 4) {
        if (tv == 1) return PersistentLaunch<Real, VAR, 1>::grid(blocks);
        if (tv == 2) return PersistentLaunch<Real, VAR, 2>::grid(blocks);
        if (tv == 3) return PersistentLaunch<Real, VAR, 3>::grid(blocks);
    }
    if (tv != 0) return cudaErrorInvalidValue;
    return PersistentLaunch<Real, VAR, 0>::grid(blocks);
}

template <int AX, typename Real, int VAR>
cudaError_t launch_sweep_batched_axis(int tv, const SweepArgs<Real> &a, const PatchGeom *pgs, const int4 *tiles,
                                      int ntiles, cudaStream_t s) {
    if constexpr (sizeof(Real) == 4) {
        if (tv == 1) return BatchedSweep<AX, Real, VAR, 1>::launch(a, pgs, tiles, ntiles, s);
        if (tv == 2) return BatchedSweep<AX, Real, VAR, 2>::launch(a, pgs, tiles, ntiles, s);
        if (tv == 3) return BatchedSweep<AX, Real, VAR, 3>::launch(a, pgs, tiles, ntiles, s);
    }
    if (tv != 0) return cudaErrorInvalidValue;
    return BatchedSweep<AX, Real, VAR, 0>::launch(a, pgs, tiles, ntiles, s);
}

template <typename Real>
cudaError_t launch_sweep_batched_impl(int axis, int variant, int tv, const SweepArgs<Real> &a, const PatchGeom *pgs,
                                      const int4 *tiles, int ntiles, cudaStream_t s) {
    if (variant == 0) {
        if (axis == 0) return launch_sweep_batched_axis<0, Real, 0>(tv, a, pgs, tiles, ntiles, s);
        if (axis == 1) return launch_sweep_batched_axis<1, Real, 0>(tv, a, pgs, tiles, ntiles, s);
        return launch_sweep_batched_axis<2, Real, 0>(tv, a, pgs, tiles, ntiles, s);
    }
    if (axis == 0) return launch_sweep_batched_axis<0, Real, 1>(tv, a, pgs, tiles, ntiles, s);
    if (axis == 1) return launch_sweep_batched_axis<1, Real, 1>(tv, a, pgs, tiles, ntiles, s);
    return launch_sweep_batched_axis<2, Real, 1>(tv, a, pgs, tiles, ntiles, s);
}

// The FP64 sweep keeps one block of 256 threads per SM (its registers), so a
// small patch fills the GPU only with shorter tiles: 8 high (256 threads, one
// face each) or 4 high (128 threads, two blocks per SM).  The float sweep
// always uses its default tile.
constexpr int kSmallTileHeights[2] = {8, 4};

// blocks of the single-patch sweep along `axis` in tiles of bx lanes x t2
inline long long sweep_blocks(int axis, int t2, int bx, int nx, int ny, int nz) {
    const long long nbx = (nx + bx - 1) / bx;
    if (axis == 2) return nbx * ny * ((nz + t2 - 1) / t2);
    return nbx * ((ny + t2 - 1) / t2) * nz;     // x- and y-sweeps: t2 pencils or faces along y
}

// Tile height of the single-patch sweep along `axis`: the default, or for
// FP64 the tallest of the shorter (32-lane) tiles that gives every SM at
// least two blocks (the shortest if none does).
template <typename Real>
inline int choose_sweep_t2(int axis, int nx, int ny, int nz, int sms) {
    const int t2d = axis == 0 ? SweepCfg<0, Real>::T2 : SweepCfg<1, Real>::T2;
    const int bxd = axis == 0 ? SweepCfg<0, Real>::BX : SweepCfg<1, Real>::BX;
    if (!std::is_same<Real, double>::value) return t2d;
    if (sweep_blocks(axis, t2d, bxd, nx, ny, nz) >= 2LL * sms) return t2d;
    for (int h : kSmallTileHeights)
        if (sweep_blocks(axis, h, 32, nx, ny, nz) >= 2LL * sms) return h;
    return kSmallTileHeights[1];
}

template <int AX, typename Real, int VAR>
cudaError_t launch_sweep_axis(int t2, const SweepArgs<Real> &a, cudaStream_t s) {
    using C = SweepCfg<AX, Real>;
    if constexpr (std::is_same<Real, double>::value) {
        if (t2 == 8) return SinglePatchSweep<AX, Real, VAR, 8, C::MINB, 1>::launch(a, s);
        if (t2 == 4) return SinglePatchSweep<AX, Real, VAR, 4, C::MINB, 1>::launch(a, s);
    }
    if (t2 != 0 && t2 != C::T2) return cudaErrorInvalidValue;
    if constexpr (std::is_same<Real, double>::value)
        if (a.dw) return launch_sweep_f64dw(AX, VAR, a, s);
    // the default tile; its shared memory is allowed by prepare_sweeps() at w5ct_init_grid
    return SinglePatchSweep<AX, Real, VAR, C::T2, C::MINB, C::FPT, C::BX>::launch(a, s);
}

template <typename Real>
cudaError_t launch_sweep_impl(int axis, int variant, int t2, const SweepArgs<Real> &a, cudaStream_t s) {
    if (variant == 0) {
        if (axis == 0) return launch_sweep_axis<0, Real, 0>(t2, a, s);
        if (axis == 1) return launch_sweep_axis<1, Real, 0>(t2, a, s);
        return launch_sweep_axis<2, Real, 0>(t2, a, s);
    }
    if (axis == 0) return launch_sweep_axis<0, Real, 1>(t2, a, s);
    if (axis == 1) return launch_sweep_axis<1, Real, 1>(t2, a, s);
    return launch_sweep_axis<2, Real, 1>(t2, a, s);
}

}  // namespace w5ct
