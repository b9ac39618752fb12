// w5ct_internal.h -- declarations shared by the translation units of libw5ct.
#pragma once
#include <cuda_runtime.h>

#include "w5ct_kernels.cuh"

namespace w5ct {

// Record the text that w5ct_last_error(NULL) returns (calls without a context).
void set_global_error(const char *text);

// Launch the characteristic sweep along `axis` (0, 1, 2) with WENO variant
// `variant` (0 = JS, 1 = Z).  Defined in w5ct_sweep32.cu / w5ct_sweep64.cu.
template <typename Real>
cudaError_t launch_sweep(int axis, int variant, const SweepArgs<Real> &a, cudaStream_t s);

// Sweep tiling per arithmetic type: faces per block in the second tile
// direction (x-sweep: pencils along y; y- and z-sweeps: faces along the
// axis) and the minimum resident blocks per SM the register budget targets.
template <typename Real>
struct SweepTuning;

// Defaults measured on GB300 at 256^3 (FP32: 2 blocks/SM of 16-high tiles,
// 1.6x faster than 1 block of 8-high tiles).
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
#define W5CT_F64_T2X 8
#endif
#ifndef W5CT_F64_T2YZ
#define W5CT_F64_T2YZ 16
#endif

template <>
struct SweepTuning<float> {
    static constexpr int T2X = W5CT_F32_T2X, T2YZ = W5CT_F32_T2YZ, MINB = W5CT_F32_MINB;
};
template <>
struct SweepTuning<double> {
    static constexpr int T2X = W5CT_F64_T2X, T2YZ = W5CT_F64_T2YZ, MINB = 1;
};

template <int AX, typename Real>
struct SweepCfg {
    static constexpr int T2 = AX == 0 ? SweepTuning<Real>::T2X : SweepTuning<Real>::T2YZ;
    static constexpr int MINB = SweepTuning<Real>::MINB;
    using TT = SweepTile<AX, T2>;
    static constexpr size_t smem = (size_t)TT::NC * NCQ * sizeof(Real);
};

// allow the dynamic shared memory of every sweep kernel of this type
template <int AX, typename Real, int VAR>
cudaError_t prepare_sweep_axis() {
    using C = SweepCfg<AX, Real>;
    cudaError_t e = cudaFuncSetAttribute(sweep_kernel<AX, Real, VAR, C::T2, C::MINB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(sweep_batched_kernel<AX, Real, VAR, C::T2, C::MINB>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem);
}

template <typename Real>
cudaError_t prepare_sweeps_impl() {
    cudaError_t e;
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
template <typename Real>
cudaError_t launch_sweep_batched(int axis, int variant, const SweepArgs<Real> &a, const PatchGeom *pgs,
                                 const int4 *tiles, int ntiles, cudaStream_t s);

// tile heights of the sweep along each axis for this arithmetic type
template <typename Real>
inline int sweep_t2(int axis) {
    return axis == 0 ? SweepTuning<Real>::T2X : SweepTuning<Real>::T2YZ;
}

template <int AX, typename Real, int VAR>
cudaError_t launch_sweep_batched_axis(const SweepArgs<Real> &a, const PatchGeom *pgs, const int4 *tiles, int ntiles,
                                      cudaStream_t s) {
    using C = SweepCfg<AX, Real>;
    sweep_batched_kernel<AX, Real, VAR, C::T2, C::MINB><<<ntiles, dim3(32, 8), C::smem, s>>>(a, pgs, tiles);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_sweep_batched_impl(int axis, int variant, const SweepArgs<Real> &a, const PatchGeom *pgs,
                                      const int4 *tiles, int ntiles, cudaStream_t s) {
    if (variant == 0) {
        if (axis == 0) return launch_sweep_batched_axis<0, Real, 0>(a, pgs, tiles, ntiles, s);
        if (axis == 1) return launch_sweep_batched_axis<1, Real, 0>(a, pgs, tiles, ntiles, s);
        return launch_sweep_batched_axis<2, Real, 0>(a, pgs, tiles, ntiles, s);
    }
    if (axis == 0) return launch_sweep_batched_axis<0, Real, 1>(a, pgs, tiles, ntiles, s);
    if (axis == 1) return launch_sweep_batched_axis<1, Real, 1>(a, pgs, tiles, ntiles, s);
    return launch_sweep_batched_axis<2, Real, 1>(a, pgs, tiles, ntiles, s);
}

template <int AX, typename Real, int VAR>
cudaError_t launch_sweep_axis(const SweepArgs<Real> &a, cudaStream_t s) {
    using C = SweepCfg<AX, Real>;
    constexpr int T2 = C::T2;
    constexpr int MINB = C::MINB;
    using TT = typename C::TT;
    const size_t smem = C::smem;     // allowed by prepare_sweeps() at w5ct_init_grid
    const dim3 block(32, 8);
    dim3 grid;
    if (AX == 0 || AX == 1)
        grid = dim3((a.nx + 31) / 32, (a.ny + TT::BY - 1) / TT::BY, a.nz);
    else
        grid = dim3((a.nx + 31) / 32, a.ny, (a.nz + TT::BZ - 1) / TT::BZ);
    sweep_kernel<AX, Real, VAR, T2, MINB><<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_sweep_impl(int axis, int variant, const SweepArgs<Real> &a, cudaStream_t s) {
    if (variant == 0) {
        if (axis == 0) return launch_sweep_axis<0, Real, 0>(a, s);
        if (axis == 1) return launch_sweep_axis<1, Real, 0>(a, s);
        return launch_sweep_axis<2, Real, 0>(a, s);
    }
    if (axis == 0) return launch_sweep_axis<0, Real, 1>(a, s);
    if (axis == 1) return launch_sweep_axis<1, Real, 1>(a, s);
    return launch_sweep_axis<2, Real, 1>(a, s);
}

}  // namespace w5ct
