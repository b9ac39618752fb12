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

template <int AX, typename Real, int VAR>
cudaError_t launch_sweep_axis(const SweepArgs<Real> &a, cudaStream_t s) {
    constexpr int T2 = AX == 0 ? SweepTuning<Real>::T2X : SweepTuning<Real>::T2YZ;
    constexpr int MINB = SweepTuning<Real>::MINB;
    using TT = SweepTile<AX, T2>;
    const size_t smem = (size_t)TT::NC * NCQ * sizeof(Real);
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(sweep_kernel<AX, Real, VAR, T2, MINB>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
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
