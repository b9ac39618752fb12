// w5ct_sweep32.cu -- instantiations of the characteristic sweep kernel for
// Real = float (one translation unit per arithmetic type, compiled in parallel).
#include "w5ct_internal.h"

namespace w5ct {

template <int AX, int VAR>
static cudaError_t launch_axis(const SweepArgs<float> &a, cudaStream_t s) {
    constexpr int T2 = kSweepT2;
    using TT = SweepTile<AX, T2>;
    const size_t smem = (size_t)TT::NC * NCQ * sizeof(float);
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(sweep_kernel<AX, float, VAR, T2>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const dim3 block(32, T2);
    dim3 grid;
    if (AX == 0 || AX == 1)
        grid = dim3((a.nx + 31) / 32, (a.ny + TT::BY - 1) / TT::BY, a.nz);
    else
        grid = dim3((a.nx + 31) / 32, a.ny, (a.nz + TT::BZ - 1) / TT::BZ);
    sweep_kernel<AX, float, VAR, T2><<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
}

template <>
cudaError_t launch_sweep<float>(int axis, int variant, const SweepArgs<float> &a, cudaStream_t s) {
    if (variant == 0) {
        if (axis == 0) return launch_axis<0, 0>(a, s);
        if (axis == 1) return launch_axis<1, 0>(a, s);
        return launch_axis<2, 0>(a, s);
    }
    if (axis == 0) return launch_axis<0, 1>(a, s);
    if (axis == 1) return launch_axis<1, 1>(a, s);
    return launch_axis<2, 1>(a, s);
}

}  // namespace w5ct
