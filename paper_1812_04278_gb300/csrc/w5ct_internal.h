// w5ct_internal.h -- declarations shared by the translation units of libw5ct.
#pragma once
#include <cuda_runtime.h>

#include "w5ct_kernels.cuh"

namespace w5ct {

// tile height of the sweep kernels (pencils along y for the x-sweep, faces
// along the axis for the y- and z-sweeps)
constexpr int kSweepT2 = 8;

// Launch the characteristic sweep along `axis` (0, 1, 2) with WENO variant
// `variant` (0 = JS, 1 = Z).  Defined in w5ct_sweep32.cu / w5ct_sweep64.cu.
template <typename Real>
cudaError_t launch_sweep(int axis, int variant, const SweepArgs<Real> &a, cudaStream_t s);

}  // namespace w5ct
