// w5ct_sweep32.cu -- the characteristic sweep kernels for Real = float (one
// translation unit per arithmetic type, compiled in parallel).
#include "w5ct_internal.h"

namespace w5ct {

template <>
cudaError_t launch_sweep<float>(int axis, int variant, const SweepArgs<float> &a, cudaStream_t s) {
    return launch_sweep_impl<float>(axis, variant, a, s);
}

template <>
cudaError_t prepare_sweeps<float>() {
    return prepare_sweeps_impl<float>();
}

template <>
cudaError_t launch_sweep_batched<float>(int axis, int variant, int tv, const SweepArgs<float> &a, const PatchGeom *pgs,
                                     const int4 *tiles, int ntiles, cudaStream_t s) {
    return launch_sweep_batched_impl<float>(axis, variant, tv, a, pgs, tiles, ntiles, s);
}

}  // namespace w5ct
