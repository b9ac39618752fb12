// w5ct_sweep64.cu -- the characteristic sweep kernels for Real = double (one
// translation unit per arithmetic type, compiled in parallel).
#include "w5ct_internal.h"

namespace w5ct {

template <>
cudaError_t launch_sweep<double>(int axis, int variant, const SweepArgs<double> &a, cudaStream_t s) {
    return launch_sweep_impl<double>(axis, variant, a, s);
}

template <>
cudaError_t prepare_sweeps<double>() {
    return prepare_sweeps_impl<double>();
}

template <>
cudaError_t launch_sweep_batched<double>(int axis, int variant, int tv, const SweepArgs<double> &a, const PatchGeom *pgs,
                                     const int4 *tiles, int ntiles, cudaStream_t s) {
    return launch_sweep_batched_impl<double>(axis, variant, tv, a, pgs, tiles, ntiles, s);
}

}  // namespace w5ct
