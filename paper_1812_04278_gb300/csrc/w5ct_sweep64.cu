// w5ct_sweep64.cu -- the characteristic sweep kernels for Real = double (one
// translation unit per arithmetic type, compiled in parallel).
#include "w5ct_internal.h"

namespace w5ct {

template <>
cudaError_t launch_sweep<double>(int axis, int variant, int t2, const SweepArgs<double> &a, cudaStream_t s) {
    return launch_sweep_impl<double>(axis, variant, t2, a, s);
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

template <>
cudaError_t launch_sweep_persistent<double>(int variant, int tv, const SweepArgs<double> (&a)[3], const PatchGeom *pgs,
                                        const int4 *items, int nitems, int *counter, int blocks, cudaStream_t s) {
    return variant == 0 ? launch_sweep_persistent_v<double, 0>(tv, a, pgs, items, nitems, counter, blocks, s)
                        : launch_sweep_persistent_v<double, 1>(tv, a, pgs, items, nitems, counter, blocks, s);
}

template <>
cudaError_t persistent_grid<double>(int variant, int tv, int &blocks) {
    return variant == 0 ? persistent_grid_v<double, 0>(tv, blocks) : persistent_grid_v<double, 1>(tv, blocks);
}

}  // namespace w5ct
