// w5ct_sweep32.cu -- the characteristic sweep kernels for Real = float (one
// translation unit per arithmetic type, compiled in parallel).
#include "w5ct_internal.h"

namespace w5ct {

template <>
cudaError_t launch_sweep<float>(int axis, int variant, int t2, const SweepArgs<float> &a, cudaStream_t s) {
    return launch_sweep_impl<float>(axis, variant, t2, a, s);
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

template <>
cudaError_t launch_sweep_persistent<float>(int variant, int tv, const SweepArgs<float> (&a)[3], const PatchGeom *pgs,
                                        const int4 *items, int nitems, int *counter, int blocks, cudaStream_t s) {
    return variant == 0 ? launch_sweep_persistent_v<float, 0>(tv, a, pgs, items, nitems, counter, blocks, s)
                        : launch_sweep_persistent_v<float, 1>(tv, a, pgs, items, nitems, counter, blocks, s);
}

template <>
cudaError_t persistent_grid<float>(int variant, int tv, int &blocks) {
    return variant == 0 ? persistent_grid_v<float, 0>(tv, blocks) : persistent_grid_v<float, 1>(tv, blocks);
}

}  // namespace w5ct
