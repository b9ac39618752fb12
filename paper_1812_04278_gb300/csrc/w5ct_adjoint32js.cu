// w5ct_adjoint32js.cu -- the adjoint sweep kernels for B = float, WENO variant
// 0 (one translation unit per arithmetic type and variant, compiled in
// parallel).
#include "w5ct_adjoint.cuh"

namespace w5ct {

template <>
cudaError_t launch_adj_sweep<float, 0>(int axis, const AdjSweepArgs<float> &a, cudaStream_t s) {
    return launch_adj_sweep_impl<float, 0>(axis, a, s);
}

}  // namespace w5ct
