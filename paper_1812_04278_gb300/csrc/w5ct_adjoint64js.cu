// w5ct_adjoint64js.cu -- the adjoint sweep kernels for B = double, WENO variant
// 0 (one translation unit per arithmetic type and variant, compiled in
// parallel).
#include "w5ct_adjoint.cuh"

namespace w5ct {

template <>
cudaError_t launch_adj_sweep<double, 0>(int axis, const AdjSweepArgs<double> &a, cudaStream_t s) {
    return launch_adj_sweep_impl<double, 0>(axis, a, s);
}

}  // namespace w5ct
