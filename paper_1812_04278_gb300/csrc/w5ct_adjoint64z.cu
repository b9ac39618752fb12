// w5ct_adjoint64z.cu -- the adjoint sweep kernels for B = double, WENO variant
// 1 (one translation unit per arithmetic type and variant, compiled in
// parallel).
#include "w5ct_adjoint.cuh"

namespace w5ct {

template <>
cudaError_t launch_adj_sweep<double, 1>(int axis, const AdjSweepArgs<double> &a, cudaStream_t s) {
    return launch_adj_sweep_impl<double, 1>(axis, a, s);
}

}  // namespace w5ct
