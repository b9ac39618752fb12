// w5ct_fused64.cu -- the fused persistent step kernel for Real = double (one
// translation unit per arithmetic type, compiled in parallel; see
// w5ct_fused.cuh).
#include "w5ct_fused.cuh"

namespace w5ct {

template <>
cudaError_t launch_fused_step<double>(int variant, const FusedArgs<double> &A, int blocks, cudaStream_t s) {
    return variant == 0 ? launch_fused_impl<double, 0>(A, blocks, s) : launch_fused_impl<double, 1>(A, blocks, s);
}

template <>
cudaError_t fused_grid<double>(int variant, int &blocks, size_t &smem) {
    return variant == 0 ? fused_grid_impl<double, 0>(blocks, smem) : fused_grid_impl<double, 1>(blocks, smem);
}

}  // namespace w5ct
