// w5ct_sweep32.cu -- the characteristic sweep kernel for Real = float (one
// translation unit per arithmetic type, compiled in parallel).
#include "w5ct_internal.h"

namespace w5ct {

template <>
cudaError_t launch_sweep<float>(int axis, int variant, const SweepArgs<float> &a, cudaStream_t s) {
    return launch_sweep_impl<float>(axis, variant, a, s);
}

}  // namespace w5ct
