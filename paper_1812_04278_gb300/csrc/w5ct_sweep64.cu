// w5ct_sweep64.cu -- the characteristic sweep kernel for Real = double (one
// translation unit per arithmetic type, compiled in parallel).
#include "w5ct_internal.h"

namespace w5ct {

template <>
cudaError_t launch_sweep<double>(int axis, int variant, const SweepArgs<double> &a, cudaStream_t s) {
    return launch_sweep_impl<double>(axis, variant, a, s);
}

}  // namespace w5ct
