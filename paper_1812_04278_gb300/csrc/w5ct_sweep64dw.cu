// w5ct_sweep64dw.cu -- the FP64 single-patch sweep kernels of the default
// tiles with the WENO part of every characteristic field's flux in
// double-word arithmetic (w5ct_physics.cuh, weno_field): the smoothness
// indicators, the nonlinear weights and the two interpolants of the LF-split
// differences run on the FP32 pipe, while the cell box, the eigenvectors,
// the projections, the split itself, the back-projection and every stored
// value stay in IEEE double.  A translation unit of its own so that it compiles in
// parallel with the other sweeps.
#include "w5ct_internal.h"

namespace w5ct {

namespace {
template <int AX, int VAR>
using DwSweep = SinglePatchSweep<AX, double, VAR, SweepCfg<AX, double>::T2, SweepCfg<AX, double>::MINB,
                                 SweepCfg<AX, double>::FPT, SweepCfg<AX, double>::BX, true>;
}  // namespace

cudaError_t launch_sweep_f64dw(int axis, int variant, const SweepArgs<double> &a, cudaStream_t s) {
    if (variant == 0) {
        if (axis == 0) return DwSweep<0, 0>::launch(a, s);
        if (axis == 1) return DwSweep<1, 0>::launch(a, s);
        return DwSweep<2, 0>::launch(a, s);
    }
    if (axis == 0) return DwSweep<0, 1>::launch(a, s);
    if (axis == 1) return DwSweep<1, 1>::launch(a, s);
    return DwSweep<2, 1>::launch(a, s);
}

cudaError_t prepare_sweeps_f64dw() {
    cudaError_t e;
    if ((e = DwSweep<0, 0>::prepare()) != cudaSuccess) return e;
    if ((e = DwSweep<1, 0>::prepare()) != cudaSuccess) return e;
    if ((e = DwSweep<2, 0>::prepare()) != cudaSuccess) return e;
    if ((e = DwSweep<0, 1>::prepare()) != cudaSuccess) return e;
    if ((e = DwSweep<1, 1>::prepare()) != cudaSuccess) return e;
    return DwSweep<2, 1>::prepare();
}

}  // namespace w5ct
