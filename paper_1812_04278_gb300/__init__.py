"""GB300-native fifth-order WENO + constrained-transport ideal MHD
(the hot path of Donnert et al., "WENO-Wombat", arXiv:1812.04278).

Submodules:
  ``w5ct``        -- ctypes binding of the CUDA C-ABI library ``libw5ct.so``;
  ``adjoint``     -- the rollout-misfit gradient as a torch.autograd.Function;
  ``inputs``      -- seeded synthetic initial conditions;
  ``diagnostics`` -- host-side analysis of states (RMS, modes, decay rates);
  ``build``       -- the nvcc build step of the library.
The binding loads the CUDA library when it is imported and raises if the
library is missing: there is no CPU fallback.
"""
__all__ = ["w5ct", "adjoint", "inputs", "diagnostics", "build"]
