"""Wave diagnostics of the paper's convergence tests (host-side analysis of
states returned by the solver; not part of a step).

* decay_rate (Sec. 4.1, Eq. decay_rate): tau_D = -(1/t) log(dB(t) / dB(0)),
  dB the root-mean-square fluctuation of a field component in the frame of
  the wave vector; sensitive to numerical dissipation only, not dispersion.
* eigenmode_amplitudes: the amplitudes of the seven linear MHD modes in
  one Fourier mode of the state; the decay of one wave family, free of the
  small other waves (same wave vector) that the CT update's dispersion
  excites and that make an RMS of B rise and fall.
* transverse_flux_rms (Sec. 4.2): RMS over the cells of
  sqrt((B_1 v_1)^2 + (B_2 v_2)^2) with 1, 2 the transverse directions of
  the wave frame; the robust dissipation measure of the polarised Alfven
  wave.
"""
from __future__ import annotations

import numpy as np

from . import inputs


def rms_fluctuation(field, e) -> float:
    """RMS about the mean of the component of a (3, nz, ny, nx) vector field
    along the unit vector e."""
    f = np.tensordot(np.asarray(e, dtype=np.float64), field, axes=(0, 0))
    return float(np.sqrt(np.mean((f - f.mean()) ** 2)))


def mode_amplitude(field, e, kint) -> float:
    """Amplitude of the Fourier mode k = 2 pi kint (unit box, cell centres) of
    the component of a (3, nz, ny, nx) vector field along e: the decay of one
    wave without the other waves that an RMS also sees."""
    f = np.tensordot(np.asarray(e, dtype=np.float64), field, axes=(0, 0))
    nz, ny, nx = f.shape
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    z = (np.arange(nz) + 0.5) / nz
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    ph = 2 * np.pi * (kint[0] * X + kint[1] * Y + kint[2] * Z)
    return float(2.0 * abs(np.mean(f * np.exp(-1j * ph))))


def eigenmode_amplitudes(cons, bcell, kint, rho, B_wave, P, gamma=inputs.GAMMA):
    """|L_m . dQ_k| for the seven modes m of linear_mhd_modes (sorted by
    speed) about a state at rest (rho, wave-frame field B_wave, P): dQ_k is
    the complex amplitude of the Fourier mode k = 2 pi kint (unit box) of the
    conserved perturbation in the wave frame (rho, m_par, m_p1, m_p2, B_p1,
    B_p2, E), the field taken at the cell centres."""
    khat, e1, e2 = inputs.wave_frame(kint)
    _, vecs = inputs.linear_mhd_modes(rho, 0.0, B_wave[0], B_wave[1], B_wave[2], P, gamma)
    left = np.linalg.inv(vecs.T)
    nz, ny, nx = cons.shape[1:]
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    z = (np.arange(nz) + 0.5) / nz
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    w = np.exp(-2j * np.pi * (kint[0] * X + kint[1] * Y + kint[2] * Z))
    m = cons[1:4]
    comps = [cons[0], np.tensordot(khat, m, 1), np.tensordot(e1, m, 1), np.tensordot(e2, m, 1),
             np.tensordot(e1, bcell, 1), np.tensordot(e2, bcell, 1), cons[4]]
    dq = np.array([2.0 * np.mean(f * w) for f in comps])
    return np.abs(left @ dq)


def decay_rate(d0: float, dt_: float, t: float) -> float:
    """tau_D = -(1/t) log(d(t) / d(0))."""
    return -np.log(dt_ / d0) / t


def transverse_flux_rms(cons, bcell, e1, e2) -> float:
    """RMS of sqrt((B_1 v_1)^2 + (B_2 v_2)^2) with B_k = B . e_k and v_k the
    velocity along e_k."""
    v = cons[1:4] / cons[0]
    b1, b2 = np.tensordot(e1, bcell, axes=(0, 0)), np.tensordot(e2, bcell, axes=(0, 0))
    v1, v2 = np.tensordot(e1, v, axes=(0, 0)), np.tensordot(e2, v, axes=(0, 0))
    return float(np.sqrt(np.mean((b1 * v1) ** 2 + (b2 * v2) ** 2)))
