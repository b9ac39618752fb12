"""Pins of the oracle's characteristic WENO flux (Sec. 2.2, Eq. FWENO).

The paper writes the flux as a central term plus two phi_N corrections of
split flux differences.  These tests compare it with the textbook form of
the same schemes -- the sum of an upwind reconstruction of F+ and a
downwind reconstruction of F- from three third-order candidate stencils
(Jiang & Shu 1996; Borges et al. 2008 for WENO-Z) -- and with closed forms.
In the paper's scaling IS_k = 12 beta_k, so eps in the textbook form is
eps/12.
"""
import numpy as np
import pytest

import oracle as O


def textbook_upwind(f, eps, variant):
    """Reconstruction of f at i+1/2 from f[i-2..i+2] (array index 0..4)."""
    f0, f1, f2, f3, f4 = f
    q = np.array([(2 * f0 - 7 * f1 + 11 * f2) / 6.0,
                  (-f1 + 5 * f2 + 2 * f3) / 6.0,
                  (2 * f2 + 5 * f3 - f4) / 6.0])
    b = np.array([13.0 / 12.0 * (f0 - 2 * f1 + f2) ** 2 + 0.25 * (f0 - 4 * f1 + 3 * f2) ** 2,
                  13.0 / 12.0 * (f1 - 2 * f2 + f3) ** 2 + 0.25 * (f1 - f3) ** 2,
                  13.0 / 12.0 * (f2 - 2 * f3 + f4) ** 2 + 0.25 * (3 * f2 - 4 * f3 + f4) ** 2])
    d = np.array([0.1, 0.6, 0.3])
    if variant == O.WENO_JS:
        a = d / (eps + b) ** 2
    else:
        tau = abs(b[0] - b[2])
        a = d * (1.0 + (tau / (eps + b)) ** 2)
    w = a / a.sum()
    return float(w @ q)


def textbook_flux(Fs, qs, alpha, variant, eps):
    fp = 0.5 * (np.asarray(Fs) + alpha * np.asarray(qs))
    fm = 0.5 * (np.asarray(Fs) - alpha * np.asarray(qs))
    # F- at i+1/2 is the mirror image: reconstruct from f[i+3..i-1]
    return textbook_upwind(fp[0:5], eps, variant) + textbook_upwind(fm[5:0:-1], eps, variant)


@pytest.mark.parametrize("variant", [O.WENO_JS, O.WENO_Z])
def test_matches_textbook_form(variant):
    cfg = O.make_config(weno_variant=variant)
    eps = (cfg.eps_js if variant == O.WENO_JS else cfg.eps_z) / 12.0
    rng = np.random.default_rng(100 + variant)
    for trial in range(400):
        kind = trial % 4
        if kind == 0:      # random data
            Fs, qs = rng.normal(size=6), rng.normal(size=6)
        elif kind == 1:    # smooth data
            x = np.arange(6) * rng.uniform(0.05, 0.6)
            Fs = np.sin(x + rng.uniform(0, 6)) * rng.uniform(0.1, 3)
            qs = np.cos(x + rng.uniform(0, 6)) * rng.uniform(0.1, 3)
        elif kind == 2:    # discontinuity
            j = rng.integers(1, 6)
            Fs = np.where(np.arange(6) < j, rng.normal(), rng.normal())
            qs = np.where(np.arange(6) < j, rng.normal(), rng.normal())
        else:              # tiny amplitude on a background
            Fs = 1.0 + 1e-6 * rng.normal(size=6)
            qs = 2.0 + 1e-6 * rng.normal(size=6)
        alpha = rng.uniform(0.0, 3.0)
        got = O.weno_char_flux(Fs, qs, alpha, cfg)
        ref = textbook_flux(Fs, qs, alpha, variant, eps)
        scale = max(np.abs(Fs).max(), alpha * np.abs(qs).max(), 1e-300)
        assert abs(got - ref) <= 2e-14 * scale, (trial, got, ref)


def test_linear_weights_closed_forms():
    """Smooth data of tiny amplitude: JS weights equal the linear weights to
    O(IS/eps), so the flux equals the fifth-order upwind formula (alpha such
    that F- = 0) and the sixth-order central formula (alpha = 0)."""
    cfg = O.make_config(weno_variant=O.WENO_JS)
    h = 0.3
    x = (np.arange(6) - 2) * h
    A = 1e-7
    F = A * np.sin(1.3 * x + 0.4)
    # alpha = 0: F+ = F- = F/2 -> (F_{i-2} - 8F_{i-1} + 37F_i + 37F_{i+1} - 8F_{i+2} + F_{i+3})/60
    got = O.weno_char_flux(F, np.zeros(6), 0.0, cfg)
    ref = (F[0] - 8 * F[1] + 37 * F[2] + 37 * F[3] - 8 * F[4] + F[5]) / 60.0
    assert abs(got - ref) < 1e-6 * A
    # q = F, alpha = 1: F- = 0 -> (2F_{i-2} - 13F_{i-1} + 47F_i + 27F_{i+1} - 3F_{i+2})/60
    got = O.weno_char_flux(F, F, 1.0, cfg)
    ref = (2 * F[0] - 13 * F[1] + 47 * F[2] + 27 * F[3] - 3 * F[4]) / 60.0
    assert abs(got - ref) < 1e-6 * A


@pytest.mark.parametrize("variant", [O.WENO_JS, O.WENO_Z, O.WENO_Z_PRINTED])
def test_constant_data_is_exact(variant):
    cfg = O.make_config(weno_variant=variant)
    got = O.weno_char_flux(np.full(6, 2.5), np.full(6, -1.0), 1.7, cfg)
    assert got == 2.5


def test_phi_n_linear_weight_limit():
    """phi_N with the linear weights (1,6,3)/10 is (a - 3b + 3c - d)/30."""
    cfg = O.make_config(weno_variant=O.WENO_JS)
    a, b, c, d = 1e-9 * np.array([0.3, -0.2, 0.7, 0.1])
    assert abs(O.phi_n(a, b, c, d, cfg) - (a - 3 * b + 3 * c - d) / 30.0) < 1e-6 * 1e-9


def test_essentially_non_oscillatory():
    """A step between i and i+1: the upwind flux stays within the data range
    to O(eps) (no Gibbs overshoot)."""
    cfg = O.make_config(weno_variant=O.WENO_JS)
    F = np.array([0.0, 0.0, 0.0, 1.0, 1.0, 1.0])
    got = O.weno_char_flux(F, F, 1.0, cfg)     # pure upwind (F- = 0)
    assert -1e-9 <= got <= 1e-3
    F = np.array([0.0, 0.0, 1.0, 1.0, 1.0, 1.0])
    got = O.weno_char_flux(F, F, 1.0, cfg)
    assert 1.0 - 1e-3 <= got <= 1.0 + 1e-9
