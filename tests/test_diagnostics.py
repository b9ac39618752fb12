"""Host-side wave diagnostics against their closed forms."""
import numpy as np

from paper_1812_04278_gb300 import diagnostics as D


def test_rms_fluctuation_of_a_sine_is_amplitude_over_sqrt2():
    n = 64
    x = (np.arange(n) + 0.5) / n
    f = np.zeros((3, 1, 1, n))
    f[1, 0, 0] = 3.0 + 0.2 * np.sin(2 * np.pi * x)        # mean removed
    assert abs(D.rms_fluctuation(f, (0, 1, 0)) - 0.2 / np.sqrt(2)) < 1e-15
    assert D.rms_fluctuation(f, (1, 0, 0)) == 0.0


def test_decay_rate_of_an_exponential():
    tau = 0.37
    assert abs(D.decay_rate(2.0, 2.0 * np.exp(-tau * 1.5), 1.5) - tau) < 1e-15


def test_transverse_flux_rms_of_a_polarised_wave():
    """B_perp = v_perp = a (sin, cos): (B1 v1)^2 + (B2 v2)^2 = a^4 (sin^4 +
    cos^4), whose mean over a period is 3 a^4 / 4."""
    n, a = 256, 0.1
    ph = 2 * np.pi * (np.arange(n) + 0.5) / n
    cons = np.zeros((5, 1, 1, n))
    cons[0] = 2.0
    cons[2, 0, 0] = 2.0 * a * np.sin(ph)
    cons[3, 0, 0] = 2.0 * a * np.cos(ph)
    b = np.zeros((3, 1, 1, n))
    b[0] = 1.0
    b[1, 0, 0] = a * np.sin(ph)
    b[2, 0, 0] = a * np.cos(ph)
    got = D.transverse_flux_rms(cons, b, np.array([0.0, 1, 0]), np.array([0.0, 0, 1]))
    assert abs(got - np.sqrt(0.75) * a * a) < 1e-15


def test_mode_amplitude_picks_one_mode():
    n = 16
    x = (np.arange(n) + 0.5) / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    f = np.zeros((3, n, n, n))
    f[2] = 0.3 * np.sin(2 * np.pi * (X + 2 * Y + 2 * Z) + 0.4) + 0.1 * np.cos(2 * np.pi * 3 * X) + 5.0
    assert abs(D.mode_amplitude(f, (0, 0, 1), (1, 2, 2)) - 0.3) < 1e-14
    assert abs(D.mode_amplitude(f, (0, 0, 1), (3, 0, 0)) - 0.1) < 1e-14


def test_eigenmode_amplitudes_of_a_pure_mode():
    """A single linear mode set up by inputs.plane_wave_state projects onto
    that mode only, with its amplitude."""
    from paper_1812_04278_gb300 import inputs as I
    Bw = (1.0, np.sqrt(2.0), 0.5)
    _, vecs = I.linear_mhd_modes(1.0, 0.0, *Bw, 1.0)
    for m in (0, 1, 2, 6):
        cons, bface = I.plane_wave_state((16, 16, 16), (1.0, 1.0, 1.0), (1, 2, 2), 1.0, (0.0, 0.0, 0.0), Bw, 1.0,
                                         vecs[m], 1e-6)
        bc = I.face_to_cell_6th(bface)
        a = D.eigenmode_amplitudes(cons, bc, (1, 2, 2), 1.0, Bw, 1.0)
        assert abs(a[m] - 1e-6) < 2e-8, (m, a)
        others = np.delete(a, m)
        assert others.max() < 2e-8, (m, a)
