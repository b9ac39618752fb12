"""The seeded input generators deliver the recipes they state (CPU only):
discretely divergence-free face fields, the stated density, pressure, rms
Mach number, mean field and field-perturbation level, solenoidal k^-5/3
velocities confined to the stated band, and the batch, blast and Alfven-wave
set-ups with their documented numbers."""
import numpy as np

from paper_1812_04278_gb300 import inputs as I

G = I.GAMMA


def primitives(cons, bface):
    rho = cons[0]
    v = cons[1:4] / rho
    Bc = I.face_to_cell_6th(bface)
    P = (G - 1.0) * (cons[4] - 0.5 * rho * np.sum(v * v, axis=0) - 0.5 * np.sum(Bc * Bc, axis=0))
    return rho, v, P


def div_b(bface):
    nz, ny, nx = bface.shape[1:]
    return ((bface[0] - np.roll(bface[0], 1, axis=2)) * nx + (bface[1] - np.roll(bface[1], 1, axis=1)) * ny
            + (bface[2] - np.roll(bface[2], 1, axis=0)) * nz)


def shell_spectrum(v):
    n = v.shape[1]
    F = np.fft.fftn(v, axes=(1, 2, 3)) / n ** 3
    k = np.fft.fftfreq(n, 1.0 / n)
    KZ, KY, KX = np.meshgrid(k, k, k, indexing="ij")
    K = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    e = 0.5 * np.sum(np.abs(F) ** 2, axis=0)
    div = np.abs(KX * F[0] + KY * F[1] + KZ * F[2])
    return K, e, div, np.sqrt(np.sum(np.abs(F) ** 2, axis=0)) * np.maximum(K, 1.0)


def test_turbulence_recipe():
    n = 64
    cons, bface = I.turbulent_state(n, seed=1812, seed_b=1813, mach=1.0, beta=1.0, dB_frac=0.1, kmin=2, kmax=32)
    rho, v, P = primitives(cons, bface)
    B0 = np.sqrt(2.0 / G)
    assert np.all(rho == 1.0)
    assert np.abs(P - 1.0 / G).max() < 1e-12
    assert abs(np.sqrt(np.mean(np.sum(v * v, axis=0))) - 1.0) < 1e-12          # rms Mach 1 at c_s = 1
    mean_b = bface.reshape(3, -1).mean(axis=1)
    assert np.allclose(mean_b, [B0, 0.0, 0.0], atol=1e-12)
    db = bface - mean_b[:, None, None, None]
    assert abs(np.sqrt(np.mean(np.sum(db * db, axis=0))) - 0.1 * B0) < 1e-12
    assert np.abs(div_b(bface)).max() < 1e-11
    K, e, div, scale = shell_spectrum(v)
    live = e > 1e-12 * e.max()                                                # modes that carry energy
    assert (div[live] / scale[live]).max() < 1e-9                             # solenoidal
    out = (K < 2 - 1e-9) | (K > 32 + 1e-9)
    assert e[out].sum() < 1e-20 * e.sum()                                     # band 2 <= |k| <= 32
    shells = np.arange(4, 31)
    E = np.array([e[(K >= s - 0.5) & (K < s + 0.5)].sum() for s in shells])
    slope = np.polyfit(np.log(shells), np.log(E), 1)[0]
    assert abs(slope - (-5.0 / 3.0)) < 0.2, slope


def test_batch_recipe():
    spec = I.patch_batch_spec(512, seed=1803)
    assert spec == I.patch_batch_spec(512, seed=1803)                        # seeded
    assert sum(int(np.prod(s["shape"])) for s in spec) == 23_908_864
    for s in spec:
        assert all(n in I.PATCH_SIZES for n in s["shape"])
        assert 0.5 <= s["mach"] <= 3.0 and 0.1 <= s["beta"] <= 10.0
        assert abs(np.linalg.norm(s["B_dir"]) - 1.0) < 1e-12
        assert s["dx"] == tuple(1.0 / n for n in s["shape"])
    s = next(x for x in spec if min(x["shape"]) == 16)
    cons, bface = I.patch_state(s)
    rho, v, P = primitives(cons, bface)
    assert np.abs(P - 1.0 / G).max() < 1e-12
    assert abs(np.sqrt(np.mean(np.sum(v * v, axis=0))) - s["mach"]) < 1e-12
    assert np.abs(div_b(bface)).max() < 1e-11


def test_blast_recipe():
    n = 32
    cons, bface = I.blast_turbulence_state(n)
    rho, v, P = primitives(cons, bface)
    X, Y, Z, _ = I.cell_centres((n, n, n))
    inside = (X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2 < 0.05 ** 2
    assert inside.sum() > 0
    assert np.abs(P[inside] - 100.0).max() < 1e-10 and np.abs(P[~inside] - 0.1).max() < 1e-12
    mean_b = bface.reshape(3, -1).mean(axis=1)
    assert np.allclose(mean_b, np.ones(3) / np.sqrt(3.0), atol=1e-12)
    assert abs(np.sqrt(np.mean(np.sum(v * v, axis=0))) - 5.0 * np.sqrt(G * 0.1)) < 1e-12
    assert np.abs(div_b(bface)).max() < 1e-10


def test_alfven_wave_with_overpressure_recipe():
    n = 32
    shape, dx = (n, n, n), (1.0 / n,) * 3
    rho, v, P, A, B0 = I.cpaw_overpressure(shape)
    cons, bface = I.ic_from_potential(rho, v, P, A, B0, dx)
    assert np.all(rho == 1.0)
    assert np.abs(np.sqrt(np.sum(v * v, axis=0)) - 0.1).max() < 1e-14      # |v_perp| = amplitude
    khat = np.array([1.0, 2.0, 2.0]) / 3.0
    assert np.abs(np.tensordot(khat, v, axes=(0, 0))).max() < 1e-15        # transverse
    # 10x peak on 0.1 about the box centre (the nearest cell centres sit
    # sqrt(3)/64 from it, where the Gaussian of radius 0.1 is 0.93)
    assert 0.9 < P.max() <= 1.0 and abs(P.min() - 0.1) < 1e-6
    X, Y, Z, _ = I.cell_centres(shape)
    r2 = (X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2
    assert P.flat[np.argmax(P)] == P.max() and r2.flat[np.argmax(P)] == r2.min()
    assert np.allclose(bface.reshape(3, -1).mean(axis=1), khat, atol=1e-12)
    assert np.abs(div_b(bface)).max() < 1e-12
