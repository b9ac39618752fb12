"""Seeded synthetic initial conditions for the WENO5-CT MHD solver.

This module builds problem set-ups only: it holds none of the scheme's
arithmetic (no fluxes, eigenvectors, WENO, CT or RK).  Both the CUDA path
and the CPU oracle take their inputs from here, so the same arrays go to
both sides.  All arrays are float64 numpy arrays shaped
``(n_fields, nz, ny, nx)`` with x fastest:

* ``cons``  = (rho, m_x, m_y, m_z, E) at cell centres,
* ``bface`` = (b_x at (i+1/2, j, k), b_y at (i, j+1/2, k), b_z at (i, j, k+1/2)).

Grid (Sec. 2 of the paper): cell centres at (i + 1/2) dx, faces at i dx,
periodic in every direction.  Face fields are built from an edge-centred
vector potential with the first-order discrete curl (Sec. 4.1), so their
discrete divergence vanishes up to rounding.  The total energy uses Eq. (P),
E = P/(gamma-1) + (rho v^2 + B^2)/2, with the cell-centred field taken from
the faces by the sixth-order interpolation the paper uses for initial
conditions (Sec. 4.14, weights (3,-25,150,150,-25,3)/256).
"""
from __future__ import annotations

import numpy as np

GAMMA = 5.0 / 3.0

# --------------------------------------------------------------------------
# basic helpers
# --------------------------------------------------------------------------


def _shift(a: np.ndarray, axis_xyz: int, s: int) -> np.ndarray:
    """a[..., i+s] along the x (0), y (1) or z (2) axis, periodic."""
    ax = a.ndim - 1 - axis_xyz
    return np.roll(a, -s, axis=ax)


def curl_edges_to_faces(Ax, Ay, Az, dx):
    """First-order discrete curl of an edge vector potential.

    Ax at (i, j+1/2, k+1/2), Ay at (i+1/2, j, k+1/2), Az at (i+1/2, j+1/2, k);
    returns (b_x, b_y, b_z) on the forward faces."""
    hx, hy, hz = dx
    bx = (Az - _shift(Az, 1, -1)) / hy - (Ay - _shift(Ay, 2, -1)) / hz
    by = (Ax - _shift(Ax, 2, -1)) / hz - (Az - _shift(Az, 0, -1)) / hx
    bz = (Ay - _shift(Ay, 0, -1)) / hx - (Ax - _shift(Ax, 1, -1)) / hy
    return bx, by, bz


def face_to_cell_6th(bface: np.ndarray) -> np.ndarray:
    """Sixth-order face -> centre interpolation used for initial conditions."""
    w = np.array([3.0, -25.0, 150.0, 150.0, -25.0, 3.0]) / 256.0
    out = np.zeros_like(bface)
    for d in range(3):
        b = bface[d]
        acc = np.zeros_like(b)
        for o, wt in zip(range(-3, 3), w):      # faces i-5/2 .. i+5/2 = index i-3 .. i+2
            acc += wt * _shift(b, d, o)
        out[d] = acc
    return out


def energy(rho, v, P, Bc, gamma=GAMMA):
    """Eq. (P): total energy from primitives and the cell-centred field."""
    return P / (gamma - 1.0) + 0.5 * rho * np.sum(v * v, axis=0) + 0.5 * np.sum(Bc * Bc, axis=0)


def assemble(rho, v, P, bface, gamma=GAMMA, Bc=None):
    """Conserved cell state from primitives and face fields."""
    if Bc is None:
        Bc = face_to_cell_6th(bface)
    cons = np.stack([rho, rho * v[0], rho * v[1], rho * v[2], energy(rho, v, P, Bc, gamma)])
    return np.ascontiguousarray(cons), np.ascontiguousarray(bface)


def cell_centres(shape, L=(1.0, 1.0, 1.0)):
    nx, ny, nz = shape
    dx = (L[0] / nx, L[1] / ny, L[2] / nz)
    x = (np.arange(nx) + 0.5) * dx[0]
    y = (np.arange(ny) + 0.5) * dx[1]
    z = (np.arange(nz) + 0.5) * dx[2]
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z, dx


# --------------------------------------------------------------------------
# uniform and plane-wave states
# --------------------------------------------------------------------------


def uniform_state(shape, rho=1.0, v=(0.0, 0.0, 0.0), B=(0.0, 0.0, 0.0), P=1.0, gamma=GAMMA):
    nx, ny, nz = shape
    o = np.ones((nz, ny, nx))
    vv = np.stack([o * v[0], o * v[1], o * v[2]])
    bface = np.stack([o * B[0], o * B[1], o * B[2]])
    Bc = bface.copy()
    return assemble(o * rho, vv, o * P, bface, gamma, Bc=Bc)


def linear_mhd_modes(rho, v_par, B_par, B_perp1, B_perp2, P, gamma=GAMMA):
    """Plane-wave modes of the ideal-MHD equations linearised about a
    uniform state, written in the wave frame (par, perp1, perp2).

    The primitive-variable system (rho, v_par, v_p1, v_p2, B_p1, B_p2, P)
    of the textbook ideal-MHD equations is diagonalised numerically;
    each eigenvector is mapped to conserved-variable perturbations
    (rho, m_par, m_p1, m_p2, B_p1, B_p2, E) to first order and scaled to
    unit Euclidean norm with a non-negative first non-zero entry.
    Returns (speeds, vectors) sorted by speed (ascending)."""
    A = np.zeros((7, 7))
    v, Bn, By, Bz = v_par, B_par, B_perp1, B_perp2
    # rho_t + v rho_x + rho u_x = 0
    A[0, 0] = v; A[0, 1] = rho
    # u_t + v u_x + P_x/rho + (By By_x + Bz Bz_x)/rho = 0
    A[1, 1] = v; A[1, 6] = 1.0 / rho; A[1, 4] = By / rho; A[1, 5] = Bz / rho
    # (vy)_t + v vy_x - Bn By_x/rho = 0
    A[2, 2] = v; A[2, 4] = -Bn / rho
    A[3, 3] = v; A[3, 5] = -Bn / rho
    # By_t + By u_x - Bn vy_x + v By_x = 0
    A[4, 1] = By; A[4, 2] = -Bn; A[4, 4] = v
    A[5, 1] = Bz; A[5, 3] = -Bn; A[5, 5] = v
    # P_t + gamma P u_x + v P_x = 0
    A[6, 1] = gamma * P; A[6, 6] = v
    lam, X = np.linalg.eig(A)
    lam = lam.real
    X = X.real
    order = np.argsort(lam)
    lam, X = lam[order], X[:, order]
    out = np.zeros((7, 7))
    for m in range(7):
        d = X[:, m]
        drho, du, dvy, dvz, dBy, dBz, dP = d
        vel = np.array([v, 0.0, 0.0])
        dvel = np.array([du, dvy, dvz])
        dm = vel * drho + rho * dvel
        dE = dP / (gamma - 1.0) + 0.5 * (vel @ vel) * drho + rho * (vel @ dvel) + By * dBy + Bz * dBz
        c = np.array([drho, dm[0], dm[1], dm[2], dBy, dBz, dE])
        c /= np.linalg.norm(c)
        nz_ = np.nonzero(np.abs(c) > 1e-12)[0]
        if len(nz_) and c[nz_[0]] < 0:
            c = -c
        out[m] = c
    return lam, out


def wave_frame(khat):
    """Right-handed orthonormal frame (par, perp1, perp2) with par = khat,
    perp1 = normalise(z x khat) (or y x khat if khat is along z)."""
    k = np.asarray(khat, dtype=np.float64)
    k = k / np.linalg.norm(k)
    ref = np.array([0.0, 0.0, 1.0]) if abs(k[2]) < 0.9 else np.array([0.0, 1.0, 0.0])
    p1 = np.cross(ref, k)
    p1 /= np.linalg.norm(p1)
    p2 = np.cross(k, p1)
    return k, p1, p2


def plane_wave_state(shape, L, kint, rho0, v_wave, B_wave, P0, dQ_wave, amp, gamma=GAMMA):
    """Uniform background plus amp * dQ * sin(k.x) in conserved variables
    (the paper's linear-wave set-up, Sec. 4.1: the perturbation is added
    once per conserved component).

    kint      integer wave numbers per box length, k = 2 pi kint / L;
    v_wave, B_wave  background velocity / field in the wave frame;
    dQ_wave   conserved perturbation (rho, m_par, m_p1, m_p2, B_p1, B_p2, E).
    Face fields: uniform background plus the discrete curl of the edge
    vector potential of the perturbation."""
    nx, ny, nz = shape
    L = tuple(float(l) for l in L)
    kvec = 2.0 * np.pi * np.asarray(kint, dtype=np.float64) / np.asarray(L)
    kmag = np.linalg.norm(kvec)
    par, p1, p2 = wave_frame(kvec)
    R = np.stack([par, p1, p2], axis=1)            # columns: frame vectors in lab coords
    v_lab = R @ np.asarray(v_wave, dtype=np.float64)
    B_lab = R @ np.asarray(B_wave, dtype=np.float64)
    X, Y, Z, dx = cell_centres(shape, L)
    ph = kvec[0] * X + kvec[1] * Y + kvec[2] * Z
    s = np.sin(ph)
    dQ = np.asarray(dQ_wave, dtype=np.float64)
    dm_lab = R @ dQ[1:4]
    dB_lab = dQ[4] * p1 + dQ[5] * p2
    rho = rho0 + amp * dQ[0] * s
    m = np.stack([rho0 * v_lab[i] + amp * dm_lab[i] * s for i in range(3)])
    Bc_bg = B_lab
    v2 = float(v_lab @ v_lab)
    E0 = P0 / (gamma - 1.0) + 0.5 * rho0 * v2 + 0.5 * float(Bc_bg @ Bc_bg)
    E = E0 + amp * dQ[6] * s
    # edge vector potential of the perturbation: dA = -(amp/k) cos(k.x) (dB_p2 p1 - dB_p1 p2)
    a_vec = -(amp / kmag) * (dQ[5] * p1 - dQ[4] * p2)
    hx, hy, hz = dx
    # edge positions: Ax at (i, j+1/2, k+1/2), Ay at (i+1/2, j, k+1/2),
    # Az at (i+1/2, j+1/2, k); X, Y, Z are the cell centres
    def phase(x, y, z):
        return kvec[0] * x + kvec[1] * y + kvec[2] * z
    Ax = a_vec[0] * np.cos(phase(X, Y + 0.5 * hy, Z + 0.5 * hz))
    Ay = a_vec[1] * np.cos(phase(X + 0.5 * hx, Y, Z + 0.5 * hz))
    Az = a_vec[2] * np.cos(phase(X + 0.5 * hx, Y + 0.5 * hy, Z))
    bx, by, bz = curl_edges_to_faces(Ax, Ay, Az, dx)
    bface = np.stack([bx + B_lab[0], by + B_lab[1], bz + B_lab[2]])
    cons = np.stack([rho, m[0], m[1], m[2], E])
    return np.ascontiguousarray(cons), np.ascontiguousarray(bface)


def fast_wave_config(shape=(32, 32, 32), amp=1e-6, gamma=GAMMA):
    """Fast magnetosonic eigenmode of amplitude 1e-6 along (1,2,2)/3 with
    wavelength 1/3 in the unit box: rho=1, P=1, v=0, B=(1, sqrt2, 1/2) in the
    wave frame (par, perp1, perp2)."""
    Bw = (1.0, np.sqrt(2.0), 0.5)
    lam, vecs = linear_mhd_modes(1.0, 0.0, *Bw, 1.0, gamma)
    dQ = vecs[6]      # fastest forward mode
    return plane_wave_state(shape, (1.0, 1.0, 1.0), (1, 2, 2), 1.0, (0.0, 0.0, 0.0), Bw, 1.0,
                            dQ, amp, gamma)


# --------------------------------------------------------------------------
# random spectral fields (turbulence-like states)
# --------------------------------------------------------------------------


def _kgrid(shape):
    nx, ny, nz = shape
    kx = np.fft.fftfreq(nx) * nx
    ky = np.fft.fftfreq(ny) * ny
    kz = np.fft.rfftfreq(nz) * nz
    KX, KY, KZ = np.meshgrid(kx, ky, kz, indexing="ij")
    return KX, KY, KZ


def random_spectral_vector(shape, rng, kmin, kmax, slope_amp, solenoidal=True):
    """Gaussian random-phase vector field with mode amplitude |k|^slope_amp
    for kmin <= |k| <= kmax (integer wave numbers), real, zero mean.
    Returned in Fourier space (3, nx, ny, nz//2+1) on the (x, y, z) grid."""
    KX, KY, KZ = _kgrid(shape)
    K = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    mask = (K >= kmin) & (K <= kmax)
    amp = np.zeros_like(K)
    amp[mask] = K[mask] ** slope_amp
    F = np.empty((3,) + K.shape, dtype=np.complex128)
    for c in range(3):
        F[c] = (rng.standard_normal(K.shape) + 1j * rng.standard_normal(K.shape)) * amp
    if solenoidal:
        Ks = np.where(K > 0, K, 1.0)
        kd = (KX * F[0] + KY * F[1] + KZ * F[2]) / Ks ** 2
        F[0] -= KX * kd
        F[1] -= KY * kd
        F[2] -= KZ * kd
    return F, (KX, KY, KZ)


def _irfft(Fc, shape, shift=(0.0, 0.0, 0.0)):
    """Inverse transform of one component; shift = offsets in cells at
    which the field is sampled (x, y, z).  Output (nz, ny, nx)."""
    nx, ny, nz = shape
    KX, KY, KZ = _kgrid(shape)
    ph = np.exp(2j * np.pi * (KX * shift[0] / nx + KY * shift[1] / ny + KZ * shift[2] / nz))
    f = np.fft.irfftn(Fc * ph, s=(nx, ny, nz), axes=(0, 1, 2))
    return np.ascontiguousarray(np.transpose(f, (2, 1, 0)))


def turbulent_state(N, seed=1812, seed_b=1813, mach=1.0, beta=1.0, dB_frac=0.1, kmin=2, kmax=32,
                    rho0=1.0, gamma=GAMMA, B_dir=(1.0, 0.0, 0.0), P0=None, shape=None):
    """Turbulence-like periodic state in the unit box:
    rho = rho0, P = P0 (default 1/gamma, so c_s = 1), mean field B0 * B_dir
    with beta = 2 P / B0^2; solenoidal Gaussian random-phase velocity with
    energy spectrum k^-5/3 (mode amplitude |k|^-11/6) for kmin <= |k| <= kmax,
    scaled to rms Mach number `mach`; field perturbation dB = curl A on the
    edges with the same k^-5/3 spectrum for dB, scaled to rms |dB| =
    dB_frac * B0."""
    shape = (N, N, N) if shape is None else tuple(shape)
    nx, ny, nz = shape
    if P0 is None:
        P0 = 1.0 / gamma
    cs = np.sqrt(gamma * P0 / rho0)
    B0 = np.sqrt(2.0 * P0 / beta)
    bdir = np.asarray(B_dir, dtype=np.float64)
    bdir = bdir / np.linalg.norm(bdir)
    dx = (1.0 / nx, 1.0 / ny, 1.0 / nz)

    rng = np.random.default_rng(seed)
    Fv, _ = random_spectral_vector(shape, rng, kmin, kmax, -11.0 / 6.0, solenoidal=True)
    v = np.stack([_irfft(Fv[c], shape) for c in range(3)])
    v *= mach * cs / np.sqrt(np.mean(np.sum(v * v, axis=0)))

    rng_b = np.random.default_rng(seed_b)
    FA, (KX, KY, KZ) = random_spectral_vector(shape, rng_b, kmin, kmax, -11.0 / 6.0 - 1.0, solenoidal=True)
    # edges relative to the cell centre of index (i, j, k), in cells:
    # Ax at (0, 1/2, 1/2), Ay at (1/2, 0, 1/2), Az at (1/2, 1/2, 0)
    Ax = _irfft(FA[0], shape, (0.0, 0.5, 0.5))
    Ay = _irfft(FA[1], shape, (0.5, 0.0, 0.5))
    Az = _irfft(FA[2], shape, (0.5, 0.5, 0.0))
    bx, by, bz = curl_edges_to_faces(Ax, Ay, Az, dx)
    db = np.stack([bx, by, bz])
    rms = np.sqrt(np.mean(np.sum(db * db, axis=0)))
    db *= (dB_frac * B0 / rms) if rms > 0 else 0.0
    bface = db + (B0 * bdir)[:, None, None, None]
    rho = np.full((nz, ny, nx), rho0)
    P = np.full((nz, ny, nx), P0)
    return assemble(rho, v, P, bface, gamma)


def random_smooth_state(shape, seed, mach=0.5, beta=1.0, dB_frac=0.3, drho=0.2, kmax=3,
                        gamma=GAMMA, B_dir=(1.0, 0.5, -0.3)):
    """Small smooth random state for parity tests: a few low Fourier modes
    in velocity, density, pressure and the vector potential; O(1) values in
    every field."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    cons, bface = turbulent_state(None, seed=int(rng.integers(1 << 30)), seed_b=int(rng.integers(1 << 30)),
                                  mach=mach, beta=beta, dB_frac=dB_frac, kmin=1, kmax=kmax,
                                  gamma=gamma, B_dir=B_dir, shape=shape)
    X, Y, Z, _ = cell_centres(shape)
    a = rng.uniform(0, 2 * np.pi, 6)
    rho = 1.0 + drho * np.sin(2 * np.pi * X + a[0]) * np.cos(2 * np.pi * Y + a[1]) \
        + 0.5 * drho * np.sin(2 * np.pi * Z + a[2])
    P = (1.0 / gamma) * (1.0 + drho * np.cos(2 * np.pi * (X + Y) + a[3]) + 0.5 * drho * np.sin(2 * np.pi * Z + a[4]))
    v = cons[1:4] / cons[0]
    return assemble(rho, v, P, bface, gamma)


def analytic_smooth_state(shape, seed=0, amp=0.2, gamma=GAMMA, dtype=np.float64):
    """Large smooth state without FFTs (for grids where spectral synthesis is
    too slow): a few separable sine modes in rho, v and P and an edge vector
    potential A_i = a sin(2 pi (k.x) + phi) sampled at the edges, plus a
    uniform mean field.  All fields O(1); div b = 0 to rounding."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    ph = rng.uniform(0, 2 * np.pi, 16)
    hx, hy, hz = 1.0 / nx, 1.0 / ny, 1.0 / nz
    x = ((np.arange(nx) + 0.5) * hx)[None, None, :]
    y = ((np.arange(ny) + 0.5) * hy)[None, :, None]
    z = ((np.arange(nz) + 0.5) * hz)[:, None, None]
    tp = 2 * np.pi
    rho = 1.0 + amp * np.sin(tp * x + ph[0]) * np.cos(tp * y + ph[1]) + 0.5 * amp * np.sin(tp * z + ph[2])
    P = (1.0 / gamma) * (1.0 + amp * np.cos(tp * y + ph[3]) * np.sin(tp * z + ph[4]) + 0.5 * amp * np.cos(tp * x + ph[5]))
    v = np.empty((3, nz, ny, nx), dtype=np.float64)
    v[0] = 0.5 * np.sin(tp * y + ph[6]) + 0.3 * np.cos(tp * z + ph[7]) + 0 * x
    v[1] = 0.5 * np.sin(tp * z + ph[8]) + 0.3 * np.cos(tp * x + ph[9]) + 0 * y
    v[2] = 0.5 * np.sin(tp * x + ph[10]) + 0.3 * np.cos(tp * y + ph[11]) + 0 * z
    a = 0.3 / tp
    # edges: Ax (i, j+1/2, k+1/2), Ay (i+1/2, j, k+1/2), Az (i+1/2, j+1/2, k)
    Ax = a * np.sin(tp * (y + 0.5 * hy) + ph[12]) * np.cos(tp * (z + 0.5 * hz) + ph[13]) + 0 * x
    Ay = a * np.sin(tp * (z + 0.5 * hz) + ph[14]) * np.cos(tp * (x + 0.5 * hx) + ph[15]) + 0 * y
    Az = a * np.sin(tp * (x + 0.5 * hx) + ph[12]) * np.cos(tp * (y + 0.5 * hy) + ph[14]) + 0 * z
    bx, by, bz = curl_edges_to_faces(Ax, Ay, Az, (hx, hy, hz))
    bface = np.stack([bx + 0.8, by + 0.4, bz - 0.5])
    del Ax, Ay, Az, bx, by, bz
    cons, bface = assemble(rho, v, P, bface, gamma)
    return cons.astype(dtype, copy=False), bface.astype(dtype, copy=False)


def blast_turbulence_state(N, seed=1815, seed_b=1816, mach=5.0, p_amb=0.1, p_blast=100.0, r_blast=0.05,
                           dB_frac=0.1, kmin=2, kmax=32, gamma=GAMMA):
    """Magnetised blast in a turbulent background (the paper's blast test,
    Sec. 4.16, in a turbulent medium): rho = 1, ambient P = p_amb, uniform
    field B = (1, 1, 1)/sqrt3 (beta = 2 p_amb / |B|^2), solenoidal k^-5/3
    velocity at rms Mach `mach` with respect to the ambient sound speed, a
    10% rms field perturbation, and P = p_blast inside r < r_blast of the
    box centre (top hat at cell centres)."""
    shape = (N, N, N)
    B0 = 1.0
    beta = 2.0 * p_amb / B0 ** 2
    cons, bface = turbulent_state(N, seed=seed, seed_b=seed_b, mach=mach, beta=beta, dB_frac=dB_frac, kmin=kmin,
                                  kmax=min(kmax, N // 2 - 1), gamma=gamma, B_dir=(1.0, 1.0, 1.0), P0=p_amb)
    X, Y, Z, _ = cell_centres(shape)
    r2 = (X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2
    inside = r2 < r_blast ** 2
    # raise the pressure inside the sphere: E grows by (p_blast - p_amb)/(gamma - 1)
    cons[4] += np.where(inside, (p_blast - p_amb) / (gamma - 1.0), 0.0)
    return cons, bface


PATCH_SIZES = (16, 24, 32, 48, 64)


def patch_batch_spec(npatch=512, seed=1803, sizes=PATCH_SIZES, mach=(0.5, 3.0), beta=(0.1, 10.0)):
    """Sizes and turbulence parameters of a batch of independent periodic
    patches: each of (nx, ny, nz) drawn uniformly from `sizes`, rms Mach
    uniform in `mach`, beta log-uniform in `beta`, mean field along a random
    unit vector, and two seeds per patch for its velocity and field draws.
    Every patch is a unit box (dx = 1/nx, dy = 1/ny, dz = 1/nz)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(npatch):
        shape = tuple(int(s) for s in rng.choice(np.asarray(sizes), size=3))
        m = float(rng.uniform(mach[0], mach[1]))
        b = float(np.exp(rng.uniform(np.log(beta[0]), np.log(beta[1]))))
        d = rng.standard_normal(3)
        d = d / np.linalg.norm(d)
        s1, s2 = (int(v) for v in rng.integers(1 << 30, size=2))
        out.append(dict(shape=shape, dx=tuple(1.0 / n for n in shape), mach=m, beta=b, B_dir=tuple(float(v) for v in d),
                        seed=s1, seed_b=s2))
    return out


def patch_state(spec, gamma=GAMMA, dB_frac=0.1, kmin=2):
    """Turbulent state of one patch of patch_batch_spec: rho = 1, P = 1/gamma,
    k^-5/3 velocity and field perturbation for kmin <= |k| <= max(kmin, min(n)/8)
    (wavelengths of at least 8 cells, as 2 <= k <= 32 on a 256^3 grid)."""
    kmax = max(kmin, min(spec["shape"]) // 8)
    return turbulent_state(None, seed=spec["seed"], seed_b=spec["seed_b"], mach=spec["mach"], beta=spec["beta"],
                           dB_frac=dB_frac, kmin=kmin, kmax=kmax, gamma=gamma, B_dir=spec["B_dir"],
                           shape=spec["shape"])


# --------------------------------------------------------------------------
# parametrised initial state (the adjoint workload)
# --------------------------------------------------------------------------


def ic_from_potential(rho, v, P, A, B0, dx, gamma=GAMMA):
    """Conserved state and face field from primitive fields and an edge
    vector potential: b = curl A + B0 (first-order discrete curl, edges as in
    curl_edges_to_faces), E from Eq. (P) with the sixth-order face -> centre
    interpolation of Sec. 4.14."""
    bx, by, bz = curl_edges_to_faces(A[0], A[1], A[2], dx)
    bface = np.stack([bx + B0[0], by + B0[1], bz + B0[2]])
    return assemble(rho, v, P, bface, gamma)


def cpaw_overpressure(shape, amp=0.1, kint=(1, 2, 2), p0=0.1, peak=10.0, r0=0.1, rho0=1.0):
    """Primitive fields and edge vector potential of a circularly polarised
    Alfven wave (Sec. 4.2 set-up: rho = 1, B_par = 1, P = 0.1, v_perp =
    B_perp = amp (sin phi, cos phi) in the wave frame) travelling along
    k = 2 pi kint in the unit box, plus a Gaussian overpressure
    P = p0 (1 + (peak - 1) exp(-r^2 / r0^2)) about the box centre.  The
    transverse field comes from A = (amp/|k|) (e1 sin phi + e2 cos phi) on the
    edges, so b = curl A + B0 is discretely divergence free.  Returns
    (rho, v, P, A, B0)."""
    nx, ny, nz = shape
    khat, e1, e2 = wave_frame(kint)
    kvec = 2.0 * np.pi * np.asarray(kint, dtype=np.float64)
    kmag = np.linalg.norm(kvec)
    X, Y, Z, dx = cell_centres(shape)
    ph = kvec[0] * X + kvec[1] * Y + kvec[2] * Z
    v = amp * (np.sin(ph)[None] * e1[:, None, None, None] + np.cos(ph)[None] * e2[:, None, None, None])
    r2 = (X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2
    P = p0 * (1.0 + (peak - 1.0) * np.exp(-r2 / r0 ** 2))
    rho = np.full((nz, ny, nx), rho0)
    hx, hy, hz = dx
    # edges: A_x at (i, j+1/2, k+1/2), A_y at (i+1/2, j, k+1/2), A_z at (i+1/2, j+1/2, k) from the centre
    shifts = [(0.0, 0.5 * hy, 0.5 * hz), (0.5 * hx, 0.0, 0.5 * hz), (0.5 * hx, 0.5 * hy, 0.0)]
    A = np.empty((3, nz, ny, nx))
    for c, (sx, sy, sz) in enumerate(shifts):
        phe = kvec[0] * (X + sx) + kvec[1] * (Y + sy) + kvec[2] * (Z + sz)
        a = (amp / kmag) * (np.sin(phe) * e1[c] + np.cos(phe) * e2[c])
        A[c] = a
    B0 = tuple(float(x) for x in khat)
    return rho, np.ascontiguousarray(v), P, A, B0


# --------------------------------------------------------------------------
# robustness problems (Secs. 4.3, 4.5, 4.14)
# --------------------------------------------------------------------------


def field_loop(shape=(128, 64, 1), L=(2.0, 1.0, 1.0), A0=1e-3, rc=0.3, v=(2.0, 1.0, 0.0), rho=1.0, P=1.0,
               gamma=GAMMA):
    """Magnetic field loop advection (Sec. 4.14): periodic L_x x L_y box,
    uniform rho, v, P, and b = curl (0, 0, A_z) with A_z = A0 (rc - r) for
    r < rc (0 outside) about the box centre, on the edges (i+1/2, j+1/2);
    cell field by the sixth-order interpolation (Sec. 4.14).  Returns
    (cons, bface, dx)."""
    nx, ny, nz = shape
    dx = (L[0] / nx, L[1] / ny, L[2] / nz)
    X, Y, Z, _ = cell_centres(shape, L)
    r = np.sqrt((X + 0.5 * dx[0] - 0.5 * L[0]) ** 2 + (Y + 0.5 * dx[1] - 0.5 * L[1]) ** 2)
    Az = np.where(r < rc, A0 * (rc - r), 0.0)
    zero = np.zeros_like(Az)
    bx, by, bz = curl_edges_to_faces(zero, zero, Az, dx)
    bface = np.stack([bx, by, bz])
    o = np.ones((nz, ny, nx))
    vv = np.stack([o * v[0], o * v[1], o * v[2]])
    cons, bface = assemble(rho * o, vv, P * o, bface, gamma)
    return cons, bface, dx


def magnetic_energy(bface, dx):
    """1/2 sum of the squared face fields times the cell volume."""
    return 0.5 * float(np.sum(bface * bface)) * dx[0] * dx[1] * dx[2]


# Riemann problems as printed (primitive U = (rho, v_x, v_y, v_z, B_x, B_y, B_z, P)).
_S4PI = np.sqrt(4.0 * np.pi)
# Sec. 4.3 prints seven entries for the left state; read as (rho, v_x, v_y,
# B_x, B_y, B_z, P) with v_z = 0 (the right state has all eight).
RJ2A = dict(left=(1.08, 1.2, 0.01, 0.0, 2.0 / _S4PI, 3.6 / _S4PI, 2.0 / _S4PI, 0.95),
            right=(1.0, 0.0, 0.0, 0.0, 2.0 / _S4PI, 4.0 / _S4PI, 2.0 / _S4PI, 1.0), gamma=5.0 / 3.0, t_end=0.2)
# Sec. 4.5, as printed (both densities 0.125), gamma = 2.
BRIO_WU = dict(left=(0.125, 0.0, 0.0, 0.0, 0.75, 1.0, 0.0, 1.0),
               right=(0.125, 0.0, 0.0, 0.0, 0.75, -1.0, 0.0, 0.1), gamma=2.0, t_end=0.08)


def shock_tube(problem, n, transverse=(4, 4)):
    """Riemann problem along x on a periodic box of length 2 (n cells along
    x, `transverse` cells in y and z, unit cross-section): the left state on
    [0, 0.5) and [1.5, 2), the right state on [0.5, 1.5), so that the
    interface at x = 0.5 is the printed problem and the one at 1.5 its
    reverse; until t_end their waves stay apart.  B_x is the same on both
    sides, so the face field is divergence free.  Returns (cons, bface, dx,
    gamma)."""
    ny, nz = transverse
    shape = (n, ny, nz)
    L = (2.0, 1.0, 1.0)
    dx = (L[0] / n, L[1] / ny, L[2] / nz)
    X, _, _, _ = cell_centres(shape, L)
    left = (X < 0.5) | (X >= 1.5)
    UL, UR = np.asarray(problem["left"]), np.asarray(problem["right"])
    U = np.where(left[None], UL[:, None, None, None], UR[:, None, None, None])
    rho, v, Bc, P = U[0], U[1:4], U[4:7], U[7]
    # fields vary along x only: b_y, b_z on their faces equal the cell values,
    # b_x is uniform
    bface = np.stack([np.full_like(rho, UL[4]), Bc[1], Bc[2]])
    cons, bface = assemble(rho, v, P, bface, problem["gamma"], Bc=Bc)
    return cons, bface, dx, problem["gamma"]
