"""Element-wise checks of the adjoint against the oracle (libw5ct through the
C ABI; the oracle has no adjoint, so its central differences stand in).

On a tiny periodic grid, 8 x 6 x 5 cells (ragged against every tile; the
5-cell axis makes the six-point stencil wrap onto itself, so two stencil
slots of one face hold the same cell and the adjoint must add both), every
component of the gradient is compared with the oracle's central difference
in that component alone:

* the rollout misfit (two fixed-dt RK4 + CT steps, Secs. 2.1, 2.3) with
  respect to each of the 240 densities, 720 velocities and 720 edge
  potentials, through the autograd rollout (per-step checkpoints);
* one step's vector-Jacobian product <lam, S'(x) e_i> for each of the 1920
  components of (q, b) (w5ct_adjoint_step).

Each difference is taken with steps h and h/4 and combined by Richardson
extrapolation, c = (16 c(h/4) - c(h)) / 15; |c(h/4) - c(h)| bounds what is
left of its truncation error.  Where that estimate is small (the regular
components: all of them for WENO-JS) the bar is 1e-6 of the largest
component.  WENO-Z with eps_Z = 1e-40 has points of very large curvature
where a characteristic field is nearly uniform (its weights are a ratio of
tiny smoothness indicators); there the difference itself is uncertain, and
the bar is widened by its own error estimate, component by component.
The FP32-bulk gradient (float face arithmetic, double accumulation) is held
to an element-wise bound of 2e-4 of the largest component.
"""
import numpy as np
import pytest

import _oracle_fd as fd

pytestmark = pytest.mark.gpu

SHAPE = (8, 6, 5)
NSTEPS = 2
H = 1e-6
TOL = 1e-6          # FP64, relative to the largest gradient component
TOL32 = 2e-4        # FP32-bulk
REG = 1e-7          # |c(h/4) - c(h)| below REG * max|g|: a regular component


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_1812_04278_gb300 import build
    build.build()
    from paper_1812_04278_gb300 import adjoint, inputs, w5ct
    oracle.build()
    return dict(torch=torch, O=oracle, I=inputs, W=w5ct, A=adjoint)


def problem(env):
    """Smooth fields of a few low Fourier modes (every field varies, so no
    WENO-Z weight is a 0/0 ratio), an oblique mean field, a target that
    differs from the state, and dt = half the oracle's CFL step."""
    I, O = env["I"], env["O"]
    nx, ny, nz = SHAPE
    dx = tuple(1.0 / n for n in SHAPE)
    X, Y, Z, _ = I.cell_centres(SHAPE)
    rng = np.random.default_rng(2024)
    tp = 2 * np.pi

    def modes(amp, n=3):
        f = np.zeros((nz, ny, nx))
        for _ in range(n):
            k = rng.integers(-1, 2, 3)
            ph = rng.uniform(0, tp)
            f += amp * rng.uniform(0.5, 1) * np.sin(tp * (k[0] * X + k[1] * Y + k[2] * Z) + ph)
        return f

    rho = 1.0 + modes(0.1)
    P = 0.6 + modes(0.05)
    v = np.stack([modes(0.3) for _ in range(3)])
    A = np.stack([modes(0.03) for _ in range(3)])
    B0 = (0.8, -0.5, 0.6)
    tc, tb = I.ic_from_potential(np.ones_like(rho), np.zeros_like(v), np.full_like(P, 0.6), 0.5 * A, B0, dx)
    q, b = I.ic_from_potential(rho, v, P, A, B0, dx)
    o = O.Oracle(SHAPE, dx, O.make_config())
    o.set_state(q, b)
    dt = 0.5 * o.cfl_dt()
    lam = np.random.default_rng(7)
    return dict(shape=SHAPE, dx=dx, rho=rho, v=v, P=P, A=A, B0=B0, tc=tc, tb=tb, q=q, b=b, dt=dt,
                nsteps=NSTEPS, lq=lam.standard_normal(q.shape), lb=lam.standard_normal(b.shape))


def cuda(env, *arrs):
    torch = env["torch"]
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


def solver(env, pb, precision, variant):
    W, torch = env["W"], env["torch"]
    return W.Solver(SHAPE, pb["dx"], W.make_config(precision=precision, weno_variant=variant),
                    stream=torch.cuda.current_stream().cuda_stream)


def rollout_gradient(env, pb, precision, variant):
    A = env["A"]
    s = solver(env, pb, precision, variant)
    rho, v, Av = (t.requires_grad_() for t in cuda(env, pb["rho"], pb["v"], pb["A"]))
    P, tc, tb = cuda(env, pb["P"], pb["tc"], pb["tb"])
    L = A.rollout_misfit(rho, v, Av, s, P, pb["B0"], tc, tb, pb["dt"], NSTEPS)
    L.backward()
    g = np.concatenate([rho.grad.cpu().numpy().ravel(), v.grad.cpu().numpy().ravel(), Av.grad.cpu().numpy().ravel()])
    s.close()
    return g


def compare(g, c1, c4, tol):
    """(max error / max|c|, number of regular components); asserts the bars."""
    cR = (16.0 * c4 - c1) / 15.0
    err = np.abs(c4 - c1)
    m = np.abs(cR).max()
    regular = err <= REG * m
    bar = tol * m + np.where(regular, 0.0, err)
    dev = np.abs(g - cR)
    worst = int(np.argmax(dev - bar))
    assert np.all(dev <= bar), (worst, g[worst], cR[worst], err[worst], m)
    return float(dev[regular].max() / m), int(regular.sum())


@pytest.fixture(scope="module")
def fd_rollout(env):
    pb = problem(env)
    return pb, {v: fd.central_differences("rollout", pb, v, H) for v in (0, 1)}


@pytest.mark.parametrize("variant", [0, 1])
def test_rollout_gradient_elementwise_vs_oracle(env, fd_rollout, variant):
    pb, fds = fd_rollout
    c1, c4 = fds[variant]
    g = rollout_gradient(env, pb, 0, variant)
    assert g.shape == c1.shape == (1680,)
    rel, nreg = compare(g, c1, c4, TOL)
    assert rel <= TOL
    if variant == 0:
        assert nreg == g.size          # WENO-JS: every component is regular
    else:
        assert nreg >= 0.9 * g.size


@pytest.mark.parametrize("variant", [0, 1])
def test_step_adjoint_elementwise_vs_oracle(env, variant):
    W = env["W"]
    pb = problem(env)
    c1, c4 = fd.central_differences("step", pb, variant, H)
    s = solver(env, pb, 0, variant)
    s.set_state(pb["q"], pb["b"])
    lq, lb = cuda(env, pb["lq"], pb["lb"])
    torch = env["torch"]
    oq, ob = torch.empty_like(lq), torch.empty_like(lb)
    W.w5ct_adjoint_step(s.ctx, pb["dt"], lq, lb, oq, ob)
    g = np.concatenate([oq.cpu().numpy().ravel(), ob.cpu().numpy().ravel()])
    assert g.shape == c1.shape == (1920,)
    rel, nreg = compare(g, c1, c4, TOL)
    assert rel <= TOL and nreg >= 0.9 * g.size
    s.close()


def test_fp32_rollout_gradient_elementwise_vs_oracle(env, fd_rollout):
    pb, fds = fd_rollout
    c1, c4 = fds[0]
    g = rollout_gradient(env, pb, 1, 0)
    cR = (16.0 * c4 - c1) / 15.0
    rel = np.abs(g - cR).max() / np.abs(cR).max()
    assert rel <= TOL32, rel
