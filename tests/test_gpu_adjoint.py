"""Adjoint of the step and of the rollout misfit (libw5ct through the C ABI).

Checked against central finite differences of the GPU path itself and of
the CPU oracle (which has no adjoint of its own): a directional derivative
g . delta from the adjoint must equal (L(x + h delta) - L(x - h delta)) / 2h
to 1e-6 relative in FP64.  The step map is smooth away from the branches of
max(), |.| and the eps_B switches, which random directions do not hit at
h = 1e-6 on these states.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SHAPE = (16, 12, 10)       # nx, ny, nz: ragged against every tile, three axes differ
NSTEPS = 3
H = 1e-6


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


def problem(env, shape=SHAPE, texture=0.02):
    """CPAW + overpressure parameters, the target (the wave without the
    overpressure) and a fixed dt from the oracle's CFL condition.

    WENO-Z with eps_Z = 1e-40 is not differentiable where a characteristic
    field is locally constant (its weights are a 0/0 ratio there, so the
    step is only directionally differentiable and a central difference sees
    the nonlinear weights of the perturbation); the CPAW has uniform rho and
    P.  The finite-difference checks therefore add a smooth texture of
    relative amplitude `texture` to rho and P, so that every field varies by
    far more than the perturbation h * delta."""
    I, O = env["I"], env["O"]
    dx = tuple(1.0 / n for n in shape)
    rho, v, P, A, B0 = I.cpaw_overpressure(shape)
    P_wave = I.cpaw_overpressure(shape, peak=1.0)[2]
    if texture:
        X, Y, Z, _ = I.cell_centres(shape)
        ph = np.random.default_rng(42).uniform(0, 2 * np.pi, 6)
        tp = 2 * np.pi
        rho = rho * (1 + texture * (np.sin(tp * X + ph[0]) + np.sin(tp * Y + ph[1]) + np.sin(tp * Z + ph[2])) / 3)
        f = 1 + texture * (np.cos(tp * X + ph[3]) + np.cos(tp * Y + ph[4]) + np.cos(tp * Z + ph[5])) / 3
        P, P_wave = P * f, P_wave * f
    tc, tb = I.ic_from_potential(rho, v, P_wave, A, B0, dx)
    cons, bface = I.ic_from_potential(rho, v, P, A, B0, dx)
    o = O.Oracle(shape, dx, O.make_config())
    o.set_state(cons, bface)
    dt = 0.5 * o.cfl_dt()
    return dict(shape=shape, dx=dx, rho=rho, v=v, P=P, A=A, B0=B0, tc=tc, tb=tb, dt=dt)


def directions(shape, seed):
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((nz, ny, nx)) * 0.05, rng.standard_normal((3, nz, ny, nx)) * 0.05,
            rng.standard_normal((3, nz, ny, nx)) * 0.002)


def cuda(env, *arrs):
    torch = env["torch"]
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


def solver(env, pb, precision=0, variant=1):
    W, torch = env["W"], env["torch"]
    return W.Solver(pb["shape"], pb["dx"], W.make_config(precision=precision, weno_variant=variant),
                    stream=torch.cuda.current_stream().cuda_stream)


def gpu_gradient(env, pb, s, nsteps=NSTEPS):
    torch, A = env["torch"], env["A"]
    rho, v, Av = (t.requires_grad_() for t in cuda(env, pb["rho"], pb["v"], pb["A"]))
    P, tc, tb = cuda(env, pb["P"], pb["tc"], pb["tb"])
    L = A.rollout_misfit(rho, v, Av, s, P, pb["B0"], tc, tb, pb["dt"], nsteps)
    L.backward()
    return float(L.detach()), rho.grad.cpu().numpy(), v.grad.cpu().numpy(), Av.grad.cpu().numpy()


def gpu_value(env, pb, s, d, h, nsteps=NSTEPS):
    A = env["A"]
    rho, v, Av, P, tc, tb = cuda(env, pb["rho"] + h * d[0], pb["v"] + h * d[1], pb["A"] + h * d[2], pb["P"],
                                 pb["tc"], pb["tb"])
    return A.rollout_value(rho, v, Av, s, P, pb["B0"], tc, tb, pb["dt"], nsteps)


def oracle_value(env, pb, d, h, nsteps=NSTEPS, variant=1):
    I, O = env["I"], env["O"]
    cons, bface = I.ic_from_potential(pb["rho"] + h * d[0], pb["v"] + h * d[1], pb["P"], pb["A"] + h * d[2],
                                      pb["B0"], pb["dx"])
    o = O.Oracle(pb["shape"], pb["dx"], O.make_config(weno_variant=variant))
    o.set_state(cons, bface)
    for _ in range(nsteps):
        o.step(pb["dt"])
    c, b = o.get_state()[:2]
    dV = np.prod(pb["dx"])
    return 0.5 * dV * (np.sum((c - pb["tc"]) ** 2) + np.sum((b - pb["tb"]) ** 2))


def dot(grads, d):
    return float(np.sum(grads[0] * d[0]) + np.sum(grads[1] * d[1]) + np.sum(grads[2] * d[2]))


def test_ic_map_matches_inputs(env):
    W, I, torch = env["W"], env["I"], env["torch"]
    pb = problem(env)
    rho, v, P, A = cuda(env, pb["rho"], pb["v"], pb["P"], pb["A"])
    nz, ny, nx = pb["rho"].shape
    cons = torch.empty((5, nz, ny, nx), dtype=torch.float64, device="cuda")
    bface = torch.empty((3, nz, ny, nx), dtype=torch.float64, device="cuda")
    W.w5ct_ic_from_potential(pb["shape"], pb["dx"], 5.0 / 3.0, pb["B0"], rho, v, P, A, cons, bface)
    c_ref, b_ref = I.ic_from_potential(pb["rho"], pb["v"], pb["P"], pb["A"], pb["B0"], pb["dx"])
    assert np.abs(cons.cpu().numpy() - c_ref).max() <= 1e-13 * np.abs(c_ref).max()
    assert np.abs(bface.cpu().numpy() - b_ref).max() <= 1e-13 * np.abs(b_ref).max()


def test_ic_adjoint_is_the_transpose(env):
    """<lam, IC'(x) d> = <IC'(x)^T lam, d>: the IC map is quadratic, so the
    central difference is its exact derivative up to rounding."""
    W, I, torch = env["W"], env["I"], env["torch"]
    pb = problem(env)
    d = directions(pb["shape"], 5)
    rng = np.random.default_rng(6)
    nz, ny, nx = pb["rho"].shape
    lc, lbf = rng.standard_normal((5, nz, ny, nx)), rng.standard_normal((3, nz, ny, nx))
    h = 1e-4
    cp, bp = I.ic_from_potential(pb["rho"] + h * d[0], pb["v"] + h * d[1], pb["P"], pb["A"] + h * d[2], pb["B0"], pb["dx"])
    cm, bm = I.ic_from_potential(pb["rho"] - h * d[0], pb["v"] - h * d[1], pb["P"], pb["A"] - h * d[2], pb["B0"], pb["dx"])
    lhs = (np.sum(lc * (cp - cm)) + np.sum(lbf * (bp - bm))) / (2 * h)
    rho, v, A = cuda(env, pb["rho"], pb["v"], pb["A"])
    _, bface = I.ic_from_potential(pb["rho"], pb["v"], pb["P"], pb["A"], pb["B0"], pb["dx"])
    bf, lcg, lbg = cuda(env, bface, lc, lbf)
    lr, lv, lA, lb = (torch.empty_like(t) for t in (rho, v, v, bf))
    W.w5ct_ic_from_potential_adjoint(pb["shape"], pb["dx"], rho, v, bf, lcg, lbg, lr, lv, lA, lb)
    rhs = dot((lr.cpu().numpy(), lv.cpu().numpy(), lA.cpu().numpy()), d)
    assert abs(lhs - rhs) <= 1e-9 * abs(lhs), (lhs, rhs)


@pytest.mark.parametrize("variant", [0, 1])
def test_step_adjoint_is_the_transpose(env, variant):
    """One step: <lam', (S(x + h d) - S(x - h d)) / 2h> = <S'(x)^T lam', d>
    for random lam' and d in (q, b) space."""
    W, I, torch = env["W"], env["I"], env["torch"]
    pb = problem(env)
    cons, bface = I.ic_from_potential(pb["rho"], pb["v"], pb["P"], pb["A"], pb["B0"], pb["dx"])
    rng = np.random.default_rng(7 + variant)
    dq, db = rng.standard_normal(cons.shape) * 1e-2, rng.standard_normal(bface.shape) * 1e-2
    lq, lb = rng.standard_normal(cons.shape), rng.standard_normal(bface.shape)
    s = solver(env, pb, 0, variant)
    h = 1e-6

    def step_of(c, b):
        s.set_state(c, b)
        s.step(pb["dt"])
        return s.get_state()[:2]

    cp, bp = step_of(cons + h * dq, bface + h * db)
    cm, bm = step_of(cons - h * dq, bface - h * db)
    lhs = (np.sum(lq * (cp - cm)) + np.sum(lb * (bp - bm))) / (2 * h)
    s.set_state(cons, bface)
    lqg, lbg = cuda(env, lq, lb)
    oq, ob = torch.empty_like(lqg), torch.empty_like(lbg)
    W.w5ct_adjoint_step(s.ctx, pb["dt"], lqg, lbg, oq, ob)
    rhs = float(np.sum(oq.cpu().numpy() * dq) + np.sum(ob.cpu().numpy() * db))
    assert abs(lhs - rhs) <= 1e-6 * abs(lhs), (lhs, rhs)
    # the adjoint leaves the state as it was: a step now equals a step before
    c1, b1 = s.get_state()[:2]
    assert np.array_equal(c1, cons) and np.array_equal(b1, bface)
    s.close()


@pytest.mark.parametrize("variant", [0, 1])
def test_rollout_gradient_matches_gpu_and_oracle_fd(env, variant):
    pb = problem(env)
    s = solver(env, pb, 0, variant)
    L, *grads = gpu_gradient(env, pb, s)
    assert L > 0
    d = directions(pb["shape"], 11 + variant)
    gd = dot(grads, d)
    fd_gpu = (gpu_value(env, pb, s, d, H) - gpu_value(env, pb, s, d, -H)) / (2 * H)
    fd_ora = (oracle_value(env, pb, d, H, variant=variant) - oracle_value(env, pb, d, -H, variant=variant)) / (2 * H)
    assert abs(gd - fd_gpu) <= 1e-6 * abs(fd_gpu), (gd, fd_gpu)
    assert abs(gd - fd_ora) <= 1e-6 * abs(fd_ora), (gd, fd_ora)
    s.close()


def test_fp32_gradient_close_to_fp64(env):
    pb = problem(env)
    s64 = solver(env, pb, 0)
    s32 = solver(env, pb, 1)
    _, *g64 = gpu_gradient(env, pb, s64)
    _, *g32 = gpu_gradient(env, pb, s32)
    for a, b in zip(g64, g32):
        assert np.abs(a - b).max() <= 1e-3 * np.abs(a).max()
    s64.close()
    s32.close()


def test_adjoint_rejects_batches(env):
    W, torch = env["W"], env["torch"]
    b = W.Batch([(8, 8, 8), (8, 8, 8)], [(0.125,) * 3] * 2, W.make_config(),
                stream=torch.cuda.current_stream().cuda_stream)
    I = env["I"]
    c, f = I.random_smooth_state((8, 8, 8), seed=1)
    b.set_state(0, c, f)
    b.set_state(1, c, f)
    lq = torch.zeros((5, 8, 8, 8) , dtype=torch.float64, device="cuda")
    lb = torch.zeros((3, 8, 8, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(W.W5ctError) as e:
        W.w5ct_adjoint_step(b.ctx, 0.01, lq, lb, lq.clone(), lb.clone())
    assert e.value.code == W.W5CT_ERR_UNSUPPORTED
    b.close()
