"""Host logic of adjoint.RolloutMisfit (no GPU): the forward pass keeps the
state at the start of every step, the backward pass runs the steps' adjoints
in reverse order from those checkpoints, swaps its buffers correctly and
scales by the incoming gradient.  The library calls are replaced by a fake
whose step is nonlinear and couples neighbouring cells (q <- q + dt sin(Sq),
S a periodic shift), so that the step Jacobians do not commute: an adjoint
applied at the wrong checkpoint or in the wrong order gives the wrong
gradient.  The gradient is compared with central differences of the same
fake pipeline."""
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def adjoint():
    from paper_1812_04278_gb300 import build
    build.build()                      # the binding imports the library
    from paper_1812_04278_gb300 import adjoint as mod
    return mod


class FakeSolver:
    def __init__(self, shape, dx):
        self.shape, self.dx = shape, dx
        self.cfg = types.SimpleNamespace(gamma=5.0 / 3.0)
        self.ctx = self
        self.q = self.b = None

    def set_state(self, q, b):
        self.q, self.b = q.clone(), b.clone()

    def step(self, dt):
        self.q = self.q + dt * torch.sin(torch.roll(self.q, 1, dims=-1))
        self.b = self.b + dt * torch.cos(torch.roll(self.b, 1, dims=-2))


def make_fake_w5(dV):
    def ic(shape, dx, gamma, B0, rho, v, P, A, cons, bface, stream):
        cons[0] = rho
        cons[1:4] = rho * v
        cons[4] = P + 0.5 * rho * (v * v).sum(0)
        bface.copy_(A + torch.tensor(B0, dtype=A.dtype)[:, None, None, None])

    def get_state(ctx, q, b, bc, on_device):
        q.copy_(ctx.q)
        b.copy_(ctx.b)

    def misfit(ctx, tc, tb, lq, lb):
        dq, db = ctx.q - tc, ctx.b - tb
        lq.copy_(dV * dq)
        lb.copy_(dV * db)
        return float(0.5 * dV * ((dq * dq).sum() + (db * db).sum()))

    def adjoint_step(ctx, dt, lq, lb, oq, ob):
        # the transpose of the step's Jacobian at the context's current state:
        # J = I + dt diag(f'(Sq)) S, J^T lam = lam + dt S^T (f'(Sq) lam)
        cq = torch.cos(torch.roll(ctx.q, 1, dims=-1))
        sb = -torch.sin(torch.roll(ctx.b, 1, dims=-2))
        oq.copy_(lq + dt * torch.roll(cq * lq, -1, dims=-1))
        ob.copy_(lb + dt * torch.roll(sb * lb, -1, dims=-2))

    def ic_adjoint(shape, dx, rho, v, bface, lq, lb, lam_rho, lam_v, lam_A, lam_bt, stream):
        lam_rho.copy_(lq[0] + (lq[1:4] * v).sum(0) + 0.5 * lq[4] * (v * v).sum(0))
        lam_v.copy_(lq[1:4] * rho + lq[4] * rho * v)
        lam_A.copy_(lb)
        lam_bt.copy_(lb)

    return types.SimpleNamespace(w5ct_ic_from_potential=ic, w5ct_get_state=get_state, w5ct_misfit=misfit,
                                 w5ct_adjoint_step=adjoint_step, w5ct_ic_from_potential_adjoint=ic_adjoint)


def test_rollout_gradient_matches_central_differences(monkeypatch, adjoint):
    shape = (4, 3, 2)
    grid = (shape[2], shape[1], shape[0])
    dV = 1.0 / 24
    monkeypatch.setattr(adjoint, "w5", make_fake_w5(dV))
    monkeypatch.setattr(torch.cuda, "current_stream", lambda: types.SimpleNamespace(cuda_stream=0))
    g = torch.Generator().manual_seed(3)
    rho = 1.0 + 0.1 * torch.rand(grid, generator=g, dtype=torch.float64)
    v = 0.3 * torch.randn((3,) + grid, generator=g, dtype=torch.float64)
    A = 0.2 * torch.randn((3,) + grid, generator=g, dtype=torch.float64)
    P = 0.6 + 0.1 * torch.rand(grid, generator=g, dtype=torch.float64)
    tc = torch.randn((5,) + grid, generator=g, dtype=torch.float64)
    tb = torch.randn((3,) + grid, generator=g, dtype=torch.float64)
    B0, dt, nsteps = (1.0, 0.5, -0.2), 0.3, 4
    s = FakeSolver(shape, (0.25, 1 / 3, 0.5))
    r, vv, aa = (t.clone().requires_grad_(True) for t in (rho, v, A))
    L = adjoint.rollout_misfit(r, vv, aa, s, P, B0, tc, tb, dt, nsteps)
    (3.0 * L).backward()                                   # an incoming gradient of 3
    dr, dv, dA = (torch.randn(t.shape, generator=g, dtype=torch.float64) for t in (rho, v, A))
    h = 1e-6

    def value(sign):
        return adjoint.rollout_value(rho + sign * h * dr, v + sign * h * dv, A + sign * h * dA, s, P, B0, tc, tb,
                                     dt, nsteps)

    fd = 3.0 * (value(1) - value(-1)) / (2 * h)
    ad = float((r.grad * dr).sum() + (vv.grad * dv).sum() + (aa.grad * dA).sum())
    assert abs(ad - fd) <= 1e-7 * abs(fd), (ad, fd)
