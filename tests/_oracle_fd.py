"""Central differences of the CPU oracle, one input component at a time, for
the element-wise checks of the adjoint (tests/test_gpu_adjoint_elementwise.py).

Two scalar functions of a small periodic problem are differenced:

* the rollout misfit L(rho, v, A) = 1/2 dV |state_n - target|^2 after n
  steps of fixed dt from the state that (rho, v, P, A, B0) define (b = curl A
  + B0, E from Eq. P), as the adjoint's autograd rollout computes it;
* the projection <lam_q, q1> + <lam_b, b1> of one step (q1, b1) = S(q, b).

For every input component x_i, the values at x_i +- h and x_i +- h/4 are
returned, so that the caller can form central differences at two step
sizes, their Richardson extrapolation and an estimate of the error.  The
evaluations run in processes started with `spawn` (never forked from a
process that has touched the GPU), each running the oracle on one thread.
Only the oracle and the problem set-ups of `inputs` are used here.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

_W: dict = {}


def _init(problem: dict, variant: int):
    import oracle
    from paper_1812_04278_gb300 import inputs as I
    oracle.set_num_threads(1)
    _W["p"] = problem
    _W["I"] = I
    _W["o"] = oracle.Oracle(problem["shape"], problem["dx"], oracle.make_config(weno_variant=variant))


def _rollout(rho, v, A):
    p, I, o = _W["p"], _W["I"], _W["o"]
    cons, bface = I.ic_from_potential(rho, v, p["P"], A, p["B0"], p["dx"])
    o.set_state(cons, bface)
    for _ in range(p["nsteps"]):
        o.step(p["dt"])
    c, b = o.get_state()[:2]
    dV = float(np.prod(p["dx"]))
    return 0.5 * dV * (float(np.sum((c - p["tc"]) ** 2)) + float(np.sum((b - p["tb"]) ** 2)))


def _step_projection(q, b):
    p, o = _W["p"], _W["o"]
    o.set_state(q, b)
    o.step(p["dt"])
    c1, b1 = o.get_state()[:2]
    return float(np.sum(p["lq"] * c1)) + float(np.sum(p["lb"] * b1))


def _task(args):
    """Values at x_f[i] + s for s in steps (fields f of the kind's inputs)."""
    kind, f, i, steps = args
    p = _W["p"]
    names = ("rho", "v", "A") if kind == "rollout" else ("q", "b")
    out = []
    for s in steps:
        x = [p[n].copy() for n in names]
        x[f].reshape(-1)[i] += s
        out.append(_rollout(*x) if kind == "rollout" else _step_projection(*x))
    return out


def central_differences(kind: str, problem: dict, variant: int, h: float, workers: int | None = None):
    """For every component of the inputs of `kind` ("rollout": rho, v, A;
    "step": q, b) in field order, C order within a field: returns (c1, c4),
    the central differences with steps h and h/4."""
    names = ("rho", "v", "A") if kind == "rollout" else ("q", "b")
    steps = (h, -h, h / 4, -h / 4)
    tasks = [(kind, f, i, steps) for f, n in enumerate(names) for i in range(problem[n].size)]
    nw = workers or max(1, min(16, os.cpu_count() or 1))
    ctx = mp.get_context("spawn")
    with ctx.Pool(nw, initializer=_init, initargs=(problem, variant)) as pool:
        vals = np.array(pool.map(_task, tasks, chunksize=max(1, len(tasks) // (4 * nw))))
    c1 = (vals[:, 0] - vals[:, 1]) / (2 * h)
    c4 = (vals[:, 2] - vals[:, 3]) / (2 * (h / 4))
    return c1, c4
