"""Robustness problems on the CPU oracle (Secs. 4.3, 4.5, 4.13, 4.14).

Pins of the oracle against what the paper reports for them:
* field loop advection (Sec. 4.14): WENO5 keeps more than 90% of the loop's
  magnetic energy through t = 2 (checked at 128 x 64, where this oracle keeps
  94%; at 64 x 32 it keeps 88.6%, below the paper's figure); the energy kept
  grows with the WENO epsilon, which sets that figure at 64 x 32;
* Riemann problems (Secs. 4.3, 4.5): no non-physical state without floors to
  the paper's end times, conservation and div b at round-off, including the
  degenerate transverse field of the Brio-Wu problem.
"""
import numpy as np
import pytest

import oracle
from paper_1812_04278_gb300 import inputs as I


@pytest.fixture(scope="module", autouse=True)
def built():
    oracle.build()


def advance_to(o, t_end, marks=()):
    t, n, out = 0.0, 0, []
    marks = list(marks)
    while t < t_end - 1e-12:
        stop = marks[0] if marks else t_end
        dt = min(o.cfl_dt(), stop - t)
        o.step(dt)
        t += dt
        n += 1
        if marks and abs(t - marks[0]) < 1e-12:
            out.append(o.get_state())
            marks.pop(0)
    return n, out


@pytest.mark.slow
def test_field_loop_keeps_ninety_percent_of_its_energy():
    shape = (128, 64, 1)
    cons, bface, dx = I.field_loop(shape)
    o = oracle.Oracle(shape, dx, oracle.make_config(weno_variant=oracle.WENO_JS))
    o.set_state(cons, bface)
    E0 = I.magnetic_energy(bface, dx)
    _, states = advance_to(o, 2.0, marks=(0.5, 1.0, 1.5, 2.0))
    E = [I.magnetic_energy(s[1], dx) / E0 for s in states]
    assert E[-1] > 0.90, E
    assert all(a >= b for a, b in zip(E, E[1:])), E        # dissipation only
    assert o.div_b_norm()[0] < 1e-12


def test_field_loop_dissipation_falls_as_the_weno_epsilon_grows():
    """The loop's field (|B| = 1e-3) makes the smoothness indicators of its
    characteristic fields comparable to the WENO epsilon (Sec. 2.2, 1e-6):
    a larger epsilon pulls the weights towards the linear ones and the
    energy lost by t = 0.5 at 64 x 32 must fall.  This is the sensitivity
    that decides whether the lowest resolution of Sec. 4.14 keeps 90%."""
    shape = (64, 32, 1)
    cons, bface, dx = I.field_loop(shape)
    E0 = I.magnetic_energy(bface, dx)
    kept = []
    for eps in (2.5e-7, 1e-6, 4e-6):
        o = oracle.Oracle(shape, dx, oracle.make_config(weno_variant=oracle.WENO_JS, eps_js=eps))
        o.set_state(cons, bface)
        _, states = advance_to(o, 0.5, marks=(0.5,))
        kept.append(I.magnetic_energy(states[-1][1], dx) / E0)
    assert kept[0] < kept[1] < kept[2], kept
    assert 0.85 < kept[1] < 0.95, kept


@pytest.mark.parametrize("name", ["RJ2A", "BRIO_WU"])
def test_riemann_problems_stay_physical_and_conservative(name):
    prob = getattr(I, name)
    cons, bface, dx, gamma = I.shock_tube(prob, 128, transverse=(2, 2))
    shape = (128, 2, 2)
    o = oracle.Oracle(shape, dx, oracle.make_config(gamma=gamma))
    o.set_state(cons, bface)
    tot0 = o.conserved_totals()
    advance_to(o, prob["t_end"])
    assert o.status()[1] == 0
    c, b = o.get_state()[:2]
    assert np.isfinite(c).all() and c[0].min() > 0
    tot = o.conserved_totals()
    scale = np.abs(cons).sum() * np.prod(dx)
    assert np.abs(tot - tot0).max() <= 1e-13 * scale
    assert o.div_b_norm()[0] < 1e-12
    # the solution stays one-dimensional
    assert np.abs(c - c[:, :1, :1, :]).max() <= 1e-12 * np.abs(c).max()
