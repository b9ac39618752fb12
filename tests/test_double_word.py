"""The double-word (float pair) arithmetic of the FP64 sweep's WENO form,
restated on the CPU in binary32 and checked against exact results and
against the oracle's phi_N (Sec. 2.2).

Each operation is written as the kernel does it (w5ct_physics.cuh: TwoSum,
Fast2Sum, TwoProd, the one-sided double-word sum, products, the division by
a refined reciprocal and one correction, the conversions to and from
double), with numpy float32 scalars for every rounded step.  An FMA is
emulated by forming the product and sum in float64 and rounding once to
float32 (the product of two floats is exact in float64, so only the rare
double rounding of the sum differs from a fused operation); the hardware's
approximate reciprocal is replaced by the correctly rounded one before the
same Newton step.  These checks fix the accuracy the kernel's form reaches
(errors of order 2^-48 of the operands), independently of the GPU, where
tests/test_gpu_fp64_dw.py holds the kernel itself to the oracle.
"""
import numpy as np
import pytest

import oracle as ora

f32 = np.float32


def fma32(a, b, c):
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def fast2sum(a, b):
    s = f32(a + b)
    return s, f32(b - f32(s - a))


def twosum(a, b):
    s = f32(a + b)
    bv = f32(s - a)
    av = f32(s - bv)
    return s, f32(f32(a - av) + f32(b - bv))


def twoprod(a, b):
    p = f32(a * b)
    return p, fma32(a, b, -p)


def dw_add(x, y):
    sh, sl = twosum(x[0], y[0])
    return fast2sum(sh, f32(sl + f32(x[1] + y[1])))


def dw_neg(x):
    return (f32(-x[0]), f32(-x[1]))


def dw_sub(x, y):
    return dw_add(x, dw_neg(y))


def dw_mul_f(x, y):
    ch, cl = twoprod(x[0], y)
    return fast2sum(ch, fma32(x[1], y, cl))


def dw_mul(x, y):
    ch, cl = twoprod(x[0], y[0])
    t = fma32(x[0], y[1], f32(x[1] * y[0]))
    return fast2sum(ch, f32(cl + t))


def dw_div(x, y):
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        r = f32(1.0 / np.float64(y[0])) if y[0] != 0 else f32(np.inf)
        r = fma32(r, fma32(-y[0], r, f32(1.0)), r)
        q = f32(x[0] * r)
        yq = dw_mul_f(y, q)
        ph, pl = twosum(x[0], f32(-yq[0]))
        d = f32(ph + f32(f32(pl - yq[1]) + x[1]))
        return fast2sum(q, f32(d * r))


def dw_from_double(x):
    """The kernel's integer-pipe conversion: hi = x truncated to 24
    significand bits, lo = the next 29 bits rounded to 24, renormalised."""
    u = int(np.array(x, dtype=np.float64).view(np.uint64))
    hw, lw = u >> 32, u & 0xFFFFFFFF
    sgn = hw & 0x80000000
    e = (hw >> 20) & 0x7FF
    hb = (sgn | (((e - 896) & 0x1FF) << 23) | ((hw & 0xFFFFF) << 3) | (lw >> 29)) & 0xFFFFFFFF
    m = f32(lw & 0x1FFFFFFF)
    scale = np.array(((e - 948) & 0x1FF) << 23, dtype=np.uint32).view(np.float32) if e > 948 else f32(0)
    lo = f32(m * scale)
    h = np.array(hb, dtype=np.uint32).view(np.float32).item()
    lo = f32(-lo) if sgn else lo
    if e <= 948:
        lo = f32(0)
    if e <= 896:
        h = 0.0
    if e >= 1151:
        h, lo = (-np.inf if sgn else np.inf), f32(0)
    return fast2sum(f32(h), lo)


def dw_value(x):
    return np.float64(x[0]) + np.float64(x[1])


def phi_dw(a, b, c, d, eps3, Z):
    """3 phi_N as the double-word kernel form computes it."""
    two = f32(2.0)
    x0, y0, z0 = dw_sub(a, b), dw_sub(b, c), dw_sub(c, d)
    x1 = dw_sub(x0, (f32(two * b[0]), f32(two * b[1])))
    y1 = dw_add(b, c)
    z1 = dw_add(z0, (f32(two * c[0]), f32(two * c[1])))
    k = (f32(4.33333349), f32(-1.58945719e-07))

    def ind(p, q):
        s = dw_add(dw_add(dw_mul(k, dw_mul(p, p)), dw_mul(q, q)), eps3)
        return (f32(0), f32(0)) if s[0] < f32(1.17549435e-38) else s

    s = [ind(x0, x1), ind(y0, y1), ind(z0, z1)]
    sm = s[0]
    for sk in s[1:]:
        if sk[0] < sm[0]:
            sm = sk
    one = (f32(1), f32(0))
    r = [one if (sk[0] == sm[0] and sk[1] == sm[1]) else dw_div(sm, sk) for sk in s]
    e = [dw_mul(rk, rk) for rk in r]
    if Z:
        tau = dw_sub(s[0], s[2])
        if tau[0] < 0:
            tau = dw_neg(tau)
        R = (f32(0), f32(0)) if tau[0] == 0 else dw_div(tau, sm)
        if R[0] <= f32(1e18):
            R2 = dw_mul(R, R)
            e = [dw_add(one, dw_mul(R2, ek)) for ek in e]
    D = dw_add(dw_add(e[0], dw_mul_f(e[1], f32(6))), dw_mul_f(e[2], f32(3)))
    inv = dw_div(one, D)
    w0 = dw_mul(e[0], inv)
    w2 = dw_add(dw_mul_f(dw_mul(e[2], inv), f32(1.5)), (f32(-0.25), f32(0)))
    return dw_add(dw_mul(w0, dw_sub(x0, y0)), dw_mul(w2, dw_sub(y0, z0)))


def test_conversion_keeps_48_bits():
    rng = np.random.default_rng(3)
    for x in rng.normal(0, 1, 2000) * 10.0 ** rng.integers(-15, 15, 2000):
        h, l = dw_from_double(x)
        assert abs(l) <= abs(h) * 2.0 ** -24 + 1e-300
        assert abs(dw_value((h, l)) - x) <= 2.0 ** -47 * abs(x)
    assert dw_value(dw_from_double(0.0)) == 0.0
    assert dw_value(dw_from_double(1e-40)) == 0.0          # below float's normal range


@pytest.mark.parametrize("op", ["add", "mul", "div"])
def test_operations_reach_double_word_accuracy(op):
    """Relative error of the kernel's sums (on operands of one sign), products
    and quotients against the float64 result of the exact pair values."""
    rng = np.random.default_rng({"add": 5, "mul": 6, "div": 7}[op])
    worst = 0.0
    for _ in range(3000):
        a, b = rng.uniform(0.1, 10, 2) * 10.0 ** rng.integers(-8, 8, 2)
        x, y = dw_from_double(a), dw_from_double(b)
        xa, ya = dw_value(x), dw_value(y)
        if op == "add":
            got, want = dw_value(dw_add(x, y)), xa + ya
        elif op == "mul":
            got, want = dw_value(dw_mul(x, y)), xa * ya
        else:
            got, want = dw_value(dw_div(x, y)), xa / ya
        worst = max(worst, abs(got - want) / abs(want))
    assert worst < 2.0 ** -44, worst


@pytest.mark.parametrize("Z", [0, 1])
def test_double_word_phi_n_equals_the_oracle(Z):
    """The kernel's double-word phi_N from double stencil differences, in
    binary32 pairs, against the oracle's phi_N: within 1e-13 of the
    stencil's scale (the conversion alone contributes 2^-48)."""
    rng = np.random.default_rng(11 + Z)
    cfg = ora.make_config(weno_variant=Z)
    eps = cfg.eps_z if Z else cfg.eps_js
    e3 = dw_from_double(eps / 3.0)
    worst = 0.0
    cases = [rng.normal(0.0, 1.0, 4) * rng.choice([1e-6, 1e-3, 1.0, 1e3]) for _ in range(400)]
    cases += [np.array(v, dtype=float) for v in
              ([1.0, 0, 0, 0], [0, 0, 0, 1.0], [1.0, 1.0, 1.0, 1.0], [2.0, 0, 0, -1.0], [0, 0, 0, 0],
               [1e-21, -2e-21, 3e-21, 1.0], [1.0, 1.0 + 1e-12, 1.0 - 1e-12, 1.0])]
    for v in cases:
        got = dw_value(phi_dw(*(dw_from_double(t) for t in v), e3, Z)) / 3.0
        want = ora.phi_n(*v, cfg)
        worst = max(worst, abs(got - want) / max(np.abs(v).max(), 1e-300))
    assert worst < 1e-13, worst
