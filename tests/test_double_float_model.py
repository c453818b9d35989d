"""Error bound of the double-float products with the inverse factor, checked
on the host: the published error-free transformations (Dekker's product
through an FMA, Knuth's TwoSum) restated with numpy float32 operations in
the order the S products use them — four accumulator pairs per lane, 32
lanes, a pairwise tree across the lanes — against the exact rational sum.
The design claims an error of order 2^-44 of the row's sum of magnitudes
(about 2^-53 for FP64); this pins that claim independently of the GPU."""
from fractions import Fraction

import numpy as np
import pytest

f32 = np.float32


def fma32(a, b, c):
    # a*b is exact in float64 (24 + 24 bits); for the operand sizes below the
    # float64 sum is exact too, so one rounding to float32 is the FMA's
    return f32(float(a) * float(b) + float(c))


def split(x):
    h = f32(x)
    return h, f32(x - float(h))


def mac(h, l, s, x):
    p = f32(s[0] * x[0])
    e = fma32(s[0], x[0], -p)
    t = fma32(s[0], x[1], fma32(s[1], x[0], e))
    sm = f32(h + p)
    bb = f32(sm - h)
    err = f32(f32(h - f32(sm - bb)) + f32(p - bb))
    return sm, f32(l + f32(err + t))


def add(a, b):
    s = f32(a[0] + b[0])
    bb = f32(s - a[0])
    err = f32(f32(a[0] - f32(s - bb)) + f32(b[0] - bb))
    l = f32(err + f32(a[1] + b[1]))
    h = f32(s + l)
    return h, f32(l - f32(h - s))


def df_row(svals, xvals):
    """One row as a warp computes it: lane k takes entries k, k+32, ...; within
    a lane, chunks of 4 x 32 go to accumulator u, the tail to accumulator 0."""
    n = len(svals)
    sp = [split(v) for v in svals]
    xp = [split(v) for v in xvals]
    lanes = []
    for lane in range(32):
        acc = [(f32(0), f32(0))] * 4
        p = lane
        while p + 96 < n:
            for u in range(4):
                acc[u] = mac(acc[u][0], acc[u][1], sp[p + 32 * u], xp[p + 32 * u])
            p += 128
        while p < n:
            acc[0] = mac(acc[0][0], acc[0][1], sp[p], xp[p])
            p += 32
        lanes.append(add(add(acc[0], acc[1]), add(acc[2], acc[3])))
    while len(lanes) > 1:
        lanes = [add(lanes[i], lanes[i + 1]) for i in range(0, len(lanes), 2)]
    h, l = lanes[0]
    return float(h) + float(l)


@pytest.mark.parametrize("n,seed", [(37, 0), (280, 1), (358, 2), (700, 3)])
def test_double_float_dot_within_2e44_of_exact(n, seed):
    rng = np.random.default_rng(seed)
    # inverse-factor-like magnitudes: entries spread over a few decades with
    # both signs, right-hand sides of mixed sign (cancellation in the sum)
    s = rng.standard_normal(n) * 10.0 ** rng.uniform(-3, 0, n)
    x = rng.standard_normal(n) * 10.0 ** rng.uniform(0, 3, n)
    # the stored operands are the double-float splits of these FP64 values
    sp = [split(v) for v in s]
    xp = [split(v) for v in x]
    s_rep = [float(h) + float(l) for h, l in sp]
    x_rep = [float(h) + float(l) for h, l in xp]
    exact = sum(Fraction(a) * Fraction(b) for a, b in zip(s_rep, x_rep))
    mag = float(sum(abs(Fraction(a) * Fraction(b)) for a, b in zip(s_rep, x_rep)))
    got = df_row(s, x)
    err = abs(Fraction(got) - exact)
    assert float(err) <= 4.0 * 2.0 ** -44 * mag, (float(err) / mag)
    # and the representation error of a split value is below 2^-48 of it
    for v, r in zip(s[:50], s_rep[:50]):
        assert abs(r - v) <= 2.0 ** -47 * abs(v)
