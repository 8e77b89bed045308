"""Accuracy of the float-float exp(-x) used for the AO values of the mixed
path (Cody-Waite reduction by ln 2 split in three parts, a 25-entry table of
exp(-j/32) in float pairs (Tang's table method), a Taylor series of the
remaining factor), emulated step by step in float32 arithmetic and compared
with FP64 exp of the same float-pair argument: relative error below 2^-42
for 0 <= x < 70 (the AO screening keeps g >= 1e-8, i.e. x below ~20 for the
contraction coefficients in use).  The ln 2 split constants are read from
the CUDA source."""
import math
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
f = np.float32


def _hexfloats():
    src = open(os.path.join(ROOT, "paper_1209_6630_gb300", "csrc", "ff_math.cuh")).read()
    l1 = re.search(r"kL1\s*=\s*(0x[0-9a-fA-Fp.+-]+)f", src).group(1)
    l2 = re.search(r"kL2\s*=\s*make_float2\((0x[0-9a-fA-Fp.+-]+)f,\s*(0x[0-9a-fA-Fp.+-]+)f\)", src)
    return f(float.fromhex(l1)), (f(float.fromhex(l2.group(1))), f(float.fromhex(l2.group(2))))


L1, L2 = _hexfloats()


def fma(a, b, c):          # a*b is exact in float64; one rounding to float32 after the add (a close stand-in)
    return f(float(a) * float(b) + float(c))


def two_sum(a, b):
    s = f(a + b)
    bb = f(s - a)
    return s, f(f(a - f(s - bb)) + f(b - bb))


def fast_two_sum(a, b):
    s = f(a + b)
    return s, f(b - f(s - a))


def add(a, b):
    s, e = two_sum(a[0], b[0])
    return fast_two_sum(s, f(e + f(a[1] + b[1])))


def neg(a):
    return (f(-a[0]), f(-a[1]))


def mul(a, b):
    p = f(a[0] * b[0])
    e = fma(a[1], b[0], fma(a[0], b[1], fma(a[0], b[0], -p)))
    return fast_two_sum(p, e)


def mulf(a, b):
    p = f(a[0] * b)
    return fast_two_sum(p, fma(a[1], b, fma(a[0], b, -p)))


def pair(v):
    h = f(v)
    return (h, f(v - float(h)))


TABLE = [pair(math.exp(-j / 32.0)) for j in range(-12, 13)]


def exp_neg(x):
    if not x[0] < 87:
        return (f(0), f(0))
    kf = f(np.rint(f(x[0] * f(1.44269504088896340736))))
    rh, rl = two_sum(f(x[0] - f(kf * L1)), x[1])
    r = add((rh, rl), neg(mulf(L2, kf)))
    jf = f(np.rint(f(r[0] * f(32))))
    sh, sl = two_sum(f(r[0] - f(jf * f(0.03125))), r[1])
    s = sh
    tail = f(s * s * s * f(f(-1 / 6) + s * f(f(1 / 24) + s * f(f(-1 / 120) + s * f(1 / 720)))))
    s2 = mul((sh, sl), (sh, sl))
    p = add((f(1), f(0)), neg((sh, sl)))
    p = add(p, (f(0.5 * s2[0]), f(0.5 * s2[1])))
    p = add(p, (tail, f(0)))
    e = mul(p, TABLE[int(jf) + 12])
    sc = f(2.0 ** (-int(kf)))
    return (f(e[0] * sc), f(e[1] * sc))


def test_ln2_split():
    # L1 + L2 carries ln 2 at least to FP64 precision (checked in FP64 arithmetic)
    assert abs((float(L1) + float(L2[0])) + float(L2[1]) - math.log(2.0)) <= 2.0 ** -53
    # kf * L1 exact in FP32 for every reduction index kf <= 126 (x < 87)
    for kf in range(127):
        assert float(f(f(kf) * L1)) == kf * float(L1)


def test_exp_neg_relative_error():
    rng = np.random.default_rng(5)
    xs = np.concatenate([rng.uniform(0, 70, 4000), rng.uniform(0, 1, 1000), [0.0, 1e-8, 0.5 * math.log(2), 20.0]])
    worst = 0.0
    for x in xs:
        xp = pair(x)
        xv = float(xp[0]) + float(xp[1])
        ref = math.exp(-xv)
        h, l = exp_neg(xp)
        worst = max(worst, abs(float(h) + float(l) - ref) / ref)
    assert worst < 2.0 ** -42, math.log2(worst)
