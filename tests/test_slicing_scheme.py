"""The exact-slice arithmetic behind the tensor-core products (C1/C5 and the
Gauss-Jordan updates), restated from its definition in numpy and checked
against the bounds the kernels rely on:

* a value with |x| < 2^E is cut into S slices s_j = q_j 2^(E - 7(j+1)), q_j
  integer with |q_0| <= 128 and |q_j| <= 65 (j >= 1): each q_j has at most
  8 significant bits, so every slice is exact in BF16;
* the remainder after S slices is below 2^(E - 7 S - 1);
* the products of one order d = i + j, summed over K terms, stay within 2^24
  units of 2^-7(d+2), so an FP32 accumulator adds them exactly: for the
  Gauss-Jordan updates (S = 7, K = 32, every order 0..6 in its own
  accumulator) always; for C1/C5 (S = 6, orders 0..2 in their own
  accumulators) up to K = 804 terms, and in the 1024-AO chunks an order sum
  can pass 2^24 units only with more than ~800 terms near the row and column
  maxima of equal sign, and then stays below 2^25 units: rounded by at most
  one unit (2^-28 of the row-column scale for d = 2).
The slice counts, slice width and K are read from the CUDA sources."""
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1209_6630_gb300", "csrc")


def _const(fname, name):
    src = open(os.path.join(CSRC, fname)).read()
    m = re.search(r"constexpr\s+(?:int|uint32_t)\s+" + name + r"\s*=\s*([^;]+);", src)
    assert m, name
    return m.group(1).strip()


S_C15 = int(_const("qmc_internal.cuh", "kC15Slices"))
BITS = int(_const("qmc_internal.cuh", "kC15SliceBits"))
S_GT = int(_const("k_gj_tc.cu", "kGtSl").replace("kC15Slices", str(S_C15)))
K_GT = int(_const("k_gj_tc.cu", "kGtB"))
K_C15 = int(_const("k_c15_tc.cu", "kChunkSteps")) * 64          # K steps of 64 AOs per exact chunk


def _exp_bound(x):
    """Smallest-ish E with 2^E > 1.001 |x| (the kernels' bound, from the FP32 exponent)."""
    y = np.float32(abs(x) * np.float32(1.001))
    return int(np.frexp(np.float64(y))[1]) if y > 0 else -126


def _slices(x, E, S):
    """q_j of the definition, computed exactly in float64 from a float pair value."""
    r = np.ldexp(np.float64(x), -E)
    q = []
    for j in range(S):
        qj = np.rint(np.ldexp(r, BITS * (j + 1)))
        q.append(int(qj))
        r = r - np.ldexp(qj, -BITS * (j + 1))
    return q, r


def _bf16_exact(q):
    q = abs(q)
    while q and q % 2 == 0:
        q //= 2
    return q < 256


def test_slice_bounds_and_reconstruction():
    rng = np.random.default_rng(7)
    for S in (S_C15, S_GT):
        worst = 0.0
        for _ in range(4000):
            hi = np.float32(rng.standard_normal() * 10.0 ** rng.uniform(-6, 6))
            lo = np.float32(np.float64(hi) * rng.uniform(-2 ** -24, 2 ** -24))
            x = np.float64(hi) + np.float64(lo)
            mx = abs(x) * rng.uniform(1.0, 1e4) if rng.random() < 0.5 else abs(x)   # row max >= |x|
            E = _exp_bound(np.float32(mx))
            assert abs(x) < 2.0 ** E
            q, r = _slices(x, E, S)
            assert abs(q[0]) <= 2 ** BITS and all(abs(v) <= 2 ** (BITS - 1) + 1 for v in q[1:]), q
            assert all(_bf16_exact(v) for v in q)
            worst = max(worst, abs(r))
        assert worst <= 2.0 ** (-BITS * S - 1), (S, worst)


def _order_bound(S, K, d):
    tot = 0
    for i in range(max(0, d - S + 1), min(d, S - 1) + 1):
        j = d - i
        tot += (2 ** BITS if i == 0 else 2 ** (BITS - 1) + 1) * (2 ** BITS if j == 0 else 2 ** (BITS - 1) + 1)
    return tot * K


def test_exact_order_sums():
    # Gauss-Jordan updates: every kept order 0..S-1 has its own accumulator over K = 32
    for d in range(S_GT):
        assert _order_bound(S_GT, K_GT, d) <= 2 ** 24, d
    # C1/C5: orders 0, 1, 2 in their own accumulators; exact up to K = 804 terms
    k_exact = min(2 ** 24 // _order_bound(S_C15, 1, d) for d in range(3))
    assert k_exact == 804, k_exact
    # the 1024-AO chunks: worst case below 2^25 units, i.e. at most one unit of rounding
    for d in range(3):
        assert _order_bound(S_C15, K_C15, d) < 2 ** 25, d
    # and the dropped orders d >= S contribute below ~2^-47 of the update (worst case 2^-42)
    dropped = sum(_order_bound(S_GT, K_GT, d) * 2.0 ** (-BITS * (d + 2)) for d in range(S_GT, 2 * S_GT - 1))
    assert dropped < 2.0 ** -42, dropped


def _bf16_rn(x):
    """Round an FP32 value to BF16 (8 significant bits), ties to even, from the definition."""
    b = np.array([x], dtype=np.float32).view(np.uint32)[0]
    lsb = (b >> 16) & 1
    r = (b + 0x7FFF + lsb) & 0xFFFF0000
    return np.array([r], dtype=np.uint32).view(np.float32)[0]


def test_three_way_bf16_split_is_exact():
    # the adjoint's operands: hi = rn(x), mid = rn(x - hi), lo = rn(x - hi - mid), x = hi + mid + lo
    rng = np.random.default_rng(11)
    for _ in range(20000):
        x = np.float32(rng.standard_normal() * 10.0 ** rng.uniform(-20, 20))
        hi = _bf16_rn(x)
        r1 = np.float32(x - hi)                          # exact in FP32
        mid = _bf16_rn(r1)
        r2 = np.float32(r1 - mid)
        lo = _bf16_rn(r2)
        assert np.float64(hi) + np.float64(mid) + np.float64(lo) == np.float64(x), x
        assert np.float32(lo) == r2                      # the last slice loses nothing
