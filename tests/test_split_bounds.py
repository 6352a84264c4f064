"""The arithmetic the split-operand tensor-core products rely on (block
build and LU trailing updates), checked on the host:

* a double x with |x| < 2^e becomes round(x 2^(62-e)), written as nine
  balanced base-128 digits a_s (|a_s| <= 65, exact in bf16) with
  x ~ 2^e sum_s a_s 2^-(6+7s), off by at most 2^(e-63);
* the products of one diagonal s + t = d sum exactly in FP32 (below 2^24)
  for the inner ranges the kernels use: chunks of 192 in the build, 32 in
  the LU;
* the diagonals' integer sums (d <= 3 shifted by 7(3-d) and scaled by
  2^(E-21), d >= 4 shifted by 7(8-d) and scaled by 2^(E-56)) weigh each
  diagonal by 2^(E-7d) and fit in 64-bit integers for inner ranges up to
  3 x 256.
A digit routine that dropped the balancing, a bound that let a diagonal's
FP32 sum round, or a wrong shift would fail here."""
import math
import random

import numpy as np


def digits(x, e, n=9):
    """Balanced base-128 digits of round(x 2^(62-e)), most significant first."""
    r = round(x * 2.0 ** (62 - e)) if abs(x) < 2.0 ** 1000 else 0
    r = int(r)
    out = []
    for _ in range(n - 1):
        dg = r & 127
        if dg >= 64:
            dg -= 128
        out.append(dg)
        r = (r - dg) >> 7
    out.append(r)
    return out[::-1]


def test_balanced_digits_reconstruct_within_half_an_ulp_of_2_62():
    rng = random.Random(3)
    for _ in range(20000):
        x = rng.uniform(-1, 1) * 2.0 ** rng.randint(-30, 30)
        if x == 0.0:
            continue
        e = math.frexp(x)[1]  # |x| < 2^e
        a = digits(x, e)
        assert all(abs(d) <= 65 for d in a)
        assert all(float(np.float32(d)) == d for d in a)  # bf16 holds |d| <= 256 exactly too
        rec = sum(d * 2.0 ** (e - 6 - 7 * s) for s, d in enumerate(a))
        assert abs(rec - x) <= 2.0 ** (e - 63)


def test_diagonal_sums_stay_exact_in_fp32():
    # per diagonal at most 9 digit pairs; |a| <= 65, |b| <= 65
    for K in (192, 32):
        assert 9 * K * 65 * 65 < 2 ** 24
    # a worst case summed in FP32 equals the exact integer
    K = 192
    prods = np.full(9 * K, 65 * 65, dtype=np.int64)
    acc = np.float32(0)
    for p in prods:
        acc = np.float32(acc + np.float32(p))
    assert int(acc) == int(prods.sum())


def test_integer_fold_weights_and_headroom():
    # the weight of diagonal d relative to 2^E: 2^shift x 2^scale = 2^(-7d)
    for d in range(9):
        shift, scale = (7 * (3 - d), -21) if d < 4 else (7 * (8 - d), -56)
        assert shift + scale == -7 * d
    # headroom: |diagonal sum| <= (d + 1) K 65^2 for inner ranges up to 3 x 256;
    # the d <= 3 sum converts to double exactly, the d >= 4 sum fits in int64
    K = 768
    hi = sum((d + 1) * K * 65 * 65 * 2 ** (7 * (3 - d)) for d in range(4))
    lo = sum((d + 1) * K * 65 * 65 * 2 ** (7 * (8 - d)) for d in range(4, 9))
    assert hi < 2 ** 53 and lo < 2 ** 62
