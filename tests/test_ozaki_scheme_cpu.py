"""The arithmetic facts the FP64 emulation on the BF16 tensor cores rests on (Ozaki splitting with
balanced base-128 digits), checked on the CPU in exact integer and rational arithmetic, apart from
the kernel:

* a value |x| < sigma / 2, truncated towards zero to 56 fraction bits of sigma, is exactly eight
  balanced base-128 digits, the seven lower ones in [-64, 63] and the leading one in [-65, 65];
  each digit is exact in BF16;
* the fixed-point value of a + b is the sum of those of a and b, within 2^-55 sigma of a + b;
* a diagonal of the digit products (at most 8 pairs, |t u| <= 65^2) accumulates exactly in FP32 for
  384 K values: 8 * 65^2 * 384 < 2^24;
* dropping the diagonals s + r >= 10 and the truncations cost below 2^-54.5 sigma tau per K value
  and real product, so a product of K terms is within K 2^-54.5 sigma tau of the exact one.
No GPU."""
from fractions import Fraction

import numpy as np
import pytest

FRAC = 56
S = 8


def fixed(x):
    """x (|x| < 1/2, a double) truncated towards zero to FRAC fraction bits, as an integer."""
    return int(np.ldexp(x, FRAC))   # scaling by 2^56 is exact; int() truncates towards zero


def digits(v):
    """Balanced base-128 digits t_1..t_S of the integer v (weight 2^(56 - 7 s)), t_1 leading."""
    out = []
    for _ in range(S - 1):
        d = ((v + 64) % 128) - 64
        out.append(d)
        v = (v - d) // 128
    out.append(v)
    return out[::-1]


def _samples(rng, n):
    x = rng.uniform(-0.5, 0.5, n)
    x[:8] = [np.nextafter(0.5, 0), -np.nextafter(0.5, 0), 0.0, 2.0 ** -60, -2.0 ** -57, 2.0 ** -1000,
             0.25, -0.375]
    return x


def test_balanced_digits_are_exact_and_bounded():
    rng = np.random.default_rng(1)
    torch = pytest.importorskip("torch")
    for x in _samples(rng, 4000):
        v = fixed(x)
        assert abs(Fraction(x) - Fraction(v, 2 ** FRAC)) < Fraction(1, 2 ** FRAC)
        t = digits(v)
        assert sum(d * 128 ** (S - 1 - s) for s, d in enumerate(t)) == v
        assert -65 <= t[0] <= 65 and all(-64 <= d <= 63 for d in t[1:])
    # every digit value is exact in BF16
    vals = torch.arange(-65, 66, dtype=torch.float32)
    assert torch.equal(vals.to(torch.bfloat16).to(torch.float32), vals)


def test_sum_operand_is_the_exact_sum_of_the_fixed_points():
    rng = np.random.default_rng(2)
    a, b = rng.uniform(-0.5, 0.5, 4000), rng.uniform(-0.5, 0.5, 4000)
    keep = np.abs(a + b) < 0.5          # sigma bounds all three operands: re, im and re + im
    for x, y in zip(a[keep], b[keep]):
        v = fixed(x) + fixed(y)
        assert abs(Fraction(x) + Fraction(y) - Fraction(v, 2 ** FRAC)) < Fraction(2, 2 ** FRAC)
        t = digits(v)
        assert -65 <= t[0] <= 65 and all(-64 <= d <= 63 for d in t[1:])


def test_fp32_diagonal_accumulation_is_exact_for_384_k_values():
    assert 8 * 65 ** 2 * 384 < 2 ** 24
    rng = np.random.default_rng(3)
    for extreme in (False, True):
        if extreme:
            p = np.full((384, 8), 65 * 65, np.int64)
        else:
            p = rng.integers(-65, 66, (384, 8)) * rng.integers(-65, 66, (384, 8))
        acc = np.float32(0.0)
        for k in range(384):
            for q in range(8):
                acc = np.float32(acc + np.float32(p[k, q]))
        assert int(acc) == int(p.sum())
    # one more chunk of worst-case odd products would no longer be exact
    assert 2 * 8 * 65 ** 2 * 384 > 2 ** 24


def test_dropped_diagonals_and_truncation_stay_below_the_stated_bound():
    # truncation: 2^-56 per operand times |other| < 1/2, two operands
    trunc = Fraction(2, 2 ** FRAC) * Fraction(1, 2)
    # dropped diagonals d = s + r >= 10 with s, r in 1..8, so both digits are non-leading
    # (|t| <= 64); digit s carries the weight 2^(-7 s) of sigma, a pair 2^(-7 (s + r))
    drop = sum(Fraction(64 * 64, 2 ** (7 * (s + r)))
               for s in range(1, S + 1) for r in range(1, S + 1) if s + r >= 10)
    total = trunc + drop
    assert float(drop) < 2 ** -55.15 and float(total) < 2 ** -54.5


def _emulated_dot(x, y):
    """The kept digit products (diagonals s + r <= S + 1) of x . y, exactly."""
    tx = [digits(fixed(v)) for v in x]
    ty = [digits(fixed(v)) for v in y]
    acc = Fraction(0)
    for k in range(len(x)):
        for s in range(S):
            for r in range(S):
                if (s + 1) + (r + 1) <= S + 1:
                    acc += Fraction(tx[k][s] * ty[k][r], 2 ** (7 * (s + 1) + 7 * (r + 1)))
    return acc


def test_emulated_dot_product_is_within_k_times_the_bound():
    rng = np.random.default_rng(4)
    for K in (16, 384, 1000):
        x = rng.uniform(-0.5, 0.5, K) * (2.0 ** -rng.integers(0, 40, K))   # a row spanning 2^-40..1
        y = rng.uniform(-0.5, 0.5, K)
        exact = sum(Fraction(a) * Fraction(b) for a, b in zip(x, y))
        assert abs(float(_emulated_dot(x, y) - exact)) < K * 2.0 ** -54.5
    # the bound nearly attained: every digit of both operands large and of one sign, so the dropped
    # diagonals of all K terms add up (the value has 53 bits, so nothing is truncated)
    v = float(sum(Fraction(63, 2 ** (7 * s)) for s in range(1, S + 1)))
    assert fixed(v) == Fraction(v) * 2 ** FRAC
    K = 384
    x = np.full(K, v)
    err = abs(float(_emulated_dot(x, x) - K * Fraction(v) ** 2))
    assert K * 2.0 ** -56 < err < K * 2.0 ** -54.5
