"""The arithmetic of the mixed mode's digit cutter (rid_probe_tc.cu,
digit_words_fp), emulated step for step in numpy float32 (round to nearest
even, subnormals kept, as the kernel's __fadd_rn / __fmul_rn / FMA steps) and
checked against exact rational arithmetic.

For a float x in a chunk with exponent e (|x| < 2^e):
  t = x 2^(8-e) (two exact scalings when 2^(8-e) is not a normal float),
  for s = 0..6: d_s = (t + M_s) - M_s with M_s = 1.5 2^(23-8s), t = t - d_s.
Claims the kernel relies on (the exact-slice argument needs them):
  * every d_s is exact in BF16 (the low 16 bits of its float32 are zero),
    d_0 is an integer in [-256, 256] and d_s a multiple of 2^(-8s) with
    |d_s| <= 128 2^(-8s);
  * sum_s d_s is x 2^(8-e) rounded to the grid 2^-48 (within half a grid
    step; a tie goes the way the last digit's rounding takes it);
  * away from ties, the sum equals the integer cutter's (rid_tc_digits.cuh:
    round |x| 2^(56-e) half up, sign applied), so the two cutters feed the
    same value to the products.
No GPU: this pins the steps, not the kernel (the GPU tests compare the
kernel's X with the oracle)."""
from fractions import Fraction

import numpy as np

F32 = np.float32


def exp_of(x):
    """e with 2^(e-1) <= |x| < 2^e; None for zero."""
    if x == 0:
        return None
    return int(np.frexp(np.float64(x))[1])


def pow2(k):
    return F32(np.ldexp(np.float64(1.0), k))


def cut(x, e):
    """The kernel's steps for one real value, in float32."""
    x = F32(x)
    p = 8 - e
    if p <= 127:
        t = F32(x * pow2(p))
    else:                                         # chunks of subnormal floats
        p1 = p >> 1
        t = F32(F32(x * pow2(p1)) * pow2(p - p1))
    digits = []
    for s in range(7):
        M = F32(1.5) * pow2(23 - 8 * s)
        d = F32(F32(t + M) - M)
        digits.append(d)
        if s < 6:
            t = F32(t - d)
    return digits


def integer_cutter_value(x, e):
    """round(|x| 2^(56-e)) half up, with x's sign, as a rational multiple of 2^-48."""
    q = abs(Fraction(float(x))) * Fraction(2) ** (56 - e)
    n = int(q + Fraction(1, 2))                   # floor(q + 1/2): half up
    v = Fraction(n, 2 ** 48)
    return -v if x < 0 else v


def chunk_values(rng, size):
    """float32 values over the whole range: log-uniform magnitudes, signs,
    zeros and subnormals."""
    mag = np.ldexp(rng.random(size) + 0.5, rng.integers(-160, 120, size))
    x = (np.where(rng.random(size) < 0.5, -1.0, 1.0) * mag).astype(np.float32)
    x[rng.random(size) < 0.05] = 0.0
    return x


def check_value(x, e):
    d = cut(x, e)
    for s, v in enumerate(d):
        bits = np.frombuffer(np.float32(v).tobytes(), dtype=np.uint32)[0]
        assert bits & 0xFFFF == 0, (x, e, s, v)                    # exact in BF16
        q = Fraction(float(v)) * Fraction(2) ** (8 * s)
        assert q.denominator == 1, (x, e, s, v)                    # a multiple of 2^(-8s)
        assert abs(q) <= (256 if s == 0 else 128), (x, e, s, v)
    total = sum(Fraction(float(v)) for v in d)
    exact = Fraction(float(x)) * Fraction(2) ** (8 - e)
    assert abs(total - exact) <= Fraction(1, 2 ** 49), (x, e)
    if abs(total - exact) < Fraction(1, 2 ** 49):
        assert total == integer_cutter_value(x, e), (x, e)
    return total


def test_digits_of_random_chunks():
    rng = np.random.default_rng(7)
    for _ in range(40):
        x = chunk_values(rng, 256)
        exps = [exp_of(v) for v in x if v != 0]
        if not exps:
            continue
        e = max(exps)
        for v in x:
            check_value(v, e)


def test_digits_of_narrow_chunks():
    """Chunks whose values share an exponent range (the common case): every
    value is then exact in the 56 bits, so the digits sum to x 2^(8-e)."""
    rng = np.random.default_rng(8)
    for scale in (-140, -100, -20, 0, 30, 120):
        x = (rng.standard_normal(256) * 2.0 ** scale).astype(np.float32)
        e = max(exp_of(v) for v in x if v != 0)
        for v in x:
            total = check_value(v, e)
            assert total == Fraction(float(v)) * Fraction(2) ** (8 - e)


def test_digits_at_the_edges():
    """The largest value of a chunk (t just below 256), ties of the last digit,
    the smallest subnormal, and chunk exponents whose scale 2^(8-e) needs two
    steps."""
    big = np.nextafter(F32(2.0) ** 20, F32(0))           # |x| just below 2^20
    check_value(big, 20)
    check_value(-big, 20)
    tiny = np.float32(np.ldexp(1.0, -149))
    check_value(tiny, -148)                                # a chunk of one subnormal: t = 128
    check_value(tiny, 0)                                   # far below the chunk maximum: all digits 0
    assert all(v == 0 for v in cut(tiny, 0))
    # a value exactly half a grid step above a grid point of 2^-48 (relative to e):
    # x = 2^(e-8) (1 + 2^-49) needs 50 significant bits, so build it from a
    # float with its bits 49 positions below the chunk maximum
    e = 10
    half = np.float32(np.ldexp(1.0, e - 8 - 49))           # t contribution 2^-49: a tie at the last digit
    check_value(half, e)
    for e in (-119, -120, -130, -148):                    # two-step scaling
        x = np.float32(np.ldexp(0.75, e))
        d = cut(x, e)
        assert sum(Fraction(float(v)) for v in d) == Fraction(float(x)) * Fraction(2) ** (8 - e)
