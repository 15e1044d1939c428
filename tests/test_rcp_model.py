"""A host model of the element kernels' FP64 reciprocal (element.cuh,
rcp_pos), which scales the gradient products by 1 / (6 |det J|).

For y = m 2^k with m in [1, 2): an FP32 reciprocal of m truncated to 24 bits
(IEEE round to nearest, as __frcp_rn) seeds r; one third-order Newton step
r + r (e + e^2) with e = 1 - m r, each step one fused multiply-add; then
2^-k goes back into the exponent.  The model runs those operations with
exact rational products and one rounding per FMA, and checks the result
against the exact reciprocal: within one ulp everywhere, the correctly
rounded value nearly always, and exact on powers of two.  The GPU test
(test_gpu_rcp.py) holds the device helper to CUDA's division.
"""
import random
import struct
from fractions import Fraction

import numpy as np


def _bits(x):
    return struct.unpack("<q", struct.pack("<d", x))[0]


def _dbl(b):
    return struct.unpack("<d", struct.pack("<q", b))[0]


def _fma(a, b, c):
    return float(Fraction(a) * Fraction(b) + Fraction(c))  # one rounding (Python rounds Fractions correctly)


def rcp_model(y):
    b = _bits(y)
    ex = (b >> 52) & 0x7FF
    if b < 0 or ex < 1023 - 1000 or ex > 1023 + 1000:
        return 1.0 / y
    m = _dbl((b & 0x000FFFFFFFFFFFFF) | 0x3FF0000000000000)
    mf = np.frombuffer(struct.pack("<I", 0x3F800000 | ((b >> 29) & 0x7FFFFF)), dtype=np.float32)[0]
    r = float(np.float32(1.0) / mf)
    e = _fma(-m, r, 1.0)
    r = _fma(r, _fma(e, e, e), r)
    return _dbl(_bits(r) - ((ex - 1023) << 52))


def _ulps(a, b):
    return abs(_bits(a) - _bits(b))


def test_seed_error_bound():
    # the FP32 seed of m in [1, 2) is within 2^-22 of 1 / m (truncation to 24
    # bits, then a rounded reciprocal): the Newton step's e^3 term is < 2^-66
    rng = random.Random(7)
    worst = 0.0
    for _ in range(20000):
        m = rng.uniform(1.0, 2.0)
        b = _bits(m)
        mf = np.frombuffer(struct.pack("<I", 0x3F800000 | ((b >> 29) & 0x7FFFFF)), dtype=np.float32)[0]
        r = float(np.float32(1.0) / mf)
        worst = max(worst, abs(float(1 - Fraction(m) * Fraction(r))))
    assert worst < 2.0 ** -22


def test_within_one_ulp_and_nearly_always_rounded():
    rng = random.Random(11)
    ys = [1.0, 1.5, 3.0, 6.0, 1 - 2.0 ** -53, 1 + 2.0 ** -52, 2 - 2.0 ** -52, 2.0 ** -1000, 2.0 ** 1000]
    ys += [rng.uniform(1.0, 2.0) for _ in range(4000)]
    ys += [rng.uniform(1.0, 2.0) * 2.0 ** rng.randint(-990, 990) for _ in range(4000)]
    exact = 0
    for y in ys:
        want = float(Fraction(1) / Fraction(y))
        got = rcp_model(y)
        assert _ulps(got, want) <= 1, y
        exact += got == want
    assert exact / len(ys) > 0.999


def test_powers_of_two_exact_and_fallback_is_the_division():
    for k in range(-1000, 1001, 7):
        assert rcp_model(2.0 ** k) == 2.0 ** -k
    for y in (2.0 ** -1001, 2.0 ** 1001, 1e-310, 5e-324, 1.7e308, -2.0, float("inf")):
        assert rcp_model(y) == 1.0 / y
    # scaling by a power of two scales the result exactly (same mantissa path)
    rng = random.Random(3)
    for _ in range(500):
        y, k = rng.uniform(1.0, 2.0), rng.randint(-900, 900)
        assert rcp_model(y * 2.0 ** k) == rcp_model(y) * 2.0 ** -k
