"""The pivot reciprocal square root of the FP64 q x q core, checked on the CPU: an FP32 estimate y0 of
1 / sqrt(d) (good to a few FP32 ulps) refined by one step of the series (1 - r)^(-1/2) = 1 + r/2 +
3 r^2 / 8 + ..., r = 1 - d y0^2, evaluated as the kernel does it (t = d y0; r = fma(-t, y0, 1);
c = fma(3/8, r, 1/2); yr = y0 r; y = fma(yr, c, y0)), each operation rounded once to binary64.
The result must be within a few binary64 ulps of 1 / sqrt(d) over the range the kernel uses it for."""
import math
from fractions import Fraction

import numpy as np


def _rn(x: Fraction) -> float:
    return float(x)  # Fraction -> float rounds to nearest (ties to even)


def _mul(a, b):
    return _rn(Fraction(a) * Fraction(b))


def _fma(a, b, c):
    return _rn(Fraction(a) * Fraction(b) + Fraction(c))


def _pivot_rsqrt(d: float, y0: float) -> float:
    t = _mul(d, y0)
    r = _fma(-t, y0, 1.0)
    c = _fma(0.375, r, 0.5)
    yr = _mul(y0, r)
    return _fma(yr, c, y0)


def _exact_rsqrt(d: float) -> Fraction:
    # 1 / sqrt(d) to ~120 bits: integer square root of d scaled by 4^k
    f = Fraction(d)
    k = 240
    num = f.numerator * (1 << (2 * k)) // f.denominator
    s = math.isqrt(num)  # ~ sqrt(d) 2^k
    return Fraction(1 << k, s)


def _ulps(y: float, exact: Fraction) -> float:
    err = abs(Fraction(y) - exact)
    return float(err / Fraction(math.ulp(float(exact))))


def test_one_cubic_step_reaches_binary64_accuracy():
    rng = np.random.default_rng(11)
    ds = [1e-30, 3.7e-21, 1e-8, 0.5, 1.0, 2.0, 3.0, 1234.5, 16384.0, 6.02e23, 9.99e29]
    ds += list(10.0 ** rng.uniform(-30, 30, size=200))
    worst = 0.0
    for d in ds:
        d = float(d)
        base = np.float32(1.0) / np.sqrt(np.float32(d))
        for shift in (-2, -1, 0, 1, 2):  # an FP32 estimate off by up to two FP32 ulps
            y32 = base
            for _ in range(abs(shift)):
                y32 = np.nextafter(y32, np.float32(np.inf if shift > 0 else -np.inf))
            y = _pivot_rsqrt(d, float(y32))
            worst = max(worst, _ulps(y, _exact_rsqrt(d)))
    assert worst <= 2.0, worst


def test_series_step_gains_the_cube_of_the_estimate_error():
    # without rounding, the step leaves the error of the r^3 term: a 2^-20 estimate gives ~2^-57
    d = Fraction(7 / 3)  # the binary64 value nearest 7/3, so that exact below is its 1 / sqrt
    exact = _exact_rsqrt(float(d))
    y0 = exact * (1 + Fraction(1, 1 << 20))
    r = 1 - d * y0 * y0
    y = y0 + y0 * r * (Fraction(1, 2) + Fraction(3, 8) * r)
    rel = abs(y - exact) / exact
    assert rel < Fraction(1, 1 << 54), float(rel)
