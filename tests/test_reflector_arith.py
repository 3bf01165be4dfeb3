"""The seeded reflector scalars of the Householder steps (hh_reflector in csrc/la.cuh), emulated
exactly on the CPU and checked against their error bounds.

For a column with squared norm d and pivot entry x_k the kernels form nrm = sqrt(d) and
beta = 2 / ||v||^2, ||v||^2 = (d - x_k^2) + v_k^2 with v_k = x_k + sign(x_k) nrm, from single-precision
seeds (rsqrt.approx / rcp.approx of the mantissa, exponents handled on the integer side) refined by one
third-order step each.  The emulation follows the same bit manipulation and the same sequence of FP64
operations, with every FMA rounded once from its exact value, and seeds equal to the correctly rounded
single-precision results moved by up to 4 ulp (the hardware approximations are within 2).  The checks:
nrm within 2 ulp of the correctly rounded square root, and beta ||v||^2 = 2 within 8 ulp, which is what
keeps H = I - beta v v' orthogonal to rounding.  Exponents outside [-1000, 1000] take the library path.
"""
import math
import struct
from fractions import Fraction

import numpy as np
import pytest


def f64_bits(x):
    return struct.unpack("<q", struct.pack("<d", x))[0]


def bits_f64(b):
    return struct.unpack("<d", struct.pack("<q", b))[0]


def f32_bits(x):
    return struct.unpack("<i", struct.pack("<f", x))[0]


def bits_f32(b):
    return struct.unpack("<f", struct.pack("<i", b))[0]


def fma(a, b, c):
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def mul(a, b):
    return float(Fraction(a) * Fraction(b))


def add(a, b):
    return float(Fraction(a) + Fraction(b))


def seed(value, ulps):
    """Correctly rounded float32 of value, moved by ulps units in the last place."""
    f = np.float32(value)
    step = np.float32(np.inf) if ulps > 0 else np.float32(0.0)
    for _ in range(abs(ulps)):
        f = np.nextafter(f, step)
    return float(f)


def hh_reflector(d, xk, u1=0, u2=0):
    db = f64_bits(d)
    dh = db >> 32
    ex = ((dh >> 20) & 0x7FF) - 1023
    if ex < -1000 or ex > 1000:
        return None
    odd = ex & 1
    h = (ex - odd) >> 1
    m23 = ((dh & 0xFFFFF) << 3) | ((db & 0xFFFFFFFF) >> 29)
    mf = bits_f32(((127 + odd) << 23) | m23)
    yf = f32_bits(seed(1.0 / math.sqrt(mf), u1))
    hi = ((((yf >> 23) & 0xFF) + (1023 - 127) - h) << 20) | ((yf & 0x7FFFFF) >> 3)
    y0 = bits_f64((hi << 32) | ((yf & 7) << 29))
    dx = fma(-xk, xk, d)
    t = mul(d, y0)
    e = fma(-t, y0, 1.0)
    p = fma(0.375, e, 0.5)
    nrm = fma(mul(t, e), p, t)
    neg = xk < 0.0  # sign(x_k) with sign(0) = +1, also for -0
    shift = -nrm if neg else nrm
    vk = add(xk, shift)
    q = fma(vk, vk, dx)
    qb = f64_bits(q)
    qh = qb >> 32
    g = ((qh >> 20) & 0x7FF) - 1023
    n23 = ((qh & 0xFFFFF) << 3) | ((qb & 0xFFFFFFFF) >> 29)
    rf = f32_bits(seed(1.0 / bits_f32((127 << 23) | n23), u2))
    rhi = ((((rf >> 23) & 0xFF) + (1023 - 127) - g) << 20) | ((rf & 0x7FFFFF) >> 3)
    rlo = (rf & 7) << 29
    r0 = bits_f64((rhi << 32) | rlo)
    r2 = bits_f64(((rhi + (1 << 20)) << 32) | rlo)
    f = fma(-q, r0, 1.0)
    beta = fma(r2, fma(f, f, f), r2)
    return nrm, shift, vk, beta, q


def ulp(x):
    return math.ulp(abs(x))


@pytest.mark.parametrize("u1,u2", [(0, 0), (4, -4), (-4, 4), (3, 3), (-3, -3)])
def test_reflector_scalars_within_their_bounds(u1, u2):
    rng = np.random.default_rng(11)
    for _ in range(300):
        e = int(rng.integers(-480, 480))
        x = rng.standard_normal(6) * 2.0 ** e
        d = float(np.dot(x, x))
        xk = float(x[0])
        out = hh_reflector(d, xk, u1, u2)
        assert out is not None
        nrm, shift, vk, beta, q = out
        ref = math.sqrt(d)
        assert abs(nrm - ref) <= 2 * ulp(ref), (d, nrm, ref)
        assert abs(shift) == nrm and (shift > 0) == (xk >= 0)
        # beta ||v||^2 = 2 for the v actually formed
        prod = Fraction(beta) * Fraction(q)
        assert abs(float(prod) - 2.0) <= 8 * ulp(2.0), (d, xk, float(prod))


def test_extreme_exponents_take_the_library_path():
    assert hh_reflector(0.0, 0.0) is None
    assert hh_reflector(5e-324, 0.0) is None                 # subnormal
    assert hh_reflector(2.0 ** -1010, 2.0 ** -506) is None   # below 2^-1000
    assert hh_reflector(2.0 ** 1010, 2.0 ** 505) is None     # above 2^1000
    assert hh_reflector(2.0 ** -1000, 2.0 ** -501) is not None
