"""Exact single- and double-precision arithmetic on rationals, in pure Python.

Used only by the tests, to brute-force tiny dwell maps without any C
compiler, libm or hardware FMA in the loop: every operation is carried out
exactly on ``fractions.Fraction`` values and then rounded once to the
nearest float32 (ties to even), which is what IEEE 754 prescribes for a
single-precision add, multiply and fused multiply-add.  The ``*64``
functions do the same with rounding to the nearest binary64 value (53-bit
significand), for the double-precision maps of deep zooms.
"""
from fractions import Fraction
import struct

_HALF = Fraction(1, 2)


def _round(q, bits, emin, emax):
    """Round the rational ``q`` to the nearest binary floating-point value
    with a ``bits``-bit significand, smallest normal exponent ``emin`` and
    overflow threshold 2**emax (ties to even)."""
    q = Fraction(q)
    if q == 0:
        return Fraction(0)
    sign = -1 if q < 0 else 1
    a = -q if q < 0 else q
    e = a.numerator.bit_length() - a.denominator.bit_length()
    # normalise so that 2**e <= a < 2**(e+1)
    while Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    quantum_exp = max(e - (bits - 1), emin - (bits - 1))   # subnormals below 2**emin
    scaled = a / Fraction(2) ** quantum_exp
    fl = scaled.numerator // scaled.denominator
    rem = scaled - fl
    if rem > _HALF or (rem == _HALF and fl % 2 == 1):
        fl += 1
    res = fl * Fraction(2) ** quantum_exp
    if res >= Fraction(2) ** emax:
        raise OverflowError("overflow in a brute-force case")
    return sign * res


def rn32(q):
    """Round the rational ``q`` to the nearest float32 (ties to even)."""
    return _round(q, 24, -126, 128)


def rn64(q):
    """Round the rational ``q`` to the nearest binary64 double (ties to even)."""
    return _round(q, 53, -1022, 1024)


def f32(x):
    """The float32 value nearest to a Python number, as a Fraction."""
    return rn32(Fraction(x))


def to_float(q):
    """A Fraction that is a float32 value, back to a Python float (exact)."""
    v = float(q)
    assert struct.unpack("f", struct.pack("f", v))[0] == v
    return v


def dwell(cr, ci, max_dwell, le=False):
    """Dwell by exact rounding: the same definition as the C reference,
    restated independently (continue while |z|^2 < 4, one update per pass)."""
    cr, ci = f32(cr), f32(ci)
    zr = zi = Fraction(0)
    d = 0
    while d < max_dwell:
        zi2 = rn32(zi * zi)
        m = rn32(zr * zr + zi2)
        if not (m <= 4 if le else m < 4):
            break
        t = rn32(-zi * zi + cr)
        nzr = rn32(zr * zr + t)
        nzi = rn32(rn32(zr + zr) * zi + ci)
        zr, zi = nzr, nzi
        d += 1
    return d


def pixel_c(window, n, px, py):
    re_min, re_max, im_min, im_max = (f32(v) for v in window)
    dx = rn32(rn32(re_max - re_min) / n)
    dy = rn32(rn32(im_max - im_min) / n)
    return rn32(px * dx + re_min), rn32(py * dy + im_min)


def exhaustive(window, n, max_dwell):
    out = [[0] * n for _ in range(n)]
    for py in range(n):
        for px in range(n):
            cr, ci = pixel_c(window, n, px, py)
            out[py][px] = dwell(cr, ci, max_dwell)
    return out


# --------------------------------------------------------------------------
# double precision: the same definitions with every operation rounded once
# to binary64
# --------------------------------------------------------------------------
def f64(x):
    """The double nearest to a Python number, as a Fraction."""
    return rn64(Fraction(x))


def dwell64(cr, ci, max_dwell, le=False):
    """Dwell with each operation rounded once to double."""
    cr, ci = f64(cr), f64(ci)
    zr = zi = Fraction(0)
    d = 0
    while d < max_dwell:
        zi2 = rn64(zi * zi)
        m = rn64(zr * zr + zi2)
        if not (m <= 4 if le else m < 4):
            break
        t = rn64(-zi * zi + cr)
        nzr = rn64(zr * zr + t)
        nzi = rn64(rn64(zr + zr) * zi + ci)
        zr, zi = nzr, nzi
        d += 1
    return d


def pixel_c64(window, n, px, py):
    re_min, re_max, im_min, im_max = (f64(v) for v in window)
    dx = rn64(rn64(re_max - re_min) / n)
    dy = rn64(rn64(im_max - im_min) / n)
    return rn64(px * dx + re_min), rn64(py * dy + im_min)


def exhaustive64(window, n, max_dwell):
    out = [[0] * n for _ in range(n)]
    for py in range(n):
        for px in range(n):
            cr, ci = pixel_c64(window, n, px, py)
            out[py][px] = dwell64(cr, ci, max_dwell)
    return out


# --------------------------------------------------------------------------
# float-float: a value is (hi, lo), two float32 values; every float
# operation below is rounded once (rn32), the fused multiply-adds included
# --------------------------------------------------------------------------
def _fast_two_sum(a, b):
    s = rn32(a + b)
    return s, rn32(b - rn32(s - a))


def _two_sum(a, b):
    s = rn32(a + b)
    bb = rn32(s - a)
    return s, rn32(rn32(a - rn32(s - bb)) + rn32(b - bb))


def ff_add(x, y):
    s, e = _two_sum(x[0], y[0])
    return _fast_two_sum(s, rn32(e + rn32(x[1] + y[1])))


def ff_mul(x, y):
    p = rn32(x[0] * y[0])
    e = rn32(x[0] * y[0] - p)
    e = rn32(x[0] * y[1] + e)
    e = rn32(x[1] * y[0] + e)
    return _fast_two_sum(p, e)


def ff_sqr(x):
    p = rn32(x[0] * x[0])
    e = rn32(x[0] * x[0] - p)
    e = rn32(rn32(x[0] + x[0]) * x[1] + e)
    return _fast_two_sum(p, e)


def ff_from_double(v):
    v = f64(v)
    hi = rn32(v)
    return hi, rn32(v - hi)


def dwell_ff(cr, ci, max_dwell, le=False):
    """Dwell in float-float arithmetic with c given in double."""
    cr, ci = ff_from_double(cr), ff_from_double(ci)
    zr = zi = (Fraction(0), Fraction(0))
    d = 0
    while d < max_dwell:
        zr2, zi2 = ff_sqr(zr), ff_sqr(zi)
        m = rn32(zr2[0] + zi2[0])
        if not (m <= 4 if le else m < 4):
            break
        nzr = ff_add(zr2, ff_add(cr, (-zi2[0], -zi2[1])))
        p = ff_mul(zr, zi)
        nzi = ff_add((2 * p[0], 2 * p[1]), ci)
        zr, zi = nzr, nzi
        d += 1
    return d
