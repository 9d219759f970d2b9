"""IEEE-754 helpers written from the standard's definitions.

Oracle (test infrastructure only).  Everything here works on exact Python
integers and fractions; no rounding happens except in the one explicit
round-to-nearest-even step of ``round_scaled``.
"""
import math
from fractions import Fraction

# (significand bits incl. the hidden bit, minimum exponent of the LSB, maximum
# unbiased exponent) for the two IEEE binary formats the emulation produces.
BINARY64 = (53, -1074, 1023)
BINARY32 = (24, -149, 127)


def ilogb(x):
    """floor(log2 |x|) for finite nonzero x (the unit in the first place)."""
    if x == 0 or not math.isfinite(x):
        raise ValueError("ilogb of zero or non-finite")
    _, e = math.frexp(x)          # x = f * 2**e with 0.5 <= |f| < 1, exact
    return e - 1


def split_float(x):
    """Exact decomposition x = sign * m * 2**e with integer m >= 0."""
    f = Fraction(x)
    sign = -1 if (f < 0 or (f == 0 and math.copysign(1.0, x) < 0)) else 1
    num, den = abs(f.numerator), f.denominator
    e = 0
    while den > 1:                # den is a power of two for any float
        den >>= 1
        e -= 1
    return sign, num, e


def round_scaled(num, exp2, fmt=BINARY64):
    """Round-to-nearest-even of the exact value num * 2**exp2 into ``fmt``.

    ``num`` is any Python integer.  Subnormal results round once at the
    subnormal LSB; results beyond the largest finite value become +-inf.
    Returns a Python float (binary64); binary32 results are exactly
    representable in it.
    """
    prec, min_lsb, max_exp = fmt
    if num == 0:
        return 0.0
    sign = -1.0 if num < 0 else 1.0
    mag = abs(num)
    lead = mag.bit_length() - 1 + exp2          # exponent of the leading bit
    lsb = max(lead - (prec - 1), min_lsb)       # exponent of the result's LSB
    sh = lsb - exp2
    if sh <= 0:
        q = mag << (-sh)
    else:
        q = mag >> sh
        rem = mag - (q << sh)
        half = 1 << (sh - 1)
        if rem > half or (rem == half and (q & 1)):
            q += 1
    if q == 0:
        return sign * 0.0
    # q * 2**lsb is exactly representable in binary64 for both formats
    if q.bit_length() - 1 + lsb > max_exp:
        return sign * math.inf
    return sign * math.ldexp(float(q), lsb)


def exact_to_binary64(v):
    """RN-even of an exact rational (Fraction or int) into binary64."""
    v = Fraction(v)
    if v == 0:
        return 0.0
    # bring to num * 2**e with enough extra bits, keeping a sticky bit so the
    # integer rounding below sees the true position of the remainder
    n, d = v.numerator, v.denominator
    shift = 64 + d.bit_length() - abs(n).bit_length() + 60
    shift = max(shift, 0)
    qt, rem = divmod(abs(n) << shift, d)
    qt = (qt << 1) | (1 if rem else 0)          # sticky
    r = round_scaled(qt, -shift - 1, BINARY64)
    return -r if n < 0 else r


def fma64(a, b, c):
    """Exact fused multiply-add a*b + c rounded once (IEEE 754 fusedMultiplyAdd)."""
    if not (math.isfinite(a) and math.isfinite(b) and math.isfinite(c)):
        return a * b + c                         # non-finite: same as unfused
    exact = Fraction(a) * Fraction(b) + Fraction(c)
    if exact == 0:
        prod_neg = (math.copysign(1.0, a) * math.copysign(1.0, b)) < 0
        c_neg = math.copysign(1.0, c) < 0
        prod_zero = (a == 0 or b == 0)
        if prod_zero and c == 0 and prod_neg and c_neg:
            return -0.0
        return 0.0
    return exact_to_binary64(exact)
