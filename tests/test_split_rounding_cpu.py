"""The residue step of the split kernel, checked exhaustively on the CPU.

For every exact float integer |z| < 2^23 (a sum of chunk products) and
modulus p, the split forms the symmetric residue (Section II, ties rounded
up) in float32 as
    q = rint(RN(z * RN(1/p))),   r = z - q p   (one fused multiply-add),
then moves r into [-p/2, p/2) by at most one subtraction or addition of p;
the Karatsuba sum plane applies the same correction to the sum of two
residues.  This is right only if the rounded quotient leaves |r| <= 3p/2 and
z - q p is exact, which rests on a rounding argument (|r| <= p/2 + 1).
This test replays the float32 steps with exact integer arithmetic
(round-to-nearest-even written out) over every z in (-2^23, 2^23) for every
modulus the plans use and checks the result against the definition.
"""
import math

import numpy as np
import pytest

from oracle.moduli import choose_moduli


def _inv_p(p):
    # the plan's RN(1/p): the double quotient rounded to float32
    m, e = math.frexp(float(np.float32(1.0 / p)))     # value = m 2^e, 0.5 <= m < 1
    return int(m * 2 ** 24), 24 - e                  # value = mi 2^-sh


def _rne_shift(a, sh):
    """Round-half-even of a / 2^sh for int64 arrays a and shifts sh >= 1 (array or scalar)."""
    fl = a >> sh
    rem = a - (fl << sh)
    half = np.left_shift(1, sh - 1)
    return fl + (rem > half) + ((rem == half) & (fl & 1))


def _quotient(z, mi, sh):
    """rint(RN_float32(z mi 2^-sh)) for int64 z with |z| < 2^23."""
    n = np.abs(z) * mi                               # exact, < 2^47
    bits = np.frexp(n.astype(np.float64))[1]         # bit length of n (exact: n < 2^53)
    drop = np.maximum(bits - 24, 0)                  # RN to 24 significant bits
    m = np.where(drop > 0, _rne_shift(n, np.maximum(drop, 1)), n)
    # value = m 2^(drop - sh); sh > drop for every z here (the quotient is below 2^23)
    assert np.all(sh - drop >= 1)
    q = _rne_shift(m, sh - drop)
    return np.where(z < 0, -q, q)


def _correct(r, p):
    r = np.where(2 * r >= p, r - p, r)
    return np.where(2 * r < -p, r + p, r)


def _check_definition(z, out, p):
    assert np.all((out - z) % p == 0)
    assert np.all(2 * out >= -p) and np.all(2 * out < p)


@pytest.mark.parametrize("p", choose_moduli(20))
def test_residue_step_is_the_symmetric_remainder(p):
    mi, sh = _inv_p(p)
    lim = 2 ** 23
    step = 1 << 21
    worst = 0
    for lo in range(-lim + 1, lim, step):
        z = np.arange(lo, min(lo + step, lim), dtype=np.int64)
        r = z - _quotient(z, mi, sh) * p             # |z - q p| < 2^24: exact in float32
        worst = max(worst, int(np.abs(2 * r).max()))
        _check_definition(z, _correct(r, p), p)
    # the rounded quotient leaves |r| <= p/2 + 1, so one correction suffices
    assert worst <= p + 2


@pytest.mark.parametrize("p", choose_moduli(20))
def test_karatsuba_sum_correction(p):
    # every sum of two symmetric residues
    a = np.arange(-(p // 2), (p + 1) // 2, dtype=np.int64)
    s = (a[:, None] + a[None, :]).ravel()
    _check_definition(s, _correct(s, p), p)
