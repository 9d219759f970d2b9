"""The residue step of the split kernel, checked exhaustively on the CPU.

The split forms, for every exact float integer |z| < 2^23 and modulus p, the
symmetric residue (Section II, ties rounded up) in two float32 steps:
    q = RN(z * RN(1/p) + 1.5 2^23) - 1.5 2^23,   r = z - q p
    f = RN((r + 1/4) * RN(1/p) + 1.5 2^23) - 1.5 2^23,   result r - f p
and applies the second step alone to the Karatsuba sum of two residues
(|s| <= p).  Its correctness rests on a rounding argument (q within
1/2 + 1/(2p) of z/p; (r + 1/4)/p at least 1/(4p) from a half-integer).
This test replays both steps with exact integer arithmetic (float32
round-to-nearest-even of a fused product-sum, written out) over every
z in (-2^23, 2^23) for every modulus the plans use, and checks the result
against the definition.
"""
import math

import numpy as np
import pytest

from oracle.moduli import choose_moduli

ROUND = 3 * 2 ** 22                  # 1.5 2^23


def _inv_p(p):
    # the plan's RN(1/p): the double quotient rounded to float32
    m, e = math.frexp(float(np.float32(1.0 / p)))     # value = m 2^e, 0.5 <= m < 1
    mi = int(m * 2 ** 24)
    return mi, 24 - e                                # value = mi 2^-sh


def _rne_shift(a, sh):
    """Round-half-even of a / 2^sh for int64 arrays a (sh >= 1)."""
    fl = a >> sh
    rem = a - (fl << sh)
    half = 1 << (sh - 1)
    return fl + (rem > half) + ((rem == half) & (fl & 1))


def _fused_round(num, sh):
    """RN(num 2^-sh + 1.5 2^23) - 1.5 2^23 in float32 (|num 2^-sh| < 2^22):
    the sum lies in [2^23, 2^24), where float32 spacing is 1 and 1.5 2^23
    is even, so this is round-half-even of num 2^-sh."""
    return _rne_shift(num, sh)


def _fix(r, p, mi, sh):
    f = _fused_round((4 * r + 1) * mi, sh + 2)      # (r + 1/4) RN(1/p), exact product
    return r - f * p


def _sym_mod_step(z, p, mi, sh):
    q = _fused_round(z * mi, sh)
    r = z - q * p
    return _fix(r, p, mi, sh), r


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
        out, r = _sym_mod_step(z, p, mi, sh)
        worst = max(worst, int(np.abs(2 * r).max()))
        _check_definition(z, out, p)
    # the first step alone already lands within p/2 + 1/2
    assert worst <= p + 1


@pytest.mark.parametrize("p", choose_moduli(20))
def test_karatsuba_sum_correction(p):
    mi, sh = _inv_p(p)
    # every sum of two symmetric residues, and the whole range |s| <= p + 1
    s = np.arange(-p - 1, p + 2, dtype=np.int64)
    _check_definition(s, _fix(s, p, mi, sh), p)
