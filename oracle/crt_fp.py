"""The paper's floating-point CRT reconstruction (Section II, eq.
CRTaccumulation, and the double-double reduction described in Section IV-A).

Oracle (test infrastructure only).  Each weight w_l = (P/p_l) q_l is split into
s_l1 + s_l2: s_l1 holds its upper (53 - 7 - ceil(log2 N)) bits and s_l2 the rest
rounded to double.  Readings:

* "upper bits" are taken on a common grid 2^g, g = bitlength(P) - (46 - ceil(log2 N)),
  which is what makes every s_l1 E'_l and their sum exact in double
  (|E'_l| <= 2^7, N terms).
* S2 = sum_l s_l2 E'_l accumulates with fma in ascending l.
* ZGEMM: with P = P_h + P_l (P_h = RN(P), P_l = RN(P - P_h)),
    r  = rint((S1 + S2) / P_h)
    (ph, pe) = r P_h exactly (pe = fma(r, P_h, -ph))
    (hi, lo) = TwoSum(S1, -ph)
    lo = ((lo - pe) - r P_l) + S2       (fma for r P_l: lo = fma(-r, P_l, lo - pe) + S2)
    c' = hi + lo
  CGEMM (double only): S = sum_l RN(w_l) E'_l (fma, ascending l),
    r = rint(S / RN(P)),  c' = fma(-r, RN(P), S).
* Step VI: out = RN(c' 2^-(x_i + y_j)) (ldexp of a double, one rounding when the
  result is subnormal), then the same alpha/beta sequence as the exact path.
"""
import math

import numpy as np

from . import fp
from .moduli import Plan


def split_weights(plan):
    N = plan.N
    g = plan.P.bit_length() - (46 - math.ceil(math.log2(N)))
    s1, s2 = [], []
    for w in plan.w:
        hi = (w >> g) << g if g > 0 else w
        s1.append(float(hi))                      # <= 46 significant bits: exact
        s2.append(fp.exact_to_binary64(w - hi))
    return s1, s2, g


def two_sum(a, b):
    s = a + b
    bb = s - a
    return s, (a - (s - bb)) + (b - bb)


def reconstruct_z(Ep, plan):
    """c' (a double) from the residues E'_l of one entry (list of ints), ZGEMM form."""
    s1, s2, _ = split_weights(plan)
    S1 = 0.0
    for l, e in enumerate(Ep):
        S1 = S1 + s1[l] * float(e)                # exact by construction
    S2 = 0.0
    for l, e in enumerate(Ep):
        S2 = fp.fma64(s2[l], float(e), S2)
    Ph = float(plan.P)                            # RN(P): CPython int->float is correctly rounded
    Pl = fp.exact_to_binary64(plan.P - int(Ph))
    r = float(round((S1 + S2) / Ph))              # round-half-even, like rint
    ph = r * Ph
    pe = fp.fma64(r, Ph, -ph)
    hi, lo = two_sum(S1, -ph)
    lo = fp.fma64(-r, Pl, lo - pe) + S2
    return hi + lo


def reconstruct_c(Ep, plan):
    """c' from the residues of one entry, CGEMM form (double precision)."""
    S = 0.0
    for l, e in enumerate(Ep):
        S = fp.fma64(float(plan.w[l]), float(e), S)
    Pd = float(plan.P)
    r = float(round(S / Pd))
    return fp.fma64(-r, Pd, S)


def unscale(c, e2):
    """RN(c 2^e2) for a double c."""
    if c == 0.0 or not math.isfinite(c):
        return c * 1.0
    sign, num, e = fp.split_float(c)
    return sign * fp.round_scaled(num, e + e2)


def outputs(em, single=False, alpha=(1.0, 0.0), beta=(0.0, 0.0), C_in=None):
    """Step V-v..VI of the paper's floating-point CRT for every entry of an
    oracle Emulation `em` (uses its residues E'_l and exponents)."""
    plan = em.plan
    m, n = em.m, em.n
    o = np.zeros((m, n), dtype=np.complex128)
    rec = reconstruct_c if single else reconstruct_z
    for i in range(m):
        for j in range(n):
            if em.flag_a[i] or em.flag_b[j]:
                o[i, j] = complex(np.nan, np.nan)
                continue
            e2 = -(int(em.x[i]) + int(em.y[j]))
            cr = rec([int(v) for v in em.Eprime[:, 0, i, j]], plan)
            ci = rec([int(v) for v in em.Eprime[:, 1, i, j]], plan)
            o[i, j] = complex(unscale(cr, e2), unscale(ci, e2))
    ar, ai = float(alpha[0]), float(alpha[1])
    br, bi = float(beta[0]), float(beta[1])
    if (ar, ai, br, bi) != (1.0, 0.0, 0.0, 0.0):
        res = np.zeros_like(o)
        for i in range(m):
            for j in range(n):
                orr, oi = o[i, j].real, o[i, j].imag
                tr = fp.fma64(ar, orr, -(ai * oi))
                ti = fp.fma64(ar, oi, ai * orr)
                if br != 0.0 or bi != 0.0:
                    cr, ci = float(np.real(C_in[i, j])), float(np.imag(C_in[i, j]))
                    tr = fp.fma64(br, cr, fp.fma64(-bi, ci, tr))
                    ti = fp.fma64(br, ci, fp.fma64(bi, cr, ti))
                res[i, j] = complex(tr, ti)
        o = res
    return o.astype(np.complex64) if single else o


def outputs_real(em, single=False, alpha=1.0, beta=0.0, C_in=None):
    """Steps V-v..VI of the floating-point CRT for a real emulation `em`
    (oracle.emulate_real.RealEmulation): the DGEMM form (S1 + S2, double-double
    reduction) for binary64 output, the single double sum for binary32."""
    from .emulate_real import finish_real
    plan = em.plan
    rec = reconstruct_c if single else reconstruct_z
    o = np.zeros((em.m, em.n), dtype=np.float64)
    for i in range(em.m):
        for j in range(em.n):
            if em.flag_a[i] or em.flag_b[j]:
                o[i, j] = np.nan
                continue
            c = rec([int(v) for v in em.Eprime[:, i, j]], plan)
            o[i, j] = unscale(c, -(int(em.x[i]) + int(em.y[j])))
    return finish_real(o, alpha, beta, C_in, fp.BINARY32 if single else fp.BINARY64)


__all__ = ["split_weights", "reconstruct_z", "reconstruct_c", "outputs", "outputs_real", "Plan"]
