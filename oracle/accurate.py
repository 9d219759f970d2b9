"""Accurate-mode scaling vectors (Section III-B, eqs. mu-accu / nu-accu).

Oracle (test infrastructure only).

Steps, in the paper's order:

1. Pre-scaling: mu-bar_i = 2^(5 - e_i) with e_i the unit in the first place
   of the largest |entry| of row i of A-hat (Re and Im of row i of op(A)), so
   the integer parts of the scaled row fit in 6 bits; likewise nu-bar_j for
   the columns of B-hat.
2. Ceiling: A-bar_R = ceil(|mu-bar A_R|), A-bar_I = ceil(|mu-bar A_I|),
   B-bar_R, B-bar_I likewise: integers in [0, 64], upper bounds of the
   pre-scaled magnitudes.
3. Bound product: C-bar_I = A-bar_I B-bar_R + A-bar_R B-bar_I and
   C-bar_R = C-bar_I + (A-bar_R - A-bar_I)(B-bar_R - B-bar_I)
   (= A-bar_R B-bar_R + A-bar_I B-bar_I); real input: C-bar = A-bar B-bar.
4. mu_i = mu-bar_i 2^floor(P'_accu - delta log2 max_j max(C-bar_R, C-bar_I)_ij),
   P'_accu = log2(P-1)/2 - 0.5; nu_j with the maximum over i.

Readings:
* As in fast mode (R5), the floor is decided exactly instead of through
  single-precision log2 with a round-down delta: since 2^(2 P'_accu) = (P-1)/2,
  E_i = max{E : 4^E max(M_i, 1) <= (P-1)/2} with M_i the row maximum of step 4,
  and x_i = 5 - e_i + E_i.  This satisfies condition (cond) exactly:
  sum_h |a'_ih||b'_hj| <= 2^(E_i + F_j) C-bar_ij <= sqrt(4^E_i M_i 4^F_j N_j)
  <= (P-1)/2.  max(M_i, 1) covers rows whose bound products are all zero.
* A row of op(A) (column of op(B)) holding Inf or NaN is flagged as in fast
  mode (its output row/column is NaN) and enters steps 2-3 as zeros, so it
  does not lower the other rows' scales.
* An all-zero row gets e_i = 0 (as in fast mode).
"""
import math

import numpy as np

from .emulate import int_matmul
from .scaling import NONFINITE

PRE_BITS = 5            # mu-bar = 2^(5 - e): scaled magnitudes below 2^6


def exponent_accu(M, P):
    """Largest integer E with 4^E * max(M, 1) <= (P - 1) / 2 (exact)."""
    M = max(int(M), 1)
    X = P - 1                      # 4^E * M <= X / 2  <=>  2 * 4^E * M <= X
    if 2 * M <= X:
        Q = X // (2 * M)
        return (Q.bit_length() - 1) // 2
    t = 1
    while 2 * M > X * 4 ** t:
        t += 1
    return -t


def prescale(V):
    """Step 1-2 for the rows of V (rows x entries, float64): (e, flag, Vbar),
    Vbar = ceil(|V| 2^(5 - e)) as int64 (zero on flagged rows)."""
    V = np.asarray(V, dtype=np.float64)
    rows = V.shape[0]
    e = np.zeros(rows, dtype=np.int64)
    flag = np.zeros(rows, dtype=bool)
    Vbar = np.zeros(V.shape, dtype=np.int64)
    for r in range(rows):
        v = V[r]
        if not np.all(np.isfinite(v)):
            flag[r] = True
            continue
        a = np.abs(v)
        amax = a.max() if a.size else 0.0
        if amax == 0.0:
            continue
        e[r] = math.frexp(float(amax))[1] - 1
        sc = np.ldexp(a, PRE_BITS - int(e[r]))     # exact power-of-two scaling (or underflow to 0)
        # ceil of |v| 2^(5-e); a nonzero entry that underflows has ceiling 1
        Vbar[r] = np.where(a != 0, np.maximum(np.ceil(sc), 1.0), 0.0).astype(np.int64)
    return e, flag, Vbar


def accurate_exponents(A, B, P, real=False):
    """x (rows of op(A)), y (columns of op(B)) and the intermediates.

    A: m x k, B: k x n after op(), complex (or real with real=True).
    Returns a dict with x, y, flag_a, flag_b, e_a, e_b, the A-bar / B-bar
    planes, C-bar products, row/column maxima M, Ncol and E, F.
    """
    A = np.asarray(A)
    B = np.asarray(B)
    m, k = A.shape
    n = B.shape[1]
    if real:
        e_a, fa, Abar = prescale(A.real.astype(np.float64))
        e_b, fb, BbarT = prescale(B.real.T.astype(np.float64))
        Cbar = int_matmul(Abar, BbarT.T)
        CR = CI = Cbar
        planes = {"A": Abar, "B": BbarT.T}
    else:
        # the pre-scaling exponent of a row of A-hat covers Re and Im together
        e_a, fa, hatA = prescale(np.concatenate([A.real, A.imag], axis=1))
        e_b, fb, hatB = prescale(np.concatenate([B.real.T, B.imag.T], axis=1))
        AR, AI = hatA[:, :k], hatA[:, k:]
        BR, BI = hatB[:, :k].T, hatB[:, k:].T
        CI = int_matmul(AI, BR) + int_matmul(AR, BI)
        CR = CI + int_matmul(AR - AI, BR - BI)
        planes = {"AR": AR, "AI": AI, "BR": BR, "BI": BI}
    both = np.maximum(CR, CI)
    M = both.max(axis=1) if n else np.zeros(m, dtype=np.int64)
    Ncol = both.max(axis=0) if m else np.zeros(n, dtype=np.int64)
    E = np.array([exponent_accu(v, P) for v in M], dtype=np.int64)
    F = np.array([exponent_accu(v, P) for v in Ncol], dtype=np.int64)
    x = np.where(fa, NONFINITE, PRE_BITS - e_a + E)
    y = np.where(fb, NONFINITE, PRE_BITS - e_b + F)
    return dict(x=x, y=y, flag_a=fa, flag_b=fb, e_a=e_a, e_b=e_b, CR=CR, CI=CI, M=M, Ncol=Ncol, E=E, F=F,
                **planes)


__all__ = ["exponent_accu", "prescale", "accurate_exponents", "PRE_BITS"]
