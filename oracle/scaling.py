"""Fast-mode scaling vectors (Section III-B, eqs. mu-fast and nu-fast).

Oracle (test infrastructure only).

The complex matrices enter through their real 2x2 block forms (Section III,
eq. complex-matrix-representation).  Row i of A-hat holds Re A(i,:) and
Im A(i,:) (with a sign that does not matter here), and rows i and i+m have
equal norms, so one scaling exponent serves both (Section III-B).  Likewise
column j of B-hat holds Re B(:,j) and Im B(:,j).

The paper bounds sum_h |a'_ih||b'_hj| by Cauchy-Schwarz and picks
mu_i = 2^(floor(P'_fast - max(1, log2 ||t_i||)) - e_i), with
e_i = floor(log2 max_h |a-hat_ih|) (ilogb) and P'_fast = log2(P-1)/2 - 1.5.

Readings taken here (the paper is ambiguous or implementation-specific):

* The norm is taken of the row normalised by its unit in the first place,
  t_h = a-hat_ih * 2^-e_i, so that the bound is scale invariant.  Read
  literally with the raw row the formula breaks condition (cond) for rows of
  small magnitude.
* The paper evaluates log2 with __log2f, a round-down delta and round-down
  FMA, which no CPU can reproduce.  Here the same inequality is decided
  exactly: since 2^(2 P'_fast) = (P-1)/8, the exponent
      E_i = floor(P'_fast - max(1, 0.5 log2 sum_h t_h^2))
  is the largest integer E with 4^E * max(4, sum_h t_h^2) <= (P-1)/8.
* sum_h t_h^2 is replaced by the upper bound sum_h ceil(|t_h| 2^15)^2 / 2^30,
  an exact integer that every evaluation order gives alike.  Multiplying by
  2^30: E_i = max{E : 4^E * max(2^32, S_i) <= (P-1) * 2^27},
  S_i = sum_h ceil(|t_h| * 2^15)^2.
* An all-zero row gets e_i = 0.  A row holding Inf or NaN is flagged; its
  output row is NaN (the paper is silent on non-finite inputs).

Then x_i = E_i - e_i and mu_i = 2^x_i (stored as an int16 exponent, Section
III-C).  |trunc(a-hat_ih mu_i)| <= |t_h| 2^E_i < 2^(E_i+1).
"""
import math

import numpy as np

SUM_FRAC_BITS = 15          # t is quantised up to a multiple of 2^-15
NONFINITE = -32768          # int16 marker for a flagged row/column


def exponent_E(S, P):
    """Largest integer E with 4^E * max(2^32, S) <= (P-1) * 2^27."""
    M = max(1 << 32, int(S))
    X = (P - 1) << 27
    if X >= M:
        Q = X // M                  # 4^E <= X/M  <=>  4^E <= floor(X/M) for E >= 0
        return (Q.bit_length() - 1) // 2
    t = 1
    while X * (4 ** t) < M:          # smallest t with M <= X * 4^t, E = -t
        t += 1
    return -t


def vector_exponents(V, P):
    """Scaling exponents for each row of V (shape rows x entries, float64).

    V's row r holds every real entry of one row of A-hat (or one column of
    B-hat): the 2k values Re and Im.  Returns (x, e, S, E, flag) per row, with
    x = E - e the exponent of mu (or nu), or NONFINITE when flagged.
    """
    V = np.asarray(V, dtype=np.float64)
    rows = V.shape[0]
    x = np.zeros(rows, dtype=np.int64)
    e_out = np.zeros(rows, dtype=np.int64)
    E_out = np.zeros(rows, dtype=np.int64)
    S_out = [0] * rows
    flag = np.zeros(rows, dtype=bool)
    for r in range(rows):
        v = V[r]
        if not np.all(np.isfinite(v)):
            flag[r] = True
            x[r] = NONFINITE
            continue
        a = np.abs(v)
        amax = a.max() if a.size else 0.0
        e = math.frexp(float(amax))[1] - 1 if amax != 0 else 0
        # ceil(|t| 2^15) with t = v 2^-e: ldexp is an exact power-of-two
        # scaling whenever the result is normal; any nonzero entry whose scaled
        # value is below 1 (including one that underflows) has ceiling 1.
        sc = np.ldexp(a, SUM_FRAC_BITS - e)
        qt = np.where(a != 0, np.maximum(np.ceil(sc), 1.0), 0.0)
        # each square <= 2^32 and there are <= 2^18 of them: the float64 sum
        # of these integers is exact in any order
        S = int(np.sum(qt * qt))
        E = exponent_E(S, P)
        e_out[r], E_out[r], S_out[r] = e, E, S
        x[r] = E - e
    return x, e_out, S_out, E_out, flag


def row_vectors(A):
    """Rows of A-hat for complex A (m x k): [Re A(i,:), Im A(i,:)]."""
    return np.concatenate([A.real, A.imag], axis=1)


def col_vectors(B):
    """Columns of B-hat for complex B (k x n), one per row of the result."""
    return np.concatenate([B.real.T, B.imag.T], axis=1)
