"""Exact references that do not go through the CRT.

Oracle (test infrastructure only).

* ``scaled_integer_product``: the exact complex integer product A'B' of the
  truncated matrices of Algorithm 1 Step IV, computed by splitting every
  integer into 21-bit limbs and forming exact limb products.  Section II states
  that, under condition (cond), the CRT of Steps V-v/V-vi returns exactly this.
* ``complex_product_entries``: the exact complex product AB of the original
  floating-point inputs at chosen entries, rounded once to binary64.  The
  paper measures errors against a double-double product (Section IV-A); the
  correctly rounded exact product used here is at least as accurate.
"""
import math

import numpy as np

LIMB_BITS = 21


def _limbs(V):
    """Split exact-integer float64 values into signed 21-bit limbs (int64)."""
    V = np.asarray(V, dtype=np.float64)
    sign = np.where(V < 0, -1, 1).astype(np.int64)
    mag = np.abs(V)
    nbits = int(np.max(np.frexp(mag)[1], initial=0))
    count = max(1, -(-nbits // LIMB_BITS))
    out = []
    base = float(1 << LIMB_BITS)
    rest = mag.copy()
    for _ in range(count):
        lo = np.fmod(rest, base)                 # exact for float64 integers
        out.append(sign * lo.astype(np.int64))
        rest = (rest - lo) / base                # exact: rest - lo is a multiple of base
    return out


def _exact_matmul(X, Y):
    """Exact integer product of exact-integer float64 matrices -> object array."""
    k = X.shape[1]
    lx, ly = _limbs(X), _limbs(Y)
    use_float = k <= (1 << 10)                   # 2^42 * 2^10 < 2^53: BLAS is exact
    acc = np.zeros((X.shape[0], Y.shape[1]), dtype=object)
    acc[...] = 0
    for s, xs in enumerate(lx):
        for t, yt in enumerate(ly):
            if use_float:
                prod = np.rint(xs.astype(np.float64) @ yt.astype(np.float64)).astype(np.int64)
            else:
                prod = xs @ yt                   # int64: 2^42 * k < 2^63 for k <= 2^17
            shift = LIMB_BITS * (s + t)
            acc = acc + np.vectorize(lambda v, sh=shift: int(v) << sh, otypes=[object])(prod)
    return acc


def scaled_integer_product(Ar, Ai, Br, Bi):
    """Exact (A'_R + i A'_I)(B'_R + i B'_I) as two object arrays of ints."""
    rr = _exact_matmul(Ar, Br)
    ii = _exact_matmul(Ai, Bi)
    ri = _exact_matmul(Ar, Bi)
    ir = _exact_matmul(Ai, Br)
    return rr - ii, ri + ir


def _two_product(a, b):
    """Error-free product a*b = p + e (Dekker with Veltkamp splitting)."""
    p = a * b
    c = 134217729.0 * a
    ah = c - (c - a)
    al = a - ah
    c = 134217729.0 * b
    bh = c - (c - b)
    bl = b - bh
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return p, e


def complex_product_entries(A, B, rows, cols):
    """Correctly rounded (AB)_ij at (rows[t], cols[t]); A: m x k, B: k x n."""
    A = np.asarray(A, dtype=np.complex128)
    B = np.asarray(B, dtype=np.complex128)
    out = np.zeros(len(rows), dtype=np.complex128)
    for t, (i, j) in enumerate(zip(rows, cols)):
        ar, ai = A[i].real.copy(), A[i].imag.copy()
        br, bi = B[:, j].real.copy(), B[:, j].imag.copy()
        p1, e1 = _two_product(ar, br)
        p2, e2 = _two_product(ai, bi)
        p3, e3 = _two_product(ar, bi)
        p4, e4 = _two_product(ai, br)
        re = math.fsum(np.concatenate([p1, e1, -p2, -e2]))
        im = math.fsum(np.concatenate([p3, e3, p4, e4]))
        out[t] = complex(re, im)
    return out


def real_product_entries(A, B, rows, cols):
    """Correctly rounded (AB)_ij of real matrices at (rows[t], cols[t])."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    out = np.zeros(len(rows), dtype=np.float64)
    for t, (i, j) in enumerate(zip(rows, cols)):
        p, e = _two_product(A[i].copy(), B[:, j].copy())
        out[t] = math.fsum(np.concatenate([p, e]))
    return out
