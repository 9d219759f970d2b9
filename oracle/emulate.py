"""Ozaki-II complex GEMM emulation, step by step (Algorithm 1 with the
Karatsuba product of Section III-A and the fast-mode scaling of Section III-B).

Oracle (test infrastructure only).

Steps, in the paper's order and notation:

  III   scaling exponents x_i (mu_i = 2^x_i) and y_j (nu_j = 2^y_j)   [scaling.py]
  IV    A' = trunc(diag(mu) A), B' = trunc(B diag(nu)), per real and imaginary part
  V-i   (A'_l) = mod(A', p_l) for the real part, the imaginary part, and
        mod(A'_R + A'_I, p_l) for the Karatsuba sum (Section III-A: the sums
        are reduced modulo p_l before the products are formed)
  V-ii  likewise for B'
  V-iii D_l = A'_R,l B'_R,l,  E_l = A'_I,l B'_I,l,  F_l = A'_S,l B'_S,l  (eq. karatsuba)
  V-iv  E'_R,l = mod(D_l - E_l, p_l),  E'_I,l = mod(F_l - D_l - E_l, p_l)
  V-v   S = sum_l (P/p_l) q_l E'_l
  V-vi  c' = mod(S, P)
  VI    C = diag(mu)^-1 C' diag(nu)^-1, then alpha*C + beta*C_in

mod(x, p) is the symmetric remainder x - p*round(x/p) of Section II.  Reading:
ties (x/p = j + 1/2, possible only for even p) round up, so residues lie in
[-p/2, p/2 - 1] for even p and in [-(p-1)/2, (p-1)/2] for odd p; for p = 256
that is the int8 range.

Reading of Step VI: the exact integer c' is scaled by 2^-(x_i + y_j) and
rounded once to nearest-even binary64.  For complex64 output that binary64
value (after alpha/beta) is rounded once more to binary32.  alpha/beta, which
the paper does not discuss, use this fixed IEEE sequence:
  t_r = fma(alpha_r, o_r, -(alpha_i * o_i)),  t_i = fma(alpha_r, o_i, alpha_i * o_r)
  u_r = fma(beta_r, c_r, fma(-beta_i, c_i, t_r)), u_i = fma(beta_r, c_i, fma(beta_i, c_r, t_i))
applied only when (alpha, beta) != (1, 0); beta = 0 never reads C_in.
"""
import numpy as np

from . import fp
from .moduli import Plan
from .scaling import NONFINITE, col_vectors, row_vectors, vector_exponents


def apply_op(X, op):
    """op(X) for op in 'N', 'T', 'C' (BLAS transpose / conjugate transpose)."""
    op = op.upper()
    if op == "N":
        return X
    if op == "T":
        return X.T
    if op == "C":
        return X.conj().T
    raise ValueError(op)


def sym_mod(x, p):
    """Symmetric remainder mod(x, p) of Section II (ties round up), exact.

    ``x`` is an int64 array, an object array of Python ints, or an int.
    """
    if isinstance(x, np.ndarray) and x.dtype != object:
        r = np.remainder(x.astype(np.int64), p)          # floor mod, in [0, p)
        return np.where(2 * r >= p, r - p, r)
    if isinstance(x, np.ndarray):
        r = np.array([v % p for v in x.ravel()], dtype=object).reshape(x.shape)
        return np.where(2 * r >= p, r - p, r)
    r = x % p
    return r - p if 2 * r >= p else r


def truncate(V, x):
    """Step IV: trunc(V * 2^x) per row; exact (power-of-two scaling, then trunc).

    Returns float64 arrays holding exact integers (|a'| < 2^(E+1) <= 2^100);
    rows flagged NONFINITE become zero.
    """
    V = np.asarray(V, dtype=np.float64)
    xs = np.where(x == NONFINITE, 0, x).astype(np.int64)
    out = np.trunc(np.ldexp(V, xs[:, None]))
    out[x == NONFINITE, :] = 0.0
    out[~np.isfinite(out)] = 0.0
    return out


def residues(Vint, p):
    """Step V-i/ii: symmetric residues of exact-integer float64 values."""
    if np.max(np.abs(Vint), initial=0.0) < 2.0 ** 62:
        return sym_mod(Vint.astype(np.int64), p).astype(np.int64)
    obj = np.array([int(v) for v in Vint.ravel()], dtype=object).reshape(Vint.shape)
    return sym_mod(obj, p).astype(np.int64)


def int_matmul(X, Y):
    """Exact product of small-integer matrices (|entries| <= 128, k <= 2^17).

    Every partial sum is an integer below 2^31 < 2^53, so the float64 matrix
    product is exact whatever order the library sums in.
    """
    return np.rint(X.astype(np.float64) @ Y.astype(np.float64)).astype(np.int64)


def to_pyint(Vint):
    return np.array([int(v) for v in Vint.ravel()], dtype=object).reshape(Vint.shape)


class Emulation:
    """All intermediate and final values of one emulated complex GEMM.

    A: m x k complex, B: k x n complex, both AFTER applying op().
    out_fmt: fp.BINARY64 (ZGEMM) or fp.BINARY32 (CGEMM).
    """

    def __init__(self, A, B, N, alpha=(1.0, 0.0), beta=(0.0, 0.0), C_in=None,
                 out_fmt=fp.BINARY64, keep_residue_planes=True, plan=None, scaling="fast"):
        A = np.asarray(A)
        B = np.asarray(B)
        self.m, self.k = A.shape
        self.n = B.shape[1]
        self.plan = plan if plan is not None else Plan(N)
        P = self.plan.P
        # Step III: fast mode, or accurate mode (accurate.py)
        if scaling == "accurate":
            from .accurate import accurate_exponents
            self.accu = accurate_exponents(A, B, P)
            self.x, self.y = self.accu["x"], self.accu["y"]
            self.flag_a, self.flag_b = self.accu["flag_a"], self.accu["flag_b"]
        elif scaling == "fast":
            self.x, self.e_a, self.S_a, self.E_a, self.flag_a = vector_exponents(row_vectors(A), P)
            self.y, self.e_b, self.S_b, self.E_b, self.flag_b = vector_exponents(col_vectors(B), P)
        else:
            raise ValueError(scaling)
        # Step IV
        self.Ar = truncate(A.real, self.x)
        self.Ai = truncate(A.imag, self.x)
        self.Br = truncate(B.real.T, self.y).T
        self.Bi = truncate(B.imag.T, self.y).T
        # Step V
        m, n = self.m, self.n
        self.DEF = np.zeros((N, 3, m, n), dtype=np.int64)
        self.Eprime = np.zeros((N, 2, m, n), dtype=np.int64)
        self.planesA = np.zeros((N, 3, m, self.k), dtype=np.int64) if keep_residue_planes else None
        self.planesB = np.zeros((N, 3, n, self.k), dtype=np.int64) if keep_residue_planes else None
        for l, p in enumerate(self.plan.p):
            aR, aI = residues(self.Ar, p), residues(self.Ai, p)
            bR, bI = residues(self.Br, p), residues(self.Bi, p)
            aS, bS = sym_mod(aR + aI, p), sym_mod(bR + bI, p)
            D = int_matmul(aR, bR)
            E = int_matmul(aI, bI)
            F = int_matmul(aS, bS)
            self.DEF[l, 0], self.DEF[l, 1], self.DEF[l, 2] = sym_mod(D, p), sym_mod(E, p), sym_mod(F, p)
            self.Eprime[l, 0] = sym_mod(D - E, p)
            self.Eprime[l, 1] = sym_mod(F - D - E, p)
            if keep_residue_planes:
                self.planesA[l, 0], self.planesA[l, 1], self.planesA[l, 2] = aR, aI, aS
                self.planesB[l, 0], self.planesB[l, 1], self.planesB[l, 2] = bR.T, bI.T, bS.T
        # Step V-v / V-vi: exact CRT with Python integers
        self.cR = self._crt(self.Eprime[:, 0])
        self.cI = self._crt(self.Eprime[:, 1])
        # Step VI and alpha/beta
        self.out = self._unscale(out_fmt, alpha, beta, C_in)

    def _crt(self, Ep):
        P = self.plan.P
        S = np.zeros(Ep.shape[1:], dtype=object)
        S[...] = 0
        for l, w in enumerate(self.plan.w):
            S = S + to_pyint(Ep[l]) * w
        return sym_mod(S, P)

    def _unscale(self, out_fmt, alpha, beta, C_in):
        m, n = self.m, self.n
        o = np.zeros((m, n), dtype=np.complex128)
        for i in range(m):
            for j in range(n):
                if self.flag_a[i] or self.flag_b[j]:
                    o[i, j] = complex(np.nan, np.nan)
                    continue
                s = -(int(self.x[i]) + int(self.y[j]))
                o[i, j] = complex(fp.round_scaled(int(self.cR[i, j]), s),
                                  fp.round_scaled(int(self.cI[i, j]), s))
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
                        cr = float(np.real(C_in[i, j]))
                        ci = float(np.imag(C_in[i, j]))
                        tr = fp.fma64(br, cr, fp.fma64(-bi, ci, tr))
                        ti = fp.fma64(br, ci, fp.fma64(bi, cr, ti))
                    res[i, j] = complex(tr, ti)
            o = res
        if out_fmt == fp.BINARY32:
            return o.astype(np.complex64)        # one RN-even binary64 -> binary32
        return o


def emulate(A, B, N, opA="N", opB="N", **kw):
    """Emulated op(A) op(B) (alpha/beta/C_in via keywords); returns Emulation."""
    return Emulation(apply_op(np.asarray(A), opA), apply_op(np.asarray(B), opB), N, **kw)


def emulate_entries(A, B, N, rows, cols, out_fmt=fp.BINARY64, xy=None):
    """Emulated result at the sampled entries (rows[t], cols[t]) only.

    Uses x_i, y_j and the truncated integers of Steps III-IV for the sampled
    rows and columns, and the exact integer dot product for c'; by the CRT and
    condition (cond) that is the value Steps V-v/V-vi reconstruct (the
    full-pipeline equality is checked on small sizes by the tests).
    A: m x k and B: k x n complex, after op().  Returns complex values.
    xy: optional scaling vectors (x over all m rows, y over all n columns), for
    instance the accurate mode's, which depend on whole rows and columns of the
    bound product; by default the fast-mode exponents of the sampled rows and
    columns.
    """
    P = Plan(N).P
    rows = np.asarray(rows)
    cols = np.asarray(cols)
    ur, inv_r = np.unique(rows, return_inverse=True)
    uc, inv_c = np.unique(cols, return_inverse=True)
    Asub = np.asarray(A)[ur, :]
    Bsub = np.asarray(B)[:, uc]
    if xy is None:
        x, *_ = vector_exponents(row_vectors(Asub), P)
        y, *_ = vector_exponents(col_vectors(Bsub), P)
    else:
        x, y = np.asarray(xy[0])[ur], np.asarray(xy[1])[uc]
    Ar, Ai = to_pyint(truncate(Asub.real, x)), to_pyint(truncate(Asub.imag, x))
    Br, Bi = to_pyint(truncate(Bsub.real.T, y)), to_pyint(truncate(Bsub.imag.T, y))
    out = np.zeros(len(rows), dtype=np.complex128)
    for t in range(len(rows)):
        a, b = inv_r[t], inv_c[t]
        if x[a] == NONFINITE or y[b] == NONFINITE:
            out[t] = complex(np.nan, np.nan)
            continue
        cr = int(np.dot(Ar[a], Br[b]) - np.dot(Ai[a], Bi[b]))
        ci = int(np.dot(Ar[a], Bi[b]) + np.dot(Ai[a], Br[b]))
        s = -(int(x[a]) + int(y[b]))
        out[t] = complex(fp.round_scaled(cr, s), fp.round_scaled(ci, s))
    if out_fmt == fp.BINARY32:
        return out.astype(np.complex64)
    return out
