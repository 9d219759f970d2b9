"""Ozaki-II emulation of a REAL matrix product (DGEMM / SGEMM), step by step.

Oracle (test infrastructure only).

Algorithm 1 as Section II states it for real matrices (the scheme the paper
extends to complex products, and the one its real-valued comparison of
Section IV-C runs): one residue product per modulus, no Karatsuba
combination.  Steps, in the paper's order and notation:

  III   scaling exponents x_i (rows of A) and y_j (columns of B), fast mode:
        the row vector is the k real entries of A(i,:)            [scaling.py]
  IV    A' = trunc(diag(mu) A),  B' = trunc(B diag(nu))
  V-i   A'_l = mod(A', p_l);  V-ii  B'_l = mod(B', p_l)
  V-iii E_l = A'_l B'_l;      V-iv  E'_l = mod(E_l, p_l)
  V-v   S = sum_l (P/p_l) q_l E'_l;  V-vi  c' = mod(S, P)
  VI    C = diag(mu)^-1 C' diag(nu)^-1, then alpha*C + beta*C_in

Fast mode (Section II): |c'_ij| <= ||a'_i|| ||b'_j|| by Cauchy-Schwarz on
k-vectors, and the exponent rule of Section III-B (the same formula the
complex rows use) keeps that product within (P-1)/8, so condition (cond)
holds.

Readings (the paper gives no real-domain alpha/beta): with (alpha, beta) !=
(1, 0) the output is t = RN(alpha * o) and, when beta != 0, u = fma(beta, c, t)
in binary64; binary32 output rounds that binary64 value once more.  op C
equals op T for real matrices, as in BLAS.
"""
import numpy as np

from . import fp
from .emulate import int_matmul, residues, sym_mod, to_pyint, truncate
from .moduli import Plan
from .scaling import NONFINITE, vector_exponents


def apply_op_real(X, op):
    op = op.upper()
    if op == "N":
        return X
    if op in ("T", "C"):
        return X.T
    raise ValueError(op)


class RealEmulation:
    """All intermediate and final values of one emulated real GEMM.

    A: m x k, B: k x n (float64 or float32 values), both AFTER op().
    out_fmt: fp.BINARY64 (DGEMM) or fp.BINARY32 (SGEMM).
    """

    def __init__(self, A, B, N, alpha=1.0, beta=0.0, C_in=None, out_fmt=fp.BINARY64, plan=None, scaling="fast"):
        A = np.asarray(A, dtype=np.float64)
        B = np.asarray(B, dtype=np.float64)
        self.m, self.k = A.shape
        self.n = B.shape[1]
        self.plan = plan if plan is not None else Plan(N)
        P = self.plan.P
        # Step III on the real rows of A and columns of B: fast or accurate mode
        if scaling == "accurate":
            from .accurate import accurate_exponents
            self.accu = accurate_exponents(A, B, P, real=True)
            self.x, self.y = self.accu["x"], self.accu["y"]
            self.flag_a, self.flag_b = self.accu["flag_a"], self.accu["flag_b"]
        elif scaling == "fast":
            self.x, self.e_a, self.S_a, self.E_a, self.flag_a = vector_exponents(A, P)
            self.y, self.e_b, self.S_b, self.E_b, self.flag_b = vector_exponents(B.T, P)
        else:
            raise ValueError(scaling)
        # Step IV
        self.Ai = truncate(A, self.x)
        self.Bi = truncate(B.T, self.y).T
        # Step V
        m, n = self.m, self.n
        self.Eprime = np.zeros((N, m, n), dtype=np.int64)
        self.planesA = np.zeros((N, m, self.k), dtype=np.int64)
        self.planesB = np.zeros((N, n, self.k), dtype=np.int64)
        for l, p in enumerate(self.plan.p):
            a, b = residues(self.Ai, p), residues(self.Bi, p)
            self.planesA[l], self.planesB[l] = a, b.T
            self.Eprime[l] = sym_mod(int_matmul(a, b), p)
        # Step V-v / V-vi: exact CRT with Python integers
        S = np.zeros((m, n), dtype=object)
        S[...] = 0
        for l, w in enumerate(self.plan.w):
            S = S + to_pyint(self.Eprime[l]) * w
        self.c = sym_mod(S, P)
        # Step VI and alpha/beta
        self.out = self._unscale(out_fmt, alpha, beta, C_in)

    def _unscale(self, out_fmt, alpha, beta, C_in):
        m, n = self.m, self.n
        o = np.zeros((m, n), dtype=np.float64)
        for i in range(m):
            for j in range(n):
                if self.flag_a[i] or self.flag_b[j]:
                    o[i, j] = np.nan
                    continue
                o[i, j] = fp.round_scaled(int(self.c[i, j]), -(int(self.x[i]) + int(self.y[j])))
        return finish_real(o, alpha, beta, C_in, out_fmt)


def finish_real(o, alpha, beta, C_in, out_fmt):
    """alpha/beta step of the real path (module docstring) and the output format."""
    a, b = float(alpha), float(beta)
    if (a, b) != (1.0, 0.0):
        res = np.zeros_like(o)
        for i in range(o.shape[0]):
            for j in range(o.shape[1]):
                t = a * float(o[i, j])
                if b != 0.0:
                    t = fp.fma64(b, float(C_in[i, j]), t)
                res[i, j] = t
        o = res
    if out_fmt == fp.BINARY32:
        return o.astype(np.float32)             # one RN-even binary64 -> binary32
    return o


def emulate_real(A, B, N, opA="N", opB="N", **kw):
    """Emulated op(A) op(B) for real matrices; returns a RealEmulation."""
    return RealEmulation(apply_op_real(np.asarray(A), opA), apply_op_real(np.asarray(B), opB), N, **kw)


def emulate_real_entries(A, B, N, rows, cols, out_fmt=fp.BINARY64, xy=None):
    """Emulated real result at sampled entries, from Steps III-IV of the sampled
    rows/columns and the exact integer dot product for c' (equal to the CRT
    result by the CRT and condition (cond)).  A: m x k, B: k x n after op().
    xy: optional scaling vectors over all rows and columns (as in
    emulate_entries); by default the fast-mode exponents of the samples."""
    P = Plan(N).P
    rows = np.asarray(rows)
    cols = np.asarray(cols)
    ur, inv_r = np.unique(rows, return_inverse=True)
    uc, inv_c = np.unique(cols, return_inverse=True)
    Asub = np.asarray(A, dtype=np.float64)[ur, :]
    Bsub = np.asarray(B, dtype=np.float64)[:, uc]
    if xy is None:
        x, *_ = vector_exponents(Asub, P)
        y, *_ = vector_exponents(Bsub.T, P)
    else:
        x, y = np.asarray(xy[0])[ur], np.asarray(xy[1])[uc]
    Ai = to_pyint(truncate(Asub, x))
    Bi = to_pyint(truncate(Bsub.T, y))
    out = np.zeros(len(rows), dtype=np.float64)
    for t in range(len(rows)):
        a, b = inv_r[t], inv_c[t]
        if x[a] == NONFINITE or y[b] == NONFINITE:
            out[t] = np.nan
            continue
        c = int(np.dot(Ai[a], Bi[b]))
        out[t] = fp.round_scaled(c, -(int(x[a]) + int(y[b])))
    if out_fmt == fp.BINARY32:
        return out.astype(np.float32)
    return out


__all__ = ["RealEmulation", "emulate_real", "emulate_real_entries", "finish_real", "apply_op_real"]
