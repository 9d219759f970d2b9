"""Error metrics.

Oracle (test infrastructure only).

* ``max_rel_error``: the maximum componentwise relative error of Section IV-A,
  max_ij max(|Re d|/|Re c|, |Im d|/|Im c|) against a high-accuracy product c.
* ``max_normalised_error``: max_ij max(|Re d|, |Im d|) / ((|A_R|+|A_I|)(|B_R|+|B_I|))_ij,
  the reading of "error normalised by |A||B|" used for the tolerances.
"""
import numpy as np


def max_rel_error(approx, ref):
    approx = np.asarray(approx, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    with np.errstate(divide="ignore", invalid="ignore"):
        er = np.abs(approx.real - ref.real) / np.abs(ref.real)
        ei = np.abs(approx.imag - ref.imag) / np.abs(ref.imag)
    er = np.where(ref.real == 0, np.where(approx.real == 0, 0.0, np.inf), er)
    ei = np.where(ref.imag == 0, np.where(approx.imag == 0, 0.0, np.inf), ei)
    return float(np.max(np.maximum(er, ei), initial=0.0))


def abs_bound_entries(A, B, rows, cols):
    """((|A_R|+|A_I|)(|B_R|+|B_I|))_ij at the given entries."""
    A = np.asarray(A)
    B = np.asarray(B)
    out = np.zeros(len(rows))
    for t, (i, j) in enumerate(zip(rows, cols)):
        a = np.abs(A[i].real) + np.abs(A[i].imag)
        b = np.abs(B[:, j].real) + np.abs(B[:, j].imag)
        out[t] = float(a @ b)
    return out


def max_normalised_error(approx, ref, bound):
    approx = np.asarray(approx, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    d = np.maximum(np.abs(approx.real - ref.real), np.abs(approx.imag - ref.imag))
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(bound > 0, d / bound, np.where(d == 0, 0.0, np.inf))
    return float(np.max(r, initial=0.0))
