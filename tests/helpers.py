"""Shared test helpers: device transfer of column-major matrices and
oracle/GPU comparison utilities."""
import numpy as np
import torch

from paper_2512_08321_gb300 import emu


def dev(A, ld=None):
    """Column-major numpy matrix -> CUDA tensor holding the same storage
    (shape (cols, ld), C-contiguous); rows beyond A's are zero padding."""
    A = np.asarray(A)
    rows, cols = A.shape
    ld = ld or max(rows, 1)
    buf = np.zeros((cols, ld), dtype=A.dtype)
    buf[:, :rows] = A.T
    return torch.from_numpy(buf).cuda()


def host(T, rows):
    """Inverse of dev(): the rows x cols column-major matrix."""
    return T.cpu().numpy()[:, :rows].T.copy()


def same_bits(a, b):
    """Bitwise equality of complex or real arrays, NaN == NaN (any payload)."""
    a = np.asarray(a)
    b = np.asarray(b)
    if a.shape != b.shape or a.dtype != b.dtype:
        return False
    wide = a.dtype in (np.complex128, np.float64)
    fa = a.view(np.float64 if wide else np.float32)
    fb = b.view(np.float64 if wide else np.float32)
    both_nan = np.isnan(fa) & np.isnan(fb)
    ia = fa.view(np.int64 if fa.dtype == np.float64 else np.int32)
    ib = fb.view(np.int64 if fb.dtype == np.float64 else np.int32)
    return bool(np.all((ia == ib) | both_nan))


def mismatch_report(a, b, k=5):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    bad = np.nonzero(~((a == b) | (np.isnan(a) & np.isnan(b))))[0]
    return f"{len(bad)} mismatches, first: " + ", ".join(f"[{i}] {a[i]!r} vs {b[i]!r}" for i in bad[:k])


def run_gemm(A, B, N, opA="N", opB="N", alpha=1.0, beta=0.0, C=None, single=False, engine=None,
             lda=None, ldb=None, ldc=None):
    """Emulated op(A) op(B) on the GPU through the C ABI; returns numpy."""
    if engine is not None:
        emu.check(emu.emu_set_engine(engine, 0), "emu_set_engine")
    m = A.shape[0] if opA == "N" else A.shape[1]
    k = A.shape[1] if opA == "N" else A.shape[0]
    n = B.shape[1] if opB == "N" else B.shape[0]
    dt = np.complex64 if single else np.complex128
    dA = dev(A.astype(dt), lda)
    dB = dev(B.astype(dt), ldb)
    Cin = np.zeros((m, n), dtype=dt) if C is None else C.astype(dt)
    dC = dev(Cin, ldc)
    emu.gemm(dA, dB, dC, m, n, k, N, opA, opB, alpha, beta, lda=dA.shape[1], ldb=dB.shape[1],
             ldc=dC.shape[1])
    torch.cuda.synchronize()
    return host(dC, m)


def run_real(A, B, N, opA="N", opB="N", alpha=1.0, beta=0.0, C=None, single=False, lda=None, ldb=None, ldc=None):
    """Emulated real op(A) op(B) (DGEMM / SGEMM) through the C ABI; returns numpy."""
    m = A.shape[0] if opA == "N" else A.shape[1]
    k = A.shape[1] if opA == "N" else A.shape[0]
    n = B.shape[1] if opB == "N" else B.shape[0]
    dt = np.float32 if single else np.float64
    dA = dev(A.astype(dt), lda)
    dB = dev(B.astype(dt), ldb)
    Cin = np.zeros((m, n), dtype=dt) if C is None else C.astype(dt)
    dC = dev(Cin, ldc)
    emu.gemm(dA, dB, dC, m, n, k, N, opA, opB, alpha, beta, lda=dA.shape[1], ldb=dB.shape[1],
             ldc=dC.shape[1])
    torch.cuda.synchronize()
    return host(dC, m)
