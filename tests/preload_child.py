"""Child process of tests/test_gpu_preload.py, run with the interposer in
LD_PRELOAD: calls cuBLAS GEMM routines the way an application linked to cuBLAS
does (symbols resolved in the global scope, where the preloaded interposer
comes first), checks the results bit for bit against the CPU oracle with the
interposer's moduli counts, and prints one JSON line."""
import ctypes
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import fp  # noqa: E402
from oracle.emulate import emulate  # noqa: E402
from oracle.emulate_real import emulate_real  # noqa: E402
from paper_2512_08321_gb300.workloads import paper_matrix, paper_matrix_real  # noqa: E402


def load(names):
    for nm in names:
        try:
            return ctypes.CDLL(nm, mode=ctypes.RTLD_GLOBAL)
        except OSError:
            continue
    raise OSError(f"none of {names} could be loaded")


cudart = load(["libcudart.so.13", "/usr/local/cuda/lib64/libcudart.so.13", "libcudart.so"])
cublas = load(["libcublas.so.13", "/usr/local/cuda/lib64/libcublas.so.13", "libcublas.so"])
glob = ctypes.CDLL(None)                     # global scope: what an application's references bind to
shim = ctypes.CDLL(os.environ["LD_PRELOAD"].split(":")[0])
vp = ctypes.c_void_p


class F2(ctypes.Structure):
    _fields_ = [("x", ctypes.c_float), ("y", ctypes.c_float)]


class D2(ctypes.Structure):
    _fields_ = [("x", ctypes.c_double), ("y", ctypes.c_double)]


def ck(r, what):
    if r != 0:
        raise RuntimeError(f"{what} returned {r}")


def to_dev(a):
    a = np.asfortranarray(a)
    p = vp()
    ck(cudart.cudaMalloc(ctypes.byref(p), ctypes.c_size_t(max(a.nbytes, 16))), "cudaMalloc")
    ck(cudart.cudaMemcpy(p, a.ctypes.data_as(vp), ctypes.c_size_t(a.nbytes), 1), "cudaMemcpy H2D")
    return p


def from_dev(p, shape, dtype):
    out = np.empty(shape, dtype=dtype, order="F")
    ck(cudart.cudaDeviceSynchronize(), "sync")
    ck(cudart.cudaMemcpy(out.ctypes.data_as(vp), p, ctypes.c_size_t(out.nbytes), 2), "cudaMemcpy D2H")
    return out


def same(a, b):
    a, b = np.ascontiguousarray(a), np.ascontiguousarray(b)
    if a.shape != b.shape or a.dtype != b.dtype:
        return False
    wide = a.dtype in (np.float64, np.complex128)
    ia = a.view(np.int64 if wide else np.int32)
    ib = b.view(np.int64 if wide else np.int32)
    return bool(np.array_equal(ia, ib))


NZ = int(os.environ.get("OZAKI2_EMU_MODULI_Z", "15"))
NC = int(os.environ.get("OZAKI2_EMU_MODULI_C", "8"))
ND = int(os.environ.get("OZAKI2_EMU_MODULI_D", "16"))
NS = int(os.environ.get("OZAKI2_EMU_MODULI_S", "8"))
res = {}
h = vp()
ck(cublas.cublasCreate_v2(ctypes.byref(h)), "cublasCreate")
res["resolves_to_interposer"] = (ctypes.cast(glob.cublasZgemm_v2, vp).value ==
                                 ctypes.cast(shim.cublasZgemm_v2, vp).value)

m, n, k = 130, 97, 150
# ZGEMM (op T, op N), alpha/beta complex
A = paper_matrix(k, m, 1.0, 501)
B = paper_matrix(k, n, 1.0, 502)
C0 = paper_matrix(m, n, 1.0, 503)
dA, dB, dC = to_dev(A), to_dev(B), to_dev(C0)
al, be = D2(0.5, -1.0), D2(2.0, 0.25)
ck(glob.cublasZgemm_v2(h, 1, 0, m, n, k, ctypes.byref(al), dA, k, dB, k, ctypes.byref(be), dC, m), "Zgemm_v2")
got = from_dev(dC, (m, n), np.complex128)
ref = emulate(A, B, NZ, "T", "N", alpha=(0.5, -1.0), beta=(2.0, 0.25), C_in=C0).out
res["zgemm_v2"] = same(got, ref)

# CGEMM (op C, op T)
A32 = paper_matrix(k, m, 0.5, 504).astype(np.complex64)
B32 = paper_matrix(n, k, 0.5, 505).astype(np.complex64)
dA, dB, dC = to_dev(A32), to_dev(B32), to_dev(np.zeros((m, n), np.complex64))
alf, bef = F2(1.0, 0.0), F2(0.0, 0.0)
ck(glob.cublasCgemm_v2(h, 2, 1, m, n, k, ctypes.byref(alf), dA, k, dB, n, ctypes.byref(bef), dC, m), "Cgemm_v2")
got = from_dev(dC, (m, n), np.complex64)
ref = emulate(A32.astype(np.complex128), B32.astype(np.complex128), NC, "C", "T", out_fmt=fp.BINARY32).out
res["cgemm_v2"] = same(got, ref)

# DGEMM and SGEMM
Ad = paper_matrix_real(m, k, 1.0, 506)
Bd = paper_matrix_real(k, n, 1.0, 507)
dA, dB, dC = to_dev(Ad), to_dev(Bd), to_dev(np.zeros((m, n)))
a_, b_ = ctypes.c_double(1.5), ctypes.c_double(0.0)
ck(glob.cublasDgemm_v2(h, 0, 0, m, n, k, ctypes.byref(a_), dA, m, dB, k, ctypes.byref(b_), dC, m), "Dgemm_v2")
res["dgemm_v2"] = same(from_dev(dC, (m, n), np.float64), emulate_real(Ad, Bd, ND, alpha=1.5).out)
As, Bs = Ad.astype(np.float32), Bd.astype(np.float32)
dA, dB, dC = to_dev(As), to_dev(Bs), to_dev(np.zeros((m, n), np.float32))
a32, b32 = ctypes.c_float(1.0), ctypes.c_float(0.0)
ck(glob.cublasSgemm_v2(h, 0, 0, m, n, k, ctypes.byref(a32), dA, m, dB, k, ctypes.byref(b32), dC, m), "Sgemm_v2")
res["sgemm_v2"] = same(from_dev(dC, (m, n), np.float32),
                       emulate_real(As.astype(np.float64), Bs.astype(np.float64), NS, out_fmt=fp.BINARY32).out)

# GemmEx, complex128 with 64F compute, scalars in device memory
dA, dB, dC = to_dev(A), to_dev(B), to_dev(np.zeros((m, n), np.complex128))
dal = to_dev(np.array([1.0 + 0.0j]))
dbe = to_dev(np.array([0.0 + 0.0j]))
ck(cublas.cublasSetPointerMode_v2(h, 1), "pointer mode")
ck(glob.cublasGemmEx(h, 1, 0, m, n, k, dal, dA, 5, k, dB, 5, k, dbe, dC, 5, m, 70, -1), "GemmEx")
ck(cublas.cublasSetPointerMode_v2(h, 0), "pointer mode")
res["gemmex_device_scalars"] = same(from_dev(dC, (m, n), np.complex128), emulate(A, B, NZ, "T", "N").out)

# forwarded: k above 2^17 goes to cuBLAS itself
kk = (1 << 17) + 64
Af = np.ones((2, kk)) * 0.5
Bf = np.ones((kk, 2)) * 0.25
dA, dB, dC = to_dev(Af), to_dev(Bf), to_dev(np.zeros((2, 2)))
a_, b_ = ctypes.c_double(1.0), ctypes.c_double(0.0)
ck(glob.cublasDgemm_v2(h, 0, 0, 2, 2, kk, ctypes.byref(a_), dA, 2, dB, kk, ctypes.byref(b_), dC, 2), "Dgemm fwd")
res["forwarded_large_k"] = bool(np.all(from_dev(dC, (2, 2), np.float64) == 0.125 * kk))

# legacy API (no handle; stream set by cublasSetKernelStream), if this cuBLAS has it
try:
    legacy = glob.cublasZgemm
    legacy.restype = None
    legacy.argtypes = [ctypes.c_char, ctypes.c_char, ctypes.c_int, ctypes.c_int, ctypes.c_int, D2, vp, ctypes.c_int,
                       vp, ctypes.c_int, D2, vp, ctypes.c_int]
    if hasattr(cublas, "cublasInit"):
        cublas.cublasInit()
    dA, dB, dC = to_dev(A), to_dev(B), to_dev(np.zeros((m, n), np.complex128))
    legacy(b"T", b"N", m, n, k, D2(1.0, 0.0), dA, k, dB, k, D2(0.0, 0.0), dC, m)
    res["legacy_zgemm"] = same(from_dev(dC, (m, n), np.complex128), emulate(A, B, NZ, "T", "N").out)
except AttributeError:
    res["legacy_zgemm"] = "absent"

calls = shim.ozaki2_preload_calls
calls.restype = ctypes.c_uint64
res["emulated"] = [int(calls(r, 1)) for r in range(6)]
res["forwarded"] = [int(calls(r, 0)) for r in range(6)]
print(json.dumps(res), flush=True)
