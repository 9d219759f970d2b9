"""The C-ABI library loads and exports every symbol include/*.h declares; the
host-side plan and argument checks agree with the oracle.  No GPU needed:
nothing here launches device work."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from oracle.moduli import Plan
from oracle.scaling import exponent_E
from paper_2512_08321_gb300 import emu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"\b(emu_[a-z0-9_]+)\s*\(", txt):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(emu.LIB_PATH):
        from paper_2512_08321_gb300.build import build
        build()
    return emu.lib()


def test_exports_every_declared_symbol(L):
    decl = declared_functions()
    assert len(decl) >= 15
    for name in decl:
        assert hasattr(L, name), name
    assert decl == set(emu.exported_names())


def test_version(L):
    assert "sm_103a" in emu.emu_version()


@pytest.mark.parametrize("N", [2, 3, 6, 9, 14, 16, 17, 20, 24])
def test_plan_matches_oracle(L, N):
    st, mod, q, P, limbs = emu.emu_plan_info(N)
    ref = Plan(N)
    assert st == emu.EMU_OK
    assert mod == ref.p and q == ref.q and P == ref.P
    assert 2 ** (32 * limbs - 1) > 2 * ref.P             # c' + {-P, 0, P} fits the two's-complement limbs


@pytest.mark.parametrize("N", [2, 5, 8, 14, 20, 24])
def test_plan_exponent_matches_oracle(L, N):
    P = Plan(N).P
    rng = np.random.default_rng(N)
    Ss = [0, 1, 2 ** 32 - 1, 2 ** 32, 2 ** 32 + 1, 2 ** 50, 2 ** 50 - 1, 3 * 2 ** 40]
    Ss += [int(v) for v in rng.integers(0, 2 ** 50, 200)]
    for S in Ss:
        assert emu.emu_plan_exponent(N, S) == exponent_E(S, P), S


def test_plan_range(L):
    assert emu.emu_plan_info(1)[0] == emu.EMU_ERR_MODULI_RANGE
    assert emu.emu_plan_info(25)[0] == emu.EMU_ERR_MODULI_RANGE


def test_argument_checks_before_device_work(L):
    # rejected synchronously, before any CUDA call
    Z = 0
    st = emu.emu_zgemm("N", "N", -1, 4, 4, 1.0, Z, 4, Z, 4, 0.0, Z, 4, 14, 0)
    assert st == emu.EMU_ERR_INVALID_ARG and emu.emu_last_bad_param() == 3
    st = emu.emu_zgemm("N", "N", 4, 4, 4, 1.0, Z, 3, Z, 4, 0.0, Z, 4, 14, 0)
    assert st == emu.EMU_ERR_INVALID_ARG and emu.emu_last_bad_param() == 8
    st = emu.emu_zgemm("T", "N", 4, 4, 5, 1.0, Z, 4, Z, 5, 0.0, Z, 4, 14, 0)
    assert st == emu.EMU_ERR_INVALID_ARG and emu.emu_last_bad_param() == 8
    st = emu.emu_cgemm("N", "C", 4, 6, 4, 1.0, Z, 4, Z, 5, 0.0, Z, 4, 8, 0)
    assert st == emu.EMU_ERR_INVALID_ARG and emu.emu_last_bad_param() == 10
    st = emu.emu_zgemm("N", "N", 4, 4, 4, 1.0, Z, 4, Z, 4, 0.0, Z, 3, 14, 0)
    assert st == emu.EMU_ERR_INVALID_ARG and emu.emu_last_bad_param() == 13
    assert emu.emu_zgemm("N", "N", 4, 4, 4, 1.0, Z, 4, Z, 4, 0.0, Z, 4, 1, 0) == emu.EMU_ERR_MODULI_RANGE
    assert emu.emu_zgemm("N", "N", 4, 4, 4, 1.0, Z, 4, Z, 4, 0.0, Z, 4, 25, 0) == emu.EMU_ERR_MODULI_RANGE
    k = 2 ** 17 + 1
    assert emu.emu_zgemm("N", "N", 4, 4, k, 1.0, Z, 4, Z, k, 0.0, Z, 4, 14, 0) == emu.EMU_ERR_K_TOO_LARGE
    assert emu.emu_zgemm(7, "N", 4, 4, 4, 1.0, Z, 4, Z, 4, 0.0, Z, 4, 14, 0) == emu.EMU_ERR_INVALID_ARG
    assert emu.emu_last_bad_param() == 1
    # quick return: empty output touches nothing
    assert emu.emu_zgemm("N", "N", 0, 4, 4, 1.0, Z, 1, Z, 4, 0.0, Z, 1, 14, 0) == emu.EMU_OK
    assert emu.emu_set_engine(1, 100) == emu.EMU_ERR_INVALID_ARG
    assert emu.emu_set_engine(9, 0) == emu.EMU_ERR_INVALID_ARG


def test_workspace_query(L):
    b14 = emu.emu_workspace_bytes(0, 1000, 900, 700, 14)
    b16 = emu.emu_workspace_bytes(0, 1000, 900, 700, 16)
    assert 0 < b14 < b16
    assert emu.emu_workspace_bytes(0, -1, 900, 700, 14) == 0


INTERPOSED = ["cublasSgemm_v2", "cublasDgemm_v2", "cublasCgemm_v2", "cublasZgemm_v2", "cublasSgemm_v2_64",
              "cublasDgemm_v2_64", "cublasCgemm_v2_64", "cublasZgemm_v2_64", "cublasGemmEx", "cublasSgemm",
              "cublasDgemm", "cublasCgemm", "cublasZgemm", "cublasSetKernelStream"]


def test_preload_interposer_exports(L):
    import ctypes
    from paper_2512_08321_gb300 import build as B
    if not os.path.exists(B.PRELOAD):
        B.build_preload()
    txt = open(os.path.join(ROOT, "include", "ozaki2_preload.h")).read()
    shim = ctypes.CDLL(B.PRELOAD)
    for name in INTERPOSED:
        assert name in txt, name
        assert hasattr(shim, name), name
    calls = shim.ozaki2_preload_calls
    calls.restype = ctypes.c_uint64
    assert [calls(r, e) for r in range(-1, 7) for e in (0, 1)] == [0] * 16


@pytest.mark.parametrize("N", [2, 5, 12, 15, 24])
def test_plan_exponent_accu_matches_oracle(L, N):
    from oracle.accurate import exponent_accu
    P = Plan(N).P
    rng = np.random.default_rng(100 + N)
    Ms = [0, 1, 2, 3, 63, 64, 4095, 4096, 2 ** 30, 2 ** 31 - 1] + [int(v) for v in rng.integers(0, 2 ** 31, 200)]
    for M in Ms:
        assert emu.emu_plan_exponent_accu(N, M) == exponent_accu(M, P), M
    assert emu.emu_plan_exponent_accu(N, 2 ** 35) == -100000


def _prototypes():
    """name -> parameter list of every function declared in include/ozaki2_emu.h"""
    txt = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "ozaki2_emu.h")).read(), flags=re.S)
    txt = re.sub(r"//[^\n]*", "", txt)
    return {m.group(1): m.group(2) for m in re.finditer(r"\b(emu_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", txt, flags=re.S)}


def _c_kind(param):
    p = " ".join(param.split())
    if p in ("", "void"):
        return None
    if "*" in p or "[" in p or re.search(r"\b(cudaStream_t|emu_grouped_t)\b", p):
        return "pointer"
    if re.search(r"\b(int64_t|long long)\b", p):
        return "int64"
    if re.search(r"\b(uint64_t|size_t)\b", p):
        return "uint64"
    if re.search(r"\bdouble\b", p):
        return "double"
    if re.search(r"\bfloat\b", p):
        return "float"
    if re.search(r"\b(u?int(32_t)?|unsigned( int)?|emu_[a-z_]+_t)\b", p):
        return "int32"
    raise AssertionError(f"unclassified parameter: {p}")


def _py_kind(t):
    if t in (ctypes.c_void_p, ctypes.c_char_p) or (isinstance(t, type) and issubclass(t, ctypes._Pointer)):
        return "pointer"
    for kind, types in (("int64", (ctypes.c_int64, ctypes.c_longlong)), ("uint64", (ctypes.c_uint64, ctypes.c_size_t)),
                        ("double", (ctypes.c_double,)), ("float", (ctypes.c_float,)),
                        ("int32", (ctypes.c_int, ctypes.c_uint, ctypes.c_int32, ctypes.c_uint32))):
        if t in types:
            return kind
    raise AssertionError(f"unclassified ctypes type: {t}")


def test_binding_signatures_match_the_header():
    """Every ctypes signature of the binding has the header's parameter count and kinds, in order."""
    protos = _prototypes()
    assert set(protos) == set(emu.exported_names())
    for name, _res, args in emu._SIGS:
        want = [k for k in (_c_kind(p) for p in protos[name].split(",")) if k is not None]
        assert [_py_kind(a) for a in args] == want, name
