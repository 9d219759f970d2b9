"""GPU parity of the real-matrix emulation (DGEMM / SGEMM) and of column
blocking: bit for bit against the CPU oracle through the C ABI.  Shapes span
several tiles with ragged tails."""
import numpy as np
import pytest
import torch

from oracle import fp
from oracle.crt_fp import outputs_real
from oracle.emulate_real import RealEmulation, apply_op_real, emulate_real
from paper_2512_08321_gb300 import emu
from paper_2512_08321_gb300.workloads import paper_matrix, paper_matrix_real

from .helpers import mismatch_report, run_gemm, run_real, same_bits

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _restore():
    yield
    emu.emu_set_engine(emu.EMU_ENGINE_AUTO, 512)
    emu.emu_set_tuning(emu.EMU_TUNE_NBLOCK, 0)
    emu.emu_set_crt_mode(emu.EMU_CRT_EXACT)
    emu.emu_set_workspace(None, 0)


def _mats(m, n, k, opA, opB, phi, seed, single):
    A = paper_matrix_real(m, k, phi, seed) if opA == "N" else paper_matrix_real(k, m, phi, seed)
    B = paper_matrix_real(k, n, phi, seed + 1) if opB == "N" else paper_matrix_real(n, k, phi, seed + 1)
    if single:
        A, B = A.astype(np.float32), B.astype(np.float32)
    return A, B


def _oracle(A, B, N, opA, opB, single, **kw):
    fmt = fp.BINARY32 if single else fp.BINARY64
    return emulate_real(A.astype(np.float64), B.astype(np.float64), N, opA, opB, out_fmt=fmt, **kw)


@pytest.mark.parametrize("single", [False, True])
@pytest.mark.parametrize("opA,opB", [("N", "N"), ("T", "N"), ("N", "T"), ("C", "C")])
def test_real_bitexact(single, opA, opB):
    N = 8 if single else 16
    m, n, k = 300, 260, 333
    A, B = _mats(m, n, k, opA, opB, 1.5, 40, single)
    ref = _oracle(A, B, N, opA, opB, single).out
    got = run_real(A, B, N, opA, opB, single=single)
    assert got.dtype == (np.float32 if single else np.float64)
    assert same_bits(got, ref), mismatch_report(got, ref)


@pytest.mark.parametrize("single", [False, True])
def test_real_alpha_beta_and_lds(single):
    m, n, k = 129, 257, 200
    A, B = _mats(m, n, k, "N", "N", 1.0, 41, single)
    C = paper_matrix_real(m, n, 1.0, 43).astype(np.float32 if single else np.float64)
    ref = _oracle(A, B, 12, "N", "N", single, alpha=-1.25, beta=0.5, C_in=C.astype(np.float64)).out
    got = run_real(A, B, 12, alpha=-1.25, beta=0.5, C=C, single=single, lda=m + 7, ldb=k + 3, ldc=m + 16)
    assert same_bits(got, ref), mismatch_report(got, ref)


@pytest.mark.parametrize("N", [2, 5, 20, 24])
def test_real_moduli_extremes(N):
    A, B = _mats(70, 90, 150, "N", "N", 2.0, 44, False)
    ref = _oracle(A, B, N, "N", "N", False).out
    got = run_real(A, B, N)
    assert same_bits(got, ref), mismatch_report(got, ref)


def test_real_edge_cases():
    # zero row, Inf and NaN, subnormals, huge range; k = 1; k = 0 with beta
    A, B = _mats(40, 33, 64, "N", "N", 1.0, 45, False)
    A[3] = 0.0
    A[5, 7] = np.inf
    B[9, 4] = np.nan
    A[8] *= 1e-310
    B[:, 11] *= 1e300
    ref = _oracle(A, B, 14, "N", "N", False).out
    got = run_real(A, B, 14)
    assert same_bits(got, ref), mismatch_report(got, ref)
    a1, b1 = A[:, :1].copy(), B[:1].copy()
    assert same_bits(run_real(a1, b1, 14), _oracle(a1, b1, 14, "N", "N", False).out)
    C = paper_matrix_real(40, 33, 1.0, 46)
    a0, b0 = np.zeros((40, 0)), np.zeros((0, 33))
    got0 = run_real(a0, b0, 14, alpha=2.0, beta=-3.0, C=C)
    assert same_bits(got0, np.array([[fp.fma64(-3.0, C[i, j], 0.0) for j in range(33)] for i in range(40)]))


def test_real_i8_engine():
    A, B = _mats(150, 70, 300, "T", "N", 1.0, 47, False)
    emu.check(emu.emu_set_engine(emu.EMU_ENGINE_I8, 0), "engine")
    got = run_real(A, B, 13, "T", "N")
    ref = _oracle(A, B, 13, "T", "N", False).out
    assert same_bits(got, ref), mismatch_report(got, ref)


@pytest.mark.parametrize("single", [False, True])
def test_real_paper_fp_crt(single):
    N = 7 if single else 16
    A, B = _mats(100, 70, 120, "N", "N", 1.0, 48, single)
    em = RealEmulation(A.astype(np.float64), B.astype(np.float64), N)
    ref = outputs_real(em, single=single)
    emu.check(emu.emu_set_crt_mode(emu.EMU_CRT_PAPER_FP64), "crt mode")
    got = run_real(A, B, N, single=single)
    assert same_bits(got, ref), mismatch_report(got, ref)


def _complex(m, n, k, seed, single):
    A = paper_matrix(m, k, 1.0, seed)
    B = paper_matrix(k, n, 1.0, seed + 1)
    return (A.astype(np.complex64), B.astype(np.complex64)) if single else (A, B)


@pytest.mark.parametrize("kind", ["z", "c", "d", "s"])
def test_column_blocking_bitidentical(kind):
    # blocks of 128 columns (ragged last block) against one pass, all four types
    m, n, k = 190, 3 * 128 + 45, 150
    single = kind in "cs"
    if kind in "zc":
        A, B = _complex(m, n, k, 50, single)
        one = run_gemm(A, B, 11, single=single)
        emu.check(emu.emu_set_tuning(emu.EMU_TUNE_NBLOCK, 128), "nblock")
        blk = run_gemm(A, B, 11, single=single)
    else:
        A, B = _mats(m, n, k, "N", "T", 1.0, 51, single)
        one = run_real(A, B, 11, "N", "T", single=single)
        emu.check(emu.emu_set_tuning(emu.EMU_TUNE_NBLOCK, 128), "nblock")
        blk = run_real(A, B, 11, "N", "T", single=single)
    assert emu.emu_get_tuning(emu.EMU_TUNE_NBLOCK) == 128
    assert same_bits(blk, one), mismatch_report(blk, one)


def test_automatic_blocking_in_small_caller_workspace():
    # a caller workspace too small for one pass: the library picks column blocks that fit
    m, n, k, N = 200, 1000, 300, 12
    A, B = _complex(m, n, k, 52, False)
    full = emu.emu_workspace_bytes(emu.EMU_DTYPE_Z, m, n, k, N)
    one = run_gemm(A, B, N)
    ws = torch.empty(full // 2, dtype=torch.uint8, device="cuda")
    emu.check(emu.emu_set_workspace(ws.data_ptr(), ws.numel()), "workspace")
    blk = run_gemm(A, B, N)
    emu.emu_set_workspace(None, 0)
    assert same_bits(blk, one), mismatch_report(blk, one)
    # too small even for one block of 128 columns
    emu.check(emu.emu_set_workspace(ws.data_ptr(), 4096), "workspace")
    dA = torch.zeros((k, m), dtype=torch.complex128, device="cuda")
    dB = torch.zeros((n, k), dtype=torch.complex128, device="cuda")
    dC = torch.zeros((n, m), dtype=torch.complex128, device="cuda")
    st = emu.emu_zgemm("N", "N", m, n, k, 1.0, dA.data_ptr(), m, dB.data_ptr(), k, 0.0, dC.data_ptr(), m, N)
    assert st == emu.EMU_ERR_WORKSPACE


def test_real_workspace_bytes_and_invalid_nblock():
    z = emu.emu_workspace_bytes(emu.EMU_DTYPE_Z, 1000, 900, 700, 14)
    d = emu.emu_workspace_bytes(emu.EMU_DTYPE_D, 1000, 900, 700, 14)
    assert 0 < d < z
    assert emu.emu_workspace_bytes(7, 1000, 900, 700, 14) == 0
    assert emu.emu_set_tuning(emu.EMU_TUNE_NBLOCK, 100) == emu.EMU_ERR_INVALID_ARG
    assert emu.emu_set_tuning(emu.EMU_TUNE_NBLOCK, 256) == emu.EMU_OK


@pytest.mark.parametrize("N", [2, 3])
@pytest.mark.parametrize("single", [False, True])
def test_single_limb_crt_complex(N, single):
    # N = 2, 3: P < 2^31, the CRT runs on one 32-bit limb
    A, B = _complex(90, 70, 80, 53, single)
    from oracle.emulate import emulate
    ref = emulate(A.astype(np.complex128), B.astype(np.complex128), N,
                  out_fmt=fp.BINARY32 if single else fp.BINARY64).out
    got = run_gemm(A, B, N, single=single)
    assert same_bits(got, ref), mismatch_report(got, ref)
