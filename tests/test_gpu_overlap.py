"""Overlapped column blocks (EMU_TUNE_OVERLAP = 1, for n >= 2048): the next
block's exponents and planes and the previous block's CRT run on a second
stream beside each block's residue products (in accurate scaling every
exponent comes first, from the bound products).
Results must be bit-identical to the phases run one after another, and to
the oracle on sampled entries."""
import numpy as np
import pytest

from oracle import fp
from oracle.emulate import apply_op, emulate_entries
from oracle.emulate_real import emulate_real_entries
from paper_2512_08321_gb300 import emu
from paper_2512_08321_gb300.workloads import paper_matrix, paper_matrix_real

from .helpers import mismatch_report, run_gemm, run_real, same_bits

pytestmark = pytest.mark.gpu


def _with_overlap(on, fn):
    emu.check(emu.emu_set_tuning(emu.EMU_TUNE_OVERLAP, 1 if on else 0), "overlap")
    try:
        return fn()
    finally:
        emu.emu_set_tuning(emu.EMU_TUNE_OVERLAP, -1)


@pytest.mark.parametrize("single,opA,opB,nblock", [(False, "N", "N", 0), (False, "T", "C", 0),
                                                    (True, "C", "N", 0), (False, "N", "T", 512)])
def test_overlapped_blocks_complex(single, opA, opB, nblock):
    m, n, k, N = 200, 2048 + 333, 96, 12          # three column blocks, the last one ragged
    A = paper_matrix(m, k, 1.0, 500) if opA == "N" else paper_matrix(k, m, 1.0, 500)
    B = paper_matrix(k, n, 1.0, 501) if opB == "N" else paper_matrix(n, k, 1.0, 501)
    C = paper_matrix(m, n, 1.0, 502)
    al, be = complex(0.5, 1.0), complex(-1.0, 0.25)
    try:
        emu.check(emu.emu_set_tuning(emu.EMU_TUNE_NBLOCK, nblock), "nblock")
        run = lambda: run_gemm(A, B, N, opA, opB, alpha=al, beta=be, C=C, single=single)
        got = _with_overlap(True, run)
        serial = _with_overlap(False, run)
    finally:
        emu.emu_set_tuning(emu.EMU_TUNE_NBLOCK, 0)
    assert same_bits(got, serial), mismatch_report(got, serial)
    # sampled entries against the oracle (alpha = 1, beta = 0 there: compare the product part)
    plain = _with_overlap(True, lambda: run_gemm(A, B, N, opA, opB, single=single))
    Ao = apply_op(A.astype(np.complex64 if single else np.complex128).astype(np.complex128), opA)
    Bo = apply_op(B.astype(np.complex64 if single else np.complex128).astype(np.complex128), opB)
    rng = np.random.default_rng(5)
    rows = np.concatenate([[0, m - 1], rng.integers(0, m, 30)])
    cols = np.concatenate([[0, 1023, 1024, 2047, 2048, n - 1], rng.integers(0, n, 26)])
    want = emulate_entries(Ao, Bo, N, rows, cols, out_fmt=fp.BINARY32 if single else fp.BINARY64)
    assert same_bits(plain[rows, cols], want), mismatch_report(plain[rows, cols], want)


@pytest.mark.parametrize("single", [False, True])
def test_overlapped_blocks_real(single):
    m, n, k, N = 150, 3 * 1024 + 5, 80, 10
    A = paper_matrix_real(m, k, 1.0, 510)
    B = paper_matrix_real(k, n, 1.0, 511)
    run = lambda: run_real(A, B, N, single=single)
    got = _with_overlap(True, run)
    serial = _with_overlap(False, run)
    assert same_bits(got, serial), mismatch_report(got, serial)
    dt = np.float32 if single else np.float64
    rng = np.random.default_rng(6)
    rows = rng.integers(0, m, 24)
    cols = np.concatenate([[0, 1024, 2048, n - 1], rng.integers(0, n, 20)])
    want = emulate_real_entries(A.astype(dt).astype(np.float64), B.astype(dt).astype(np.float64), N, rows, cols,
                                out_fmt=fp.BINARY32 if single else fp.BINARY64)
    assert same_bits(got[rows, cols], want), mismatch_report(got[rows, cols], want)


@pytest.mark.parametrize("real", [False, True], ids=["complex", "real"])
def test_overlapped_blocks_accurate(real):
    """Accurate scaling: the bound products of all column blocks give every
    exponent first, then the blocks overlap as in fast scaling; bit-identical
    to one phase after another and to the oracle on sampled entries."""
    from oracle.accurate import accurate_exponents
    from oracle.moduli import Plan
    m, n, k, N = 180, 2048 + 200, 300, 13
    if real:
        A, B = paper_matrix_real(m, k, 2.0, 520), paper_matrix_real(k, n, 2.0, 521)
        run = lambda: run_real(A, B, N)
    else:
        A, B = paper_matrix(m, k, 2.0, 522), paper_matrix(k, n, 2.0, 523)
        run = lambda: run_gemm(A, B, N)
    emu.check(emu.emu_set_scaling(emu.EMU_SCALING_ACCURATE), "scaling")
    try:
        got = _with_overlap(True, run)
        serial = _with_overlap(False, run)
    finally:
        emu.emu_set_scaling(emu.EMU_SCALING_FAST)
    assert same_bits(got, serial), mismatch_report(got, serial)
    ex = accurate_exponents(A, B, Plan(N).P, real=real)
    rng = np.random.default_rng(8)
    rows = np.concatenate([[0, m - 1], rng.integers(0, m, 22)])
    cols = np.concatenate([[0, 1024, 2047, 2048, n - 1], rng.integers(0, n, 19)])
    entries = emulate_real_entries if real else emulate_entries
    want = entries(A, B, N, rows, cols, xy=(ex["x"], ex["y"]))
    assert same_bits(got[rows, cols], want), mismatch_report(got[rows, cols], want)


def test_overlap_knob():
    assert emu.emu_get_tuning(emu.EMU_TUNE_OVERLAP) == -1         # default: on for the real GEMMs only
    assert emu.emu_set_tuning(emu.EMU_TUNE_OVERLAP, 2) == emu.EMU_ERR_INVALID_ARG


def test_tolerance_call_with_overlap():
    """emu_zgemm_tol hands its precomputed exponent sums to the GEMM; with the
    overlapped column blocks (n >= 2048) the result equals the plain call with
    the N it chose, bit for bit."""
    import torch
    from .helpers import dev, host
    m, n, k = 300, 2048 + 200, 150
    A = paper_matrix(m, k, 1.0, 520)
    B = paper_matrix(k, n, 1.0, 521)
    dA, dB = dev(A), dev(B)
    dC = dev(np.zeros((m, n), dtype=np.complex128))
    st, N = _with_overlap(True, lambda: emu.emu_zgemm_tol("N", "N", m, n, k, 1.0, dA.data_ptr(), m, dB.data_ptr(),
                                                          k, 0.0, dC.data_ptr(), m, 1e-10,
                                                          torch.cuda.current_stream()))
    emu.check(st, "zgemm_tol")
    torch.cuda.synchronize()
    got = host(dC, m)
    want = _with_overlap(False, lambda: run_gemm(A, B, N))
    assert same_bits(got, want), mismatch_report(got, want)
