"""GPU parity of accurate-mode scaling (Section III-B, eqs. mu-accu / nu-accu):
exponents and results bit for bit against the CPU oracle for all four element
types, the exact bound products across several k chunks, column blocking,
edge cases, and the CRT's range correction near |c'| = P/2."""
import numpy as np
import pytest
import torch

from oracle import fp
from oracle.crt_fp import outputs, outputs_real
from oracle.emulate import Emulation, apply_op
from oracle.emulate_real import RealEmulation, apply_op_real
from paper_2512_08321_gb300 import emu
from paper_2512_08321_gb300.workloads import paper_matrix, paper_matrix_real

from .helpers import mismatch_report, run_gemm, run_real, same_bits

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _accurate():
    pair = emu.emu_get_tuning(emu.EMU_TUNE_BOUND_PAIR)
    emu.check(emu.emu_set_scaling(emu.EMU_SCALING_ACCURATE), "scaling")
    yield
    emu.emu_set_scaling(emu.EMU_SCALING_FAST)
    emu.emu_set_crt_mode(emu.EMU_CRT_EXACT)
    emu.emu_set_tuning(emu.EMU_TUNE_NBLOCK, 0)
    emu.emu_set_tuning(emu.EMU_TUNE_BOUND_PAIR, pair)


def _cplx(m, n, k, opA, opB, phi, seed, single):
    A = paper_matrix(m, k, phi, seed) if opA == "N" else paper_matrix(k, m, phi, seed)
    B = paper_matrix(k, n, phi, seed + 1) if opB == "N" else paper_matrix(n, k, phi, seed + 1)
    if single:
        A, B = A.astype(np.complex64), B.astype(np.complex64)
    return A, B


def _real(m, n, k, opA, opB, phi, seed, single):
    A = paper_matrix_real(m, k, phi, seed) if opA == "N" else paper_matrix_real(k, m, phi, seed)
    B = paper_matrix_real(k, n, phi, seed + 1) if opB == "N" else paper_matrix_real(n, k, phi, seed + 1)
    if single:
        A, B = A.astype(np.float32), B.astype(np.float32)
    return A, B


def test_scaling_switch():
    assert emu.emu_get_scaling() == emu.EMU_SCALING_ACCURATE
    assert emu.emu_set_scaling(7) == emu.EMU_ERR_INVALID_ARG


@pytest.mark.parametrize("single", [False, True])
@pytest.mark.parametrize("opA,opB", [("N", "N"), ("C", "T")])
def test_complex_accurate_bitexact(single, opA, opB):
    N = 7 if single else 13
    A, B = _cplx(300, 260, 333, opA, opB, 2.0, 80, single)
    em = Emulation(apply_op(A.astype(np.complex128), opA), apply_op(B.astype(np.complex128), opB), N,
                   scaling="accurate", out_fmt=fp.BINARY32 if single else fp.BINARY64, keep_residue_planes=False)
    got = run_gemm(A, B, N, opA, opB, single=single)
    assert same_bits(got, em.out), mismatch_report(got, em.out)


@pytest.mark.parametrize("single", [False, True])
@pytest.mark.parametrize("opA,opB", [("N", "N"), ("T", "N")])
def test_real_accurate_bitexact(single, opA, opB):
    N = 7 if single else 14
    A, B = _real(300, 260, 333, opA, opB, 2.0, 82, single)
    em = RealEmulation(apply_op_real(A.astype(np.float64), opA), apply_op_real(B.astype(np.float64), opB), N,
                       scaling="accurate", out_fmt=fp.BINARY32 if single else fp.BINARY64)
    got = run_real(A, B, N, opA, opB, single=single)
    assert same_bits(got, em.out), mismatch_report(got, em.out)


@pytest.mark.parametrize("real", [False, True])
def test_bound_products_over_many_chunks(real):
    # k = 5000: the bound accumulation restarts every 4096 (complex C-bar_I runs over 2k: 3 chunks)
    if real:
        A, B = _real(70, 150, 5000, "N", "N", 1.0, 84, False)
        ref = RealEmulation(A, B, 12, scaling="accurate").out
        got = run_real(A, B, 12)
    else:
        A, B = _cplx(70, 150, 5000, "N", "N", 1.0, 86, False)
        ref = Emulation(A, B, 12, scaling="accurate", keep_residue_planes=False).out
        got = run_gemm(A, B, 12)
    assert same_bits(got, ref), mismatch_report(got, ref)


@pytest.mark.parametrize("N", [2, 24])
def test_moduli_extremes(N):
    A, B = _cplx(90, 70, 120, "N", "N", 3.0, 88, False)
    ref = Emulation(A, B, N, scaling="accurate", keep_residue_planes=False).out
    assert same_bits(run_gemm(A, B, N), ref)


def test_edge_cases():
    A, B = _cplx(40, 33, 64, "N", "N", 1.0, 90, False)
    A[3] = 0.0
    A[5, 7] = complex(np.inf, 0.0)
    B[9, 4] = complex(0.0, np.nan)
    A[8] *= 1e-310
    B[:, 11] *= 1e300
    ref = Emulation(A, B, 14, scaling="accurate", keep_residue_planes=False).out
    got = run_gemm(A, B, 14)
    assert same_bits(got, ref), mismatch_report(got, ref)
    Ar, Br = A.real.copy(), B.real.copy()
    refr = RealEmulation(Ar, Br, 14, scaling="accurate").out
    assert same_bits(run_real(Ar, Br, 14), refr)


@pytest.mark.parametrize("N,k", [(4, 16867), (5, 16274), (6, 15321)])
@pytest.mark.parametrize("kind", ["real", "complex"])
def test_range_correction_near_half_P(N, k, kind):
    # constant integer inputs with k chosen so that c' = M 4^E sits within 1e-4 of P/2:
    # the float quotient can round either way and the CRT must still return c'
    m, n = 16, 24
    if kind == "real":
        A, B = np.full((m, k), 3.0), np.full((k, n), 5.0)
        got = run_real(A, B, N)
        want = np.full((m, n), 15.0 * k)
    else:
        A, B = np.full((m, k), 3.0 + 0.0j), np.full((k, n), 5.0 + 0.0j)
        got = run_gemm(A, B, N)
        want = np.full((m, n), complex(15.0 * k, 0.0))
    assert same_bits(got, want), mismatch_report(got, want)


@pytest.mark.parametrize("kind", ["z", "d"])
def test_accurate_with_column_blocking(kind):
    m, n, k = 150, 3 * 128 + 45, 200
    if kind == "z":
        A, B = _cplx(m, n, k, "N", "N", 2.0, 92, False)
        one = run_gemm(A, B, 12)
        emu.check(emu.emu_set_tuning(emu.EMU_TUNE_NBLOCK, 128), "nblock")
        blk = run_gemm(A, B, 12)
    else:
        A, B = _real(m, n, k, "N", "N", 2.0, 93, False)
        one = run_real(A, B, 12)
        emu.check(emu.emu_set_tuning(emu.EMU_TUNE_NBLOCK, 128), "nblock")
        blk = run_real(A, B, 12)
    assert same_bits(blk, one), mismatch_report(blk, one)


def test_accurate_with_paper_fp_crt():
    A, B = _cplx(60, 50, 90, "N", "N", 1.0, 94, False)
    em = Emulation(A, B, 16, scaling="accurate")
    ref = outputs(em)
    emu.check(emu.emu_set_crt_mode(emu.EMU_CRT_PAPER_FP64), "crt")
    got = run_gemm(A, B, 16)
    assert same_bits(got, ref), mismatch_report(got, ref)
    Ar, Br = A.real.copy(), B.real.copy()
    emr = RealEmulation(Ar, Br, 16, scaling="accurate")
    assert same_bits(run_real(Ar, Br, 16), outputs_real(emr))


def test_accuracy_gain_over_fast_at_same_N():
    """Accurate scaling keeps more bits where its exponents exceed the fast ones.
    Over all entries the largest error sits on entries whose two total shifts
    x_i + y_j coincide, so the test compares the mean error over all entries and
    the maximum error over the entries where the accurate shift is larger (the
    exponents are the oracle's, which the GPU's equal bit for bit)."""
    A, B = _cplx(200, 180, 2000, "N", "N", 2.0, 96, False)
    exact = Emulation(A, B, 24, keep_residue_planes=False).out            # reference, far below the errors
    bound = (np.abs(A.real) + np.abs(A.imag)) @ (np.abs(B.real) + np.abs(B.imag))
    shift = {}
    for mode, name in ((emu.EMU_SCALING_FAST, "fast"), (emu.EMU_SCALING_ACCURATE, "accurate")):
        em = Emulation(A, B, 10, keep_residue_planes=False, scaling=name)
        shift[mode] = em.x[:, None] + em.y[None, :]
    errs = {}
    for mode in (emu.EMU_SCALING_FAST, emu.EMU_SCALING_ACCURATE):
        emu.check(emu.emu_set_scaling(mode), "scaling")
        got = run_gemm(A, B, 10)
        errs[mode] = np.maximum(np.abs(got.real - exact.real), np.abs(got.imag - exact.imag)) / bound
    fast, accu = errs[emu.EMU_SCALING_FAST], errs[emu.EMU_SCALING_ACCURATE]
    more = shift[emu.EMU_SCALING_ACCURATE] > shift[emu.EMU_SCALING_FAST]
    assert np.all(shift[emu.EMU_SCALING_ACCURATE] >= shift[emu.EMU_SCALING_FAST])
    assert more.sum() > more.size // 2
    # the tighter bound keeps about half a bit more on average here (k = 2000, phi = 2)
    assert accu.mean() < fast.mean() / 1.2, (accu.mean(), fast.mean())
    assert accu[more].max() < fast[more].max(), (accu[more].max(), fast[more].max())


@pytest.mark.parametrize("pair", [1, 0], ids=["sm_pairs", "one_sm"])
@pytest.mark.parametrize("case", ["complex", "real", "single", "chunks", "edges", "one"])
def test_bound_products_on_sm_pairs(case, pair):
    """The bound products on SM pairs (256-column tiles, each CTA of a pair
    holding 128 of them and loading half of the 128 rows) and on one SM
    (128-column tiles): the same exponents and results, including column
    counts that leave the odd CTA of a pair only padding."""
    emu.check(emu.emu_set_tuning(emu.EMU_TUNE_BOUND_PAIR, pair), "bound pair")
    if case == "real":
        A, B = _real(300, 520, 333, "N", "T", 2.0, 94, False)
        ref = RealEmulation(A, apply_op_real(B, "T"), 14, scaling="accurate").out
        got = run_real(A, B, 14, "N", "T")
    elif case == "single":
        A, B = _cplx(257, 300, 200, "N", "N", 1.0, 96, True)
        ref = Emulation(A.astype(np.complex128), B.astype(np.complex128), 7, scaling="accurate",
                        out_fmt=fp.BINARY32, keep_residue_planes=False).out
        got = run_gemm(A, B, 7, single=True)
    else:
        m, n, k = {"complex": (300, 600, 333), "chunks": (70, 150, 5000), "edges": (129, 100, 64),
                   "one": (1, 1, 1)}[case]
        A, B = _cplx(m, n, k, "N", "N", 2.0, 98, False)
        if case == "edges":
            A[3] = 0.0
            A[5, 7] = complex(np.inf, 0.0)
            B[9, 4] = complex(0.0, np.nan)
        ref = Emulation(A, B, 13, scaling="accurate", keep_residue_planes=False).out
        got = run_gemm(A, B, 13)
    assert same_bits(got, ref), mismatch_report(got, ref)
    assert emu.emu_stream_status() == emu.EMU_OK


@pytest.mark.parametrize("pair", [1, 0], ids=["sm_pairs", "one_sm"])
@pytest.mark.parametrize("real", [False, True], ids=["complex", "real"])
def test_bound_products_several_tiles_per_cta(real, pair):
    """4096 x 4096 outputs, k = 2100: 256 (pairs) or 512 (one SM) bound-product
    tiles, so every CTA runs several, each of three FP32 chunks (C-bar_I over 2k
    in two, the difference product in one; real input: one of two), and complex
    CTAs reuse their scratch.  The exponents come from the oracle's whole bound
    product; results bit for bit on sampled entries."""
    from oracle.accurate import accurate_exponents
    from oracle.emulate import emulate_entries
    from oracle.emulate_real import emulate_real_entries
    from oracle.moduli import Plan
    from paper_2512_08321_gb300.workloads import paper_matrix_device, paper_matrix_real_device
    emu.check(emu.emu_set_tuning(emu.EMU_TUNE_BOUND_PAIR, pair), "bound pair")
    m = n = 4096
    k, N = 2100, 13
    if real:
        A = paper_matrix_real_device(m, k, 2.0, 120, torch.float64)      # storage (k, m)
        B = paper_matrix_real_device(k, n, 2.0, 121, torch.float64)      # storage (n, k)
        C = torch.zeros((n, m), dtype=torch.float64, device="cuda")
        f = emu.emu_dgemm
    else:
        A = paper_matrix_device(m, k, 2.0, 122, torch.complex128)
        B = paper_matrix_device(k, n, 2.0, 123, torch.complex128)
        C = torch.zeros((n, m), dtype=torch.complex128, device="cuda")
        f = emu.emu_zgemm
    emu.check(f("N", "N", m, n, k, 1.0, A.data_ptr(), m, B.data_ptr(), k, 0.0, C.data_ptr(), m, N, None), "gemm")
    torch.cuda.synchronize()
    assert emu.emu_stream_status() == emu.EMU_OK
    Ah, Bh = A.t().cpu().numpy(), B.t().cpu().numpy()                   # op(A) m x k, op(B) k x n
    ex = accurate_exponents(Ah, Bh, Plan(N).P, real=real)
    rng = np.random.default_rng(11)
    rows = np.concatenate([[0, m - 1], rng.integers(0, m, 30)])
    cols = np.concatenate([[0, n - 1], rng.integers(0, n, 30)])
    got = C[torch.from_numpy(cols).cuda(), torch.from_numpy(rows).cuda()].cpu().numpy()
    entries = emulate_real_entries if real else emulate_entries
    want = entries(Ah, Bh, N, rows, cols, xy=(ex["x"], ex["y"]))
    assert np.array_equal(got.view(np.float64), want.view(np.float64))
