"""GPU parity: every stage of the CUDA path against the CPU oracle, bit for bit,
through the C ABI.  Shapes span several tiles with ragged tails."""
import numpy as np
import pytest
import torch

from oracle import fp
from oracle.emulate import apply_op, emulate
from paper_2512_08321_gb300 import emu
from paper_2512_08321_gb300.workloads import paper_matrix

from .helpers import dev, host, mismatch_report, run_gemm, same_bits

pytestmark = pytest.mark.gpu

ENGINES = {"i8": emu.EMU_ENGINE_I8, "f16": emu.EMU_ENGINE_F16}


@pytest.fixture(autouse=True)
def _restore_engine():
    yield
    emu.emu_set_engine(emu.EMU_ENGINE_AUTO, 512)


def _stages(A, B, N, opA, opB, single, fp16):
    """Run the stage entry points; return x, y, planes A/B (numpy), residues."""
    m = A.shape[0] if opA == "N" else A.shape[1]
    k = A.shape[1] if opA == "N" else A.shape[0]
    n = B.shape[1] if opB == "N" else B.shape[0]
    dt = np.complex64 if single else np.complex128
    dA, dB = dev(A.astype(dt)), dev(B.astype(dt))
    x = torch.zeros(m, dtype=torch.int16, device="cuda")
    y = torch.zeros(n, dtype=torch.int16, device="cuda")
    emu.check(emu.emu_stage_exponents(single, opA, opB, m, n, k, dA.data_ptr(), dA.shape[1],
                                      dB.data_ptr(), dB.shape[1], N, x.data_ptr(), y.data_ptr()), "exp")
    kpad = (k + 63) // 64 * 64
    pdt = torch.float16 if fp16 else torch.int8
    pa = torch.full((3 * N, m, kpad), 77, dtype=pdt, device="cuda")
    pb = torch.full((3 * N, n, kpad), 77, dtype=pdt, device="cuda")
    emu.check(emu.emu_stage_split(single, opA, opB, m, n, k, dA.data_ptr(), dA.shape[1], dB.data_ptr(),
                                  dB.shape[1], N, x.data_ptr(), y.data_ptr(), fp16, kpad,
                                  pa.data_ptr(), pb.data_ptr()), "split")
    torch.cuda.synchronize()
    return m, n, k, kpad, x, y, pa, pb


@pytest.mark.parametrize("opA,opB", [("N", "N"), ("T", "N"), ("C", "T"), ("N", "C")])
@pytest.mark.parametrize("single", [False, True])
def test_exponents_and_planes_bitexact(opA, opB, single):
    N = 9 if single else 14
    A = paper_matrix(70, 45, 1.0, 1) if opA == "N" else paper_matrix(45, 70, 1.0, 1)
    B = paper_matrix(45, 37, 1.0, 2) if opB == "N" else paper_matrix(37, 45, 1.0, 2)
    if single:
        A, B = A.astype(np.complex64), B.astype(np.complex64)
    ref = emulate(A.astype(np.complex128), B.astype(np.complex128), N, opA=opA, opB=opB)
    for fp16 in (False, True):
        m, n, k, kpad, x, y, pa, pb = _stages(A, B, N, opA, opB, single, fp16)
        assert np.array_equal(x.cpu().numpy(), ref.x.astype(np.int16))
        assert np.array_equal(y.cpu().numpy(), ref.y.astype(np.int16))
        PA = pa.cpu().numpy().astype(np.int64)
        PB = pb.cpu().numpy().astype(np.int64)
        for l in range(N):
            for c in range(3):
                assert np.array_equal(PA[3 * l + c, :, :k], ref.planesA[l, c]), (l, c)
                assert np.array_equal(PB[3 * l + c, :, :k], ref.planesB[l, c]), (l, c)
        assert np.all(PA[:, :, k:] == 0) and np.all(PB[:, :, k:] == 0)


@pytest.mark.parametrize("engine", ["i8", "f16"])
@pytest.mark.parametrize("m,n,k,N", [(130, 70, 200, 14), (64, 64, 64, 6), (257, 129, 700, 16),
                                     (5, 3, 1, 2), (33, 300, 130, 20)])
def test_residue_gemm_bitexact(engine, m, n, k, N):
    A = paper_matrix(m, k, 0.5, 11)
    B = paper_matrix(k, n, 0.5, 12)
    ref = emulate(A, B, N)
    fp16 = engine == "f16"
    m, n, k, kpad, x, y, pa, pb = _stages(A, B, N, "N", "N", False, fp16)
    ldr = (m + 15) // 16 * 16
    res = torch.full((3 * N, n, ldr), 99, dtype=torch.int8, device="cuda")
    st = emu.emu_stage_residue_gemm(ENGINES[engine], m, n, kpad, N, pa.data_ptr(), pb.data_ptr(),
                                    res.data_ptr(), ldr)
    emu.check(st, "residue_gemm")
    assert emu.emu_stream_status() == emu.EMU_OK
    R = res.cpu().numpy().astype(np.int64)
    for l in range(N):
        for c in range(3):
            got = R[3 * l + c, :, :m].T
            assert np.array_equal(got, ref.DEF[l, c]), (l, c, mismatch_report(got, ref.DEF[l, c]))


@pytest.mark.parametrize("engine", ["i8", "f16"])
def test_residue_gemm_extreme_residues(engine):
    # every residue -128 (p = 256) or the most negative symmetric residue:
    # the largest products the accumulation must carry exactly
    N, m, n, k = 4, 96, 80, 2048
    kpad = k
    fp16 = engine == "f16"
    vals = np.zeros((3 * N, 1, 1))
    plan_p = emu.emu_plan_info(N)[1]
    for l, p in enumerate(plan_p):
        vals[3 * l:3 * l + 3] = -(p // 2)
    A = np.broadcast_to(vals, (3 * N, m, k)).copy()
    B = np.broadcast_to(vals, (3 * N, n, k)).copy()
    pdt = torch.float16 if fp16 else torch.int8
    pa = torch.from_numpy(A).to(pdt).cuda()
    pb = torch.from_numpy(B).to(pdt).cuda()
    ldr = 96
    res = torch.zeros((3 * N, n, ldr), dtype=torch.int8, device="cuda")
    emu.check(emu.emu_stage_residue_gemm(ENGINES[engine], m, n, kpad, N, pa.data_ptr(), pb.data_ptr(),
                                         res.data_ptr(), ldr), "residue_gemm")
    R = res.cpu().numpy().astype(np.int64)
    for l, p in enumerate(plan_p):
        v = (p // 2) ** 2 * k
        want = v % p
        want = want - p if 2 * want >= p else want
        assert np.all(R[3 * l:3 * l + 3, :, :m] == want), (l, p)


@pytest.mark.parametrize("single", [False, True])
def test_crt_stage_bitexact(single):
    N = 8 if single else 16
    m, n, k = 100, 52, 90
    A = paper_matrix(m, k, 2.0, 21)
    B = paper_matrix(k, n, 2.0, 22)
    if single:
        A, B = A.astype(np.complex64), B.astype(np.complex64)
    ref = emulate(A.astype(np.complex128), B.astype(np.complex128), N,
                  out_fmt=fp.BINARY32 if single else fp.BINARY64)
    ldr = (m + 15) // 16 * 16
    res = np.zeros((3 * N, n, ldr), dtype=np.int8)
    for l in range(N):
        for c in range(3):
            res[3 * l + c, :, :m] = ref.DEF[l, c].T
    dres = torch.from_numpy(res).cuda()
    x = torch.from_numpy(ref.x.astype(np.int16)).cuda()
    y = torch.from_numpy(ref.y.astype(np.int16)).cuda()
    dt = np.complex64 if single else np.complex128
    dC = dev(np.zeros((m, n), dtype=dt))
    emu.check(emu.emu_stage_crt(single, m, n, N, dres.data_ptr(), ldr, x.data_ptr(), y.data_ptr(),
                                1.0, 0.0, dC.data_ptr(), m), "crt")
    torch.cuda.synchronize()
    got = host(dC, m)
    assert same_bits(got, ref.out), mismatch_report(got, ref.out)


@pytest.mark.parametrize("engine", ["i8", "f16"])
@pytest.mark.parametrize("opA,opB", [("N", "N"), ("T", "C"), ("C", "N")])
@pytest.mark.parametrize("N", [6, 14, 20])
def test_zgemm_bitexact(engine, opA, opB, N):
    m, n, k = 150, 90, 333
    A = paper_matrix(m, k, 1.0, 31 + N) if opA == "N" else paper_matrix(k, m, 1.0, 31 + N)
    B = paper_matrix(k, n, 1.0, 41 + N) if opB == "N" else paper_matrix(n, k, 1.0, 41 + N)
    ref = emulate(A, B, N, opA=opA, opB=opB, keep_residue_planes=False)
    got = run_gemm(A, B, N, opA, opB, engine=ENGINES[engine])
    assert same_bits(got, ref.out), mismatch_report(got, ref.out)


@pytest.mark.parametrize("engine", ["i8", "f16"])
def test_cgemm_bitexact(engine):
    m, n, k, N = 140, 77, 260, 8
    A = paper_matrix(m, k, 0.5, 51, np.complex64)
    B = paper_matrix(k, n, 0.5, 52, np.complex64)
    ref = emulate(A.astype(np.complex128), B.astype(np.complex128), N, out_fmt=fp.BINARY32,
                  keep_residue_planes=False)
    got = run_gemm(A, B, N, single=True, engine=ENGINES[engine])
    assert got.dtype == np.complex64
    assert same_bits(got, ref.out), mismatch_report(got, ref.out)


@pytest.mark.parametrize("single", [False, True])
def test_alpha_beta_and_leading_dims(single):
    m, n, k, N = 40, 33, 50, 10
    A = paper_matrix(m, k, 1.0, 61)
    B = paper_matrix(k, n, 1.0, 62)
    C = paper_matrix(m, n, 1.0, 63)
    dt = np.complex64 if single else np.complex128
    A, B, C = A.astype(dt), B.astype(dt), C.astype(dt)
    al, be = complex(0.75, -1.25), complex(0.5, 2.0)
    ref = emulate(A.astype(np.complex128), B.astype(np.complex128), N, alpha=(al.real, al.imag),
                  beta=(be.real, be.imag), C_in=C.astype(np.complex128),
                  out_fmt=fp.BINARY32 if single else fp.BINARY64, keep_residue_planes=False)
    got = run_gemm(A, B, N, alpha=al, beta=be, C=C, single=single, lda=m + 7, ldb=k + 3, ldc=m + 5)
    assert same_bits(got, ref.out), mismatch_report(got, ref.out)


def test_beta_zero_ignores_nan_c():
    m, n, k, N = 20, 18, 30, 12
    A = paper_matrix(m, k, 1.0, 71)
    B = paper_matrix(k, n, 1.0, 72)
    C = np.full((m, n), complex(np.nan, np.nan))
    got = run_gemm(A, B, N, C=C, alpha=complex(2.0, 0.0), beta=0.0)
    ref = emulate(A, B, N, alpha=(2.0, 0.0), keep_residue_planes=False)
    assert same_bits(got, ref.out)


def test_edge_cases():
    N = 14
    # k = 0: C = beta * C
    C = paper_matrix(5, 4, 1.0, 81)
    got = run_gemm(np.zeros((5, 0), complex), np.zeros((0, 4), complex), N, C=C, alpha=1.0,
                   beta=complex(2.0, 0.0))
    ref = emulate(np.zeros((5, 0), complex), np.zeros((0, 4), complex), N, alpha=(1.0, 0.0),
                  beta=(2.0, 0.0), C_in=C)
    assert same_bits(got, ref.out)
    # k = 1, single rows/cols, zero rows, non-finite entries, subnormals, wide range
    A = paper_matrix(37, 65, 4.0, 82)
    B = paper_matrix(65, 29, 4.0, 83)
    A[3, :] = 0
    A[5, 10] = np.inf
    B[7, 4] = complex(0, np.nan)
    A[9, :] *= 1e-300
    A[11, 7] = 5e-324
    B[:, 20] *= 1e280
    ref = emulate(A, B, N, keep_residue_planes=False)
    got = run_gemm(A, B, N)
    assert same_bits(got, ref.out), mismatch_report(got, ref.out)
    A1 = paper_matrix(1, 1, 0.0, 84)
    B1 = paper_matrix(1, 1, 0.0, 85)
    assert same_bits(run_gemm(A1, B1, N), emulate(A1, B1, N).out)


def test_integer_inputs_exact():
    rng = np.random.default_rng(3)
    A = rng.integers(-100, 101, (70, 90)) + 1j * rng.integers(-100, 101, (70, 90))
    B = rng.integers(-100, 101, (90, 50)) + 1j * rng.integers(-100, 101, (90, 50))
    got = run_gemm(A, B, 14)
    assert np.array_equal(got, A @ B)


def test_bounded_wait_reports_timeout():
    assert emu.emu_stream_status() == emu.EMU_OK
    emu.check(emu.emu_selftest_bounded_wait(2_000_000), "selftest")
    assert emu.emu_stream_status() == emu.EMU_ERR_TIMEOUT
    assert emu.emu_stream_status() == emu.EMU_OK          # read-and-clear
    # the context is still usable
    A = paper_matrix(8, 8, 0.5, 91)
    assert same_bits(run_gemm(A, A, 8), emulate(A, A, 8).out)


@pytest.mark.parametrize("single,N", [(False, 14), (False, 20), (True, 7)])
def test_paper_fp64_crt_bitexact(single, N):
    """The paper's floating-point CRT (EMU_CRT_PAPER_FP64) against the oracle's
    restatement of the same IEEE sequence, bit for bit, with alpha/beta."""
    from oracle import crt_fp
    m, n, k = 70, 45, 200
    dt = np.complex64 if single else np.complex128
    A = paper_matrix(m, k, 1.0, 301).astype(dt)
    B = paper_matrix(k, n, 1.0, 302).astype(dt)
    C = paper_matrix(m, n, 1.0, 303).astype(dt)
    em = emulate(A.astype(np.complex128), B.astype(np.complex128), N, keep_residue_planes=False)
    al, be = complex(0.5, -1.5), complex(2.0, 0.25)
    want = crt_fp.outputs(em, single=single, alpha=(al.real, al.imag), beta=(be.real, be.imag),
                          C_in=C.astype(np.complex128))
    emu.check(emu.emu_set_crt_mode(emu.EMU_CRT_PAPER_FP64), "crt mode")
    try:
        got = run_gemm(A, B, N, alpha=al, beta=be, C=C, single=single)
    finally:
        emu.emu_set_crt_mode(emu.EMU_CRT_EXACT)
    assert same_bits(got, want), mismatch_report(got, want)


@pytest.mark.parametrize("single", [False, True])
def test_outputs_across_the_subnormal_range_and_overflow(single):
    """Output magnitudes swept by exact power-of-two scalings of rows and
    columns through the normal range, the subnormals, underflow to (signed)
    zero and overflow to infinity: the CRT's integer rounding against the
    oracle's (each scaling only shifts x_i or y_j, so c' is unchanged)."""
    N = 14
    m, n, k = 24, 64, 40
    A = paper_matrix(m, k, 1.0, 401)
    B = paper_matrix(k, n, 1.0, 402)
    h = n // 2
    if single:       # complex64: normal down to 2^-126, subnormal to 2^-149, finite below 2^128
        a_lo, a_hi, b_under, b_step, b_over = -50, 58, -70, -2, 60
    else:            # complex128: normal down to 2^-1022, subnormal to 2^-1074, finite below 2^1024
        a_lo, a_hi, b_under, b_step, b_over = -480, 480, -540, -3, 520
    A[: m // 2] *= 2.0 ** a_lo
    A[m // 2:] *= 2.0 ** a_hi
    for j in range(h):                  # rows scaled by 2^a_lo: outputs near 2^(a_lo + b_under + b_step j)
        B[:, j] *= 2.0 ** (b_under + b_step * j)
    for j in range(h, n):               # rows scaled by 2^a_hi: outputs near 2^(a_hi + b_over + j - h)
        B[:, j] *= 2.0 ** (b_over + j - h)
    dt = np.complex64 if single else np.complex128
    A, B = A.astype(dt), B.astype(dt)
    ref = emulate(A.astype(np.complex128), B.astype(np.complex128), N, keep_residue_planes=False,
                  out_fmt=fp.BINARY32 if single else fp.BINARY64)
    got = run_gemm(A, B, N, single=single)
    want = ref.out
    assert same_bits(got, want), mismatch_report(got, want)
    # the sweep reached what it is for
    w = np.concatenate([want.real.ravel(), want.imag.ravel()])
    tiny = np.finfo(np.float32 if single else np.float64).tiny
    assert np.any((w != 0) & (np.abs(w) < tiny))                  # subnormal results
    assert np.any(w == 0) and np.any(np.signbit(w[w == 0]))       # underflow, with its sign
    assert np.any(np.isinf(w))                                   # overflow
