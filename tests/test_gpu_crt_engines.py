"""The two CRT kernels (Steps V-v, V-vi, VI): the sum over moduli as an exact
fp16 product with digits of the CRT weights on the tensor cores, and limb
products on the CUDA cores.  Both must give the oracle's outputs bit for bit
for every limb count (N = 2 .. 24: 1 to 6 32-bit limbs, the 32- and 64-column
layouts), real and complex, both output precisions, fast and accurate
scaling, ragged row blocks and the stage entry point."""
import numpy as np
import pytest
import torch

from oracle import fp
from oracle.emulate import Emulation, apply_op, emulate
from oracle.emulate_real import emulate_real
from paper_2512_08321_gb300 import emu
from paper_2512_08321_gb300.workloads import paper_matrix, paper_matrix_real

from .helpers import dev, host, mismatch_report, run_gemm, run_real, same_bits

pytestmark = pytest.mark.gpu

ENGINES = [1, 0]


@pytest.fixture(autouse=True)
def _restore():
    saved = emu.emu_get_tuning(emu.EMU_TUNE_CRT_ENGINE)
    yield
    emu.emu_set_tuning(emu.EMU_TUNE_CRT_ENGINE, saved)
    emu.emu_set_scaling(emu.EMU_SCALING_FAST)


def _engine(e):
    emu.check(emu.emu_set_tuning(emu.EMU_TUNE_CRT_ENGINE, e), "crt engine")


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("N", [2, 3, 5, 8, 12, 15, 16, 17, 20, 24])
def test_zgemm_every_limb_count(engine, N):
    m, n, k = 200, 70, 150                    # two row blocks, the second ragged
    A = paper_matrix(m, k, 1.5, 300 + N)
    B = paper_matrix(k, n, 1.5, 400 + N)
    ref = emulate(A, B, N, keep_residue_planes=False)
    _engine(engine)
    got = run_gemm(A, B, N)
    assert same_bits(got, ref.out), mismatch_report(got, ref.out)


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("N", [2, 6, 9, 13])
def test_cgemm_every_limb_count(engine, N):
    m, n, k = 131, 40, 97
    A = paper_matrix(m, k, 0.5, 500 + N, np.complex64)
    B = paper_matrix(k, n, 0.5, 600 + N, np.complex64)
    ref = emulate(A.astype(np.complex128), B.astype(np.complex128), N, out_fmt=fp.BINARY32,
                  keep_residue_planes=False)
    _engine(engine)
    got = run_gemm(A, B, N, single=True)
    assert same_bits(got, ref.out), mismatch_report(got, ref.out)


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("single,N", [(False, 2), (False, 15), (False, 24), (True, 4), (True, 8)])
def test_real_every_limb_count(engine, single, N):
    m, n, k = 150, 33, 120
    A = paper_matrix_real(m, k, 1.0, 700 + N)
    B = paper_matrix_real(k, n, 1.0, 800 + N)
    if single:
        A, B = A.astype(np.float32), B.astype(np.float32)
    ref = emulate_real(A.astype(np.float64), B.astype(np.float64), N,
                       out_fmt=fp.BINARY32 if single else fp.BINARY64)
    _engine(engine)
    got = run_real(A, B, N, single=single)
    assert same_bits(got, ref.out), mismatch_report(got, ref.out)


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("N", [3, 14, 20])
def test_accurate_scaling_range_fix(engine, N):
    """Accurate mode lets |c'| reach (P-1)/2, so the quotient estimate can be
    one off and the range correction runs."""
    m, n, k = 140, 60, 200
    A = paper_matrix(m, k, 2.0, 900 + N)
    B = paper_matrix(k, n, 2.0, 950 + N)
    em = Emulation(A, B, N, scaling="accurate", keep_residue_planes=False)
    _engine(engine)
    emu.check(emu.emu_set_scaling(emu.EMU_SCALING_ACCURATE), "scaling")
    got = run_gemm(A, B, N)
    assert same_bits(got, em.out), mismatch_report(got, em.out)


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("m", [1, 15, 17, 128, 129])
def test_row_block_edges_alpha_beta(engine, m):
    """Row counts at and around the 16-row storage unit and the 128-row block,
    with alpha/beta and a ldc larger than m."""
    n, k, N = 9, 40, 14
    A = paper_matrix(m, k, 1.0, 1000 + m)
    B = paper_matrix(k, n, 1.0, 1100 + m)
    C = paper_matrix(m, n, 1.0, 1200 + m)
    alpha, beta = 0.75 - 0.5j, -1.25 + 2.0j
    ref = emulate(A, B, N, alpha=(alpha.real, alpha.imag), beta=(beta.real, beta.imag), C_in=C,
                  keep_residue_planes=False)
    _engine(engine)
    got = run_gemm(A, B, N, alpha=alpha, beta=beta, C=C, ldc=m + 5)
    assert same_bits(got, ref.out), mismatch_report(got, ref.out)


@pytest.mark.parametrize("engine", ENGINES)
def test_nonfinite_rows_and_columns(engine):
    m, n, k, N = 140, 20, 64, 15
    A = paper_matrix(m, k, 1.0, 1300)
    B = paper_matrix(k, n, 1.0, 1301)
    A[5, 3] = np.inf
    A[133, 0] = np.nan
    B[7, 11] = -np.inf
    ref = emulate(A, B, N, keep_residue_planes=False)
    _engine(engine)
    got = run_gemm(A, B, N)
    assert same_bits(got, ref.out), mismatch_report(got, ref.out)


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("single", [False, True])
def test_stage_crt_both_engines(engine, single):
    N = 8 if single else 16
    m, n, k = 300, 41, 90
    A = paper_matrix(m, k, 2.0, 1400)
    B = paper_matrix(k, n, 2.0, 1401)
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
    dC = dev(np.zeros((m, n), dtype=np.complex64 if single else np.complex128))
    _engine(engine)
    emu.check(emu.emu_stage_crt(single, m, n, N, dres.data_ptr(), ldr, x.data_ptr(), y.data_ptr(),
                                1.0, 0.0, dC.data_ptr(), m), "crt")
    torch.cuda.synchronize()
    assert emu.emu_stream_status() == emu.EMU_OK
    got = host(dC, m)
    assert same_bits(got, ref.out), mismatch_report(got, ref.out)


def test_engines_agree_on_a_larger_product():
    """More items than resident blocks (each block walks several items, both
    staging buffers in turn), compared between the engines bit for bit."""
    m, n, k, N = 1000, 300, 64, 15
    A = paper_matrix(m, k, 1.0, 1500)
    B = paper_matrix(k, n, 1.0, 1501)
    _engine(0)
    ref = run_gemm(A, B, N)
    _engine(1)
    got = run_gemm(A, B, N)
    assert same_bits(got, ref), mismatch_report(got, ref)
    assert emu.emu_stream_status() == emu.EMU_OK
