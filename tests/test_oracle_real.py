"""Pins for the real-matrix oracle (DGEMM / SGEMM emulation): checks against
closed forms, exact integer arithmetic, the independently pinned complex
oracle and the correctly rounded exact product.  CPU only."""
import numpy as np
import pytest

from oracle import fp
from oracle.crt_fp import outputs_real
from oracle.emulate import emulate
from oracle.emulate_real import RealEmulation, emulate_real, emulate_real_entries
from oracle.exact import _exact_matmul, real_product_entries
from oracle.moduli import Plan
from oracle.scaling import NONFINITE
from paper_2512_08321_gb300.workloads import paper_matrix_real


def test_integer_inputs_are_exact():
    # small integers: x_i >= 0, nothing is truncated, C' = AB exactly
    rng = np.random.default_rng(1)
    A = rng.integers(-1000, 1000, size=(7, 20)).astype(np.float64)
    B = rng.integers(-1000, 1000, size=(20, 5)).astype(np.float64)
    em = RealEmulation(A, B, 8)
    assert np.all(em.x >= 0) and np.all(em.y >= 0)
    assert np.array_equal(em.out, A @ B)          # |AB| < 2^53: the float product is exact


@pytest.mark.parametrize("N", [2, 5, 14, 20])
def test_crt_equals_exact_integer_product(N):
    A = paper_matrix_real(9, 33, 1.0, 11)
    B = paper_matrix_real(33, 6, 1.0, 12)
    em = RealEmulation(A, B, N)
    exact = _exact_matmul(em.Ai, em.Bi)
    assert all(int(em.c[i, j]) == int(exact[i, j]) for i in range(9) for j in range(6))
    # condition (cond): 2 max |c'| < P with the (P-1)/8 margin
    assert 8 * max(abs(int(v)) for v in exact.ravel()) <= Plan(N).P - 1


def test_residue_products_match_exact_product_mod_p():
    A = paper_matrix_real(5, 40, 2.0, 13)
    B = paper_matrix_real(40, 4, 2.0, 14)
    em = RealEmulation(A, B, 6)
    exact = _exact_matmul(em.Ai, em.Bi)
    for l, p in enumerate(em.plan.p):
        for i in range(5):
            for j in range(4):
                r = int(exact[i, j]) % p
                r = r - p if 2 * r >= p else r
                assert em.Eprime[l, i, j] == r


@pytest.mark.parametrize("N", [6, 14])
def test_agrees_with_complex_oracle_on_real_inputs(N):
    # a complex product with zero imaginary parts has the same exponents,
    # truncations and real part: the (separately pinned) complex oracle's real
    # part equals the real oracle bit for bit
    A = paper_matrix_real(6, 25, 1.5, 15)
    B = paper_matrix_real(25, 7, 1.5, 16)
    r = RealEmulation(A, B, N).out
    c = emulate(A.astype(np.complex128), B.astype(np.complex128), N).out
    assert np.array_equal(r.view(np.uint64), np.ascontiguousarray(c.real).view(np.uint64))


def test_converges_to_correctly_rounded_product():
    A = paper_matrix_real(8, 64, 1.0, 17)
    B = paper_matrix_real(64, 8, 1.0, 18)
    rows, cols = np.meshgrid(np.arange(8), np.arange(8), indexing="ij")
    ref = real_product_entries(A, B, rows.ravel(), cols.ravel()).reshape(8, 8)
    bound = np.abs(A) @ np.abs(B)
    errs = [float(np.max(np.abs(RealEmulation(A, B, N).out - ref) / bound)) for N in (8, 10, 12, 14)]
    # two more moduli add about 15 bits per operand until the binary64 floor
    for a, b in zip(errs, errs[1:]):
        assert b < a / 64
    assert errs[-1] < 2.0 ** -49
    # with enough moduli the truncation error vanishes below half an ulp: RN(AB)
    assert np.array_equal(RealEmulation(A, B, 18).out, ref)


def test_row_scale_invariance():
    A = paper_matrix_real(4, 30, 1.0, 19)
    B = paper_matrix_real(30, 3, 1.0, 20)
    A2 = A.copy()
    A2[2] *= 2.0 ** 37
    e1, e2 = RealEmulation(A, B, 10), RealEmulation(A2, B, 10)
    assert e2.x[2] == e1.x[2] - 37
    assert np.array_equal(e2.out[2], e1.out[2] * 2.0 ** 37)
    assert np.array_equal(np.delete(e2.out, 2, 0), np.delete(e1.out, 2, 0))


def test_ops_and_alpha_beta_and_single():
    A = paper_matrix_real(20, 6, 1.0, 21)          # stored k x m for op T
    B = paper_matrix_real(9, 20, 1.0, 22)          # stored n x k for op T
    C = paper_matrix_real(6, 9, 1.0, 23)
    base = emulate_real(A, B, 12, "T", "C").out
    assert np.array_equal(base, emulate_real(A.T.copy(), B.T.copy(), 12).out)
    ab = emulate_real(A, B, 12, "T", "T", alpha=-0.75, beta=2.0, C_in=C).out
    want = np.array([[fp.fma64(2.0, C[i, j], -0.75 * base[i, j]) for j in range(9)] for i in range(6)])
    assert np.array_equal(ab, want)
    s = emulate_real(A.astype(np.float32), B.astype(np.float32), 12, "T", "T", out_fmt=fp.BINARY32).out
    assert s.dtype == np.float32
    assert np.array_equal(s, emulate_real(A.astype(np.float32).astype(np.float64),
                                          B.astype(np.float32).astype(np.float64), 12, "T", "T").out.astype(np.float32))


def test_nonfinite_rows_and_zero_rows():
    A = paper_matrix_real(5, 12, 1.0, 24)
    B = paper_matrix_real(12, 4, 1.0, 25)
    A[1, 3] = np.inf
    A[3] = 0.0
    B[5, 2] = np.nan
    em = RealEmulation(A, B, 8)
    assert em.x[1] == NONFINITE and em.y[2] == NONFINITE
    assert np.all(np.isnan(em.out[1])) and np.all(np.isnan(em.out[:, 2]))
    assert np.all(em.out[3][[0, 1, 3]] == 0.0)


def test_sampled_entries_equal_full_pipeline():
    A = paper_matrix_real(11, 50, 2.0, 26)
    B = paper_matrix_real(50, 9, 2.0, 27)
    full = RealEmulation(A, B, 13).out
    rows = [0, 3, 10, 10, 7]
    cols = [8, 0, 4, 8, 2]
    got = emulate_real_entries(A, B, 13, rows, cols)
    assert np.array_equal(got, full[rows, cols])


@pytest.mark.parametrize("N", [3, 5])
def test_paper_fp_crt_exact_when_P_small(N):
    # N * 128 * P < 2^53: every double operation of the FP CRT is exact
    A = paper_matrix_real(6, 16, 1.0, 28)
    B = paper_matrix_real(16, 5, 1.0, 29)
    em = RealEmulation(A, B, N)
    assert N * 128 * em.plan.P < 2 ** 53
    assert np.array_equal(outputs_real(em), em.out)
    assert np.array_equal(outputs_real(em, single=True), em.out.astype(np.float32))


def test_paper_fp_crt_error_bound_large_N():
    A = paper_matrix_real(6, 40, 1.0, 30)
    B = paper_matrix_real(40, 5, 1.0, 31)
    em = RealEmulation(A, B, 16)
    fpo = outputs_real(em)
    # the double-double reduction keeps c' within a few units of 2^-100 |c'|-scale
    bound = np.abs(A) @ np.abs(B)
    assert np.max(np.abs(fpo - em.out) / bound) < 1e-17
