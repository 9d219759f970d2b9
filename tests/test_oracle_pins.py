"""Pins for the CPU oracle: checks against what the paper and mathematics fix,
independent of the oracle's own code paths (brute force, closed forms,
invariants, the paper's worked example).  CPU only."""
import math
import os
from fractions import Fraction
from math import gcd

import numpy as np
import pytest

from oracle import fp
from oracle.emulate import Emulation, apply_op, emulate, emulate_entries, sym_mod
from oracle.exact import _limbs, _two_product, complex_product_entries, scaled_integer_product
from oracle.metrics import abs_bound_entries, max_normalised_error, max_rel_error
from oracle.model import model_tflops
from oracle.moduli import Plan, choose_moduli
from oracle.scaling import NONFINITE, exponent_E, row_vectors, vector_exponents
from paper_2512_08321_gb300.workloads import paper_matrix

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Steps I-II
def test_moduli_pairwise_coprime_and_bounded():
    for N in (2, 6, 14, 20, 24):
        p = choose_moduli(N)
        assert len(p) == N and all(2 <= v <= 256 for v in p)
        for a in range(N):
            for b in range(a + 1, N):
                assert gcd(p[a], p[b]) == 1


def test_moduli_greedy_is_maximal():
    # every integer in (min p, 256] that was skipped shares a factor with a kept one
    p = choose_moduli(24)
    for c in range(min(p) + 1, 257):
        if c not in p:
            assert any(gcd(c, v) > 1 for v in p if v > c)


def test_inverses_by_brute_force():
    for N in (3, 14, 24):
        plan = Plan(N)
        for pl, ql in zip(plan.p, plan.q):
            M = plan.P // pl
            brute = [q for q in range(pl) if (M * q) % pl == 1]
            assert brute == [ql]


def test_crt_bijection_tiny_moduli():
    # every integer in the symmetric range is recovered from its residues
    for moduli in ([3, 5, 7], [7, 11, 13], [4, 9, 5]):
        plan = Plan(len(moduli), moduli)
        P = plan.P
        for x in range(-(P // 2), (P + 1) // 2):
            S = sum(w * (x % p) for w, p in zip(plan.w, plan.p))
            assert sym_mod(S, P) == x


# ------------------------------------------------------ symmetric remainder
def test_sym_mod_matches_definition():
    # mod(x,p) = x - p*round(x/p) with ties rounded up (reading of Section II)
    for p in (2, 3, 7, 173, 255, 256):
        xs = np.arange(-3 * p - 5, 3 * p + 6)
        got = sym_mod(xs, p)
        for x, g in zip(xs, got):
            want = int(x) - p * math.floor(Fraction(int(x), p) + Fraction(1, 2))
            assert g == want
        lo = -(p // 2)
        hi = (p - 1) // 2
        assert got.min() == lo and got.max() == hi


def test_sym_mod_256_is_int8_cast():
    xs = np.arange(-70000, 70000, 37)
    assert np.array_equal(sym_mod(xs, 256), xs.astype(np.int64).astype(np.int8).astype(np.int64))


# ------------------------------------------------------------------ fp helpers
def test_round_scaled_matches_cpython_division():
    rng = np.random.default_rng(5)
    for _ in range(3000):
        num = int(rng.integers(-(1 << 62), 1 << 62)) * int(rng.integers(1, 1 << 40))
        e = int(rng.integers(-1200, 200))
        got = fp.round_scaled(num, e)
        want = num / (1 << -e) if e < 0 else float(num << e)   # CPython: correctly rounded
        assert got == want and math.copysign(1, got) == math.copysign(1, want)


def test_round_scaled_subnormal_and_overflow():
    assert fp.round_scaled(1, -1074) == 5e-324
    assert fp.round_scaled(1, -1075) == 0.0          # tie to even (zero)
    assert fp.round_scaled(3, -1076) == 5e-324       # 0.75 ulp -> 1 ulp
    assert fp.round_scaled(1, 1024) == math.inf
    assert fp.round_scaled((1 << 53) - 1, 971) == 1.7976931348623157e308
    assert fp.round_scaled(-1, 1024) == -math.inf


def test_round_scaled_binary32_matches_numpy_on_doubles():
    rng = np.random.default_rng(7)
    for _ in range(3000):
        mnt = int(rng.integers(1, 1 << 53))
        e = int(rng.integers(-200, 70))
        d = math.ldexp(float(mnt), e)                    # exact double
        want = float(np.float32(d))                      # RN-even double -> single
        assert fp.round_scaled(mnt, e, fp.BINARY32) == want


def test_fma_exactness():
    a = 1 + 2.0 ** -30
    b = 1 - 2.0 ** -30
    assert fp.fma64(a, b, -1.0) == -(2.0 ** -60)         # unfused gives 0
    assert a * b - 1.0 == 0.0
    assert fp.fma64(2.0, 3.0, 4.0) == 10.0
    assert math.copysign(1, fp.fma64(-0.0, 1.0, -0.0)) < 0
    assert math.copysign(1, fp.fma64(1.0, 1.0, -1.0)) > 0


def test_two_product_error_free():
    rng = np.random.default_rng(3)
    a = rng.standard_normal(200) * 1e3
    b = rng.standard_normal(200) * 1e-3
    p, e = _two_product(a, b)
    for ai, bi, pi, ei in zip(a, b, p, e):
        assert Fraction(pi) + Fraction(ei) == Fraction(ai) * Fraction(bi)


def test_limbs_reconstruct():
    rng = np.random.default_rng(1)
    v = np.trunc(rng.standard_normal(100) * 2.0 ** rng.integers(0, 99, 100))
    limbs = _limbs(v)
    for t, x in enumerate(v):
        assert sum(int(l[t]) << (21 * s) for s, l in enumerate(limbs)) == int(x)


# ------------------------------------------------------------- Step III
def test_exponent_E_is_maximal_closed_form():
    for N in (2, 6, 14, 20):
        P = Plan(N).P
        X = (P - 1) << 27
        for S in [0, 1, 1 << 32, (1 << 32) + 1, 12345678901, 1 << 50, (1 << 50) - 3]:
            E = exponent_E(S, P)
            M = max(1 << 32, S)
            assert Fraction(4) ** E * M <= X < Fraction(4) ** (E + 1) * M


def test_exponent_matches_real_formula():
    # E_i = floor(P'_fast - max(1, 0.5 log2 sum t^2)), P'_fast = log2(P-1)/2 - 1.5
    # (eqs. mu-fast/nu-fast with the normalised-row reading); the quantised sum
    # may only lower it, by at most one
    for N, phi in ((14, 0.5), (8, 2.0), (20, 1.0)):
        plan = Plan(N)
        A = paper_matrix(30, 50, phi, 11)
        V = row_vectors(A)
        x, e, S, E, flag = vector_exponents(V, plan.P)
        Pf = math.log2(plan.P - 1) / 2 - 1.5
        for r in range(V.shape[0]):
            t = V[r] * 2.0 ** -e[r]
            L = 0.5 * math.log2(float(np.sum(t * t)))
            Ereal = math.floor(Pf - max(1.0, L))
            assert E[r] in (Ereal, Ereal - 1)
            assert x[r] == E[r] - e[r]


def _cond_holds(em):
    """Condition (cond): 2 sum_h |a'_ih||b'_hj| < P, for both real products of
    the 2x2 block form (Section II), checked exactly."""
    Ar, Ai = em.Ar, em.Ai
    Br, Bi = em.Br, em.Bi
    absA = np.concatenate([np.abs(Ar), np.abs(Ai)], axis=1)
    absB = np.concatenate([np.abs(Br), np.abs(Bi)], axis=0)
    worst = 0
    for i in range(absA.shape[0]):
        row = [int(v) for v in absA[i]]
        for j in range(absB.shape[1]):
            col = [int(v) for v in absB[:, j]]
            worst = max(worst, sum(a * b for a, b in zip(row, col)))
    return 2 * worst < em.plan.P, worst


@pytest.mark.parametrize("phi", [0.0, 1.0, 4.0])
def test_condition_cond_holds(phi):
    A = paper_matrix(12, 40, phi, 21)
    B = paper_matrix(40, 9, phi, 22)
    for N in (4, 10, 16):
        em = emulate(A, B, N)
        ok, worst = _cond_holds(em)
        assert ok
        assert 8 * worst <= em.plan.P - 1                 # the (P-1)/8 margin of the bound


def test_condition_cond_tight_inputs():
    # equal-magnitude entries make Cauchy-Schwarz tight
    k = 64
    A = np.full((3, k), 1.0 + 1.0j)
    B = np.full((k, 3), -1.0 + 1.0j)
    for N in (3, 8, 14):
        em = emulate(A, B, N)
        ok, _ = _cond_holds(em)
        assert ok


def test_row_scale_invariance_bitwise():
    A = paper_matrix(8, 24, 1.0, 31)
    B = paper_matrix(24, 7, 1.0, 32)
    base = emulate(A, B, 12)
    A2 = A.copy()
    A2[3, :] *= 2.0 ** 37
    A2[5, :] *= 2.0 ** -41
    sc = emulate(A2, B, 12)
    assert sc.x[3] == base.x[3] - 37 and sc.x[5] == base.x[5] + 41
    want = base.out.copy()
    want[3, :] *= 2.0 ** 37
    want[5, :] *= 2.0 ** -41
    assert np.array_equal(sc.out, want)


def test_nonfinite_and_zero_rows():
    A = paper_matrix(5, 6, 0.5, 41)
    B = paper_matrix(6, 4, 0.5, 42)
    A[1, 2] = np.inf
    A[3, :] = 0
    B[0, 2] = complex(np.nan, 0)
    em = emulate(A, B, 8)
    assert em.flag_a[1] and em.x[1] == NONFINITE and em.flag_b[2]
    assert np.all(np.isnan(em.out[1, :].real)) and np.all(np.isnan(em.out[:, 2].imag))
    assert np.all(em.out[3, [0, 1, 3]] == 0)


# ------------------------------------------------------------- Steps IV-VI
def test_residues_in_range_and_karatsuba_identity():
    A = paper_matrix(7, 20, 1.0, 51)
    B = paper_matrix(20, 6, 1.0, 52)
    em = emulate(A, B, 10)
    cR, cI = scaled_integer_product(em.Ar, em.Ai, em.Br, em.Bi)
    for l, p in enumerate(em.plan.p):
        lo, hi = -(p // 2), (p - 1) // 2
        assert em.planesA.min() >= -128 and em.planesA.max() <= 127
        assert em.planesA[l].min() >= lo and em.planesA[l].max() <= hi
        for i in range(7):
            for j in range(6):
                # E'_l is the residue of the exact complex integer product (eq. karatsuba)
                assert em.Eprime[l, 0, i, j] == sym_mod(int(cR[i, j]), p)
                assert em.Eprime[l, 1, i, j] == sym_mod(int(cI[i, j]), p)


@pytest.mark.parametrize("N", [2, 5, 14, 20, 24])
def test_crt_equals_exact_product(N):
    A = paper_matrix(9, 33, 1.0, 60 + N)
    B = paper_matrix(33, 8, 1.0, 80 + N)
    em = emulate(A, B, N)
    cR, cI = scaled_integer_product(em.Ar, em.Ai, em.Br, em.Bi)
    assert np.all(em.cR == cR) and np.all(em.cI == cI)


def test_exact_once_enough_moduli():
    # small integers: no truncation happens, the product is an exact integer
    rng = np.random.default_rng(9)
    A = (rng.integers(-100, 101, (11, 17)) + 1j * rng.integers(-100, 101, (11, 17)))
    B = (rng.integers(-100, 101, (17, 13)) + 1j * rng.integers(-100, 101, (17, 13)))
    want = A.astype(np.complex128) @ B.astype(np.complex128)      # exact integers
    for N in (8, 14):
        em = emulate(A.astype(np.complex128), B.astype(np.complex128), N)
        assert np.array_equal(em.out, want)


def test_transpose_symmetry_bitwise():
    A = paper_matrix(6, 15, 1.0, 71)
    B = paper_matrix(15, 5, 1.0, 72)
    e1 = emulate(A, B, 12)
    e2 = emulate(B, A, 12, opA="T", opB="T")
    assert np.array_equal(e1.out.T, e2.out)


def test_conjugate_op():
    As = paper_matrix(15, 6, 1.0, 73)          # stored k x m, used as A^H (m x k)
    Bs = paper_matrix(5, 15, 1.0, 74)          # stored n x k, used as B^T
    want = emulate(As.conj().T, Bs.T, 12).out
    got = emulate(As, Bs, 12, opA="C", opB="T").out
    assert np.array_equal(got, want)
    assert np.array_equal(apply_op(As, "C"), As.conj().T)


def test_unscale_is_single_rounding_of_exact():
    A = paper_matrix(5, 9, 2.0, 81)
    B = paper_matrix(9, 4, 2.0, 82)
    em = emulate(A, B, 14)
    for i in range(5):
        for j in range(4):
            s = -(int(em.x[i]) + int(em.y[j]))
            v = Fraction(int(em.cR[i, j])) * Fraction(2) ** s
            assert em.out[i, j].real == float(v)                  # Fraction->float is RN


def test_alpha_beta_sequence():
    A = paper_matrix(4, 7, 0.5, 91)
    B = paper_matrix(7, 3, 0.5, 92)
    C = paper_matrix(4, 3, 0.5, 93)
    base = emulate(A, B, 14).out
    al, be = (0.75, -1.25), (0.5, 2.0)
    em = emulate(A, B, 14, alpha=al, beta=be, C_in=C)
    z = al[0] * base + 1j * al[1] * base
    want = (al[0] + 1j * al[1]) * base + (be[0] + 1j * be[1]) * C
    assert np.allclose(em.out, want, rtol=1e-14, atol=1e-14)
    assert not np.array_equal(em.out, z)


def test_complex64_output_single_rounding_of_binary64():
    A = paper_matrix(6, 10, 1.0, 95, np.complex64)
    B = paper_matrix(10, 5, 1.0, 96, np.complex64)
    em64 = emulate(A.astype(np.complex128), B.astype(np.complex128), 8)
    em32 = emulate(A.astype(np.complex128), B.astype(np.complex128), 8, out_fmt=fp.BINARY32)
    assert em32.out.dtype == np.complex64
    assert np.array_equal(em32.out, em64.out.astype(np.complex64))


def test_entries_path_matches_full_pipeline():
    A = paper_matrix(12, 40, 1.0, 101)
    B = paper_matrix(40, 10, 1.0, 102)
    em = emulate(A, B, 14)
    rows = np.array([0, 3, 11, 5, 5])
    cols = np.array([0, 9, 2, 5, 6])
    got = emulate_entries(A, B, 14, rows, cols)
    assert np.array_equal(got, em.out[rows, cols])


# ------------------------------------------------------------ accuracy
def test_reference_product_matches_fractions():
    A = paper_matrix(3, 6, 1.5, 111)
    B = paper_matrix(6, 3, 1.5, 112)
    rows, cols = np.meshgrid(range(3), range(3), indexing="ij")
    ref = complex_product_entries(A, B, rows.ravel(), cols.ravel())
    for t, (i, j) in enumerate(zip(rows.ravel(), cols.ravel())):
        re = sum(Fraction(A[i, h].real) * Fraction(B[h, j].real) - Fraction(A[i, h].imag) * Fraction(B[h, j].imag) for h in range(6))
        im = sum(Fraction(A[i, h].real) * Fraction(B[h, j].imag) + Fraction(A[i, h].imag) * Fraction(B[h, j].real) for h in range(6))
        assert ref[t] == complex(float(re), float(im))


def test_error_shrinks_with_moduli_then_saturates():
    # each modulus adds about log2(p_l)/2 bits to every scaled operand
    A = paper_matrix(16, 256, 1.0, 121)
    B = paper_matrix(256, 16, 1.0, 122)
    rows, cols = np.meshgrid(range(16), range(16), indexing="ij")
    rows, cols = rows.ravel(), cols.ravel()
    ref = complex_product_entries(A, B, rows, cols)
    bound = abs_bound_entries(A, B, rows, cols)
    errs = {}
    for N in (6, 8, 10, 12, 14, 16):
        out = emulate(A, B, N, keep_residue_planes=False).out
        errs[N] = max_normalised_error(out[rows, cols], ref, bound)
    for a, b in ((6, 8), (8, 10), (10, 12)):
        assert errs[b] < errs[a] / 64
    assert errs[16] <= 2.0 ** -52                          # at the binary64 rounding floor
    assert errs[14] < 1e-15


def test_truncation_error_bound():
    # |c - AB| <= per-entry bound from |a - a'/mu| < 2^-x and |b - b'/nu| < 2^-y
    A = paper_matrix(8, 64, 2.0, 131)
    B = paper_matrix(64, 8, 2.0, 132)
    em = emulate(A, B, 9)
    rows, cols = np.meshgrid(range(8), range(8), indexing="ij")
    rows, cols = rows.ravel(), cols.ravel()
    ref = complex_product_entries(A, B, rows, cols)
    for t, (i, j) in enumerate(zip(rows, cols)):
        da = 2.0 ** -int(em.x[i])
        db = 2.0 ** -int(em.y[j])
        a = np.abs(A[i].real) + np.abs(A[i].imag)
        b = np.abs(B[:, j].real) + np.abs(B[:, j].imag)
        bnd = float(np.sum(da * b + a * db + 2 * da * db)) * 1.0000001
        out = em.out[i, j]
        tol = bnd + 2.0 ** -52 * abs(out.real)
        assert abs(out.real - ref[t].real) <= tol
        assert abs(out.imag - ref[t].imag) <= bnd + 2.0 ** -52 * abs(out.imag)


def test_metrics_closed_forms():
    assert max_rel_error(np.array([1.0 + 2j]), np.array([1.0 + 2j])) == 0.0
    assert max_rel_error(np.array([1.5 + 2j]), np.array([1.0 + 2j])) == 0.5
    assert max_normalised_error(np.array([1.0 + 1.25j]), np.array([1.0 + 1j]), np.array([0.5])) == 0.5


# ------------------------------------------------------------ the model
def test_performance_model_worked_example():
    with open(os.path.join(GOLDEN, "perf_model_example.txt")) as f:
        line = [l for l in f if l.strip() and not l.startswith("#")][0].split()
    mode, dt = line[0], line[1]
    m, n, k, N, c = map(int, line[2:7])
    blo, bhi, p, want = map(float, line[7:11])
    lo = model_tflops(m, n, k, N, blo, p, c=c, dtype=dt, mode=mode)
    hi = model_tflops(m, n, k, N, bhi, p, c=c, dtype=dt, mode=mode)
    assert lo <= want * 1.05 and hi >= want * 0.95           # "approximately 120 TFLOPS"
    assert abs((lo + hi) / 2 - want) / want < 0.1
