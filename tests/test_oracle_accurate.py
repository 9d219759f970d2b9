"""Pins for the accurate-mode scaling oracle (Section III-B, eqs. mu-accu /
nu-accu): the bound identity, condition (cond) checked exactly, the exponent
rule against a direct evaluation of the paper's formula, invariants, and the
accuracy gain over fast mode.  CPU only."""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle.accurate import PRE_BITS, accurate_exponents, exponent_accu, prescale
from oracle.emulate import Emulation, emulate_entries
from oracle.emulate_real import RealEmulation, emulate_real_entries
from oracle.exact import _exact_matmul, complex_product_entries, real_product_entries
from oracle.moduli import Plan
from oracle.scaling import NONFINITE
from paper_2512_08321_gb300.workloads import paper_matrix, paper_matrix_real


def _floor_formula(M, P):
    """floor(P'_accu - 0.5 log2 max(M, 1)) with P'_accu = log2(P-1)/2 - 0.5, by
    bisection on exact rationals (no floating-point log)."""
    M = max(M, 1)
    # largest E with E <= log2(P-1)/2 - 0.5 - log2(M)/2  <=>  2^(2E+1) M <= P-1
    E = -400
    while 2 ** (2 * (E + 1) + 1) * Fraction(M) <= P - 1 if E + 1 >= 0 else \
            Fraction(2) ** (2 * (E + 1) + 1) * M <= P - 1:
        E += 1
    return E


@pytest.mark.parametrize("N", [2, 6, 14, 24])
def test_exponent_rule_matches_formula(N):
    P = Plan(N).P
    rng = np.random.default_rng(N)
    for M in [0, 1, 2, 3, 4, 5, 63, 64, 65, 4096, 2 ** 20 - 1, 2 ** 20, 2 ** 29 + 7] + list(rng.integers(1, 2 ** 30, 20)):
        assert exponent_accu(int(M), P) == _floor_formula(int(M), P), M


def test_prescale_bounds_and_width():
    V = paper_matrix_real(20, 37, 3.0, 61)
    V[4] = 0.0
    V[7, 3] = np.nan
    V[9] *= 1e-300
    e, flag, Vbar = prescale(V)
    assert flag[7] and not flag[9] and e[4] == 0
    for r in range(20):
        if flag[r] or r == 4:
            assert np.all(Vbar[r] == 0)
            continue
        sc = np.abs(V[r]) * 2.0 ** (PRE_BITS - int(e[r]))
        assert sc.max() >= 32 and sc.max() < 64            # integer part fits in 6 bits
        assert np.all(Vbar[r] >= sc) and np.all(Vbar[r] <= np.ceil(sc) + (sc == 0))   # ceiling, upper bound
        assert Vbar[r].max() <= 64


def test_bound_identity_and_real_reduction():
    A = paper_matrix(9, 40, 2.0, 62)
    B = paper_matrix(40, 7, 2.0, 63)
    acc = accurate_exponents(A, B, Plan(10).P)
    direct = acc["AR"] @ acc["BR"] + acc["AI"] @ acc["BI"]
    assert np.array_equal(acc["CR"], direct)
    assert np.array_equal(acc["CI"], acc["AI"] @ acc["BR"] + acc["AR"] @ acc["BI"])
    # real input: C-bar = A-bar B-bar; equals the complex bound with zero imaginary parts
    Ar, Br = A.real.copy(), B.real.copy()
    r = accurate_exponents(Ar, Br, Plan(10).P, real=True)
    c = accurate_exponents(Ar.astype(np.complex128), Br.astype(np.complex128), Plan(10).P)
    assert np.array_equal(r["x"], c["x"]) and np.array_equal(r["y"], c["y"])


@pytest.mark.parametrize("N,phi", [(4, 0.5), (8, 2.0), (14, 1.0), (20, 4.0)])
def test_condition_holds_exactly(N, phi):
    A = paper_matrix(12, 50, phi, 64)
    B = paper_matrix(50, 10, phi, 65)
    em = Emulation(A, B, N, scaling="accurate")
    P = em.plan.P
    abs_r = _exact_matmul(np.abs(em.Ar), np.abs(em.Br)) + _exact_matmul(np.abs(em.Ai), np.abs(em.Bi))
    abs_i = _exact_matmul(np.abs(em.Ar), np.abs(em.Bi)) + _exact_matmul(np.abs(em.Ai), np.abs(em.Br))
    worst = max(max(int(v) for v in abs_r.ravel()), max(int(v) for v in abs_i.ravel()))
    assert 2 * worst < P                          # condition (cond), Section II
    # and the scale is not wasted: one more bit on every row would break the bound for some entry
    assert 8 * worst > (P - 1) // 8


def test_accurate_result_is_the_exact_crt_and_beats_fast():
    A = paper_matrix(16, 300, 2.0, 66)
    B = paper_matrix(300, 12, 2.0, 67)
    rows, cols = np.meshgrid(np.arange(16), np.arange(12), indexing="ij")
    ref = complex_product_entries(A, B, rows.ravel(), cols.ravel()).reshape(16, 12)
    bound = (np.abs(A.real) + np.abs(A.imag)) @ (np.abs(B.real) + np.abs(B.imag))
    err = {}
    for mode in ("fast", "accurate"):
        em = Emulation(A, B, 10, scaling=mode, keep_residue_planes=False)
        cr = _exact_matmul(em.Ar, em.Br) - _exact_matmul(em.Ai, em.Bi)
        assert all(int(em.cR[i, j]) == int(cr[i, j]) for i in range(16) for j in range(12))
        d = np.maximum(np.abs(em.out.real - ref.real), np.abs(em.out.imag - ref.imag))
        err[mode] = float(np.max(d / bound))
    # the tighter bound keeps more bits at the same N
    assert err["accurate"] < err["fast"] / 2


def test_row_scale_invariance_and_flags():
    A = paper_matrix(6, 30, 1.0, 68)
    B = paper_matrix(30, 5, 1.0, 69)
    A2 = A.copy()
    A2[1] *= 2.0 ** -45
    e1, e2 = Emulation(A, B, 9, scaling="accurate"), Emulation(A2, B, 9, scaling="accurate")
    assert e2.x[1] == e1.x[1] + 45
    assert np.array_equal(e2.out[1], e1.out[1] * 2.0 ** -45)
    A3 = A.copy()
    A3[2, 4] = np.inf
    e3 = Emulation(A3, B, 9, scaling="accurate")
    assert e3.x[2] == NONFINITE and np.all(np.isnan(e3.out[2].real))
    # a flagged row enters the bound product as zeros: other rows keep their scales
    assert np.array_equal(np.delete(e3.x, 2), np.delete(e1.x, 2))


def test_real_accurate_mode():
    A = paper_matrix_real(10, 200, 3.0, 70)
    B = paper_matrix_real(200, 8, 3.0, 71)
    rows, cols = np.meshgrid(np.arange(10), np.arange(8), indexing="ij")
    ref = real_product_entries(A, B, rows.ravel(), cols.ravel()).reshape(10, 8)
    bound = np.abs(A) @ np.abs(B)
    ef = np.max(np.abs(RealEmulation(A, B, 9).out - ref) / bound)
    ea = np.max(np.abs(RealEmulation(A, B, 9, scaling="accurate").out - ref) / bound)
    assert ea < ef / 2
    em = RealEmulation(A, B, 9, scaling="accurate")
    exact = _exact_matmul(em.Ai, em.Bi)
    assert all(int(em.c[i, j]) == int(exact[i, j]) for i in range(10) for j in range(8))


def test_sampled_entries_with_accurate_exponents():
    """The sampled-entry oracle given the accurate mode's x and y (which depend
    on whole rows and columns of the bound product) equals the full accurate
    emulation, through the CRT, at those entries; complex and real."""
    A = paper_matrix(40, 150, 2.0, 72)
    B = paper_matrix(150, 36, 2.0, 73)
    rng = np.random.default_rng(3)
    rows, cols = rng.integers(0, 40, 30), rng.integers(0, 36, 30)
    em = Emulation(A, B, 11, scaling="accurate", keep_residue_planes=False)
    ex = accurate_exponents(A, B, Plan(11).P)
    got = emulate_entries(A, B, 11, rows, cols, xy=(ex["x"], ex["y"]))
    assert np.array_equal(got.view(np.float64), em.out[rows, cols].view(np.float64))
    assert np.array_equal(ex["x"], em.x) and np.array_equal(ex["y"], em.y)
    # without xy the fast-mode exponents apply, and the results differ here
    assert not np.array_equal(emulate_entries(A, B, 11, rows, cols).view(np.float64), got.view(np.float64))
    Ar, Br = A.real.copy(), B.real.copy()
    er = RealEmulation(Ar, Br, 11, scaling="accurate")
    exr = accurate_exponents(Ar, Br, Plan(11).P, real=True)
    gotr = emulate_real_entries(Ar, Br, 11, rows, cols, xy=(exr["x"], exr["y"]))
    assert np.array_equal(gotr, er.out[rows, cols])
