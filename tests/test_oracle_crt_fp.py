"""Pins for the paper's floating-point CRT (oracle.crt_fp): the common-grid
split makes S1 exact, the reconstruction equals the exact CRT while P < 2^53,
and stays within its rounding bound beyond."""
import math
import random

import numpy as np
import pytest

from oracle import crt_fp
from oracle.emulate import emulate, sym_mod
from oracle.moduli import Plan
from paper_2512_08321_gb300.workloads import paper_matrix


@pytest.mark.parametrize("N", [4, 9, 14, 20, 24])
def test_split_grid_and_exact_S1(N):
    plan = Plan(N)
    s1, s2, g = crt_fp.split_weights(plan)
    for w, a, b in zip(plan.w, s1, s2):
        ia = int(a)
        assert ia == a and ia % (1 << max(g, 0)) == 0 and ia <= w < ia + (1 << max(g, 0))
        assert abs((w - ia) - b) <= math.ulp(b) / 2
    rnd = random.Random(N)
    for _ in range(200):
        E = [rnd.randint(-(p // 2), (p - 1) // 2) for p in plan.p]
        S1 = 0.0
        for a, e in zip(s1, E):
            S1 = S1 + a * float(e)
        assert int(S1) == sum(int(a) * e for a, e in zip(s1, E))     # no rounding anywhere


def _exact_cprime(E, plan):
    return sym_mod(sum(w * e for w, e in zip(plan.w, E)), plan.P)


@pytest.mark.parametrize("N", [3, 5, 6])
def test_small_P_is_exact(N):
    # the split form is exact while P < 2^53; the double-only (complex64) form
    # only while every product and sum, up to N 2^7 P, stays below 2^53
    plan = Plan(N)
    rnd = random.Random(100 + N)
    for _ in range(300):
        c = rnd.randint(-(plan.P // 8), plan.P // 8)
        E = [sym_mod(c, p) for p in plan.p]
        assert crt_fp.reconstruct_z(E, plan) == float(c)
        got = crt_fp.reconstruct_c(E, plan)
        if N * 128 * plan.P < 2 ** 53:
            assert got == float(c)
        else:
            assert abs(got - c) <= N * 2 * math.ulp(128.0 * plan.P)


@pytest.mark.parametrize("N", [12, 16, 20])
def test_rounding_bound(N):
    plan = Plan(N)
    s1, s2, g = crt_fp.split_weights(plan)
    rnd = random.Random(200 + N)
    ulp_s2 = max(math.ulp(b) for b in s2)
    for _ in range(300):
        c = rnd.randint(-(plan.P // 8), plan.P // 8)
        E = [sym_mod(c, p) for p in plan.p]
        got = crt_fp.reconstruct_z(E, plan)
        bound = N * 128 * ulp_s2 + 4 * math.ulp(abs(float(c)) + 1.0) + 2 * N * math.ulp(float(plan.P)) * 2 ** -52
        assert abs(got - c) <= bound


def test_paper_crt_accuracy_limit():
    # the exact CRT reaches RN(exact); the paper's FP reconstruction is limited by its arithmetic
    A = paper_matrix(6, 64, 1.0, 5)
    B = paper_matrix(64, 5, 1.0, 6)
    em = emulate(A, B, 20)
    fp_out = crt_fp.outputs(em)
    assert np.max(np.abs(fp_out - em.out) / np.abs(em.out)) < 1e-12
