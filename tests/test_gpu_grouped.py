"""Grouped emulated GEMM (one persistent launch per phase over all problems,
replayed from a CUDA graph): every problem bit-exact against the oracle, for
each tile width of the residue-product launch and for the autotuned plan."""
import numpy as np
import pytest
import torch

from oracle import fp
from oracle.emulate import emulate
from paper_2512_08321_gb300 import emu
from paper_2512_08321_gb300.workloads import log_uniform_shapes, paper_matrix

from .helpers import dev, host, mismatch_report, same_bits

pytestmark = pytest.mark.gpu


def _problems(count, lo, hi, seed, single, with_ab=True):
    shapes = log_uniform_shapes(count, lo, hi, seed)
    rng = np.random.default_rng(seed)
    dt = np.complex64 if single else np.complex128
    probs = []
    for i, (m, n, k) in enumerate(shapes):
        m, n, k = int(m), int(n), int(k)
        if i == 3:
            k = 0                              # empty inner dimension
        if i == 5:
            m = 0                              # empty output: skipped
        ta = "NTC"[i % 3]
        tb = "NCT"[(i // 3) % 3]
        A = paper_matrix(m, k, 1.0, seed * 1000 + 2 * i) if ta == "N" else paper_matrix(k, m, 1.0, seed * 1000 + 2 * i)
        B = paper_matrix(k, n, 1.0, seed * 1000 + 2 * i + 1) if tb == "N" else paper_matrix(n, k, 1.0, seed * 1000 + 2 * i + 1)
        C = paper_matrix(m, n, 1.0, seed * 1000 + 999 + i)
        al = complex(rng.uniform(-2, 2), rng.uniform(-2, 2)) if (with_ab and i % 4 == 1) else 1.0
        be = complex(rng.uniform(-2, 2), rng.uniform(-2, 2)) if (with_ab and i % 4 == 2) else 0.0
        probs.append(dict(transa=ta, transb=tb, m=m, n=n, k=k, A=A.astype(dt), B=B.astype(dt),
                          C=C.astype(dt), alpha=al, beta=be))
    return probs


def _device(probs):
    out = []
    for p in probs:
        dA, dB, dC = dev(p["A"]), dev(p["B"]), dev(p["C"])
        out.append(dict(p, dA=dA, dB=dB, dC=dC, lda=dA.shape[1], ldb=dB.shape[1], ldc=dC.shape[1]))
    return out


def _args(dprobs, N):
    return emu.GroupedArgs([dict(transa=p["transa"], transb=p["transb"], m=p["m"], n=p["n"], k=p["k"],
                                 alpha=p["alpha"], beta=p["beta"], A=p["dA"].data_ptr(), lda=p["lda"],
                                 B=p["dB"].data_ptr(), ldb=p["ldb"], C=p["dC"].data_ptr(), ldc=p["ldc"])
                            for p in dprobs], N)


def _oracle(p, N, single):
    ab = dict(alpha=(complex(p["alpha"]).real, complex(p["alpha"]).imag),
              beta=(complex(p["beta"]).real, complex(p["beta"]).imag))
    return emulate(p["A"].astype(np.complex128), p["B"].astype(np.complex128), N, opA=p["transa"],
                   opB=p["transb"], C_in=p["C"].astype(np.complex128), keep_residue_planes=False,
                   out_fmt=fp.BINARY32 if single else fp.BINARY64, **ab).out


@pytest.mark.parametrize("tile", [64, 128, 256, -1, 0])
def test_grouped_bitexact(tile):
    N, single = 14, False
    probs = _problems(14, 1, 200, 11, single)
    dprobs = _device(probs)
    args = _args(dprobs, N)
    st, plan = emu.emu_grouped_create(single, args, tile)
    emu.check(st, "emu_grouped_create")
    try:
        assert emu.emu_grouped_tile(plan) in (64, 128, 256, emu.EMU_GROUPED_TILE_PER_PROBLEM)
        if tile:
            assert emu.emu_grouped_tile(plan) == tile
        assert emu.emu_grouped_kernels(plan) >= 6
        emu.check(emu.emu_grouped_run(plan), "emu_grouped_run")
        torch.cuda.synchronize()
        assert emu.emu_stream_status() == emu.EMU_OK
        for i, p in enumerate(dprobs):
            if p["m"] == 0 or p["n"] == 0:
                continue
            got = host(p["dC"], p["m"])
            want = _oracle(p, N, single)
            assert same_bits(got, want), (i, p["m"], p["n"], p["k"], mismatch_report(got, want))
    finally:
        emu.emu_grouped_destroy(plan)


def test_grouped_replay_and_cgemm():
    N, single = 8, True
    probs = _problems(10, 8, 260, 23, single, with_ab=False)
    dprobs = _device(probs)
    args = _args(dprobs, N)
    st, plan = emu.emu_grouped_create(single, args, 0)
    emu.check(st, "create")
    try:
        for _ in range(3):                     # beta = 0: every replay gives the same result
            emu.check(emu.emu_grouped_run(plan), "run")
        torch.cuda.synchronize()
        for p in dprobs:
            if p["m"] == 0 or p["n"] == 0:
                continue
            got = host(p["dC"], p["m"])
            assert same_bits(got, _oracle(p, N, single))
    finally:
        emu.emu_grouped_destroy(plan)


def test_grouped_matches_single_calls_and_one_shot():
    N = 16
    probs = _problems(9, 30, 300, 31, False)
    d1 = _device(probs)
    d2 = _device(probs)
    emu.check(emu.emu_zgemm_grouped(_args(d1, N)), "emu_zgemm_grouped")
    for p in d2:
        if p["m"] == 0 or p["n"] == 0:
            continue
        emu.gemm(p["dA"], p["dB"], p["dC"], p["m"], p["n"], p["k"], N, p["transa"], p["transb"], p["alpha"],
                 p["beta"], lda=p["lda"], ldb=p["ldb"], ldc=p["ldc"])
    torch.cuda.synchronize()
    for a, b in zip(d1, d2):
        assert torch.equal(torch.view_as_real(a["dC"]), torch.view_as_real(b["dC"]))


def test_grouped_argument_errors():
    probs = _problems(3, 4, 20, 41, False)
    d = _device(probs)
    args = _args(d, 14)
    args.lda[0] = 0
    st, plan = emu.emu_grouped_create(False, args, 0)
    assert st == emu.EMU_ERR_INVALID_ARG and not plan.value
    args = _args(d, 30)
    assert emu.emu_grouped_create(False, args, 0)[0] == emu.EMU_ERR_MODULI_RANGE
    args = _args(d, 14)
    assert emu.emu_grouped_create(False, args, 96)[0] == emu.EMU_ERR_INVALID_ARG


@pytest.mark.parametrize("engine,N,single", [(0, 14, False), (1, 14, False), (1, 20, False), (1, 8, True),
                                             (0, 8, True)])
def test_grouped_crt_engines(engine, N, single):
    """The grouped CRT phase on the tensor cores (128-row items, every limb
    layout) and on the CUDA cores: each problem bit-exact against the oracle."""
    saved = emu.emu_get_tuning(emu.EMU_TUNE_CRT_ENGINE)
    emu.check(emu.emu_set_tuning(emu.EMU_TUNE_CRT_ENGINE, engine), "crt engine")
    try:
        probs = _problems(12, 1, 300, 17 + N, single)
        dprobs = _device(probs)
        st, plan = emu.emu_grouped_create(single, _args(dprobs, N), 128)
        emu.check(st, "emu_grouped_create")
        try:
            emu.check(emu.emu_grouped_run(plan), "emu_grouped_run")
            torch.cuda.synchronize()
            assert emu.emu_stream_status() == emu.EMU_OK
            for i, p in enumerate(dprobs):
                if p["m"] == 0 or p["n"] == 0:
                    continue
                got = host(p["dC"], p["m"])
                want = _oracle(p, N, single)
                assert same_bits(got, want), (i, p["m"], p["n"], p["k"], mismatch_report(got, want))
        finally:
            emu.emu_grouped_destroy(plan)
    finally:
        emu.emu_set_tuning(emu.EMU_TUNE_CRT_ENGINE, saved)
