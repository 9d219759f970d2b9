"""Launch-configuration knobs and the autotuner: every knob value is a
different code path of the same computation, so each must give results
bit-identical to the oracle; the autotuner's choices must be valid, used,
and kept in the cache file across processes."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import fp
from oracle.emulate import emulate
from paper_2512_08321_gb300 import emu
from paper_2512_08321_gb300.workloads import paper_matrix

from .helpers import mismatch_report, run_gemm, same_bits

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

KNOBS = [(emu.EMU_TUNE_TILE_N, v) for v in (64, 128, 256)] + \
        [(emu.EMU_TUNE_GROUP, v) for v in (1, 3, 32)] + \
        [(emu.EMU_TUNE_CHUNK_K, v) for v in (64, 512, 960)] + \
        [(emu.EMU_TUNE_CRT_ROWS, v) for v in (1, 2, 4)] + \
        [(emu.EMU_TUNE_SPLIT_ELEMS, v) for v in (2, 4)]


@pytest.fixture(autouse=True)
def _defaults():
    saved = {k: emu.emu_get_tuning(k) for k in range(1, 6)}
    yield
    for k, v in saved.items():
        emu.emu_set_tuning(k, v)
    emu.emu_autotune_clear()


@pytest.mark.parametrize("key,value", KNOBS)
def test_knob_bitexact(key, value):
    m, n, k, N = 301, 170, 1100, 13
    A = paper_matrix(k, m, 1.0, 7)           # op T
    B = paper_matrix(k, n, 1.0, 8)
    ref = emulate(A, B, N, opA="T", keep_residue_planes=False)
    emu.check(emu.emu_set_tuning(key, value), "set tuning")
    got = run_gemm(A, B, N, opA="T")
    assert same_bits(got, ref.out), mismatch_report(got, ref.out)


def test_knob_bitexact_cgemm():
    m, n, k, N = 200, 99, 700, 8
    A = paper_matrix(m, k, 0.5, 9, np.complex64)
    B = paper_matrix(k, n, 0.5, 10, np.complex64)
    ref = emulate(A.astype(np.complex128), B.astype(np.complex128), N, out_fmt=fp.BINARY32,
                  keep_residue_planes=False)
    for key, value in ((emu.EMU_TUNE_CRT_ROWS, 1), (emu.EMU_TUNE_SPLIT_ELEMS, 2), (emu.EMU_TUNE_TILE_N, 128)):
        emu.check(emu.emu_set_tuning(key, value), "set tuning")
        got = run_gemm(A, B, N, single=True)
        assert same_bits(got, ref.out)


def test_invalid_knobs_rejected():
    for key, value in ((emu.EMU_TUNE_TILE_N, 96), (emu.EMU_TUNE_CHUNK_K, 1024), (emu.EMU_TUNE_CRT_ROWS, 3),
                       (emu.EMU_TUNE_SPLIT_ELEMS, 8), (99, 1)):
        assert emu.emu_set_tuning(key, value) == emu.EMU_ERR_INVALID_ARG


def test_autotune_choices_valid_and_used():
    m, n, k, N = 640, 500, 900, 14
    st, best = emu.emu_autotune_gemm(False, m, n, k, N)
    emu.check(st, "autotune")
    assert best[0] in (64, 128, 256) and 1 <= best[1] <= 64 and best[2] % 64 == 0
    assert best[3] in (1, 2, 4) and best[4] in (2, 4)
    A = paper_matrix(m, k, 1.0, 11)
    B = paper_matrix(k, n, 1.0, 12)
    ref = emulate(A, B, N, keep_residue_planes=False)
    got = run_gemm(A, B, N)                  # same shape bucket: the tuned configuration
    assert same_bits(got, ref.out)


def test_autotune_cache_file_round_trip(tmp_path):
    cache = tmp_path / "tune.txt"
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2512_08321_gb300 import emu\n"
            "st, best = emu.emu_autotune_gemm(False, 300, 200, 500, 12)\n"
            "print(st, *best)\n") % ROOT
    env = dict(os.environ, EMU_AUTOTUNE_CACHE=str(cache))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    st, *best = map(int, r.stdout.split())
    assert st == 0
    lines = [l.split() for l in cache.read_text().splitlines() if l.startswith("gemm ")]
    assert len(lines) == 1 and list(map(int, lines[0][6:])) == best
