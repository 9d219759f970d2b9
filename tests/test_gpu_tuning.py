"""Launch-configuration knobs and the autotuner: every knob value is a
different code path of the same computation, so each must give results
bit-identical to the oracle; the autotuner's choices must be valid, used,
and kept in the cache file across processes."""
import functools
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
    saved = {k: emu.emu_get_tuning(k) for k in list(range(1, 6)) + list(range(8, 14))}
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
    lines = [l.split() for l in cache.read_text().splitlines() if l.startswith("gemm3 ")]
    assert len(lines) == 1 and list(map(int, lines[0][6:11])) == best
    assert len(lines[0]) == 17


# modulus-loop schedules of the residue products: (order, pairing, kdir, band columns, chunk_k)
SCHEDULES = [(0, 0, 0, 8192, 960), (1, 0, 0, 8192, 960), (2, 0, 0, 128, 960), (2, 1, 1, 256, 64),
             (0, 2, 1, 8192, 960), (1, 1, 1, 8192, 64), (0, 1, 0, 8192, 512), (2, 2, 1, 384, 960)]


def _set_schedule(order, pairing, kdir, band, chunk):
    for key, v in ((emu.EMU_TUNE_ORDER, order), (emu.EMU_TUNE_PAIRING, pairing), (emu.EMU_TUNE_KDIR, kdir),
                   (emu.EMU_TUNE_BAND, band), (emu.EMU_TUNE_CHUNK_K, chunk)):
        emu.check(emu.emu_set_tuning(key, v), "set tuning")


@functools.lru_cache(maxsize=1)
def _schedule_case():
    m, n, k, N = 600, 520, 1100, 13
    A = paper_matrix(m, k, 1.0, 41)
    B = paper_matrix(n, k, 1.0, 42)          # op T
    return A, B, N, emulate(A, B, N, opB="T", keep_residue_planes=False).out


@pytest.mark.parametrize("order,pairing,kdir,band,chunk", SCHEDULES)
def test_schedule_bitexact(order, pairing, kdir, band, chunk):
    """Every schedule is the same computation: more units than blocks (so the
    alternating k direction is taken), ragged tiles, several column bands and
    an odd job count (N = 13: 39 jobs, the last pair single)."""
    A, B, N, ref = _schedule_case()
    _set_schedule(order, pairing, kdir, band, chunk)
    got = run_gemm(A, B, N, opB="T")
    assert same_bits(got, ref), mismatch_report(got, ref)


@pytest.mark.parametrize("order,pairing,kdir", [(1, 2, 1), (2, 1, 0)])
def test_schedule_bitexact_real_and_single(order, pairing, kdir):
    from oracle.emulate_real import emulate_real
    from paper_2512_08321_gb300.workloads import paper_matrix_real
    from .helpers import run_real
    _set_schedule(order, pairing, kdir, 128, 960)
    emu.check(emu.emu_set_tuning(emu.EMU_TUNE_TILE_N, 64), "tile")     # 24 tiles: more units than blocks
    m, n, k, N = 330, 400, 1000, 15
    A = paper_matrix_real(m, k, 1.0, 43)
    B = paper_matrix_real(k, n, 1.0, 44)
    ref = emulate_real(A, B, N)
    got = run_real(A, B, N)
    assert same_bits(got, ref.out), mismatch_report(got, ref.out)
    Ac = paper_matrix(m, k, 0.5, 45, np.complex64)
    Bc = paper_matrix(k, n, 0.5, 46, np.complex64)
    refc = emulate(Ac.astype(np.complex128), Bc.astype(np.complex128), 8, out_fmt=fp.BINARY32,
                   keep_residue_planes=False)
    assert same_bits(run_gemm(Ac, Bc, 8, single=True), refc.out)


def test_invalid_schedule_knobs_rejected():
    for key, value in ((emu.EMU_TUNE_ORDER, 3), (emu.EMU_TUNE_PAIRING, -1), (emu.EMU_TUNE_KDIR, 2),
                       (emu.EMU_TUNE_BAND, 100), (emu.EMU_TUNE_BAND, 0), (emu.EMU_TUNE_CTA_PAIR, 2),
                       (emu.EMU_TUNE_CTA_PAIR, -1)):
        assert emu.emu_set_tuning(key, value) == emu.EMU_ERR_INVALID_ARG


def test_autotuned_schedule_valid_reported_and_used():
    m, n, k, N = 1500, 2600, 700, 14
    st, best = emu.emu_autotune_gemm(False, m, n, k, N)
    emu.check(st, "autotune")
    got_sched = {nm: emu.emu_tuned_value(emu.EMU_DTYPE_Z, N, m, n, k, key)
                 for nm, key in emu.SCHEDULE_KNOBS.items()}
    assert got_sched["order"] in (0, 1, 2) and got_sched["pairing"] in (0, 1, 2) and got_sched["kdir"] in (0, 1)
    assert got_sched["band"] % 128 == 0 and got_sched["cta_pair"] in (0, 1)
    assert emu.emu_tuned_value(emu.EMU_DTYPE_Z, N, m, n, k, emu.EMU_TUNE_TILE_N) == best[0]
    assert emu.emu_tuned_value(emu.EMU_DTYPE_Z, N, m, n, k, 99) == -1
    A = paper_matrix(m, k, 1.0, 47)
    B = paper_matrix(k, n, 1.0, 48)
    rows, cols = np.arange(0, m, 97), np.arange(0, n, 131)
    from oracle.emulate import emulate_entries
    got = run_gemm(A, B, N)
    want = emulate_entries(A, B, N, np.repeat(rows, len(cols)), np.tile(cols, len(rows)))
    assert same_bits(got[np.repeat(rows, len(cols)), np.tile(cols, len(rows))], want)


def test_autotune_cache_skips_invalid_entries(tmp_path):
    """A cache line whose values the launchers would refuse is ignored: the GEMM
    of that bucket runs with the defaults and succeeds."""
    cache = tmp_path / "tune.txt"
    # dtype 0 (Z), N 12, buckets of m = 300, n = 200, k = 500 -> 9, 8, 9; chunk_k 1000 is invalid
    cache.write_text("gemm3 0 12 9 8 9 256 16 1000 4 4 0 0 0 8192 1 0\n"
                     "gemm2 0 12 9 8 9 256 16 960 4 4 0 0 0 8192 1\n")
    code = ("import sys; sys.path.insert(0, %r)\n"
            "import numpy as np, torch\n"
            "from paper_2512_08321_gb300 import emu\n"
            "from paper_2512_08321_gb300.workloads import paper_matrix\n"
            "from oracle.emulate import emulate\n"
            "from tests.helpers import run_gemm, same_bits\n"
            "A = paper_matrix(300, 500, 1.0, 1); B = paper_matrix(500, 200, 1.0, 2)\n"
            "got = run_gemm(A, B, 12)\n"
            "print(int(same_bits(got, emulate(A, B, 12, keep_residue_planes=False).out)),\n"
            "      emu.emu_tuned_value(0, 12, 300, 200, 500, emu.EMU_TUNE_CHUNK_K))\n") % ROOT
    env = dict(os.environ, EMU_AUTOTUNE_CACHE=str(cache))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    same, chunk = map(int, r.stdout.split())
    assert same == 1 and chunk == 960
    assert "ignoring invalid autotune cache entry" in r.stderr


# SM-pair tiles (256 x 256 on a cluster of two CTAs): the schedules above, then
# shapes whose second CTA of a pair holds only padding (m or n <= 128)
PAIR_SCHEDULES = [(0, 0, 0, 8192, 960), (1, 1, 1, 8192, 64), (2, 2, 1, 384, 960), (0, 2, 0, 8192, 512)]


@pytest.mark.parametrize("order,pairing,kdir,band,chunk", PAIR_SCHEDULES)
def test_pair_schedule_bitexact(order, pairing, kdir, band, chunk):
    A, B, N, ref = _schedule_case()
    _set_schedule(order, pairing, kdir, band, chunk)
    emu.check(emu.emu_set_tuning(emu.EMU_TUNE_CTA_PAIR, 1), "cta pair")
    got = run_gemm(A, B, N, opB="T")
    assert same_bits(got, ref), mismatch_report(got, ref)


@pytest.mark.parametrize("m,n,k", [(100, 300, 200), (300, 90, 130), (257, 129, 64), (1, 1, 1)])
def test_pair_edges_bitexact(m, n, k):
    N = 14
    A = paper_matrix(m, k, 1.0, 50 + m)
    B = paper_matrix(k, n, 1.0, 51 + n)
    ref = emulate(A, B, N, keep_residue_planes=False)
    emu.check(emu.emu_set_tuning(emu.EMU_TUNE_CTA_PAIR, 1), "cta pair")
    got = run_gemm(A, B, N)
    assert same_bits(got, ref.out), mismatch_report(got, ref.out)


def test_pair_real_and_single_bitexact():
    from oracle.emulate_real import emulate_real
    from paper_2512_08321_gb300.workloads import paper_matrix_real
    from .helpers import run_real
    emu.check(emu.emu_set_tuning(emu.EMU_TUNE_CTA_PAIR, 1), "cta pair")
    m, n, k, N = 530, 610, 1000, 15
    A = paper_matrix_real(m, k, 1.0, 53)
    B = paper_matrix_real(k, n, 1.0, 54)
    ref = emulate_real(A, B, N)
    got = run_real(A, B, N)
    assert same_bits(got, ref.out), mismatch_report(got, ref.out)
    Ac = paper_matrix(m, k, 0.5, 55, np.complex64)
    Bc = paper_matrix(k, n, 0.5, 56, np.complex64)
    refc = emulate(Ac.astype(np.complex128), Bc.astype(np.complex128), 8, out_fmt=fp.BINARY32,
                   keep_residue_planes=False)
    assert same_bits(run_gemm(Ac, Bc, 8, single=True), refc.out)
    assert emu.emu_stream_status() == emu.EMU_OK
