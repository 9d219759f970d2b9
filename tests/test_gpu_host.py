"""Host-buffer GEMMs (emu_?gemm_host): A, B, C in host memory (pinned and
pageable), results bit-identical to the device-buffer calls, which the
parity tests tie to the oracle."""
import numpy as np
import pytest
import torch

from paper_2512_08321_gb300 import emu
from paper_2512_08321_gb300.workloads import paper_matrix, paper_matrix_real

from .helpers import dev, host, mismatch_report, same_bits

pytestmark = pytest.mark.gpu

KINDS = {"z": (np.complex128, emu.emu_zgemm, emu.emu_zgemm_host),
         "c": (np.complex64, emu.emu_cgemm, emu.emu_cgemm_host),
         "d": (np.float64, emu.emu_dgemm, emu.emu_dgemm_host),
         "s": (np.float32, emu.emu_sgemm, emu.emu_sgemm_host)}


def _mats(kind, m, n, k, opA, opB, seed):
    dt = KINDS[kind][0]
    gen = paper_matrix if kind in "zc" else paper_matrix_real
    A = gen(m, k, 1.0, seed) if opA == "N" else gen(k, m, 1.0, seed)
    B = gen(k, n, 1.0, seed + 1) if opB == "N" else gen(n, k, 1.0, seed + 1)
    C = gen(m, n, 1.0, seed + 2)
    return A.astype(dt), B.astype(dt), C.astype(dt)


def _scal(kind, v):
    return complex(v) if kind in "zc" else float(v)


def _device_ref(kind, A, B, C, m, n, k, opA, opB, alpha, beta, N):
    f = KINDS[kind][1]
    dA, dB, dC = dev(A), dev(B), dev(C)
    emu.check(f(opA, opB, m, n, k, _scal(kind, alpha), dA.data_ptr(), dA.shape[1], dB.data_ptr(), dB.shape[1],
                _scal(kind, beta), dC.data_ptr(), dC.shape[1], N), "device call")
    torch.cuda.synchronize()
    return host(dC, m)


@pytest.mark.parametrize("kind", ["z", "c", "d", "s"])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_buffers_match_device_call(kind, pinned):
    m, n, k, N = 130, 97, 150, 9
    opA, opB = "T", "N"
    A, B, C = _mats(kind, m, n, k, opA, opB, 300)
    alpha, beta = 0.75, -1.5
    ref = _device_ref(kind, A, B, C, m, n, k, opA, opB, alpha, beta, N)
    f = KINDS[kind][2]
    if pinned:
        tA = torch.from_numpy(np.ascontiguousarray(A.T)).pin_memory()
        tB = torch.from_numpy(np.ascontiguousarray(B.T)).pin_memory()
        tC = torch.from_numpy(np.ascontiguousarray(C.T)).pin_memory()
        pa, pb, pc = tA.data_ptr(), tB.data_ptr(), tC.data_ptr()
    else:
        hA, hB, hC = np.asfortranarray(A), np.asfortranarray(B), np.asfortranarray(C.copy())
        pa, pb, pc = hA.ctypes.data, hB.ctypes.data, hC.ctypes.data
    st = f(opA, opB, m, n, k, _scal(kind, alpha), pa, A.shape[0], pb, B.shape[0], _scal(kind, beta), pc, m, N)
    emu.check(st, "host call")
    torch.cuda.synchronize()
    got = tC.numpy().T if pinned else hC
    assert same_bits(np.ascontiguousarray(got), np.ascontiguousarray(ref)), mismatch_report(got, ref)


def test_host_buffers_with_leading_dimensions_and_k0():
    m, n, k, N = 70, 50, 40, 12
    A, B, C = _mats("z", m, n, k, "N", "N", 310)
    ref = _device_ref("z", A, B, C, m, n, k, "N", "N", 1.0, 0.0, N)
    lda, ldb, ldc = m + 5, k + 3, m + 9
    hA = np.zeros((lda, k), np.complex128, order="F"); hA[:m] = A
    hB = np.zeros((ldb, n), np.complex128, order="F"); hB[:k] = B
    hC = np.full((ldc, n), 7.0 + 7.0j, np.complex128, order="F")
    emu.check(emu.emu_zgemm_host("N", "N", m, n, k, 1.0, hA.ctypes.data, lda, hB.ctypes.data, ldb, 0.0,
                                 hC.ctypes.data, ldc, N), "host call")
    torch.cuda.synchronize()
    assert same_bits(np.ascontiguousarray(hC[:m]), np.ascontiguousarray(ref))
    assert np.all(hC[m:] == 7.0 + 7.0j)                     # rows beyond m untouched
    # k = 0 with beta: C = beta C, A and B never read
    emu.check(emu.emu_zgemm_host("N", "N", m, n, 0, 1.0, None, m, None, 1, 2.0, hC.ctypes.data, ldc, N), "k=0")
    torch.cuda.synchronize()
    assert np.array_equal(hC[:m], 2.0 * ref)


def test_host_argument_errors():
    assert emu.emu_zgemm_host("N", "N", 4, 4, 4, 1.0, None, 4, None, 4, 0.0, None, 4, 12) == emu.EMU_ERR_INVALID_ARG
    assert emu.emu_zgemm_host("N", "N", 4, 4, 4, 1.0, 1, 2, 1, 4, 0.0, 1, 4, 12) == emu.EMU_ERR_INVALID_ARG


@pytest.mark.parametrize("kind", ["z", "d"])
def test_host_buffers_accurate_mode_and_blocking(kind):
    # accurate-mode scaling and column blocking run A's phases before B arrives
    m, n, k, N = 150, 3 * 128 + 20, 120, 11
    A, B, C = _mats(kind, m, n, k, "N", "N", 320)
    try:
        emu.check(emu.emu_set_scaling(emu.EMU_SCALING_ACCURATE), "scaling")
        emu.check(emu.emu_set_tuning(emu.EMU_TUNE_NBLOCK, 128), "nblock")
        ref = _device_ref(kind, A, B, C, m, n, k, "N", "N", 1.0, 0.0, N)
        f = KINDS[kind][2]
        tA = torch.from_numpy(np.ascontiguousarray(A.T)).pin_memory()
        tB = torch.from_numpy(np.ascontiguousarray(B.T)).pin_memory()
        tC = torch.zeros((n, m), dtype=tA.dtype).pin_memory()
        emu.check(f("N", "N", m, n, k, _scal(kind, 1.0), tA.data_ptr(), m, tB.data_ptr(), k, _scal(kind, 0.0),
                    tC.data_ptr(), m, N), "host call")
        torch.cuda.synchronize()
    finally:
        emu.emu_set_scaling(emu.EMU_SCALING_FAST)
        emu.emu_set_tuning(emu.EMU_TUNE_NBLOCK, 0)
    got = tC.numpy().T
    assert same_bits(np.ascontiguousarray(got), np.ascontiguousarray(ref)), mismatch_report(got, ref)


def _stored(X, ld, pinned, fill=0):
    """X (rows x cols) stored column-major with leading dimension ld in host
    memory: a pinned tensor of shape (cols, ld) or a Fortran numpy array."""
    rows, cols = X.shape
    buf = np.full((cols, ld), fill, dtype=X.dtype)
    buf[:, :rows] = X.T
    if pinned:
        t = torch.from_numpy(buf).pin_memory()
        return t, t.data_ptr(), (lambda: t.numpy().T)
    f = np.asfortranarray(buf.T)
    return f, f.ctypes.data, (lambda: f)


@pytest.mark.parametrize("kind,opB,pinned,nblock", [("c", "C", True, 0), ("z", "N", False, 0),
                                                     ("d", "T", True, 768), ("s", "N", True, 384)])
def test_host_column_blocks(kind, opB, pinned, nblock):
    # n above 2048: B and C travel in column blocks on the side stream while
    # earlier blocks compute (nblock narrower than the copy blocks in two cases);
    # padded leading dimensions make the copies strided
    m, n, k, N = 40, 3 * 1024 + 77, 64, 8
    A, B, C = _mats(kind, m, n, k, "N", opB, 330)
    alpha, beta = 1.25, -0.5
    try:
        emu.check(emu.emu_set_tuning(emu.EMU_TUNE_NBLOCK, nblock), "nblock")
        ref = _device_ref(kind, A, B, C, m, n, k, "N", opB, alpha, beta, N)
        lda, ldb, ldc = m + 1, B.shape[0] + 5, m + 3
        hA, pa, _ = _stored(A, lda, pinned)
        hB, pb, _ = _stored(B, ldb, pinned)
        hC, pc, view = _stored(C, ldc, pinned, fill=7)
        f = KINDS[kind][2]
        emu.check(f("N", opB, m, n, k, _scal(kind, alpha), pa, lda, pb, ldb, _scal(kind, beta), pc, ldc, N),
                  "host call")
        torch.cuda.synchronize()
    finally:
        emu.emu_set_tuning(emu.EMU_TUNE_NBLOCK, 0)
    got = view()
    assert same_bits(np.ascontiguousarray(got[:m]), np.ascontiguousarray(ref)), mismatch_report(got[:m], ref)
    assert np.all(got[m:] == 7)                             # padding rows untouched


def test_host_calls_on_two_streams():
    # two host-buffer calls issued back to back on different streams share the
    # staging buffers: the second waits for the first
    m, n, k, N = 64, 2600, 48, 10
    probs = [_mats("z", m, n, k, "N", "N", 340 + 10 * t) for t in range(2)]
    refs = [_device_ref("z", A, B, C, m, n, k, "N", "N", 1.0, 0.0, N) for A, B, C in probs]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = []
    for (A, B, _), s in zip(probs, streams):
        hA, pa, _ = _stored(A, m, True)
        hB, pb, _ = _stored(B, k, True)
        hC, pc, view = _stored(np.zeros((m, n), np.complex128), m, True)
        outs.append((hA, hB, hC, view))
        emu.check(emu.emu_zgemm_host("N", "N", m, n, k, 1.0, pa, m, pb, k, 0.0, pc, m, N, stream=s), "host call")
    torch.cuda.synchronize()
    for (_, _, _, view), ref in zip(outs, refs):
        assert same_bits(np.ascontiguousarray(view()), np.ascontiguousarray(ref))


def test_host_trace_records_the_pipeline():
    # two blocks of rows of A; three column blocks: a first block of half the
    # width (1024), then [1024, 3072) and the ragged [3072, 3149)
    m, n, k, N = 2304, 2048 + 1101, 32, 6
    A, B, _ = _mats("z", m, n, k, "N", "N", 350)
    hA, pa, _ = _stored(A, m, True)
    hB, pb, _ = _stored(B, k, True)
    hC, pc, view = _stored(np.zeros((m, n), np.complex128), m, True)
    ref = _device_ref("z", A, B, np.zeros((m, n), np.complex128), m, n, k, "N", "N", 1.0, 0.0, N)
    emu.check(emu.emu_host_trace_enable(1), "trace on")
    try:
        emu.check(emu.emu_zgemm_host("N", "N", m, n, k, 1.0, pa, m, pb, k, 0.0, pc, m, N), "host call")
        torch.cuda.synchronize()
        tr = emu.emu_host_trace_read()
    finally:
        emu.emu_host_trace_enable(0)
    assert same_bits(np.ascontiguousarray(view()), np.ascontiguousarray(ref))
    names = [t[0] for t in tr]
    ms = {}
    for nm, t in tr:
        ms.setdefault(nm, []).append(t)
    # side stream: the first column block, A's two blocks of rows, the other column blocks
    side_in = [nm for nm in names if nm in ("a_in", "b_in")]
    assert side_in == ["b_in", "a_in", "a_in", "b_in", "b_in"]
    assert names[0] == "start" and names[-1] == "end"
    # pinned C (beta = 0): the blocks before the last two go through the device copy and back by
    # DMA, the last two blocks' CRTs write host memory in place
    assert [len(ms.get(nm, [])) for nm in ("block_start", "block_crt", "c_out")] == [3, 3, 1]
    assert ms["start"] == [0.0] and min(t for _, t in tr) >= 0.0
    assert ms["end"][0] >= max(t for _, t in tr)             # the call ends after every step
    assert ms["block_crt"][0] >= ms["a_in"][-1]               # the first block used all of A
    for b in range(3):
        s, c = ms["block_start"][b], ms["block_crt"][b]
        assert s <= c                                        # block start, its CRT
        assert s >= ms["b_in"][b]                            # after its columns of B arrived
    assert ms["c_out"][0] >= ms["block_crt"][0]               # copied back after its CRT


@pytest.mark.parametrize("kind,opA,scaling", [("z", "N", "fast"), ("s", "T", "fast"), ("c", "C", "fast"),
                                              ("d", "N", "accurate")])
def test_host_row_blocks_of_a(kind, opA, scaling):
    # m above 2048: A arrives in blocks of rows and the first column block is
    # computed row block by row block (fast mode); padded leading dimensions,
    # a ragged last block of rows, beta != 0
    m, n, k, N = 2100, 2100, 48, 9
    A, B, C = _mats(kind, m, n, k, opA, "N", 360)
    alpha, beta = 0.5, 2.0
    try:
        if scaling == "accurate":
            emu.check(emu.emu_set_scaling(emu.EMU_SCALING_ACCURATE), "scaling")
        ref = _device_ref(kind, A, B, C, m, n, k, opA, "N", alpha, beta, N)
        lda, ldb, ldc = A.shape[0] + 3, k + 1, m + 5
        hA, pa, _ = _stored(A, lda, True)
        hB, pb, _ = _stored(B, ldb, True)
        hC, pc, view = _stored(C, ldc, True, fill=3)
        f = KINDS[kind][2]
        emu.check(f(opA, "N", m, n, k, _scal(kind, alpha), pa, lda, pb, ldb, _scal(kind, beta), pc, ldc, N),
                  "host call")
        torch.cuda.synchronize()
    finally:
        emu.emu_set_scaling(emu.EMU_SCALING_FAST)
    got = view()
    assert same_bits(np.ascontiguousarray(got[:m]), np.ascontiguousarray(ref)), mismatch_report(got[:m], ref)
    assert np.all(got[m:] == 3)
