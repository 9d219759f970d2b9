"""The allocation-free exponent entry point.

Callers that cannot let the library allocate device memory (their memory is
owned by their own pool, or they cannot accept the device-wide
synchronisation of cudaMalloc/cudaFree) use emu_stage_exponents_static, whose
scratch is a fixed array inside the library.  Its results must equal those of
emu_stage_exponents, on consecutive calls that reuse the same array.  This
file is collected last so a failure here stops a -x run only after every
other test has run."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2512_08321_gb300 import emu
from paper_2512_08321_gb300.workloads import paper_matrix

from .helpers import dev

pytestmark = pytest.mark.gpu


def _exponents(fn, A, B, N, opA="N", opB="N", single=False):
    m = A.shape[0] if opA == "N" else A.shape[1]
    k = A.shape[1] if opA == "N" else A.shape[0]
    n = B.shape[1] if opB == "N" else B.shape[0]
    dt = np.complex64 if single else np.complex128
    dA, dB = dev(A.astype(dt)), dev(B.astype(dt))
    x = torch.full((m,), 1234, dtype=torch.int16, device="cuda")
    y = torch.full((n,), 1234, dtype=torch.int16, device="cuda")
    st = fn(single, opA, opB, m, n, k, dA.data_ptr(), dA.shape[1], dB.data_ptr(), dB.shape[1], N,
            x.data_ptr(), y.data_ptr())
    emu.check(st, fn.__name__)
    torch.cuda.synchronize()
    return x.cpu().numpy(), y.cpu().numpy()


def test_static_matches_allocating_on_consecutive_calls():
    # first call: wide dynamic range and many rows; second call: small values,
    # fewer rows -- leftover scratch from the first call must not leak into it
    cases = [
        (paper_matrix(3000, 700, 4.0, 1), paper_matrix(700, 2500, 4.0, 2), 16, "N", "N", False),
        (paper_matrix(500, 300, 0.0, 3) * 1e-30, paper_matrix(200, 300, 0.5, 4), 8, "N", "T", True),
        (paper_matrix(300, 900, 1.0, 5), paper_matrix(900, 77, 1.0, 6), 14, "C", "N", False),
    ]
    for A, B, N, opA, opB, single in cases:
        if opA != "N":
            A = A.T.copy()
        xs, ys = _exponents(emu.emu_stage_exponents_static, A, B, N, opA, opB, single)
        xa, ya = _exponents(emu.emu_stage_exponents, A, B, N, opA, opB, single)
        assert np.array_equal(xs, xa) and np.array_equal(ys, ya)
    assert emu.emu_stream_status() == emu.EMU_OK


def test_static_rejects_sizes_beyond_its_array():
    big = emu.EMU_STATIC_EXP_MAX_ROWS + 1
    st = emu.emu_stage_exponents_static(0, "N", "N", big, 4, 4, 0, big, 0, 4, 14, 0, 0)
    assert st == emu.EMU_ERR_SIZE_LIMIT
    st = emu.emu_stage_exponents_static(0, "N", "N", 4, big, 4, 0, 4, 0, 4, 14, 0, 0)
    assert st == emu.EMU_ERR_SIZE_LIMIT


def _cudart():
    """The CUDA runtime already loaded into this process (by the library or torch)."""
    for name in ("libcudart.so.13", "libcudart.so.12", "libcudart.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    pytest.skip("no CUDA runtime library found by name")


_USED_MEM_CURRENT, _USED_MEM_HIGH = 7, 8      # cudaMemPoolAttrUsedMemCurrent / cudaMemPoolAttrUsedMemHigh


def _pool_attr(rt, pool, attr):
    v = ctypes.c_uint64(0)
    assert rt.cudaMemPoolGetAttribute(pool, attr, ctypes.byref(v)) == 0
    return v.value


def test_static_allocates_nothing():
    """Across a warmed-up static call neither the device's free memory nor the
    stream-ordered pool's high-water mark moves: no cudaMalloc and no
    cudaMallocAsync happened (the allocating entry point uses the latter)."""
    rt = _cudart()
    A = paper_matrix(4000, 600, 2.0, 11)
    B = paper_matrix(600, 3000, 2.0, 12)
    dA, dB = dev(A), dev(B)
    m, k = A.shape
    n = B.shape[1]
    x = torch.empty(m, dtype=torch.int16, device="cuda")
    y = torch.empty(n, dtype=torch.int16, device="cuda")

    def call():
        emu.check(emu.emu_stage_exponents_static(0, "N", "N", m, n, k, dA.data_ptr(), dA.shape[1], dB.data_ptr(),
                                                 dB.shape[1], 16, x.data_ptr(), y.data_ptr()), "static")
        torch.cuda.synchronize()

    call()                                            # modules loaded, address looked up
    dev_id = torch.cuda.current_device()
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), dev_id) == 0
    zero = ctypes.c_uint64(0)
    assert rt.cudaMemPoolSetAttribute(pool, _USED_MEM_HIGH, ctypes.byref(zero)) == 0   # reset to current
    used0 = _pool_attr(rt, pool, _USED_MEM_CURRENT)
    free0, total = ctypes.c_size_t(0), ctypes.c_size_t(0)
    assert rt.cudaMemGetInfo(ctypes.byref(free0), ctypes.byref(total)) == 0
    for _ in range(3):
        call()
    free1 = ctypes.c_size_t(0)
    assert rt.cudaMemGetInfo(ctypes.byref(free1), ctypes.byref(total)) == 0
    assert _pool_attr(rt, pool, _USED_MEM_HIGH) == used0
    assert free1.value == free0.value
    # the check itself can see an allocation: the allocating entry point raises the pool's mark
    xa = torch.empty(m, dtype=torch.int16, device="cuda")
    ya = torch.empty(n, dtype=torch.int16, device="cuda")
    emu.check(emu.emu_stage_exponents(0, "N", "N", m, n, k, dA.data_ptr(), dA.shape[1], dB.data_ptr(), dB.shape[1],
                                      16, xa.data_ptr(), ya.data_ptr()), "allocating")
    torch.cuda.synchronize()
    assert _pool_attr(rt, pool, _USED_MEM_HIGH) > used0
    assert torch.equal(xa, x) and torch.equal(ya, y)


def test_static_bad_pointer_sets_the_parameter_index():
    st = emu.emu_stage_exponents_static(0, "N", "N", 8, 8, 8, 0, 8, 0, 8, 14, 0, 0)
    assert st == emu.EMU_ERR_INVALID_ARG and emu.emu_last_bad_param() == 7
    st = emu.emu_stage_exponents_static(0, 7, "N", 8, 8, 8, 0, 8, 0, 8, 14, 0, 0)
    assert st == emu.EMU_ERR_INVALID_ARG and emu.emu_last_bad_param() == 1
    st = emu.emu_stage_exponents_static(0, "N", "N", 8, 8, 8, 0, 4, 0, 8, 14, 0, 0)
    assert st == emu.EMU_ERR_INVALID_ARG and emu.emu_last_bad_param() == 8
