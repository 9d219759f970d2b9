"""The allocation-free exponent entry point.

Callers that cannot let the library allocate device memory (their memory is
owned by their own pool, or they cannot accept the device-wide
synchronisation of cudaMalloc/cudaFree) use emu_stage_exponents_static, whose
scratch is a fixed array inside the library.  Its results must equal those of
emu_stage_exponents, on consecutive calls that reuse the same array.  This
file is collected last so a failure here stops a -x run only after every
other test has run."""
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
