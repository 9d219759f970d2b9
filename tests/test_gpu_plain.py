"""The bench's plain-emulation comparator (the paper's unfused design: int8
planes, one cuBLAS INT8 GEMM per residue product with a separate mod pass, then
the CRT) checked against the oracle and against the fused library call on the
same inputs, so the comparator's timing belongs to a correct result."""
import numpy as np
import pytest
import torch

import bench
from oracle import fp
from oracle.emulate import emulate
from paper_2512_08321_gb300 import emu
from paper_2512_08321_gb300.workloads import paper_matrix

from .helpers import same_bits

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("single,N", [(False, 14), (False, 15), (True, 8)])
def test_plain_emulation_matches_oracle_and_fused(single, N):
    m, n, k = 200, 136, 328                     # torch._int_mm needs m > 16 and n, k multiples of 8
    cdt = torch.complex64 if single else torch.complex128
    ndt = np.complex64 if single else np.complex128
    A = paper_matrix(m, k, 1.0, 31).astype(ndt)
    B = paper_matrix(k, n, 1.0, 32).astype(ndt)
    dA = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()     # storage (k, m): lda = m
    dB = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()     # storage (n, k): ldb = k
    wl = dict(m=m, n=n, k=k, N=N, single=single)
    Cp, _ = bench.plain_emulation_run(emu, torch, dA, dB, wl)
    Cf = torch.zeros((n, m), dtype=cdt, device="cuda")
    f = emu.emu_cgemm if single else emu.emu_zgemm
    emu.check(f("N", "N", m, n, k, 1.0, dA.data_ptr(), m, dB.data_ptr(), k, 0.0, Cf.data_ptr(), m, N, None), "gemm")
    torch.cuda.synchronize()
    ref = emulate(A.astype(np.complex128), B.astype(np.complex128), N, keep_residue_planes=False,
                  out_fmt=fp.BINARY32 if single else fp.BINARY64).out.astype(ndt)
    got_plain = np.ascontiguousarray(Cp.cpu().numpy().T)
    got_fused = np.ascontiguousarray(Cf.cpu().numpy().T)
    assert same_bits(got_plain, ref)
    assert same_bits(got_fused, got_plain)
