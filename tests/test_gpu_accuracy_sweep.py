"""Accuracy sweeps of the bench workloads at full size (opt-in: set
EMU_ACCURACY_SWEEP=1; several minutes, most of it native cuBLAS ZGEMM).

ZGEMM 16384^3 with phi in {0, 1, 2} and N = 12..20, CGEMM 8192^3 with phi in
{0, 0.5, 1} and N = 6..10: the normalised error of the emulation and of native
cuBLAS against the correctly rounded exact product on 4096 sampled entries
(the exact reference runs in a process pool started with `spawn`).  The
report is also written as accuracy_sweep.json into the output folder, when
that folder exists."""
import json
import multiprocessing as mp
import os

import numpy as np
import pytest
import torch

from oracle.exact import complex_product_entries
from oracle.metrics import abs_bound_entries, max_normalised_error, max_rel_error
from paper_2512_08321_gb300 import emu
from paper_2512_08321_gb300.workloads import paper_matrix_device

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(os.environ.get("EMU_ACCURACY_SWEEP") != "1",
                                 reason="opt-in full-size accuracy sweep (EMU_ACCURACY_SWEEP=1)")]

# measured figures are written as JSON into this directory when it is set and exists
OUT = os.environ.get("EMU_RESULTS_DIR", "")
SAMPLES = 4096
SWEEPS = [  # name, m=n=k, complex64, phis, moduli, tolerance
    ("zgemm16384", 16384, False, (0.0, 1.0, 2.0), tuple(range(12, 21)), 1e-15),
    ("cgemm8192", 8192, True, (0.0, 0.5, 1.0), tuple(range(6, 11)), 1e-6),
]


def _exact_chunk(args):
    Ar, Bc = args
    idx = np.arange(Ar.shape[0])
    return complex_product_entries(Ar, Bc, idx, idx)


@pytest.fixture(scope="module")
def pool():
    p = mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1))
    yield p
    p.close()
    p.join()


def test_accuracy_sweep(pool):
    report = {"samples": SAMPLES}
    for name, size, single, phis, moduli, tol in SWEEPS:
        m = n = k = size
        cdt = torch.complex64 if single else torch.complex128
        f = emu.emu_cgemm if single else emu.emu_zgemm
        rng = np.random.default_rng(11)
        rows = np.concatenate([[0, m - 1], rng.integers(0, m, SAMPLES - 2)])
        cols = np.concatenate([[0, n - 1], rng.integers(0, n, SAMPLES - 2)])
        rt, ct = torch.from_numpy(rows).cuda(), torch.from_numpy(cols).cuda()
        report[name] = {}
        for s, phi in enumerate(phis):
            A = paper_matrix_device(m, k, phi, 20260 + 10 * s, cdt)          # storage (k, m)
            B = paper_matrix_device(k, n, phi, 20261 + 10 * s, cdt)          # storage (n, k)
            Ar = A[:, rt].t().cpu().numpy().astype(np.complex128)           # sampled rows of A, in order
            Bc = B[ct, :].t().cpu().numpy().astype(np.complex128)           # sampled columns of B, in order
            chunks = [(Ar[i:i + 128], Bc[:, i:i + 128]) for i in range(0, SAMPLES, 128)]
            exact = np.concatenate(pool.map(_exact_chunk, chunks))
            idx = np.arange(SAMPLES)
            bound = abs_bound_entries(Ar, Bc, idx, idx)
            C = torch.zeros((n, m), dtype=cdt, device="cuda")
            entry = {"by_moduli": {}}
            for N in moduli:
                emu.check(f("N", "N", m, n, k, 1.0, A.data_ptr(), m, B.data_ptr(), k, 0.0, C.data_ptr(), m, N,
                            None), "gemm")
                torch.cuda.synchronize()
                assert emu.emu_stream_status() == emu.EMU_OK
                got = C[ct, rt].cpu().numpy()
                entry["by_moduli"][N] = {"max_normalised_error": max_normalised_error(got, exact, bound),
                                         "max_rel_error": max_rel_error(got, exact)}
            del C
            Cn = torch.matmul(A.t(), B.t())
            torch.cuda.synchronize()
            nat = Cn[rt, ct].cpu().numpy()
            del Cn
            entry["native"] = {"max_normalised_error": max_normalised_error(nat, exact, bound),
                               "max_rel_error": max_rel_error(nat, exact)}
            ok = [N for N in moduli if entry["by_moduli"][N]["max_normalised_error"]
                  <= max(entry["native"]["max_normalised_error"], tol)]
            entry["fewest_moduli_no_worse_than_native"] = min(ok) if ok else None
            report[name][str(phi)] = entry
            print(name, phi, json.dumps(entry), flush=True)
            # the sweep's largest N is within the stated tolerance
            assert entry["by_moduli"][moduli[-1]]["max_normalised_error"] <= tol
            del A, B
            torch.cuda.empty_cache()
    if OUT and os.path.isdir(OUT):
        with open(os.path.join(OUT, "accuracy_sweep.json"), "w") as fh:
            json.dump(report, fh, indent=1)
