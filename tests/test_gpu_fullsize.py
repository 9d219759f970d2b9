"""Full-size parity: the bench workloads (ZGEMM 16384^3, CGEMM 8192^3) in the
launch configuration bench.py times, checked bit for bit against the oracle
on sampled entries, plus the accuracy of the emulation and of native cuBLAS
against the exact product on the same entries."""
import json
import os

import numpy as np
import pytest
import torch

import bench
from oracle import fp
from oracle.emulate import emulate_entries
from oracle.exact import complex_product_entries
from oracle.metrics import abs_bound_entries, max_normalised_error, max_rel_error
from paper_2512_08321_gb300 import emu
from paper_2512_08321_gb300.workloads import paper_matrix_device

pytestmark = pytest.mark.gpu

# measured figures are written as JSON into this directory when it is set and exists
OUT = os.environ.get("EMU_RESULTS_DIR", "")


def _record(name, data):
    if OUT and os.path.isdir(OUT):
        with open(os.path.join(OUT, name), "w") as f:
            json.dump(data, f, indent=1)


@pytest.mark.parametrize("workload,moduli,tol", [("zgemm16384", (12, 14, 15, 16, 20), 1e-15),
                                                  ("cgemm8192", (6, 8, 10), 1e-6)])
def test_fullsize_sampled(workload, moduli, tol):
    wl = bench.WORKLOADS[workload]
    m, n, k, single = wl["m"], wl["n"], wl["k"], wl["single"]
    cdt = torch.complex64 if single else torch.complex128
    A = paper_matrix_device(m, k, wl["phi"], wl["seed"], cdt)          # storage (k, m)
    B = paper_matrix_device(k, n, wl["phi"], wl["seed"] + 1, cdt)      # storage (n, k)
    C = torch.zeros((n, m), dtype=cdt, device="cuda")
    rng = np.random.default_rng(7)
    S = 48
    rows = np.concatenate([[0, m - 1], rng.integers(0, m, S - 2)])
    cols = np.concatenate([[0, n - 1], rng.integers(0, n, S - 2)])
    # the sampled rows of A and columns of B, as the oracle's inputs (complex128)
    Arows = A[:, torch.from_numpy(np.unique(rows)).cuda()].t().cpu().numpy().astype(np.complex128)
    Bcols = B[torch.from_numpy(np.unique(cols)).cuda(), :].t().cpu().numpy().astype(np.complex128)
    ri = np.searchsorted(np.unique(rows), rows)
    ci = np.searchsorted(np.unique(cols), cols)
    exact = complex_product_entries(Arows, Bcols, ri, ci)
    bound = abs_bound_entries(Arows, Bcols, ri, ci)
    f = emu.emu_cgemm if single else emu.emu_zgemm
    report = {"workload": workload, "samples": S, "tolerance_normalised": tol, "by_moduli": {}}
    fmt = fp.BINARY32 if single else fp.BINARY64
    for N in moduli:
        st = f("N", "N", m, n, k, 1.0, A.data_ptr(), m, B.data_ptr(), k, 0.0, C.data_ptr(), m, N, None)
        emu.check(st, "gemm")
        torch.cuda.synchronize()
        assert emu.emu_stream_status() == emu.EMU_OK
        got = C[torch.from_numpy(cols).cuda(), torch.from_numpy(rows).cuda()].cpu().numpy()
        want = emulate_entries(Arows, Bcols, N, ri, ci, out_fmt=fmt)
        assert np.array_equal(got.view(np.float32 if single else np.float64),
                              want.view(np.float32 if single else np.float64)), f"N={N} not bit-exact"
        report["by_moduli"][N] = {"max_normalised_error": max_normalised_error(got, exact, bound),
                                  "max_rel_error": max_rel_error(got, exact)}
    # native cuBLAS on the same inputs and entries
    Cn = torch.matmul(A.t(), B.t())
    torch.cuda.synchronize()
    nat = Cn[torch.from_numpy(rows).cuda(), torch.from_numpy(cols).cuda()].cpu().numpy()
    report["native"] = {"max_normalised_error": max_normalised_error(nat, exact, bound),
                        "max_rel_error": max_rel_error(nat, exact)}
    _record(f"accuracy_{workload}.json", report)
    print(json.dumps(report))
    default_N = wl["N"]
    assert report["by_moduli"][default_N]["max_normalised_error"] <= tol
    # accuracy no worse than native at the bench's moduli count
    assert report["by_moduli"][default_N]["max_normalised_error"] <= max(report["native"]["max_normalised_error"], tol)


@pytest.mark.parametrize("workload,moduli,tol", [("dgemm16384", (12, 14, 15, 16, 18), 1e-15),
                                                  ("sgemm16384", (6, 7, 8, 10), 1e-6)])
def test_fullsize_sampled_real(workload, moduli, tol):
    from oracle.emulate_real import emulate_real_entries
    from oracle.exact import real_product_entries
    from paper_2512_08321_gb300.workloads import paper_matrix_real_device
    wl = bench.WORKLOADS[workload]
    m, n, k, single = wl["m"], wl["n"], wl["k"], wl["single"]
    dt = torch.float32 if single else torch.float64
    A = paper_matrix_real_device(m, k, wl["phi"], wl["seed"], dt)      # storage (k, m)
    B = paper_matrix_real_device(k, n, wl["phi"], wl["seed"] + 1, dt)  # storage (n, k)
    C = torch.zeros((n, m), dtype=dt, device="cuda")
    rng = np.random.default_rng(8)
    S = 48
    rows = np.concatenate([[0, m - 1], rng.integers(0, m, S - 2)])
    cols = np.concatenate([[0, n - 1], rng.integers(0, n, S - 2)])
    ur, uc = np.unique(rows), np.unique(cols)
    Arows = A[:, torch.from_numpy(ur).cuda()].t().cpu().numpy().astype(np.float64)
    Bcols = B[torch.from_numpy(uc).cuda(), :].t().cpu().numpy().astype(np.float64)
    ri, ci = np.searchsorted(ur, rows), np.searchsorted(uc, cols)
    exact = real_product_entries(Arows, Bcols, ri, ci)
    bound = abs_bound_entries(Arows, Bcols, ri, ci)
    f = emu.emu_sgemm if single else emu.emu_dgemm
    fmt = fp.BINARY32 if single else fp.BINARY64
    report = {"workload": workload, "samples": S, "tolerance_normalised": tol, "by_moduli": {}}
    for N in moduli:
        emu.check(f("N", "N", m, n, k, 1.0, A.data_ptr(), m, B.data_ptr(), k, 0.0, C.data_ptr(), m, N, None), "gemm")
        torch.cuda.synchronize()
        assert emu.emu_stream_status() == emu.EMU_OK
        got = C[torch.from_numpy(cols).cuda(), torch.from_numpy(rows).cuda()].cpu().numpy()
        want = emulate_real_entries(Arows, Bcols, N, ri, ci, out_fmt=fmt)
        assert np.array_equal(got.view(np.int32 if single else np.int64),
                              want.view(np.int32 if single else np.int64)), f"N={N} not bit-exact"
        report["by_moduli"][N] = {"max_normalised_error": max_normalised_error(got, exact, bound),
                                  "max_rel_error": max_rel_error(got, exact)}
    Cn = torch.matmul(A.t(), B.t())
    torch.cuda.synchronize()
    nat = Cn[torch.from_numpy(rows).cuda(), torch.from_numpy(cols).cuda()].cpu().numpy()
    report["native"] = {"max_normalised_error": max_normalised_error(nat, exact, bound),
                        "max_rel_error": max_rel_error(nat, exact)}
    _record(f"accuracy_{workload}.json", report)
    print(json.dumps(report))
    # the fewest listed moduli whose error is no worse than native is recorded; the bench's N must meet it
    default_N = wl["N"]
    assert report["by_moduli"][default_N]["max_normalised_error"] <= max(report["native"]["max_normalised_error"], tol)


def test_sm_pair_tiles_at_size_sampled():
    """Residue products on SM pairs (a launch form the autotuner can select) at a
    large size, bit for bit against the oracle on sampled entries."""
    m = n = k = 8192
    N = 15
    A = paper_matrix_device(m, k, 1.0, 2025, torch.complex128)      # storage (k, m)
    B = paper_matrix_device(k, n, 1.0, 2026, torch.complex128)      # storage (n, k)
    C = torch.zeros((n, m), dtype=torch.complex128, device="cuda")
    rng = np.random.default_rng(11)
    rows = np.concatenate([[0, m - 1], rng.integers(0, m, 14)])
    cols = np.concatenate([[0, n - 1], rng.integers(0, n, 14)])
    saved = emu.emu_get_tuning(emu.EMU_TUNE_CTA_PAIR)
    emu.check(emu.emu_set_tuning(emu.EMU_TUNE_CTA_PAIR, 1), "tuning")
    try:
        emu.check(emu.emu_zgemm("N", "N", m, n, k, 1.0, A.data_ptr(), m, B.data_ptr(), k, 0.0, C.data_ptr(), m,
                                N, None), "zgemm")
        torch.cuda.synchronize()
        assert emu.emu_stream_status() == emu.EMU_OK
    finally:
        emu.emu_set_tuning(emu.EMU_TUNE_CTA_PAIR, saved)
    got = C[torch.from_numpy(cols).cuda(), torch.from_numpy(rows).cuda()].cpu().numpy()
    ur, uc = np.unique(rows), np.unique(cols)
    Arows = A[:, torch.from_numpy(ur).cuda()].t().cpu().numpy()     # sampled rows of A, (r, k)
    Bcols = B[torch.from_numpy(uc).cuda(), :].t().cpu().numpy()     # sampled columns of B, (k, c)
    want = emulate_entries(Arows, Bcols, N, np.searchsorted(ur, rows), np.searchsorted(uc, cols))
    assert np.array_equal(got.view(np.uint64), np.asarray(want, dtype=np.complex128).view(np.uint64))
