#!/usr/bin/env python
"""Benchmark of the Ozaki-II emulated complex GEMM on GB300.

One step = one emulated GEMM of the workload through the C ABI (exponents,
residue split, residue products, CRT), inputs resident in HBM.  Prints one
JSON line (rank 0).  Workloads (synthetic, the paper's generator of Section
IV-A, drawn on the GPU from a fixed seed):

  zgemm16384  complex128, m = n = k = 16384, phi = 1, N = 15 moduli (default; the
              fewest moduli whose error is no worse than native cuBLAS ZGEMM here)
  cgemm8192   complex64,  m = n = k = 8192,  phi = 0.5, N = 8 moduli
  dgemm16384  float64, m = n = k = 16384, phi = 1, N = 15 (the paper's real-valued comparison)
  sgemm16384  float32, m = n = k = 16384, phi = 0.5

Inputs are larger than L2 (8.6 GB / 1.1 GB), so no flush is needed between
steps.  `--impl reference` times the CPU oracle on a bounded sample of the
same workload instead.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "emulated ZGEMM/CGEMM TFLOPS (8mnk/s) vs cuBLAS native at matched accuracy"
METRIC_REAL = "emulated DGEMM/SGEMM TFLOPS (2mnk/s) vs cuBLAS native at matched accuracy"
WORKLOADS = {
    "zgemm16384": dict(single=False, m=16384, n=16384, k=16384, phi=1.0, N=15, seed=20251208),
    "cgemm8192": dict(single=True, m=8192, n=8192, k=8192, phi=0.5, N=8, seed=20251209),
    # the paper's CGEMM size (its speed-ups over cublasCgemm are quoted at 16384^3)
    "cgemm16384": dict(single=True, m=16384, n=16384, k=16384, phi=0.5, N=8, seed=20251217),
    # real matrices (one residue product per modulus)
    "dgemm16384": dict(single=False, real=True, m=16384, n=16384, k=16384, phi=1.0, N=15, seed=20251215),
    "sgemm16384": dict(single=True, real=True, m=16384, n=16384, k=16384, phi=0.5, N=8, seed=20251216),
    # 512 uneven problems, m, n, k log-uniform in [64, 2048]: one grouped plan replayed from a CUDA graph
    "grouped512": dict(single=False, grouped=True, count=512, lo=64, hi=2048, phi=1.0, N=16, seed=20251212,
                       m=0, n=0, k=0),
    # 64 problems of the same distribution: a case small enough for profiler captures
    "grouped64": dict(single=False, grouped=True, count=64, lo=64, hi=2048, phi=1.0, N=16, seed=20251213,
                      m=0, n=0, k=0),
    # held-out inputs for the learned moduli selector (not in its training set), three targets
    "learned": dict(single=False, learned=True, shapes=[(8192, 8192, 8192), (16384, 1024, 16384)],
                    phis=[0.5, 3.0], targets=[1e-6, 1e-10, 1e-15], seed=20251214, N=0, m=0, n=0, k=0, phi=0.0),
    # small cases of the same kernels for profiler captures
    "zgemm4096": dict(single=False, m=4096, n=4096, k=4096, phi=1.0, N=14, seed=20251210),
    "zgemm8192": dict(single=False, m=8192, n=8192, k=8192, phi=1.0, N=14, seed=20251211),
}
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
CPU_SAMPLE = 256          # cpu baseline: a CPU_SAMPLE x CPU_SAMPLE output block at full k


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="zgemm16384")
    ap.add_argument("--moduli", type=int, default=0, help="override N")
    ap.add_argument("--no-native", action="store_true", help="skip the cuBLAS native comparison")
    ap.add_argument("--no-plain", action="store_true", help="skip the unfused cuBLAS-INT8 comparator")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the compact cgemm8192 and grouped512 records added to the default workload's line")
    ap.add_argument("--overlap", choices=["auto", "on", "off"], default="auto",
                    help="EMU_TUNE_OVERLAP: split and CRT of neighbouring column blocks beside the products "
                         "(auto: the library's default, on for the real GEMMs)")
    ap.add_argument("--bound-pair", choices=["auto", "on", "off"], default="auto",
                    help="EMU_TUNE_BOUND_PAIR: accurate-mode bound products on SM pairs (auto: the library's default, on)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch configuration")
    ap.add_argument("--scaling", choices=["fast", "accurate"], default="fast",
                    help="scaling vectors of Section III-B (fast or accurate mode)")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return dict(FALLBACK_PEAKS), "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples (200 ms) while the timed region runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ oracle (CPU baseline only)
def flops_per_entry(wl):
    """Real flops of one output entry per unit of k: 8 complex, 2 real."""
    return 2.0 if wl.get("real") else 8.0


def cpu_baseline(wl, repeat=1):
    """The CPU oracle as it stands, timed on a CPU_SAMPLE x CPU_SAMPLE output block
    of the workload at full k; throughput in the metric's unit (TFLOPS)."""
    import numpy as np
    from paper_2512_08321_gb300.workloads import paper_matrix, paper_matrix_real
    s = CPU_SAMPLE
    if wl.get("real"):
        from oracle.emulate_real import RealEmulation
        dt = np.float32 if wl["single"] else np.float64
        A = paper_matrix_real(s, wl["k"], wl["phi"], wl["seed"], dt).astype(np.float64)
        B = paper_matrix_real(wl["k"], s, wl["phi"], wl["seed"] + 1, dt).astype(np.float64)
        run = lambda: RealEmulation(A, B, wl["N"])
    else:
        from oracle.emulate import emulate
        dt = np.complex64 if wl["single"] else np.complex128
        A = paper_matrix(s, wl["k"], wl["phi"], wl["seed"], dt).astype(np.complex128)
        B = paper_matrix(wl["k"], s, wl["phi"], wl["seed"] + 1, dt).astype(np.complex128)
        run = lambda: emulate(A, B, wl["N"], keep_residue_planes=False)
    times = []
    for _ in range(repeat):
        t0 = time.perf_counter()
        run()
        times.append(time.perf_counter() - t0)
    t = statistics.median(times)
    return {"value": flops_per_entry(wl) * s * s * wl["k"] / t * 1e-12, "unit": "TFLOPS", "cores": os.cpu_count(),
            "kind": "oracle", "seconds_per_sample": t,
            "sample": f"{s}x{s} output block of the {wl['m']}x{wl['n']}x{wl['k']} workload at full k "
                      f"(N={wl['N']}, numpy float64 BLAS for the residue products, Python integers for the CRT)"}


def run_reference(args, wl, rank):
    if rank != 0:
        return 0
    steps = []
    for i in range(args.warmup + args.steps):
        r = cpu_baseline(wl)
        if i >= args.warmup:
            steps.append(r)
    t = statistics.mean(x["seconds_per_sample"] for x in steps)
    value = flops_per_entry(wl) * CPU_SAMPLE * CPU_SAMPLE * wl["k"] / t * 1e-12
    cb = dict(steps[-1])
    cb["value"] = value
    out = {"impl": "reference", "metric": METRIC_REAL if wl.get("real") else METRIC, "value": value, "unit": "TFLOPS", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64+int", "data": "synthetic",
           "config": {"workload": args.workload, "m": wl["m"], "n": wl["n"], "k": wl["k"], "num_moduli": wl["N"],
                      "phi": wl["phi"], "sample": cb["sample"]},
           "cpu_baseline": cb, "e2e": {"value": value, "unit": "TFLOPS", "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm
def overlap_blocks(n):
    """Column blocks of an overlapped GEMM: about eight of a multiple of 256 columns, at least 1024."""
    nb = max(1024, (-(-n // 8) + 255) // 256 * 256)
    return -(-n // nb)


def source_sha256(files):
    """sha256 over the kernel's source files, in order."""
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2512_08321_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profile_traffic(kernel_files, summary_name):
    """dram bytes per launch from the committed ncu summary, if the kernel's sources
    (its .cu file and the shared tcgen05/TMA header) are unchanged since the capture
    (their sha256 is recorded there)."""
    path = os.path.join(ROOT, "profiles", summary_name)
    try:
        kv = {}
        for ln in open(path):
            if ":" in ln and not ln.startswith("#"):
                a, b = ln.split(":", 1)
                kv[a.strip()] = b.strip()
        sha = source_sha256(kernel_files)
        if kv.get("source_sha256") != sha:
            return None
        return float(kv["dram_bytes_per_launch_full_size"])
    except Exception:
        return None


def main():
    args = parse()
    wl = dict(WORKLOADS[args.workload])
    if args.moduli:
        wl["N"] = args.moduli
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, wl, rank)
    if wl.get("grouped"):
        return run_grouped(args, wl, world, rank, local)
    if wl.get("learned"):
        return run_learned(args, wl, world, rank, local)

    import torch
    from paper_2512_08321_gb300 import emu
    from paper_2512_08321_gb300.workloads import paper_matrix_device, paper_matrix_real_device

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    emu.lib()
    emu.check(emu.emu_set_scaling(emu.EMU_SCALING_ACCURATE if args.scaling == "accurate" else emu.EMU_SCALING_FAST),
              "emu_set_scaling")
    if args.overlap != "auto":
        emu.check(emu.emu_set_tuning(emu.EMU_TUNE_OVERLAP, 1 if args.overlap == "on" else 0), "overlap")
    if args.bound_pair != "auto":
        emu.check(emu.emu_set_tuning(emu.EMU_TUNE_BOUND_PAIR, 1 if args.bound_pair == "on" else 0), "bound pair")
    m, n, k, N = wl["m"], wl["n"], wl["k"], wl["N"]
    single = wl["single"]
    real = bool(wl.get("real"))
    ppm = 1 if real else 3                      # residue products per modulus
    if real:
        cdt = torch.float32 if single else torch.float64
        gen = paper_matrix_real_device
        f = emu.emu_sgemm if single else emu.emu_dgemm
        dtype_code = emu.EMU_DTYPE_S if single else emu.EMU_DTYPE_D
    else:
        cdt = torch.complex64 if single else torch.complex128
        gen = paper_matrix_device
        f = emu.emu_cgemm if single else emu.emu_zgemm
        dtype_code = emu.EMU_DTYPE_C if single else emu.EMU_DTYPE_Z
    esz = torch.empty((), dtype=cdt).element_size()
    A = gen(m, k, wl["phi"], wl["seed"] + 1000 * rank, cdt)   # (k, m): lda = m
    B = gen(k, n, wl["phi"], wl["seed"] + 1 + 1000 * rank, cdt)
    C = torch.zeros((n, m), dtype=cdt, device="cuda")
    st = torch.cuda.current_stream()

    def step(a=A, b=B, c=C):
        s = f("N", "N", m, n, k, 1.0, a.data_ptr(), m, b.data_ptr(), k, 0.0, c.data_ptr(), m, N, st)
        if s != emu.EMU_OK:
            raise emu.EmuError(s, "gemm")

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    tuned = None
    if not args.no_autotune:
        st_t, tuned = emu.emu_autotune_gemm(dtype_code, m, n, k, N)
        emu.check(st_t, "emu_autotune_gemm")
    for _ in range(args.warmup):
        step()
    barrier()
    # ---- timed region: K steps, phase events per step
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    for row in evs:
        for e in row:
            e.record()              # materialise the CUDA events before the timed region
    torch.cuda.synchronize()
    t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = emu.emu_kernel_launches()
    with ClockSampler(local) as clk:
        time.sleep(0.3)
        barrier()
        t0e.record()
        for i in range(args.steps):
            emu.check(emu.emu_set_phase_events(evs[i]), "emu_set_phase_events")
            step()
        t1e.record()
        barrier()
        emu.emu_set_phase_events(None)
    launches = emu.emu_kernel_launches() - launches0
    status = emu.emu_stream_status(st)
    total_ms = t0e.elapsed_time(t1e)
    ms = max_over_ranks(total_ms / args.steps, dist)
    flops = flops_per_entry(wl) * m * n * k
    value = world * flops / (ms * 1e-3) * 1e-12
    ev_ms = lambda row, a, b: statistics.mean(row[i][a].elapsed_time(row[i][b]) for i in range(len(row)))
    # overlapped column blocks (EMU_TUNE_OVERLAP; by default on for the real GEMMs): the step's phase events mark
    # the planes of A and of the first block (0 -> 2), the residue products of all blocks back to
    # back (2 -> 3) and the last block's CRT (3 -> 4); the other blocks' exponents, planes and CRTs
    # run beside the products.  The per-phase times below come from one more step with overlap off.
    ov_setting = emu.emu_get_tuning(emu.EMU_TUNE_OVERLAP)
    overlapped = (ov_setting == 1 or (ov_setting < 0 and real)) and n >= 2048
    nblk = overlap_blocks(n) if overlapped else 1
    if overlapped:
        overlap_ms = {"planes_before_first_products": ev_ms(evs, 0, 2), "residue_products_all_blocks": ev_ms(evs, 2, 3),
                      "last_crt": ev_ms(evs, 3, 4)}
        t_gemm_step = overlap_ms["residue_products_all_blocks"] * 1e-3
        sev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)]]
        emu.check(emu.emu_set_tuning(emu.EMU_TUNE_OVERLAP, 0), "overlap off")
        try:
            step()
            emu.check(emu.emu_set_phase_events(sev[0]), "phase events")
            step()
            emu.emu_set_phase_events(None)
        finally:
            emu.emu_set_tuning(emu.EMU_TUNE_OVERLAP, ov_setting)
        torch.cuda.synchronize()
        pev_rows = sev
    else:
        pev_rows = evs
    phase_names = ["exponents", "split", "residue_gemm", "crt"]
    phases = {nm: ev_ms(pev_rows, p, p + 1) for p, nm in enumerate(phase_names)}
    pk, pk_src = peaks()
    if not overlapped:
        t_gemm_step = phases["residue_gemm"] * 1e-3
    gemm_flops = 2.0 * ppm * N * m * n * k
    t_gemm = t_gemm_step
    achieved = gemm_flops / t_gemm * 1e-12
    peak = float(pk.get("bf16_tflops_sustained", FALLBACK_PEAKS["bf16_tflops_sustained"]))
    traffic = profile_traffic(("k_gemm_f16.cu", "tc_common.cuh"), f"gemm_f16_{args.workload}.txt")
    roofline = {"bound": "tensor", "kernel": "gemm_f16_kernel (tcgen05.mma kind::f16, exact residue products)",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": (traffic / nblk if traffic else traffic),
                "peak_source": f"{pk_src} bf16_tflops_sustained (fp16 = bf16 rate)",
                "launches_per_step": nblk, "algorithmic_flops_per_launch": gemm_flops / nblk,
                "timing": ("the step's residue-product launches back to back on their stream (CUDA events), "
                           "divided by the launches" if overlapped else "the one launch of the step (CUDA events)")}
    hbm = float(pk.get("hbm_gbs", FALLBACK_PEAKS["hbm_gbs"]))
    byts = {"exponents": 2 * esz * k * (m + n), "split": esz * k * (m + n) + ppm * N * 2 * k * (m + n),
            "crt": ppm * N * m * n + esz * m * n}
    mem_phases = {nm: {"ms": phases[nm], "algorithmic_bytes": byts[nm],
                       "GBps": byts[nm] / (phases[nm] * 1e-3) * 1e-9,
                       "frac_of_hbm": byts[nm] / (phases[nm] * 1e-3) * 1e-9 / hbm} for nm in byts}
    out = {"metric": METRIC_REAL if real else METRIC, "value": value, "unit": "TFLOPS", "n_gpus": world,
           "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "fp16", "data": "synthetic",
           "config": {"workload": args.workload, "m": m, "n": n, "k": k,
                      "io": str(cdt).replace("torch.", ""), "num_moduli": N, "phi": wl["phi"],
                      "engine": "tcgen05 kind::f16 (exact residues), integer CRT", "scaling": args.scaling,
                      "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas{world}",
                      "seed": wl["seed"],
                      "tuning": tuning_record(emu, dtype_code, N, m, n, k, tuned)},
           "roofline": roofline, "phases_ms": phases, "memory_phases": mem_phases,
           "overlap": ({"column_blocks": nblk, "step_ms": overlap_ms,
                        "phases_ms_from": "one more step with EMU_TUNE_OVERLAP = 0 (one phase after another)"}
                       if overlapped else None),
           # the paper counts the residue products as INT8 operations (6N mnk complex, 2N mnk real):
           # their rate here, beside GB300's dense INT8 peak from its Table 1 (B300 row)
           "int8_equivalent": {"tops": gemm_flops / t_gemm * 1e-12, "table1_int8_peak_tops": 150.0,
                               "ratio_to_int8_peak": gemm_flops / t_gemm * 1e-12 / 150.0},
           "gpu_launches": int(launches), "device_status": emu.STATUS_NAMES.get(status, status),
           "clocks": clk.summary()}

    # ---- the paper's floating-point CRT on the same step (one run, phase events)
    pev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    emu.check(emu.emu_set_crt_mode(emu.EMU_CRT_PAPER_FP64), "crt mode")
    overlap_setting = emu.emu_get_tuning(emu.EMU_TUNE_OVERLAP)
    emu.check(emu.emu_set_tuning(emu.EMU_TUNE_OVERLAP, 0), "overlap off")     # phases one after another
    try:
        step()
        emu.check(emu.emu_set_phase_events(pev), "phase events")
        step()
        emu.emu_set_phase_events(None)
    finally:
        emu.emu_set_crt_mode(emu.EMU_CRT_EXACT)
        emu.emu_set_tuning(emu.EMU_TUNE_OVERLAP, overlap_setting)
    torch.cuda.synchronize()
    out["crt_modes_ms"] = {"exact_integer": phases["crt"], "paper_fp64_double_double": pev[3].elapsed_time(pev[4])}

    # ---- end to end through the C ABI with host buffers
    if not args.no_e2e:
        Ah = A.cpu().pin_memory()
        Bh = B.cpu().pin_memory()
        Ch = torch.empty(C.shape, dtype=cdt).pin_memory()
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

        fh = {emu.emu_zgemm: emu.emu_zgemm_host, emu.emu_cgemm: emu.emu_cgemm_host,
              emu.emu_dgemm: emu.emu_dgemm_host, emu.emu_sgemm: emu.emu_sgemm_host}[f]

        def e2e_step():
            # host buffers in, host buffer out: the library's copy kernel brings A and B over
            # the CPU-GPU link and the CRT writes C into host memory
            s = fh("N", "N", m, n, k, 1.0, Ah.data_ptr(), m, Bh.data_ptr(), k, 0.0, Ch.data_ptr(), m, N, st)
            if s != emu.EMU_OK:
                raise emu.EmuError(s, "host gemm")

        e2e_step()
        barrier()
        ea.record()
        for _ in range(args.steps):
            e2e_step()
        eb.record()
        barrier()
        e_ms = max_over_ranks(ea.elapsed_time(eb) / args.steps, dist)
        # one more call with the library's trace: when A, B arrived and each column block finished
        emu.emu_host_trace_enable(True)
        e2e_step()
        torch.cuda.synchronize()
        tr = emu.emu_host_trace_read()
        emu.emu_host_trace_enable(False)
        step()                                 # the device call once more (C last held the FP64-CRT result)
        torch.cuda.synchronize()
        ev = {}
        for nm, t in tr:
            ev.setdefault(nm, []).append(round(t, 2))
        trace_summary = {"a_in_done_ms": max(ev.get("a_in", [0.0])), "b_in_done_ms": max(ev.get("b_in", [0.0])),
                         "block_crt_ms": ev.get("block_crt", []), "c_out_ms": ev.get("c_out", []),
                         "end_ms": max(ev.get("end", [0.0]))}
        out["e2e"] = {"value": world * flops / (e_ms * 1e-3) * 1e-12, "unit": "TFLOPS",
                      "h2d_bytes_per_step": esz * (m * k + k * n), "d2h_bytes_per_step": esz * m * n,
                      "ms_per_step": e_ms, "call": fh.__name__ + " (pinned host A, B, C)",
                      "bitexact_vs_device_call": bool(torch.equal(Ch, C.cpu())),
                      "trace_of_one_more_call": trace_summary}
        del Ah, Bh, Ch

    # ---- comparators on the same GPU (rank 0)
    if rank == 0 and not args.no_native:
        At, Bt = A.t(), B.t()                  # op(A) m x k, op(B) k x n views of the same storage
        torch.matmul(At[:64, :64], Bt[:64, :64])
        torch.cuda.synchronize()
        na, nb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        na.record()
        torch.matmul(At, Bt)
        nb.record()
        torch.cuda.synchronize()
        nms = na.elapsed_time(nb)
        routine = {torch.complex64: "cublasCgemm", torch.complex128: "cublasZgemm",
                   torch.float32: "cublasSgemm", torch.float64: "cublasDgemm"}[cdt]
        out["native_cublas"] = {"routine": routine + " (torch.matmul)",
                                "ms": nms, "tflops": flops / (nms * 1e-3) * 1e-12,
                                "speedup_of_emulation": nms / ms,
                                "math_mode": "default (CUBLAS_EMULATION_STRATEGY %s)"
                                             % os.environ.get("CUBLAS_EMULATION_STRATEGY", "unset")}
    # the fused result the comparators are checked against: one more device call with the exact CRT,
    # snapshotted into a buffer no comparator writes
    C_fused = None
    if rank == 0 and not args.no_plain and not real:
        step()
        torch.cuda.synchronize()
        C_fused = C.clone()
    if rank == 0 and not args.no_native and not real:
        g3 = gemm3m(torch, A, B, m, n, k, single, st)
        if g3:
            g3["speedup_of_emulation"] = g3["ms"] / ms
        out["native_cublas_3m"] = g3
    if C_fused is not None:
        out["plain_emulation"] = plain_emulation(emu, torch, A, B, wl, C_fused)
        del C_fused

    # the other workloads of the hot path, measured in the same run (rank 0, default workload only)
    if rank == 0 and args.workload == "zgemm16384" and not args.no_extra:
        extra = {"cgemm8192": extra_single(emu, torch, "cgemm8192")}
        plan, g = grouped_measure(emu, torch, WORKLOADS["grouped512"], rank, 5, 3, with_loop=True)
        emu.emu_grouped_destroy(plan)
        pk2, _ = peaks()
        g["roofline_residue_gemm"] = {
            "achieved_tflops": g["gemm_flops"] / (g["phases_ms"]["residue_gemm"] * 1e-3) * 1e-12,
            "peak": float(pk2.get("bf16_tflops_sustained", FALLBACK_PEAKS["bf16_tflops_sustained"]))}
        g["roofline_residue_gemm"]["frac"] = g["roofline_residue_gemm"]["achieved_tflops"] / \
            g["roofline_residue_gemm"]["peak"]
        extra["grouped512"] = g
        out["extra_workloads"] = extra
    if rank == 0 and world == 1 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(wl)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def gemm3m(torch, A, B, m, n, k, single, stream):
    """cuBLAS's Gauss 3-multiplication complex GEMM (cublasZgemm3m / cublasCgemm3m, the paper's
    Zgemm3m comparator), called through ctypes on the same inputs; it writes into an output buffer
    of its own, so no other result is overwritten.  None if unavailable."""
    import ctypes
    C = torch.empty((n, m), dtype=A.dtype, device=A.device)
    try:
        cb = None
        for nm in ("libcublas.so.13", "libcublas.so"):
            try:
                cb = ctypes.CDLL(nm)
                break
            except OSError:
                continue
        if cb is None:
            return None
        h = ctypes.c_void_p()
        if cb.cublasCreate_v2(ctypes.byref(h)) != 0:
            return None
        cb.cublasSetStream_v2(h, ctypes.c_void_p(stream.cuda_stream))
        T = ctypes.c_float if single else ctypes.c_double
        one, zero = (T * 2)(1.0, 0.0), (T * 2)(0.0, 0.0)
        fn = cb.cublasCgemm3m if single else cb.cublasZgemm3m
        call = lambda mm, nn, kk: fn(h, 0, 0, mm, nn, kk, one, ctypes.c_void_p(A.data_ptr()), m,
                                     ctypes.c_void_p(B.data_ptr()), k, zero, ctypes.c_void_p(C.data_ptr()), m)
        # warm-up on a 64^3 corner (the full product takes tens of seconds at FP64 rates)
        if call(min(m, 64), min(n, 64), min(k, 64)) != 0:
            cb.cublasDestroy_v2(h)
            return None
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        st = call(m, n, k)
        b.record()
        torch.cuda.synchronize()
        cb.cublasDestroy_v2(h)
        if st != 0:
            return None
        ms = a.elapsed_time(b)
        return {"routine": "cublasCgemm3m" if single else "cublasZgemm3m", "ms": ms,
                "tflops": 8.0 * m * n * k / (ms * 1e-3) * 1e-12}
    except Exception:
        return None


def tuning_record(emu, dtype_code, N, m, n, k, tuned):
    """The launch configuration the timed calls used: the autotuned knobs (or the
    defaults) and the residue products' modulus-loop schedule."""
    keys = {"tile_n": emu.EMU_TUNE_TILE_N, "group": emu.EMU_TUNE_GROUP, "chunk_k": emu.EMU_TUNE_CHUNK_K,
            "crt_rows": emu.EMU_TUNE_CRT_ROWS, "split_elems": emu.EMU_TUNE_SPLIT_ELEMS}
    rec = {nm: emu.emu_tuned_value(dtype_code, N, m, n, k, key) for nm, key in keys.items()}
    rec["schedule"] = {nm: emu.emu_tuned_value(dtype_code, N, m, n, k, key) for nm, key in emu.SCHEDULE_KNOBS.items()}
    names = {0: "modulus outer", 1: "tile outer", 2: "column bands (the paper's n-blocking)"}
    rec["schedule"]["order_name"] = names.get(rec["schedule"]["order"], "?")
    rec["source"] = "autotuned (emu_autotune_gemm)" if tuned else "defaults"
    return rec


def max_over_ranks(ms, dist):
    """The step time the job reports: the maximum over ranks."""
    if dist is None:
        return ms
    import torch
    dev = "cuda" if torch.cuda.is_available() and dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_learned(args, wl, world, rank, local):
    """emu_zgemm_tol with the trained selector against the a priori rule on
    held-out inputs; accuracy is reported against the N = 24 emulation."""
    import torch
    from paper_2512_08321_gb300 import emu, moduli
    from paper_2512_08321_gb300.workloads import paper_matrix_device

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    emu.lib()
    cases = []
    for (m, n, k) in wl["shapes"]:
        for phi in wl["phis"]:
            s = wl["seed"] + m + 3 * n + 7 * k + int(100 * phi) + 1000 * rank
            A = paper_matrix_device(m, k, phi, s, torch.complex128)
            B = paper_matrix_device(k, n, phi, s + 1, torch.complex128)
            R = torch.zeros((n, m), dtype=torch.complex128, device="cuda")
            emu.check(emu.emu_zgemm("N", "N", m, n, k, 1.0, A.data_ptr(), m, B.data_ptr(), k, 0.0, R.data_ptr(),
                                    m, 24), "reference N=24")
            bound = ((A.real.abs() + A.imag.abs()).t().float() @ (B.real.abs() + B.imag.abs()).t().float()).t()
            cases.append((m, n, k, phi, A, B, R, bound.double().clamp_min(1e-300)))
    C = torch.zeros((max(c[1] for c in cases), max(c[0] for c in cases)), dtype=torch.complex128, device="cuda")
    stream = torch.cuda.current_stream()

    def run(use_learned):
        if use_learned:
            moduli.load()
        else:
            moduli.unload()
        rows, total_ms, flops = [], 0.0, 0.0
        for (m, n, k, phi, A, B, R, bound) in cases:
            for T in wl["targets"]:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record()
                st, N = emu.emu_zgemm_tol("N", "N", m, n, k, 1.0, A.data_ptr(), m, B.data_ptr(), k, 0.0,
                                          C.data_ptr(), m, T, stream)
                e1.record()
                torch.cuda.synchronize()
                emu.check(st, "emu_zgemm_tol")
                ms = e0.elapsed_time(e1)
                Cm = C.view(-1)[: n * m].view(n, m)
                d = torch.maximum((Cm.real - R.real).abs(), (Cm.imag - R.imag).abs())
                err = float((d / bound).max())
                rows.append({"m": m, "n": n, "k": k, "phi": phi, "target": T, "N": N, "ms": ms, "err_vs_N24": err,
                             "meets": err <= T})
                total_ms += ms
                flops += 8.0 * m * n * k
        return rows, total_ms, flops

    for _ in range(max(args.warmup, 1)):
        run(True)
    learned_runs = [run(True) for _ in range(args.steps)]
    apriori = run(False)
    ms = statistics.mean(r[1] for r in learned_runs)
    ms = max_over_ranks(ms, dist)
    rows, _, flops = learned_runs[-1]
    out = {"metric": METRIC, "value": world * flops / (ms * 1e-3) * 1e-12, "unit": "TFLOPS", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "fp16", "data": "synthetic",
           "config": {"workload": args.workload, "shapes": wl["shapes"], "phis": wl["phis"], "targets": wl["targets"],
                      "io": "complex128", "selector": "trained network (emu_zgemm_tol), one stream sync per call",
                      "parallelism": f"replicas{world}"},
           "learned": rows,
           "apriori": {"ms": apriori[1], "tflops": apriori[2] / (apriori[1] * 1e-3) * 1e-12, "rows": apriori[0]},
           "learned_meets_all": all(r["meets"] for r in rows),
           "apriori_meets_all": all(r["meets"] for r in apriori[0])}
    if rank == 0:
        print(json.dumps(out), flush=True)
    moduli.unload()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_grouped(args, wl, world, rank, local):
    """Batched uneven ZGEMM: one graph replay of the grouped plan per step,
    against the plain loop of per-problem emu_zgemm calls."""
    import torch
    from paper_2512_08321_gb300 import emu
    from paper_2512_08321_gb300.workloads import log_uniform_shapes, paper_matrix_device

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    N = wl["N"]
    shapes = log_uniform_shapes(wl["count"], wl["lo"], wl["hi"], wl["seed"])
    probs, tensors = [], []
    flops = 0.0
    for i, (m, n, k) in enumerate(shapes):
        m, n, k = int(m), int(n), int(k)
        s = wl["seed"] + 7919 * i + 1000003 * rank
        A = paper_matrix_device(m, k, wl["phi"], s, torch.complex128)
        B = paper_matrix_device(k, n, wl["phi"], s + 1, torch.complex128)
        C = torch.zeros((n, m), dtype=torch.complex128, device="cuda")
        tensors.append((A, B, C))
        probs.append(dict(transa="N", transb="N", m=m, n=n, k=k, A=A.data_ptr(), lda=m, B=B.data_ptr(), ldb=k,
                          C=C.data_ptr(), ldc=m))
        flops += 8.0 * m * n * k
    args_g = emu.GroupedArgs(probs, N)
    st, plan = emu.emu_grouped_create(False, args_g, 0)
    emu.check(st, "emu_grouped_create")
    stream = torch.cuda.current_stream()

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        emu.check(emu.emu_grouped_run(plan, stream), "run")
    barrier()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = emu.emu_kernel_launches()
    with ClockSampler(local) as clk:
        time.sleep(0.3)
        barrier()
        a.record()
        for _ in range(args.steps):
            emu.check(emu.emu_grouped_run(plan, stream), "run")
        b.record()
        barrier()
    ms = max_over_ranks(a.elapsed_time(b) / args.steps, dist)
    per_replay = emu.emu_grouped_kernels(plan)
    # phase times of the same plan (outside the graph), for the roofline of the residue products
    phase_runs = [emu.emu_grouped_phase_times(plan, stream)[1] for _ in range(3)]
    phases = {nm: statistics.mean(r[i] for r in phase_runs)
              for i, nm in enumerate(["exponents", "split", "residue_gemm", "crt"])}
    gemm_flops = 6.0 * N * sum(float(m) * n * k for m, n, k in shapes)
    pk, pk_src = peaks()
    peak = float(pk.get("bf16_tflops_sustained", FALLBACK_PEAKS["bf16_tflops_sustained"]))
    achieved = gemm_flops / (phases["residue_gemm"] * 1e-3) * 1e-12
    out = {"metric": METRIC, "value": world * flops / (ms * 1e-3) * 1e-12, "unit": "TFLOPS", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "fp16", "data": "synthetic",
           "config": {"workload": args.workload, "problems": wl["count"], "mnk_range": [wl["lo"], wl["hi"]],
                      "io": "complex128", "num_moduli": N, "phi": wl["phi"], "seed": wl["seed"],
                      "tile_n_autotuned": emu.emu_grouped_tile(plan), "graph_kernels_per_replay": per_replay,
                      "l2": "working set larger than L2 (no flush)", "parallelism": f"replicas{world}"},
           "roofline": {"bound": "tensor", "kernel": "gemm_f16_grouped_kernel", "achieved": achieved,
                        "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                        "peak_source": f"{pk_src} bf16_tflops_sustained",
                        "timing": "grouped phases run once more outside the graph with events"},
           "phases_ms": phases, "gpu_launches": int(per_replay * args.steps),
           "clocks": clk.summary()}
    if rank == 0 and not args.no_plain:
        # the plain per-problem loop on the same data (one emu_zgemm per problem)
        def loop():
            for (m, n, k), (A, B, C) in zip(shapes, tensors):
                s = emu.emu_zgemm("N", "N", int(m), int(n), int(k), 1.0, A.data_ptr(), int(m), B.data_ptr(), int(k),
                                  0.0, C.data_ptr(), int(m), N, stream)
                if s != emu.EMU_OK:
                    raise emu.EmuError(s, "emu_zgemm")
        loop()
        torch.cuda.synchronize()
        la, lb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        la.record()
        loop()
        lb.record()
        torch.cuda.synchronize()
        lms = la.elapsed_time(lb)
        out["plain_loop"] = {"ms": lms, "tflops": flops / (lms * 1e-3) * 1e-12,
                             "speedup_of_grouped": lms / ms,
                             "launches": 10 * len(shapes)}
    if rank == 0:
        print(json.dumps(out), flush=True)
    emu.emu_grouped_destroy(plan)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def extra_single(emu, torch, name, steps=5, warmup=3):
    """A compact record of another single-GEMM workload (cgemm8192) measured in the
    same run: autotuned, W warm-up calls, then the median of K device-timed calls
    (CUDA events on the launching stream), with the phase times of one more call."""
    from paper_2512_08321_gb300.workloads import paper_matrix_device
    wl = WORKLOADS[name]
    m, n, k, N, single = wl["m"], wl["n"], wl["k"], wl["N"], wl["single"]
    cdt = torch.complex64 if single else torch.complex128
    f = emu.emu_cgemm if single else emu.emu_zgemm
    code = emu.EMU_DTYPE_C if single else emu.EMU_DTYPE_Z
    A = paper_matrix_device(m, k, wl["phi"], wl["seed"], cdt)
    B = paper_matrix_device(k, n, wl["phi"], wl["seed"] + 1, cdt)
    C = torch.zeros((n, m), dtype=cdt, device="cuda")
    st = torch.cuda.current_stream()
    st_t, tuned = emu.emu_autotune_gemm(code, m, n, k, N)
    emu.check(st_t, "emu_autotune_gemm")

    def call():
        emu.check(f("N", "N", m, n, k, 1.0, A.data_ptr(), m, B.data_ptr(), k, 0.0, C.data_ptr(), m, N, st), name)

    for _ in range(warmup):
        call()
    torch.cuda.synchronize()
    times = []
    for _ in range(steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        call()
        b.record()
        b.synchronize()
        times.append(a.elapsed_time(b))
    pev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    emu.check(emu.emu_set_phase_events(pev), "phase events")
    call()
    emu.emu_set_phase_events(None)
    torch.cuda.synchronize()
    ms = statistics.median(times)
    flops = 8.0 * m * n * k
    return {"workload": name, "m": m, "n": n, "k": k, "num_moduli": N, "phi": wl["phi"], "io": str(cdt)[6:],
            "tflops": flops / (ms * 1e-3) * 1e-12, "ms_median": ms, "steps": steps, "warmup": warmup,
            "phases_ms": {nm: pev[i].elapsed_time(pev[i + 1])
                          for i, nm in enumerate(["exponents", "split", "residue_gemm", "crt"])},
            "tuning": tuning_record(emu, code, N, m, n, k, tuned),
            "status": emu.STATUS_NAMES.get(emu.emu_stream_status(st), "?")}


def grouped_measure(emu, torch, wl, rank, steps, warmup, with_loop, seed_offset=0):
    """The grouped workload: a plan over every problem (autotuned tile width), W warm-up
    replays of its CUDA graph, then K timed replays (CUDA events, median and mean), the
    phase times of the same plan outside the graph, and optionally the plain loop of
    per-problem emu_zgemm calls on the same data."""
    from paper_2512_08321_gb300.workloads import log_uniform_shapes, paper_matrix_device
    N = wl["N"]
    shapes = log_uniform_shapes(wl["count"], wl["lo"], wl["hi"], wl["seed"])
    probs, tensors = [], []
    flops = 0.0
    for i, (m, n, k) in enumerate(shapes):
        m, n, k = int(m), int(n), int(k)
        s = wl["seed"] + 7919 * i + 1000003 * rank + seed_offset
        A = paper_matrix_device(m, k, wl["phi"], s, torch.complex128)
        B = paper_matrix_device(k, n, wl["phi"], s + 1, torch.complex128)
        C = torch.zeros((n, m), dtype=torch.complex128, device="cuda")
        tensors.append((A, B, C))
        probs.append(dict(transa="N", transb="N", m=m, n=n, k=k, A=A.data_ptr(), lda=m, B=B.data_ptr(), ldb=k,
                          C=C.data_ptr(), ldc=m))
        flops += 8.0 * m * n * k
    st, plan = emu.emu_grouped_create(False, emu.GroupedArgs(probs, N), 0)
    emu.check(st, "emu_grouped_create")
    stream = torch.cuda.current_stream()
    try:
        for _ in range(warmup):
            emu.check(emu.emu_grouped_run(plan, stream), "run")
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in evs:
            a.record()
            emu.check(emu.emu_grouped_run(plan, stream), "run")
            b.record()
        torch.cuda.synchronize()
        times = [a.elapsed_time(b) for a, b in evs]
        phase_runs = [emu.emu_grouped_phase_times(plan, stream)[1] for _ in range(3)]
        phases = {nm: statistics.mean(r[i] for r in phase_runs)
                  for i, nm in enumerate(["exponents", "split", "residue_gemm", "crt"])}
        rec = {"problems": wl["count"], "mnk_range": [wl["lo"], wl["hi"]], "num_moduli": N, "phi": wl["phi"],
               "flops": flops, "replay_ms_median": statistics.median(times), "replay_ms_mean": statistics.mean(times),
               "tflops": flops / (statistics.median(times) * 1e-3) * 1e-12, "phases_ms": phases,
               "gemm_flops": 6.0 * N * sum(float(m) * n * k for m, n, k in shapes),
               "tile_n": emu.emu_grouped_tile(plan), "graph_kernels_per_replay": emu.emu_grouped_kernels(plan),
               "status": emu.STATUS_NAMES.get(emu.emu_stream_status(stream), "?")}
        if with_loop:
            def loop():
                for (m, n, k), (A, B, C) in zip(shapes, tensors):
                    s2 = emu.emu_zgemm("N", "N", int(m), int(n), int(k), 1.0, A.data_ptr(), int(m), B.data_ptr(),
                                       int(k), 0.0, C.data_ptr(), int(m), N, stream)
                    if s2 != emu.EMU_OK:
                        raise emu.EmuError(s2, "emu_zgemm")
            loop()
            torch.cuda.synchronize()
            la, lb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            la.record()
            loop()
            lb.record()
            torch.cuda.synchronize()
            lms = la.elapsed_time(lb)
            rec["plain_loop"] = {"ms": lms, "tflops": flops / (lms * 1e-3) * 1e-12,
                                 "speedup_of_grouped": lms / rec["replay_ms_median"], "launches": 10 * len(shapes)}
        return plan, rec
    except Exception:
        emu.emu_grouped_destroy(plan)
        raise


def plain_emulation(emu, torch, A, B, wl, C_ref):
    """The unfused pipeline of the paper's design on the same GPU: our exponent and
    split kernels (int8 planes), 3N cuBLAS INT8 GEMMs (torch._int_mm) with a
    separate mod pass, then our CRT kernel.  Timed once.  C_ref is a snapshot of
    the fused emulation's output, which the result must equal bit for bit."""
    C, pms = plain_emulation_run(emu, torch, A, B, wl)
    same = bool(torch.equal(torch.view_as_real(C), torch.view_as_real(C_ref)))
    m, n, k = wl["m"], wl["n"], wl["k"]
    return {"ms": pms, "tflops": 8.0 * m * n * k / (pms * 1e-3) * 1e-12,
            "int8_gemm": "cuBLASLt via torch._int_mm, 3N launches + torch mod pass",
            "bitexact_vs_fused": same}


def plain_emulation_run(emu, torch, A, B, wl):
    """One timed run of the unfused pipeline; returns (C, ms).  A is stored (k, m)
    and B (n, k), column-major op(A) = A.t() and op(B) = B.t() as in the bench."""
    m, n, k, N = wl["m"], wl["n"], wl["k"], wl["N"]
    single = wl["single"]
    kpad = (k + 63) // 64 * 64
    ldr = (m + 15) // 16 * 16
    st = emu.emu_plan_info(N)
    moduli = st[1]
    x = torch.empty(m, dtype=torch.int16, device="cuda")
    y = torch.empty(n, dtype=torch.int16, device="cuda")
    pa = torch.empty((3 * N, m, kpad), dtype=torch.int8, device="cuda")
    pb = torch.empty((3 * N, n, kpad), dtype=torch.int8, device="cuda")
    res = torch.empty((3 * N, n, ldr), dtype=torch.int8, device="cuda")
    C = torch.empty((n, m), dtype=torch.complex64 if single else torch.complex128, device="cuda")

    def run():
        emu.check(emu.emu_stage_exponents(single, "N", "N", m, n, k, A.data_ptr(), m, B.data_ptr(), k, N,
                                          x.data_ptr(), y.data_ptr()), "exp")
        emu.check(emu.emu_stage_split(single, "N", "N", m, n, k, A.data_ptr(), m, B.data_ptr(), k, N,
                                      x.data_ptr(), y.data_ptr(), 0, kpad, pa.data_ptr(), pb.data_ptr()), "split")
        for j in range(3 * N):
            p = moduli[j // 3]
            prod = torch._int_mm(pa[j], pb[j].t())                  # m x n int32
            r = torch.remainder(prod, p)
            r = torch.where(2 * r >= p, r - p, r).to(torch.int8)
            res[j, :, :m].copy_(r.t())
        emu.check(emu.emu_stage_crt(single, m, n, N, res.data_ptr(), ldr, x.data_ptr(), y.data_ptr(), 1.0, 0.0,
                                    C.data_ptr(), m), "crt")

    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    run()
    b.record()
    torch.cuda.synchronize()
    pms = a.elapsed_time(b)
    del pa, pb, res
    return C, pms


if __name__ == "__main__":
    sys.exit(main())
