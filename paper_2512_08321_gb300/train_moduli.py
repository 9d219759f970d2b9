"""Train the moduli-selection network on data the emulator generates.

For each synthetic problem (the paper's generator, Section IV-A, with phi in
[0, 4] and square or rectangular shapes up to 4096) the emulated GEMM runs for
every N = 4..24; its normalised error is measured over all entries against
the N = 24 result (whose own error is far below every target).  The label
for target T and moduli count N is 1 when N and every larger count meet T
(with a safety factor).  The network is trained on the GPU with the
library's forward/backward/Adam kernels, full batch.  The trained parameters
are written to moduli_mlp.json beside this file.

    python -m paper_2512_08321_gb300.train_moduli [--problems 240] [--steps 6000] [--out path]
"""
import argparse
import json
import math
import os
import time

import numpy as np
import torch

from . import emu
from .workloads import paper_matrix_device

TARGETS = (1e-6, 1e-10, 1e-15)
N_MIN, N_MAX = 4, 24
SAFETY = 0.5          # a label counts N as meeting T only when its error is <= SAFETY * T
HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_OUT = os.path.join(HERE, "moduli_mlp.json")


def training_problems(count, seed):
    """(m, n, k, phi) of the training set: mostly rectangular m, n in [32, 1024],
    k in [64, 4096]; one in eight square in [512, 4096]."""
    rng = np.random.Generator(np.random.Philox(seed))
    out = []
    for i in range(count):
        phi = float(rng.uniform(0.0, 4.0))
        if i % 8 == 7:
            s = int(np.exp(rng.uniform(np.log(512), np.log(4096))))
            m = n = k = s
        else:
            m = int(np.exp(rng.uniform(np.log(32), np.log(1024))))
            n = int(np.exp(rng.uniform(np.log(32), np.log(1024))))
            k = int(np.exp(rng.uniform(np.log(64), np.log(4096))))
        out.append((m, n, k, phi))
    return out


def normalised_error(C, R, bound):
    d = torch.maximum((C.real - R.real).abs(), (C.imag - R.imag).abs())
    return float((d / bound).max())


def problem_rows(m, n, k, phi, seed):
    """Features (per target) and the error of every N for one problem."""
    A = paper_matrix_device(m, k, phi, seed, torch.complex128)           # storage (k, m)
    B = paper_matrix_device(k, n, phi, seed + 1, torch.complex128)       # storage (n, k)
    C = torch.zeros((n, m), dtype=torch.complex128, device="cuda")

    def run(N, out):
        st = emu.emu_zgemm("N", "N", m, n, k, 1.0, A.data_ptr(), m, B.data_ptr(), k, 0.0, out.data_ptr(), m, N)
        emu.check(st, "emu_zgemm")

    R = torch.zeros_like(C)
    run(N_MAX, R)
    absA = (A.real.abs() + A.imag.abs()).t().float()        # m x k
    absB = (B.real.abs() + B.imag.abs()).t().float()        # k x n
    bound = (absA @ absB).t().double()                      # n x m like C's storage
    bound = torch.where(bound > 0, bound, torch.ones_like(bound))
    errs = []
    for N in range(N_MIN, N_MAX + 1):
        run(N, C)
        errs.append(normalised_error(C, R, bound))
    feats = []
    f = torch.zeros(64, dtype=torch.float32, device="cuda")
    for T in TARGETS:
        emu.check(emu.emu_moduli_features(False, "N", "N", m, n, k, A.data_ptr(), m, B.data_ptr(), k, T,
                                          f.data_ptr()), "features")
        feats.append(f[:39].cpu().numpy().copy())
    return feats, errs


def labels(errs, T):
    """y_t = 1 when N = 4 + t and every larger N meet SAFETY * T."""
    y = np.zeros(len(errs), dtype=np.float32)
    ok = True
    for t in range(len(errs) - 1, -1, -1):
        ok = ok and errs[t] <= SAFETY * T
        y[t] = 1.0 if ok else 0.0
    return y


def init_params(seed):
    rng = np.random.Generator(np.random.Philox(seed))
    shapes = [(64, 39), (64,), (64, 64), (64,), (21, 64), (21,)]
    parts = []
    for s in shapes:
        if len(s) == 2:
            parts.append(rng.standard_normal(s) * math.sqrt(2.0 / s[1]))
        else:
            parts.append(np.zeros(s))
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


def train(X, Y, steps, seed, lr=3e-3, log=None):
    P = emu.emu_mlp_param_count()
    th = torch.from_numpy(init_params(seed)).cuda()
    assert th.numel() == P
    g = torch.zeros(P, dtype=torch.float32, device="cuda")
    m = torch.zeros_like(g)
    v = torch.zeros_like(g)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
    Yd = torch.from_numpy(np.ascontiguousarray(Y, dtype=np.float32)).cuda()
    B = X.shape[0]
    for step in range(1, steps + 1):
        rate = lr if step <= steps * 2 // 3 else lr / 3
        emu.check(emu.emu_mlp_backward(th.data_ptr(), Xd.data_ptr(), Yd.data_ptr(), B, g.data_ptr(),
                                       loss.data_ptr()), "backward")
        emu.check(emu.emu_mlp_adam(th.data_ptr(), g.data_ptr(), m.data_ptr(), v.data_ptr(), step, rate), "adam")
        if log is not None and (step % 500 == 0 or step == 1):
            torch.cuda.synchronize()
            log.append((step, float(loss.item())))
    torch.cuda.synchronize()
    return th.cpu().numpy()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--problems", type=int, default=240)
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--seed", type=int, default=20251213)
    ap.add_argument("--out", default=DEFAULT_OUT)
    ap.add_argument("--dataset-out", default=None, help="also save features/errors (npz)")
    args = ap.parse_args()
    emu.lib()
    t0 = time.time()
    probs = training_problems(args.problems, args.seed)
    X, Y, E, meta = [], [], [], []
    for i, (m, n, k, phi) in enumerate(probs):
        feats, errs = problem_rows(m, n, k, phi, args.seed * 7 + 1000 * i)
        for T, f in zip(TARGETS, feats):
            X.append(f)
            Y.append(labels(errs, T))
        E.append(errs)
        meta.append((m, n, k, phi))
    X = np.array(X)
    Y = np.array(Y)
    t1 = time.time()
    log = []
    theta = train(X, Y, args.steps, args.seed, log=log)
    t2 = time.time()
    # training-set agreement: chosen N vs the smallest N that met SAFETY * T
    from .emu import lib as _lib  # noqa: F401
    Z = np.zeros((X.shape[0], 21), dtype=np.float32)
    Xd = torch.from_numpy(X.astype(np.float32)).cuda()
    Zd = torch.zeros((X.shape[0], 21), dtype=torch.float32, device="cuda")
    thd = torch.from_numpy(theta).cuda()
    emu.check(emu.emu_mlp_forward(thd.data_ptr(), Xd.data_ptr(), X.shape[0], Zd.data_ptr()), "forward")
    Z = Zd.cpu().numpy()
    p = 1.0 / (1.0 + np.exp(-Z))
    under = over = exact = 0
    for row, y in zip(p, Y):
        ok = row >= 0.99
        chosen = None
        for t in range(20, -1, -1):
            if not ok[t]:
                break
            chosen = N_MIN + t
        true_n = N_MIN + int(np.argmax(y)) if y.any() else None
        if chosen is None or true_n is None:
            continue
        exact += chosen == true_n
        under += chosen < true_n
        over += chosen > true_n
    summary = {"problems": len(probs), "samples": int(X.shape[0]), "steps": args.steps,
               "data_seconds": t1 - t0, "train_seconds": t2 - t1, "loss_log": log,
               "train_choice": {"exact": int(exact), "under": int(under), "over": int(over)},
               "targets": TARGETS, "safety": SAFETY, "threshold": 0.99}
    with open(args.out, "w") as f:
        json.dump({"params": [float(v) for v in theta], "train": summary}, f)
    if args.dataset_out:
        np.savez(args.dataset_out, X=X, Y=Y, E=np.array(E), meta=np.array(meta))
    print(json.dumps(summary))


if __name__ == "__main__":
    main()
