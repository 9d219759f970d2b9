"""The paper's performance model (Section III-C, fast and accurate modes).

Oracle (test infrastructure only); used to put measured phase times beside
the model.  b is the sustained memory bandwidth in B/s, p the INT8 matrix
engine throughput in op/s, c the correction term for arithmetic overhead in
memory-bound steps (Section III-C sets c = N in its heatmaps).

Fast mode, complex128 inputs:
  T = [((3N + 32 + c) k + 4)(m + n) + (16N + 16 + 2c) m n] / b + 6 N m n k / p
Fast mode, complex64 inputs:
  T = [((3N + 16 + c) k + 4)(m + n) + (16N + 8 + 2c) m n] / b + 6 N m n k / p
Accurate mode, complex128 / complex64:
  T = [((35 + 3N + c) k + 8)(m + n) + (16N + 40 + 2c) m n] / b + 6 (N+1) m n k / p
  T = [((19 + 3N + c) k + 8)(m + n) + (16N + 32 + 2c) m n] / b + 6 (N+1) m n k / p
Throughput is reported as 8 m n k / T (Section III-C).
"""


def model_time(m, n, k, N, b, p, c=None, dtype="z", mode="fast"):
    c = N if c is None else c
    if mode == "fast" and dtype == "z":
        mem = ((3 * N + 32 + c) * k + 4) * (m + n) + (16 * N + 16 + 2 * c) * m * n
        ops = 6 * N * m * n * k
    elif mode == "fast" and dtype == "c":
        mem = ((3 * N + 16 + c) * k + 4) * (m + n) + (16 * N + 8 + 2 * c) * m * n
        ops = 6 * N * m * n * k
    elif mode == "accurate" and dtype == "z":
        mem = ((35 + 3 * N + c) * k + 8) * (m + n) + (16 * N + 40 + 2 * c) * m * n
        ops = 6 * (N + 1) * m * n * k
    elif mode == "accurate" and dtype == "c":
        mem = ((19 + 3 * N + c) * k + 8) * (m + n) + (16 * N + 32 + 2 * c) * m * n
        ops = 6 * (N + 1) * m * n * k
    else:
        raise ValueError((mode, dtype))
    return mem / b + ops / p


def model_tflops(m, n, k, N, b, p, **kw):
    return 8.0 * m * n * k / model_time(m, n, k, N, b, p, **kw) * 1e-12
