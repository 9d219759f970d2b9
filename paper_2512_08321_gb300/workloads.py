"""Seeded synthetic inputs shaped like the paper's test matrices.

This module holds no arithmetic of the emulation; it only draws inputs, and it
is the one module that both the CUDA tests/bench and the CPU oracle's callers
share.

Section IV-A draws the real and imaginary parts of every entry independently
as (rand - 0.5) * exp(randn * phi), with rand uniform on (0, 1] and randn
standard normal; phi widens the exponent range.  Draws come from numpy's
counter-based Philox generator keyed by the seed.  Matrices are returned in
column-major (Fortran) order, the BLAS layout of the library's entry points.
"""
import numpy as np


def paper_matrix(rows, cols, phi, seed, dtype=np.complex128):
    """rows x cols complex matrix, Re/Im = (U(0,1] - 0.5) * exp(phi * N(0,1))."""
    rng = np.random.Generator(np.random.Philox(seed))
    parts = []
    for _ in range(2):
        u = 1.0 - rng.random((rows, cols))          # (0, 1]
        g = rng.standard_normal((rows, cols))
        parts.append((u - 0.5) * np.exp(g * phi))
    out = np.empty((rows, cols), dtype=np.complex128, order="F")
    out.real = parts[0]
    out.imag = parts[1]
    return np.asfortranarray(out.astype(dtype))


def log_uniform_shapes(count, lo, hi, seed):
    """count (m, n, k) triples drawn log-uniformly in [lo, hi] (integers)."""
    rng = np.random.Generator(np.random.Philox(seed))
    v = np.exp(rng.uniform(np.log(lo), np.log(hi + 1), size=(count, 3)))
    return np.clip(np.floor(v).astype(np.int64), lo, hi)


def paper_matrix_device(rows, cols, phi, seed, dtype, device="cuda"):
    """Same distribution as paper_matrix, drawn on the GPU (torch Philox).

    Returns the column-major rows x cols matrix as a C-contiguous
    (cols x rows) torch tensor, i.e. leading dimension `rows`.
    """
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    single = dtype in (np.complex64, "complex64", torch.complex64)
    real_t = torch.float32 if single else torch.float64
    parts = []
    for _ in range(2):
        u = 1.0 - torch.rand((cols, rows), generator=g, device=device, dtype=real_t)
        n = torch.randn((cols, rows), generator=g, device=device, dtype=real_t)
        parts.append((u - 0.5) * torch.exp(n * phi))
    return torch.complex(parts[0], parts[1])


def paper_matrix_real(rows, cols, phi, seed, dtype=np.float64):
    """rows x cols real matrix, entries (U(0,1] - 0.5) * exp(phi * N(0,1)),
    column-major."""
    rng = np.random.Generator(np.random.Philox(seed))
    u = 1.0 - rng.random((rows, cols))
    g = rng.standard_normal((rows, cols))
    return np.asfortranarray(((u - 0.5) * np.exp(g * phi)).astype(dtype))


def paper_matrix_real_device(rows, cols, phi, seed, dtype, device="cuda"):
    """Same distribution as paper_matrix_real, drawn on the GPU; returns the
    column-major rows x cols matrix as a C-contiguous (cols x rows) tensor."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    single = dtype in (np.float32, "float32", torch.float32)
    real_t = torch.float32 if single else torch.float64
    u = 1.0 - torch.rand((cols, rows), generator=g, device=device, dtype=real_t)
    n = torch.randn((cols, rows), generator=g, device=device, dtype=real_t)
    return (u - 0.5) * torch.exp(n * phi)
