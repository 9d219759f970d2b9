"""CPU reference of the moduli-selection MLP and of its input features.

Oracle (test infrastructure only).  The paper selects the number of moduli
from empirical accuracy bands (Section IV-A); the learned selector is an
addition: a fully connected network that, from features of the inputs and
the requested accuracy, estimates for each N = 4..24 the probability that N
moduli meet that accuracy.

Network (float64 here, float32 on the GPU):
    h1 = relu(W1 x + b1)      W1: 64 x 39
    h2 = relu(W2 h1 + b2)     W2: 64 x 64
    z  = W3 h2 + b3           W3: 21 x 64    (logits, z_t for N = 4 + t)
Loss: mean over the batch of sum_t BCE(sigmoid(z_t), y_t), written in the
stable form max(z, 0) - z y + log(1 + exp(-|z|)).
Optimiser: Adam (Kingma & Ba 2015) with bias correction.

Parameter vector layout (float32 on the GPU): W1 (row major), b1, W2, b2, W3, b3.

Features of one problem (op(A) m x k, op(B) k x n, complex):
    [0:16]  fraction of the 2mk real entries of A-hat whose exponent span
            d = e_i - ilogb|a_ih| (nonzero entries) falls in bin min(d, 15);
            zero entries count in bin 15
    [16:32] the same for the 2kn entries of B-hat (columns)
    [32:34] mean and max over rows of L_i = 0.5 log2(max(S_i, 1) 2^-30), S_i the
            quantised sum of squares of the exponent phase (Section III-B reading)
    [34:36] the same over columns of B-hat
    [36]    log2(k) / 17
    [37]    -log10(target) / 16
    [38]    1 for complex64 inputs, 0 for complex128
"""
import math

import numpy as np

N_IN, N_H, N_OUT = 39, 64, 21
N_MIN = 4
SHAPES = [(N_H, N_IN), (N_H,), (N_H, N_H), (N_H,), (N_OUT, N_H), (N_OUT,)]


def n_params():
    return sum(int(np.prod(s)) for s in SHAPES)


def unpack(theta):
    out, o = [], 0
    for s in SHAPES:
        c = int(np.prod(s))
        out.append(np.asarray(theta[o:o + c], dtype=np.float64).reshape(s))
        o += c
    return out


def pack(parts):
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in parts])


def forward(theta, X):
    """X: batch x 39.  Returns (logits, cache)."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    a1 = X @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    z = h2 @ W3.T + b3
    return z, (X, a1, h1, a2, h2)


def loss(z, Y):
    z = np.asarray(z, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    per = np.maximum(z, 0.0) - z * Y + np.log1p(np.exp(-np.abs(z)))
    return float(per.sum() / z.shape[0])


def backward(theta, cache, z, Y):
    """Gradient of loss(z, Y) with respect to the parameter vector."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    X, a1, h1, a2, h2 = cache
    B = z.shape[0]
    dz = (1.0 / (1.0 + np.exp(-z)) - np.asarray(Y, dtype=np.float64)) / B
    gW3 = dz.T @ h2
    gb3 = dz.sum(axis=0)
    dh2 = dz @ W3
    da2 = dh2 * (a2 > 0)
    gW2 = da2.T @ h1
    gb2 = da2.sum(axis=0)
    dh1 = da2 @ W2
    da1 = dh1 * (a1 > 0)
    gW1 = da1.T @ X
    gb1 = da1.sum(axis=0)
    return pack([gW1, gb1, gW2, gb2, gW3, gb3])


def adam_step(theta, grad, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (t counts from 1).  Returns (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def choose(z, threshold=0.99):
    """Smallest N such that every N' >= N has predicted probability >= threshold,
    or None (fallback to the a priori rule)."""
    p = 1.0 / (1.0 + np.exp(-np.asarray(z, dtype=np.float64)))
    ok = p >= threshold
    best = None
    for t in range(N_OUT - 1, -1, -1):
        if not ok[t]:
            break
        best = N_MIN + t
    return best


# ------------------------------------------------------------------ features
def _span_hist(V):
    """16-bin histogram of exponent spans over the rows of V (real entries)."""
    V = np.asarray(V, dtype=np.float64)
    cnt = np.zeros(16, dtype=np.int64)
    for r in range(V.shape[0]):
        v = np.abs(V[r])
        nz = v != 0
        if not np.any(nz):
            cnt[15] += v.size
            continue
        e = np.frexp(v[nz])[1] - 1
        d = np.minimum(e.max() - e, 15)
        cnt += np.bincount(d, minlength=16)
        cnt[15] += int((~nz).sum())
    return cnt


def _L_stats(S_list):
    L = [0.5 * math.log2(max(int(S), 1) * 2.0 ** -30) for S in S_list]
    return float(np.mean(L)), float(np.max(L))


def features(A, B, target, single=False, N_for_sums=14):
    """Feature vector of op(A) (m x k) and op(B) (k x n); see the module docstring."""
    from .moduli import Plan
    from .scaling import col_vectors, row_vectors, vector_exponents
    A = np.asarray(A)
    B = np.asarray(B)
    m, k = A.shape
    n = B.shape[1]
    RA, CB = row_vectors(A), col_vectors(B)
    ha, hb = _span_hist(RA), _span_hist(CB)
    P = Plan(N_for_sums).P
    _, _, Sa, _, _ = vector_exponents(RA, P)
    _, _, Sb, _, _ = vector_exponents(CB, P)
    f = np.zeros(N_IN)
    f[0:16] = ha / max(2 * m * k, 1)
    f[16:32] = hb / max(2 * k * n, 1)
    f[32], f[33] = _L_stats(Sa)
    f[34], f[35] = _L_stats(Sb)
    f[36] = math.log2(max(k, 1)) / 17.0
    f[37] = -math.log10(target) / 16.0
    f[38] = 1.0 if single else 0.0
    return f
