"""Moduli and CRT constants (Algorithm 1, Steps I and II; Section II).

Oracle (test infrastructure only).

Step I asks for N pairwise-coprime moduli p_l <= 256 without listing them.
Reading used here: the greedy descending choice -- walk c = 256, 255, ... and
keep c when it is coprime to every modulus kept so far.  Step II asks for the
modular inverse q_l of P/p_l modulo p_l.  The CRT of Section II then rebuilds
C' = sum_l (P/p_l) q_l C'_l, congruent to A'B' modulo P.
"""
from math import gcd, prod

MAX_MODULUS = 256          # Algorithm 1 Step I: p_l <= 256
MIN_MODULI = 2
MAX_MODULI = 24


def choose_moduli(N):
    """Step I: the first N moduli of the greedy descending pairwise-coprime set."""
    if not (1 <= N <= 40):
        raise ValueError("number of moduli out of range")
    chosen = []
    c = MAX_MODULUS
    while len(chosen) < N:
        if c < 2:
            raise ValueError("ran out of moduli")
        if all(gcd(c, p) == 1 for p in chosen):
            chosen.append(c)
        c -= 1
    return chosen


def modinv(a, p):
    """Inverse of a modulo p by the extended Euclidean algorithm (textbook)."""
    r0, r1 = a % p, p
    s0, s1 = 1, 0
    while r1:
        qt = r0 // r1
        r0, r1 = r1, r0 - qt * r1
        s0, s1 = s1, s0 - qt * s1
    if r0 != 1:
        raise ValueError("not invertible")
    return s0 % p


class Plan:
    """Steps I-II for N moduli: p_l, P = prod p_l, q_l = (P/p_l)^-1 mod p_l,
    and the CRT weights w_l = (P/p_l) q_l of Section II."""

    def __init__(self, N, moduli=None):
        self.N = N
        self.p = list(moduli) if moduli is not None else choose_moduli(N)
        if len(self.p) != N:
            raise ValueError("moduli list length differs from N")
        self.P = prod(self.p)
        self.q = [modinv(self.P // pl, pl) for pl in self.p]
        self.w = [(self.P // pl) * ql for pl, ql in zip(self.p, self.q)]

    @property
    def log2P(self):
        from math import log2
        return log2(self.P)

    def __repr__(self):
        return f"Plan(N={self.N}, p={self.p})"
