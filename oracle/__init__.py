"""CPU oracle for the Ozaki-II emulation of complex matrix multiplication.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously-correct
restatement of the method in Python (standard library big integers and
fractions, plus numpy for exact small-integer and float64 work).  Only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import it.  The CUDA library never calls it and shares no code, table or
constant with it.

Modules
-------
``moduli``    Algorithm 1 Steps I-II: moduli, P, the inverses q_l, CRT weights.
``fp``        IEEE helpers written from their definitions: ilogb, correctly
              rounded binary64/binary32 conversion of exact values, an exact fma.
``scaling``   Section III-B fast-mode scaling vectors (eqs. mu-fast / nu-fast),
              evaluated exactly.
``emulate``   Algorithm 1 Steps IV-VI with the Karatsuba product of Section
              III-A: truncation, symmetric residues, residue products, mod-p,
              CRT reconstruction, inverse scaling, alpha/beta.
``exact``     Exact references that do not use the CRT: the scaled integer
              product A'B' by limb splitting, and the exact complex product AB
              (error-free transformations + math.fsum) for error metrics.
``metrics``   The Section IV-A maximum componentwise relative error and the
              |A||B|-normalised error.
"""
