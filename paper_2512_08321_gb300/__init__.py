"""GB300-native Ozaki-II emulation of ZGEMM/CGEMM (complex GEMM via the CRT)."""
