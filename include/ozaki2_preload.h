/*
 * ozaki2_preload.h -- the LD_PRELOAD interposer libozaki2emu_preload.so.
 *
 * The paper's library is activated by adding it to LD_PRELOAD, after which an
 * application's cuBLAS GEMM calls run through the emulation with no change
 * to the application (Section III-D).  libozaki2emu_preload.so defines these
 * cuBLAS entry points with cuBLAS's own signatures (cublas_api.h, cublas.h):
 *   cublasSgemm_v2, cublasDgemm_v2, cublasCgemm_v2, cublasZgemm_v2,
 *   cublasSgemm_v2_64, cublasDgemm_v2_64, cublasCgemm_v2_64, cublasZgemm_v2_64,
 *   cublasGemmEx, and the legacy cublasSgemm, cublasDgemm, cublasCgemm,
 *   cublasZgemm with cublasSetKernelStream.
 * A call runs as emu_sgemm / emu_dgemm / emu_cgemm / emu_zgemm on the handle's
 * stream (legacy calls: the stream last given to cublasSetKernelStream) when
 *   - transa and transb are N, T or C, 0 <= k <= 2^17, no size is negative;
 *   - for cublasGemmEx, A, B and C have one type among CUDA_R_32F, CUDA_R_64F,
 *     CUDA_C_32F, CUDA_C_64F and the compute type is CUBLAS_COMPUTE_32F(_PEDANTIC)
 *     for the 32-bit types or CUBLAS_COMPUTE_64F(_PEDANTIC) for the 64-bit ones;
 *   - min(m, n, k) >= OZAKI2_EMU_MIN_DIM (default 1) and OZAKI2_EMU_DISABLE is
 *     unset, empty or "0";
 *   - the emulation accepts it (returns EMU_OK).
 * Otherwise the call goes, unchanged, to the same routine of the cuBLAS loaded
 * after the interposer.  alpha and beta in device pointer mode are copied to
 * the host on the handle's stream, which is then synchronised.
 *
 * Environment: OZAKI2_EMU_MODULI_Z / _C / _D / _S = N per element type
 * (defaults 15, 8, 16, 8); OZAKI2_EMU_TOL = a normalised accuracy target for
 * ZGEMM and CGEMM (N chosen per call by emu_zgemm_tol / emu_cgemm_tol);
 * OZAKI2_EMU_VERBOSE = 1 prints a line on the first emulated call of each routine.
 */
#ifndef OZAKI2_PRELOAD_H
#define OZAKI2_PRELOAD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Calls of routine r seen so far in this process: r = 0 Sgemm, 1 Dgemm,
 * 2 Cgemm, 3 Zgemm (the _v2 and _v2_64 forms), 4 GemmEx, 5 the legacy
 * routines; emulated != 0 counts the calls the emulation ran, 0 those that
 * went to cuBLAS.  Out-of-range r returns 0.  Host only. */
uint64_t ozaki2_preload_calls(int r, int emulated);

#ifdef __cplusplus
}
#endif

#endif /* OZAKI2_PRELOAD_H */
