// Internal definitions shared by the library's translation units.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/ozaki2_emu.h"

namespace emu {

constexpr int kMaxModuli = EMU_MAX_MODULI;
constexpr int kMaxLimbs = 6;        // 32-bit limbs of the CRT accumulator (P < 2^191)
constexpr int kPow2Table = 128;     // 2^s mod p for s in [0, 128)
constexpr int kSumFracBits = 15;    // row sums use ceil(|t| 2^15), Section III-B reading
constexpr int16_t kExpNonfinite = EMU_EXP_NONFINITE;

// Per-N constants of Algorithm 1 Steps I-II and of the exact CRT, computed on
// the host (plan.cpp) and passed to kernels by value.
struct Plan {
  int N;                                  // number of moduli
  int L;                                  // 32-bit limbs of the CRT accumulator
  int R0;                                 // offset making the CRT quotient non-negative
  int sX;                                 // X = (P-1) 2^27 ~= Xtop * 2^sX (floor)
  uint64_t Xtop;
  int p[kMaxModuli];                      // moduli
  uint32_t barrett[kMaxModuli];           // floor(2^32 / p)
  uint32_t two32[kMaxModuli];             // 2^32 mod p
  float qp[kMaxModuli];                   // q_l / p_l rounded to float
  uint32_t w[kMaxModuli][kMaxLimbs];      // w_l = (P/p_l) q_l, little endian
  uint32_t negP[kMaxLimbs];               // 2^(32L) - P
  uint32_t K[kMaxLimbs];                  // R0*P - 128*sum_l w_l  (mod 2^(32L))
  uint8_t pow2[kMaxModuli][kPow2Table];   // 2^s mod p_l
};

// Host: build (and cache) the plan of N moduli; nullptr when N is out of range.
const Plan* get_plan(int N);
int plan_exponent(const Plan& pl, uint64_t S);

// Device status word helpers (api.cu).
unsigned int* device_status_ptr();

// Launchers (one per translation unit).
cudaError_t launch_exponents(bool single, const void* X, int64_t rows, int64_t k,
                             int64_t rs, int64_t hs, const Plan& pl, int16_t* xout,
                             void* scratch, cudaStream_t st);
size_t exponents_scratch_bytes(int64_t rows);

cudaError_t launch_split(bool single, bool conj, const void* X, int64_t rows, int64_t k,
                         int64_t rs, int64_t hs, const Plan& pl, const int16_t* xexp,
                         bool fp16, int64_t kpad, void* planes, cudaStream_t st);

cudaError_t launch_gemm_i8(int64_t m, int64_t n, int64_t kpad, const Plan& pl,
                           const int8_t* planesA, const int8_t* planesB, int8_t* res,
                           int64_t ldr, cudaStream_t st);

cudaError_t launch_gemm_f16(int64_t m, int64_t n, int64_t kpad, const Plan& pl,
                            const void* planesA, const void* planesB, int8_t* res,
                            int64_t ldr, int chunk_k, unsigned int* status, cudaStream_t st);

cudaError_t launch_crt(bool single, int64_t m, int64_t n, const Plan& pl,
                       const int8_t* res, int64_t ldr, const int16_t* x, const int16_t* y,
                       double ar, double ai, double br, double bi,
                       void* C, int64_t ldc, cudaStream_t st);

cudaError_t launch_bounded_wait_selftest(int64_t limit_cycles, unsigned int* status,
                                         cudaStream_t st);

// Launch accounting (api.cu): launchers report each kernel they enqueue.
void count_launches(int n);

inline int64_t round_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

}  // namespace emu
