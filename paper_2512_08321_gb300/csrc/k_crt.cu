// K4: CRT reconstruction, inverse scaling and alpha/beta (Algorithm 1 Steps
// V-iv..VI with the Karatsuba combination of Section III-A).
//
// Per output (i, j), from the int8 residues D_l, E_l, F_l of job 3l+c:
//   E'_R,l = mod(D_l - E_l, p_l),  E'_I,l = mod(F_l - D_l - E_l, p_l)       (eq. karatsuba)
//   c' = mod(sum_l (P/p_l) q_l E'_l, P)                                     (Steps V-v, V-vi)
//   C_ij = alpha RN(c' 2^-(x_i + y_j)) + beta C_ij                          (Step VI)
// The CRT sum only needs each E'_l modulo p_l, so the exact path feeds the
// unreduced D_l - E_l and F_l - D_l - E_l (offset to be non-negative) and
// never forms the symmetric remainders; the result is the same c'.
//
// The paper evaluates the CRT sum in two double-precision parts and the final
// reduction in double-double (Section II, eq. CRTaccumulation; Section IV-A).
// GB300 has 1/62 of its FP32 rate in FP64, so here the CRT is exact integer
// arithmetic instead: with u_l = E'_l + 128 in [0, 255] and the quotient
// r = round(sum_l E'_l q_l / p_l) (an fp32 estimate is exact because
// |c'| <= (P-1)/8 keeps S/P within 1/8 of an integer),
//   c' = sum_l w_l u_l + (r + R0)(2^(32L) - P) + K   (mod 2^(32L)),
// accumulated limb by limb in 64-bit registers and carried once.  The result
// is the exact c', then rounded once to nearest-even binary64 by integer
// operations (subnormals included).  complex64 output rounds that binary64
// value (after alpha/beta) once more to binary32.
//
// Real input (DGEMM/SGEMM emulation) has one residue plane per modulus and
// one output component (crt_real_kernel).
//
// Thread mapping: 4 consecutive rows i of one column j; the residue bytes of
// those rows are one 32-bit word per job.
#include <algorithm>

#include "crt_common.cuh"

namespace emu {
namespace {

constexpr int kThreads = 128;

__device__ __forceinline__ int sym_small(int v, int p) {   // |v| <= 3 p / 2 + 1
  if (2 * v >= p) v -= p;
  if (2 * v >= p) v -= p;
  if (2 * v < -p) v += p;
  if (2 * v < -p) v += p;
  return v;
}

// Finish one part.  acc holds sum_l u_l w_l limb by limb (unnormalised), u_l
// the residues offset to be non-negative by `off` (the offset constant koff =
// R0 P - off sum_l w_l).  The quotient r = round(sum_l E'_l w_l / P) is
// estimated in float from the limbs, sum_t acc_t 2^(32 t) / P - off sum_l q_l /
// p_l (every term below 765 N: the float error stays far under the 1/8 margin
// of condition (cond)); then c' = acc + koff + (r + R0)(2^(32 L) - P) mod
// 2^(32 L), carried once, (accurate mode) range-fixed and rounded.
template <int L, bool ROBUST>
__device__ __forceinline__ double finish(const uint64_t (&acc)[L], const uint32_t* koff, float foff, const Plan& pl,
                                         int e2) {
  float est = -foff;
#pragma unroll
  for (int t = 0; t < L; ++t) est = fmaf(__ull2float_rn(acc[t]), pl.qinv[t], est);
  const uint32_t rq = static_cast<uint32_t>(static_cast<int>(rintf(est)) + pl.R0);
  uint32_t c[L];
  uint64_t carry = 0;
#pragma unroll
  for (int t = 0; t < L; ++t) {
    const uint64_t v = acc[t] + koff[t] + static_cast<uint64_t>(rq) * pl.negP[t] + carry;
    c[t] = static_cast<uint32_t>(v);
    carry = v >> 32;
  }
  if constexpr (ROBUST) fix_range<L>(c, pl);
  return round_exact<L>(c, e2);
}

// Residues of the block's rows for every job, staged in shared memory with
// asynchronous 16-byte copies issued all at once (the rows of one job are
// contiguous and the block start is 16-byte aligned), so the loads of all
// moduli are in flight together instead of one modulus at a time.
// smem[job * (kThreads * R) + r]; returns after the copies have landed.
template <int R>
__device__ __forceinline__ void stage_residues(int8_t* smem, const int8_t* __restrict__ blk, int64_t job_stride,
                                               int jobs, int64_t rows_left) {
  constexpr int kRows = kThreads * R;
  const int rows = static_cast<int>(rows_left < kRows ? rows_left : kRows);   // a multiple of 16
  const int per_job = rows / 16;
  const uint32_t s0 = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  for (int c = threadIdx.x; c < jobs * per_job; c += kThreads) {
    const int job = c / per_job, q = c - job * per_job;
    const int8_t* g = blk + job * job_stride + 16 * q;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s0 + job * kRows + 16 * q), "l"(g));
  }
  asm volatile("cp.async.commit_group;\n");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
}

template <int R>
__device__ __forceinline__ uint32_t smem_word(const int8_t* smem, int job, int r) {
  const int8_t* p = smem + job * (kThreads * R) + r;
  if constexpr (R == 4) return *reinterpret_cast<const uint32_t*>(p);
  else if constexpr (R == 2) return *reinterpret_cast<const unsigned short*>(p);
  else return static_cast<uint8_t>(*p);
}

template <int L, bool SINGLE, int kRowsPerThread, bool ROBUST = false>
__device__ __forceinline__ void crt_block(int64_t m, int64_t n, const Plan& pl, const int8_t* __restrict__ res,
                                          int64_t ldr, const int16_t* __restrict__ x, const int16_t* __restrict__ y,
                                          double ar, double ai, double br, double bi, int flags,
                                          void* __restrict__ Cv, int64_t ldc, int64_t j, int64_t iblock) {
  const int64_t i0 = (iblock * kThreads + threadIdx.x) * kRowsPerThread;
  const int N = pl.N;
  const int64_t job_stride = n * ldr;
  const int64_t row0 = iblock * kThreads * kRowsPerThread;
  extern __shared__ __align__(16) int8_t crt_smem[];
  // rows below round_up(m, 16) only: res may be a block of rows of a taller residue set
  stage_residues<kRowsPerThread>(crt_smem, res + j * ldr + row0, job_stride, 3 * N, (m + 15) / 16 * 16 - row0);
  const bool active = i0 < m;
  const int rr = threadIdx.x * kRowsPerThread;

  // exact limb accumulators for the real and imaginary parts of the thread's rows
  uint64_t accR[kRowsPerThread][L], accI[kRowsPerThread][L];
  if (active) {
#pragma unroll
  for (int q = 0; q < kRowsPerThread; ++q) {
#pragma unroll
    for (int t = 0; t < L; ++t) accR[q][t] = accI[q][t] = 0ull;
  }
  for (int l = 0; l < N; ++l) {
    uint32_t w[L];
#pragma unroll
    for (int t = 0; t < L; ++t) w[t] = pl.w[l][t];
    // bytes as D + 128, E + 128, F + 128 (unsigned)
    const uint32_t wd = smem_word<kRowsPerThread>(crt_smem, 3 * l, rr) ^ 0x80808080u;
    const uint32_t we = smem_word<kRowsPerThread>(crt_smem, 3 * l + 1, rr) ^ 0x80808080u;
    const uint32_t wf = smem_word<kRowsPerThread>(crt_smem, 3 * l + 2, rr) ^ 0x80808080u;
#pragma unroll
    for (int q = 0; q < kRowsPerThread; ++q) {
      const int d = static_cast<int>((wd >> (8 * q)) & 0xFFu);
      const int e = static_cast<int>((we >> (8 * q)) & 0xFFu);
      const int f = static_cast<int>((wf >> (8 * q)) & 0xFFu);
      const int vr = d - e;                        // D - E == E'_R,l (mod p_l), in [-255, 255]
      const int vi = f - d - e + 128;              // F - D - E == E'_I,l (mod p_l), in [-382, 383]
      const uint32_t ur = static_cast<uint32_t>(vr + 255), ui = static_cast<uint32_t>(vi + 382);
#pragma unroll
      for (int t = 0; t < L; ++t) {
        accR[q][t] = mad_wide(ur, w[t], accR[q][t]);
        accI[q][t] = mad_wide(ui, w[t], accI[q][t]);
      }
    }
  }
  }
  // the residues are consumed: the buffer now holds the unscaled outputs, which
  // are then written row-coalesced (thread t: rows t, t + 128, ...), so every
  // store instruction of a warp covers one contiguous run of C -- also when C
  // is host memory reached over the CPU-GPU link
  __syncthreads();
  double2* so = reinterpret_cast<double2*>(crt_smem);
  const int yj = y[j];
  if (active) {
#pragma unroll
    for (int q = 0; q < kRowsPerThread; ++q) {
      const int64_t i = i0 + q;
      if (i >= m) break;
      const int xi = x[i];
      double orr, oi;
      if (xi == kExpNonfinite || yj == kExpNonfinite) {
        orr = oi = __longlong_as_double(0x7FF8000000000000ll);
      } else {
        const int e2 = -(xi + yj);
        orr = finish<L, ROBUST>(accR[q], pl.KR, pl.off255, pl, e2);
        oi = finish<L, ROBUST>(accI[q], pl.KI, pl.off382, pl, e2);
      }
      so[rr + q] = make_double2(orr, oi);
    }
  }
  __syncthreads();
  const bool plain = (flags & kCrtPlain) != 0;
  const bool use_beta = (flags & kCrtBeta) != 0;
#pragma unroll
  for (int q = 0; q < kRowsPerThread; ++q) {
    const int r = q * kThreads + threadIdx.x;
    const int64_t i = row0 + r;
    if (i >= m) break;
    double orr = so[r].x, oi = so[r].y;
    const int64_t ci = j * ldc + i;
    if (!plain) {
      double tr = __fma_rn(ar, orr, -__dmul_rn(ai, oi));
      double ti = __fma_rn(ar, oi, __dmul_rn(ai, orr));
      if (use_beta) {
        double cr, cim;
        if (SINGLE) {
          const float2 cv = static_cast<const float2*>(Cv)[ci];
          cr = cv.x;
          cim = cv.y;
        } else {
          const double2 cv = static_cast<const double2*>(Cv)[ci];
          cr = cv.x;
          cim = cv.y;
        }
        tr = __fma_rn(br, cr, __fma_rn(-bi, cim, tr));
        ti = __fma_rn(br, cim, __fma_rn(bi, cr, ti));
      }
      orr = tr;
      oi = ti;
    }
    if (SINGLE)
      static_cast<float2*>(Cv)[ci] = make_float2(__double2float_rn(orr), __double2float_rn(oi));
    else
      static_cast<double2*>(Cv)[ci] = make_double2(orr, oi);
  }
}


// Real input (DGEMM/SGEMM emulation): E'_l is the residue of job l itself; one
// accumulator per row.  alpha/beta: t = RN(alpha o), then fma(beta, c, t).
template <int L, bool SINGLE, int kRowsPerThread, bool ROBUST>
__device__ __forceinline__ void crt_block_real(int64_t m, int64_t n, const Plan& pl, const int8_t* __restrict__ res,
                                               int64_t ldr, const int16_t* __restrict__ x,
                                               const int16_t* __restrict__ y, double ar, double br, int flags,
                                               void* __restrict__ Cv, int64_t ldc, int64_t j, int64_t iblock) {
  const int64_t i0 = (iblock * kThreads + threadIdx.x) * kRowsPerThread;
  const int N = pl.N;
  const int64_t job_stride = n * ldr;
  const int64_t row0 = iblock * kThreads * kRowsPerThread;
  extern __shared__ __align__(16) int8_t crt_smem[];
  stage_residues<kRowsPerThread>(crt_smem, res + j * ldr + row0, job_stride, N, (m + 15) / 16 * 16 - row0);
  const bool active = i0 < m;
  const int rr = threadIdx.x * kRowsPerThread;
  uint64_t acc[kRowsPerThread][L];
  if (active) {
#pragma unroll
  for (int q = 0; q < kRowsPerThread; ++q) {
#pragma unroll
    for (int t = 0; t < L; ++t) acc[q][t] = 0ull;
  }
  for (int l = 0; l < N; ++l) {
    uint32_t w[L];
#pragma unroll
    for (int t = 0; t < L; ++t) w[t] = pl.w[l][t];
    const uint32_t wv = smem_word<kRowsPerThread>(crt_smem, l, rr) ^ 0x80808080u;   // bytes as E' + 128
#pragma unroll
    for (int q = 0; q < kRowsPerThread; ++q) {
      const uint32_t u = (wv >> (8 * q)) & 0xFFu;
#pragma unroll
      for (int t = 0; t < L; ++t) acc[q][t] = mad_wide(u, w[t], acc[q][t]);
    }
  }
  }
  // outputs through shared memory, then written row-coalesced (as in crt_block)
  __syncthreads();
  double* so = reinterpret_cast<double*>(crt_smem);
  const int yj = y[j];
  if (active) {
#pragma unroll
    for (int q = 0; q < kRowsPerThread; ++q) {
      const int64_t i = i0 + q;
      if (i >= m) break;
      const int xi = x[i];
      so[rr + q] = (xi == kExpNonfinite || yj == kExpNonfinite) ? __longlong_as_double(0x7FF8000000000000ll)
                                                                : finish<L, ROBUST>(acc[q], pl.K, pl.off128, pl, -(xi + yj));
    }
  }
  __syncthreads();
  const bool plain = (flags & kCrtPlain) != 0;
#pragma unroll
  for (int q = 0; q < kRowsPerThread; ++q) {
    const int r = q * kThreads + threadIdx.x;
    const int64_t i = row0 + r;
    if (i >= m) break;
    double o = so[r];
    const int64_t ci = j * ldc + i;
    if (!plain) {
      double t = __dmul_rn(ar, o);
      if (flags & kCrtBeta) t = __fma_rn(br, SINGLE ? static_cast<double>(static_cast<const float*>(Cv)[ci])
                                             : static_cast<const double*>(Cv)[ci], t);
      o = t;
    }
    if (SINGLE) static_cast<float*>(Cv)[ci] = __double2float_rn(o);
    else static_cast<double*>(Cv)[ci] = o;
  }
}

template <int L, bool SINGLE, int R, bool ROBUST>
__global__ void __launch_bounds__(kThreads) crt_real_kernel(int64_t m, int64_t n, const __grid_constant__ Plan pl,
                                                            const int8_t* __restrict__ res, int64_t ldr,
                                                            const int16_t* __restrict__ x,
                                                            const int16_t* __restrict__ y, double ar, double br,
                                                            int flags, void* __restrict__ Cv, int64_t ldc) {
  crt_block_real<L, SINGLE, R, ROBUST>(m, n, pl, res, ldr, x, y, ar, br, flags, Cv, ldc, blockIdx.x, blockIdx.y);
}

template <int L, bool SINGLE, int R, bool ROBUST>
__global__ void __launch_bounds__(kThreads) crt_kernel(int64_t m, int64_t n,
                                                       const __grid_constant__ Plan pl,
                                                       const int8_t* __restrict__ res, int64_t ldr,
                                                       const int16_t* __restrict__ x,
                                                       const int16_t* __restrict__ y, double ar,
                                                       double ai, double br, double bi, int flags,
                                                       void* __restrict__ Cv, int64_t ldc) {
  crt_block<L, SINGLE, R, ROBUST>(m, n, pl, res, ldr, x, y, ar, ai, br, bi, flags, Cv, ldc, blockIdx.x,
                                  blockIdx.y);
}

// one launch over every problem of a grouped call: blocks are (column, row block) of each problem.
// Two rows per thread (256-row blocks): for the grouped workloads' small m, 512-row blocks would
// leave half the threads idle (log-uniform m in [64, 2048]: 1.50x padding against 1.22x).
constexpr int kGroupedCrtRows = 2;

template <int L, bool SINGLE>
__global__ void __launch_bounds__(kThreads) crt_grouped(const CrtProb* __restrict__ probs, int nprob,
                                                        const __grid_constant__ Plan pl) {
  int lo = 0, hi = nprob - 1;
  const long long b = blockIdx.x;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (probs[mid].block_begin <= b) lo = mid; else hi = mid - 1;
  }
  const CrtProb& c = probs[lo];
  const long long local = b - c.block_begin;
  crt_block<L, SINGLE, kGroupedCrtRows>(c.m, c.n, pl, c.res, c.ldr, c.x, c.y, c.ar, c.ai, c.br, c.bi, c.flags, c.C,
                                        c.ldc, local / c.iblocks, local % c.iblocks);
}

template <int L, int R, bool ROBUST>
void launch_lrr(bool single, bool real, dim3 grid, int64_t m, int64_t n, const Plan& pl, const int8_t* res,
                int64_t ldr, const int16_t* x, const int16_t* y, double ar, double ai, double br, double bi, void* C,
                int64_t ldc, cudaStream_t st) {
  // staged residues, then the unscaled outputs (16 or 8 bytes a row)
  const size_t sm = std::max(static_cast<size_t>(real ? 1 : 3) * pl.N * kThreads * R,
                             static_cast<size_t>(real ? 8 : 16) * kThreads * R);
  const int fl = crt_flags(ar, real ? 0.0 : ai, br, real ? 0.0 : bi);
  if (real) {
    if (single)
      crt_real_kernel<L, true, R, ROBUST><<<grid, kThreads, sm, st>>>(m, n, pl, res, ldr, x, y, ar, br, fl, C, ldc);
    else
      crt_real_kernel<L, false, R, ROBUST><<<grid, kThreads, sm, st>>>(m, n, pl, res, ldr, x, y, ar, br, fl, C, ldc);
  } else if (single) {
    max_shared_carveout(crt_kernel<L, true, R, ROBUST>);
    crt_kernel<L, true, R, ROBUST><<<grid, kThreads, sm, st>>>(m, n, pl, res, ldr, x, y, ar, ai, br, bi, fl, C, ldc);
  } else {
    max_shared_carveout(crt_kernel<L, false, R, ROBUST>);
    crt_kernel<L, false, R, ROBUST><<<grid, kThreads, sm, st>>>(m, n, pl, res, ldr, x, y, ar, ai, br, bi, fl, C, ldc);
  }
}

template <int L, int R>
cudaError_t launch_lr(bool single, int64_t m, int64_t n, const Plan& pl, const int8_t* res, int64_t ldr,
                      const int16_t* x, const int16_t* y, double ar, double ai, double br, double bi, void* C,
                      int64_t ldc, cudaStream_t st, bool real, bool robust) {
  const int64_t per_block = static_cast<int64_t>(kThreads) * R;
  if ((m + per_block - 1) / per_block > 65535) return cudaErrorInvalidValue;
  dim3 grid(static_cast<unsigned int>(n), static_cast<unsigned int>((m + per_block - 1) / per_block));
  if (robust) launch_lrr<L, R, true>(single, real, grid, m, n, pl, res, ldr, x, y, ar, ai, br, bi, C, ldc, st);
  else launch_lrr<L, R, false>(single, real, grid, m, n, pl, res, ldr, x, y, ar, ai, br, bi, C, ldc, st);
  count_launches(1);
  return cudaGetLastError();
}

template <int L>
cudaError_t launch_l(bool single, int64_t m, int64_t n, const Plan& pl, const int8_t* res,
                     int64_t ldr, const int16_t* x, const int16_t* y, double ar, double ai,
                     double br, double bi, void* C, int64_t ldc, cudaStream_t st, int rows, bool real,
                     bool robust) {
  switch (rows) {
    case 1: return launch_lr<L, 1>(single, m, n, pl, res, ldr, x, y, ar, ai, br, bi, C, ldc, st, real, robust);
    case 2: return launch_lr<L, 2>(single, m, n, pl, res, ldr, x, y, ar, ai, br, bi, C, ldc, st, real, robust);
    default: return launch_lr<L, 4>(single, m, n, pl, res, ldr, x, y, ar, ai, br, bi, C, ldc, st, real, robust);
  }
}

// ---------------------------------------------------------------------------
// The paper's floating-point reconstruction (Section II, eq. CRTaccumulation;
// Section IV-A): S1 = sum s_l1 E'_l (exact on the common grid), S2 = sum s_l2 E'_l
// (fma, ascending l), then c' = mod(S1 + S2, P) in double-double for complex128
// and S - P rint(S/P) in double for complex64.  Every step is an explicit IEEE
// intrinsic, in the same order as the oracle, so results are bitwise stable.
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
  s = __dadd_rn(a, b);
  const double bb = __dsub_rn(s, a);
  e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
}

// c' from the accumulated sums: mod(S1 + S2, P) in double-double (complex128).
__device__ __forceinline__ double fp_reduce_z(double S1, double S2, const Plan& pl) {
  const double r = rint(__ddiv_rn(__dadd_rn(S1, S2), pl.Ph));
  const double ph = __dmul_rn(r, pl.Ph);
  const double pe = __fma_rn(r, pl.Ph, -ph);
  double hi, lo;
  two_sum(S1, -ph, hi, lo);
  lo = __dadd_rn(__fma_rn(-r, pl.Pl, __dsub_rn(lo, pe)), S2);
  return __dadd_rn(hi, lo);
}

// c' = S - P rint(S / P) in double (complex64).
__device__ __forceinline__ double fp_reduce_c(double S, const Plan& pl) {
  const double r = rint(__ddiv_rn(S, pl.Ph));
  return __fma_rn(-r, pl.Ph, S);
}

// RN(c 2^e2) of a double c by integer operations (subnormal results round once).
__device__ __forceinline__ double scale_double(double c, int e2) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(c));
  const int ex = static_cast<int>((b >> 52) & 0x7FF);
  if (ex == 0x7FF) return c;
  const unsigned long long fr = b & 0xFFFFFFFFFFFFFull;
  const unsigned long long mm = ex ? (fr | (1ull << 52)) : fr;
  if (mm == 0) return c;
  const int elsb = ex ? ex - 1075 : -1074;
  uint32_t limbs[3];
  limbs[0] = static_cast<uint32_t>(mm);
  limbs[1] = static_cast<uint32_t>(mm >> 32);
  limbs[2] = 0;
  if (b >> 63) {  // two's complement negate for round_limbs
    uint32_t carry = 1;
    for (int t = 0; t < 3; ++t) {
      const uint64_t v = static_cast<uint64_t>(~limbs[t]) + carry;
      limbs[t] = static_cast<uint32_t>(v);
      carry = static_cast<uint32_t>(v >> 32);
    }
  }
  return round_limbs<3>(limbs, elsb + e2);
}

template <bool SINGLE>
__global__ void __launch_bounds__(kThreads) crt_fp_kernel(int64_t m, int64_t n, const __grid_constant__ Plan pl,
                                                          const int8_t* __restrict__ res, int64_t ldr,
                                                          const int16_t* __restrict__ x, const int16_t* __restrict__ y,
                                                          double ar, double ai, double br, double bi,
                                                          void* __restrict__ Cv, int64_t ldc) {
  const int64_t j = blockIdx.x;
  const int64_t i = static_cast<int64_t>(blockIdx.y) * kThreads + threadIdx.x;
  if (i >= m) return;
  const int N = pl.N;
  const int64_t js = n * ldr;
  const int8_t* base = res + j * ldr + i;
  // S1 = sum s_l1 E'_l (exact), S2 = sum s_l2 E'_l (fma), ascending l, both parts at once
  double s1r = 0.0, s2r = 0.0, s1i = 0.0, s2i = 0.0;
  for (int l = 0; l < N; ++l) {
    const int p = pl.p[l];
    const int d = base[(3 * l) * js], e = base[(3 * l + 1) * js], f = base[(3 * l + 2) * js];
    const double er = static_cast<double>(sym_small(d - e, p));
    const double ei = static_cast<double>(sym_small(f - d - e, p));
    if (SINGLE) {
      s1r = __fma_rn(pl.wd[l], er, s1r);
      s1i = __fma_rn(pl.wd[l], ei, s1i);
    } else {
      s1r = __dadd_rn(s1r, __dmul_rn(pl.s1[l], er));
      s1i = __dadd_rn(s1i, __dmul_rn(pl.s1[l], ei));
      s2r = __fma_rn(pl.s2[l], er, s2r);
      s2i = __fma_rn(pl.s2[l], ei, s2i);
    }
  }
  const int xi = x[i], yj = y[j];
  double orr, oi;
  if (xi == kExpNonfinite || yj == kExpNonfinite) {
    orr = oi = __longlong_as_double(0x7FF8000000000000ll);
  } else {
    const int e2 = -(xi + yj);
    orr = scale_double(SINGLE ? fp_reduce_c(s1r, pl) : fp_reduce_z(s1r, s2r, pl), e2);
    oi = scale_double(SINGLE ? fp_reduce_c(s1i, pl) : fp_reduce_z(s1i, s2i, pl), e2);
  }
  const int64_t ci = j * ldc + i;
  if (!(ar == 1.0 && ai == 0.0 && br == 0.0 && bi == 0.0)) {
    double tr = __fma_rn(ar, orr, -__dmul_rn(ai, oi));
    double ti = __fma_rn(ar, oi, __dmul_rn(ai, orr));
    if (!(br == 0.0 && bi == 0.0)) {
      double cr, cim;
      if (SINGLE) {
        const float2 cv = static_cast<const float2*>(Cv)[ci];
        cr = cv.x;
        cim = cv.y;
      } else {
        const double2 cv = static_cast<const double2*>(Cv)[ci];
        cr = cv.x;
        cim = cv.y;
      }
      tr = __fma_rn(br, cr, __fma_rn(-bi, cim, tr));
      ti = __fma_rn(br, cim, __fma_rn(bi, cr, ti));
    }
    orr = tr;
    oi = ti;
  }
  if (SINGLE)
    static_cast<float2*>(Cv)[ci] = make_float2(__double2float_rn(orr), __double2float_rn(oi));
  else
    static_cast<double2*>(Cv)[ci] = make_double2(orr, oi);
}

// The paper's floating-point CRT for real input: the DGEMM form (S1 + S2 and
// the double-double reduction) for binary64 output, one double sum for binary32.
template <bool SINGLE>
__global__ void __launch_bounds__(kThreads) crt_fp_real_kernel(int64_t m, int64_t n, const __grid_constant__ Plan pl,
                                                               const int8_t* __restrict__ res, int64_t ldr,
                                                               const int16_t* __restrict__ x,
                                                               const int16_t* __restrict__ y, double ar, double br,
                                                               void* __restrict__ Cv, int64_t ldc) {
  const int64_t j = blockIdx.x;
  const int64_t i = static_cast<int64_t>(blockIdx.y) * kThreads + threadIdx.x;
  if (i >= m) return;
  const int N = pl.N;
  const int64_t js = n * ldr;
  const int8_t* base = res + j * ldr + i;
  double s1 = 0.0, s2 = 0.0;
  for (int l = 0; l < N; ++l) {
    const double e = static_cast<double>(base[l * js]);
    if (SINGLE) {
      s1 = __fma_rn(pl.wd[l], e, s1);
    } else {
      s1 = __dadd_rn(s1, __dmul_rn(pl.s1[l], e));
      s2 = __fma_rn(pl.s2[l], e, s2);
    }
  }
  const int xi = x[i], yj = y[j];
  double o;
  if (xi == kExpNonfinite || yj == kExpNonfinite) o = __longlong_as_double(0x7FF8000000000000ll);
  else o = scale_double(SINGLE ? fp_reduce_c(s1, pl) : fp_reduce_z(s1, s2, pl), -(xi + yj));
  const int64_t ci = j * ldc + i;
  if (!(ar == 1.0 && br == 0.0)) {
    double t = __dmul_rn(ar, o);
    if (br != 0.0) t = __fma_rn(br, SINGLE ? static_cast<double>(static_cast<const float*>(Cv)[ci])
                                           : static_cast<const double*>(Cv)[ci], t);
    o = t;
  }
  if (SINGLE) static_cast<float*>(Cv)[ci] = __double2float_rn(o);
  else static_cast<double*>(Cv)[ci] = o;
}

template <int L>
cudaError_t launch_grouped_l(bool single, const CrtProb* probs, int nprob, long long blocks, const Plan& pl,
                             cudaStream_t st) {
  const unsigned int gb = static_cast<unsigned int>(blocks);
  const size_t sm = std::max(static_cast<size_t>(3) * pl.N * kThreads * kGroupedCrtRows,   // residues, outputs
                             static_cast<size_t>(16) * kThreads * kGroupedCrtRows);
  if (single) crt_grouped<L, true><<<gb, kThreads, sm, st>>>(probs, nprob, pl);
  else crt_grouped<L, false><<<gb, kThreads, sm, st>>>(probs, nprob, pl);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace

long long crt_prob_blocks(CrtProb& c) {
  const int64_t per_block = static_cast<int64_t>(kThreads) * kGroupedCrtRows;
  c.iblocks = static_cast<int>((c.m + per_block - 1) / per_block);
  c.flags = crt_flags(c.ar, c.ai, c.br, c.bi);
  return static_cast<long long>(c.n) * c.iblocks;
}

cudaError_t launch_crt_grouped(bool single, const CrtProb* probs_dev, int nprob, long long blocks, const Plan& pl,
                               cudaStream_t st) {
  if (nprob <= 0 || blocks <= 0) return cudaSuccess;
  if (blocks > 2147483647LL) return cudaErrorInvalidValue;
  switch (pl.L) {
    case 1: return launch_grouped_l<1>(single, probs_dev, nprob, blocks, pl, st);
    case 2: return launch_grouped_l<2>(single, probs_dev, nprob, blocks, pl, st);
    case 3: return launch_grouped_l<3>(single, probs_dev, nprob, blocks, pl, st);
    case 4: return launch_grouped_l<4>(single, probs_dev, nprob, blocks, pl, st);
    case 5: return launch_grouped_l<5>(single, probs_dev, nprob, blocks, pl, st);
    case 6: return launch_grouped_l<6>(single, probs_dev, nprob, blocks, pl, st);
    default: return cudaErrorInvalidValue;
  }
}

int g_crt_mode = 0;

cudaError_t launch_crt_fp(bool single, int64_t m, int64_t n, const Plan& pl, const int8_t* res, int64_t ldr,
                          const int16_t* x, const int16_t* y, double ar, double ai, double br, double bi, void* C,
                          int64_t ldc, cudaStream_t st, bool real) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  if (n > 2147483647LL || (m + kThreads - 1) / kThreads > 65535) return cudaErrorInvalidValue;
  dim3 grid(static_cast<unsigned int>(n), static_cast<unsigned int>((m + kThreads - 1) / kThreads));
  if (real) {
    if (single) crt_fp_real_kernel<true><<<grid, kThreads, 0, st>>>(m, n, pl, res, ldr, x, y, ar, br, C, ldc);
    else crt_fp_real_kernel<false><<<grid, kThreads, 0, st>>>(m, n, pl, res, ldr, x, y, ar, br, C, ldc);
  } else if (single)
    crt_fp_kernel<true><<<grid, kThreads, 0, st>>>(m, n, pl, res, ldr, x, y, ar, ai, br, bi, C, ldc);
  else
    crt_fp_kernel<false><<<grid, kThreads, 0, st>>>(m, n, pl, res, ldr, x, y, ar, ai, br, bi, C, ldc);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_crt(bool single, int64_t m, int64_t n, const Plan& pl, const int8_t* res,
                       int64_t ldr, const int16_t* x, const int16_t* y, double ar, double ai,
                       double br, double bi, void* C, int64_t ldc, cudaStream_t st, int rows, bool real,
                       bool robust) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  if (ldr % 16 || m > ldr || n > 2147483647LL || (reinterpret_cast<uintptr_t>(res) & 15u))
    return cudaErrorInvalidValue;
  switch (pl.L) {
    case 1: return launch_l<1>(single, m, n, pl, res, ldr, x, y, ar, ai, br, bi, C, ldc, st, rows, real, robust);
    case 2: return launch_l<2>(single, m, n, pl, res, ldr, x, y, ar, ai, br, bi, C, ldc, st, rows, real, robust);
    case 3: return launch_l<3>(single, m, n, pl, res, ldr, x, y, ar, ai, br, bi, C, ldc, st, rows, real, robust);
    case 4: return launch_l<4>(single, m, n, pl, res, ldr, x, y, ar, ai, br, bi, C, ldc, st, rows, real, robust);
    case 5: return launch_l<5>(single, m, n, pl, res, ldr, x, y, ar, ai, br, bi, C, ldc, st, rows, real, robust);
    case 6: return launch_l<6>(single, m, n, pl, res, ldr, x, y, ar, ai, br, bi, C, ldc, st, rows, real, robust);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace emu
