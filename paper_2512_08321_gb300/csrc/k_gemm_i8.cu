// K3 (INT8 engine): residue products on the INT8 tensor path of sm_103a,
// warp-level mma.sync.m16n8k32 s8 x s8 -> s32 (Algorithm 1 Steps V-iii/iv).
//
// For job j = 3l + c (c: D, E or F of eq. karatsuba; real input: j = l) and
// output (row, col):
//   res[j][col][row] = mod(sum_h A_j[row][h] B_j[col][h], p_l)
// INT32 accumulation is exact for k <= 2^17 (Section II).  Both operands are
// K-major int8 planes ([rows][kpad]); the output is int8 with `row`
// contiguous so the CRT phase reads it coalesced.
//
// Tiling: 64 x 64 output tile per block, BK = 64, 4 warps of 32 x 32, two
// cp.async stages.  Shared rows are padded to 80 bytes so the fragment loads
// (4 bytes per lane at row lane/4, column 4*(lane%4)) are bank-conflict free.
#include "emu_internal.h"

namespace emu {
namespace {

constexpr int BM = 64, BN = 64, BK = 64;
constexpr int kRowPad = 80;          // bytes per shared row
constexpr int kThreads = 128;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool pred) {
  const unsigned int s = static_cast<unsigned int>(__cvta_generic_to_shared(smem));
  const int n = pred ? 16 : 0;       // zero-fill when out of range
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

__device__ __forceinline__ void mma_s8(int* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ int sym_mod32(int v, uint32_t p, uint32_t bar) {
  const uint32_t u = static_cast<uint32_t>(v < 0 ? -v : v);
  const uint32_t q = __umulhi(u, bar);
  uint32_t r = u - q * p;
  if (r >= p) r -= p;
  int s = static_cast<int>(r);
  if (v < 0 && s) s = static_cast<int>(p) - s;
  if (2 * s >= static_cast<int>(p)) s -= static_cast<int>(p);
  return s;
}

__global__ void __launch_bounds__(kThreads) gemm_i8_kernel(int64_t m, int64_t n, int64_t kpad,
                                                           const __grid_constant__ Plan pl,
                                                           const int8_t* __restrict__ PA,
                                                           const int8_t* __restrict__ PB,
                                                           int8_t* __restrict__ res, int64_t ldr, int ppm) {
  __shared__ __align__(16) int8_t sA[2][BM][kRowPad];
  __shared__ __align__(16) int8_t sB[2][BN][kRowPad];
  __shared__ __align__(16) int8_t sOut[BN][BM + 16];

  const int job = blockIdx.z;
  const int l = job / ppm;
  const uint32_t p = static_cast<uint32_t>(pl.p[l]);
  const uint32_t bar = pl.barrett[l];
  const int64_t row0 = static_cast<int64_t>(blockIdx.x) * BM;
  const int64_t col0 = static_cast<int64_t>(blockIdx.y) * BN;
  const int8_t* A = PA + static_cast<int64_t>(job) * m * kpad;
  const int8_t* B = PB + static_cast<int64_t>(job) * n * kpad;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = (warp & 1) * 32, wn = (warp >> 1) * 32;
  const int g = lane >> 2, tg = lane & 3;

  int acc[2][4][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0;

  auto load_stage = [&](int s, int64_t k0) {
    // 64 rows x 64 bytes per operand = 256 chunks of 16 B; 2 per thread each
#pragma unroll
    for (int it = 0; it < 2; ++it) {
      const int c = tid + it * kThreads;
      const int rr = c >> 2, cc = (c & 3) * 16;
      const int64_t ra = row0 + rr, rb = col0 + rr;
      cp_async16(&sA[s][rr][cc], A + (ra < m ? ra : 0) * kpad + k0 + cc, ra < m);
      cp_async16(&sB[s][rr][cc], B + (rb < n ? rb : 0) * kpad + k0 + cc, rb < n);
    }
    cp_async_commit();
  };

  const int64_t nk = kpad / BK;
  if (nk > 0) load_stage(0, 0);
  for (int64_t kb = 0; kb < nk; ++kb) {
    const int s = static_cast<int>(kb & 1);
    if (kb + 1 < nk) {
      load_stage(s ^ 1, (kb + 1) * BK);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; kk += 32) {
      uint32_t af[2][4], bf[4][2];
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const int r = wm + a * 16 + g;
        af[a][0] = *reinterpret_cast<const uint32_t*>(&sA[s][r][kk + tg * 4]);
        af[a][1] = *reinterpret_cast<const uint32_t*>(&sA[s][r + 8][kk + tg * 4]);
        af[a][2] = *reinterpret_cast<const uint32_t*>(&sA[s][r][kk + 16 + tg * 4]);
        af[a][3] = *reinterpret_cast<const uint32_t*>(&sA[s][r + 8][kk + 16 + tg * 4]);
      }
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int c = wn + b * 8 + g;
        bf[b][0] = *reinterpret_cast<const uint32_t*>(&sB[s][c][kk + tg * 4]);
        bf[b][1] = *reinterpret_cast<const uint32_t*>(&sB[s][c][kk + 16 + tg * 4]);
      }
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) mma_s8(acc[a][b], af[a], bf[b]);
    }
    __syncthreads();
  }

  // epilogue: mod p -> int8, staged as [col][row] for coalesced stores
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int r = wm + a * 16 + g, c = wn + b * 8 + tg * 2;
      sOut[c][r] = static_cast<int8_t>(sym_mod32(acc[a][b][0], p, bar));
      sOut[c + 1][r] = static_cast<int8_t>(sym_mod32(acc[a][b][1], p, bar));
      sOut[c][r + 8] = static_cast<int8_t>(sym_mod32(acc[a][b][2], p, bar));
      sOut[c + 1][r + 8] = static_cast<int8_t>(sym_mod32(acc[a][b][3], p, bar));
    }
  __syncthreads();
  int8_t* out = res + static_cast<int64_t>(job) * n * ldr;
  // 64 cols x 64 rows = 256 chunks of 16 bytes
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const int c = tid + it * kThreads;
    const int cc = c >> 2, rr = (c & 3) * 16;
    const int64_t col = col0 + cc, row = row0 + rr;
    if (col < n && row < ldr)
      *reinterpret_cast<uint4*>(out + col * ldr + row) = *reinterpret_cast<const uint4*>(&sOut[cc][rr]);
  }
}

}  // namespace

cudaError_t launch_gemm_i8(int64_t m, int64_t n, int64_t kpad, const Plan& pl,
                           const int8_t* planesA, const int8_t* planesB, int8_t* res, int64_t ldr,
                           cudaStream_t st, int ppm) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  if (kpad % BK || ldr % 16 || (ppm != 1 && ppm != 3)) return cudaErrorInvalidValue;
  dim3 grid(static_cast<unsigned int>((m + BM - 1) / BM), static_cast<unsigned int>((n + BN - 1) / BN),
            static_cast<unsigned int>(ppm * pl.N));
  gemm_i8_kernel<<<grid, kThreads, 0, st>>>(m, n, kpad, pl, planesA, planesB, res, ldr, ppm);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace emu
