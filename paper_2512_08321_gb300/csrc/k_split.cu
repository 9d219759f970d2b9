// K2: truncation and residue split (Algorithm 1 Steps IV and V-i/ii, with the
// Karatsuba sum of Section III-A).
//
// For every entry v = X(r, h) (complex; conjugated for op C) of a row r with
// scaling exponent x_r:
//   a'_R = trunc(Re v 2^x_r),  a'_I = trunc(Im v 2^x_r)            (Step IV)
//   plane 3l+0 = mod(a'_R, p_l), plane 3l+1 = mod(a'_I, p_l),
//   plane 3l+2 = mod(plane 3l+0 + plane 3l+1, p_l)                 (Step V-i, eq. karatsuba)
// mod is the symmetric remainder of Section II with ties rounded up, so every
// residue fits int8 (and is exact in fp16).  Everything is integer arithmetic:
// with v = +-m 2^elsb, a' = m 2^(elsb+x) when elsb+x >= 0 (residue
// (m mod p)(2^s mod p) mod p) and m >> -(elsb+x) otherwise.
//
// Output layout: planes[(3l+c) * rows * kpad + r * kpad + h]; h in [k, kpad)
// is zero.  One block handles 32 rows x 64 h: the tile is staged through
// shared memory so global reads are coalesced whichever of r or h is
// contiguous, and every thread then writes 8 consecutive h of one row.
#include <cuda_fp16.h>

#include "emu_internal.h"

namespace emu {
namespace {

constexpr int kTileR = 32;
constexpr int kTileH = 64;
constexpr int kThreads = 256;   // 8 warps: warp w owns h in [8w, 8w+8) of the tile
constexpr int kPerThread = 8;

__device__ __forceinline__ uint32_t mod32(uint32_t x, uint32_t p, uint32_t bar) {
  const uint32_t q = __umulhi(x, bar);
  uint32_t r = x - q * p;
  return r >= p ? r - p : r;
}

// Decoded magnitude of one real part: residue base value V (< 2^53), shift s
// (>= 0: multiply by 2^s; < 0: already shifted), sign.
struct Part {
  uint32_t lo, hi;
  int s;        // >= 0: a' = V 2^s, V = m; < 0 means a' = V (already truncated)
  bool neg;
  bool zero;
};

template <bool SINGLE>
__device__ __forceinline__ Part decode(uint64_t bits, int x) {
  Part pt;
  int ex;
  uint64_t m;
  int elsb;
  if (SINGLE) {
    const uint32_t b = static_cast<uint32_t>(bits);
    pt.neg = (b >> 31) != 0;
    ex = (b >> 23) & 0xFF;
    const uint32_t fr = b & 0x7FFFFFu;
    m = ex ? (fr | 0x800000u) : fr;
    elsb = ex ? ex - 150 : -149;
  } else {
    pt.neg = (bits >> 63) != 0;
    ex = static_cast<int>((bits >> 52) & 0x7FF);
    const uint64_t fr = bits & 0xFFFFFFFFFFFFFull;
    m = ex ? (fr | (1ull << 52)) : fr;
    elsb = ex ? ex - 1075 : -1074;
  }
  const int s = elsb + x;
  uint64_t V;
  if (s >= 0) {
    V = m;
    pt.s = s;
  } else {
    V = (-s >= 64) ? 0ull : (m >> (-s));
    pt.s = -1;
  }
  pt.zero = (V == 0);
  pt.lo = static_cast<uint32_t>(V);
  pt.hi = static_cast<uint32_t>(V >> 32);
  return pt;
}

// symmetric residue of one part modulo p (ties up)
__device__ __forceinline__ int residue(const Part& pt, uint32_t p, uint32_t bar, uint32_t two32,
                                       const uint8_t* pow2) {
  if (pt.zero) return 0;
  uint32_t r = mod32(pt.lo, p, bar);
  r = mod32(pt.hi * two32 + r, p, bar);
  // s < 128 whenever x comes from the exponent phase (|a'| < 2^(E+1)); the
  // mask only keeps a caller-supplied exponent inside the table
  if (pt.s >= 0) r = mod32(r * static_cast<uint32_t>(pow2[pt.s & (kPow2Table - 1)]), p, bar);
  int v = static_cast<int>(r);
  if (pt.neg && v) v = static_cast<int>(p) - v;
  if (2 * v >= static_cast<int>(p)) v -= static_cast<int>(p);
  return v;
}

__device__ __forceinline__ int sym_small(int v, int p) {   // |v| <= 256
  if (2 * v >= p) v -= p;
  if (2 * v < -p) v += p;
  return v;
}

template <typename T>
struct Store8;
template <>
struct Store8<int8_t> {
  __device__ static void put(int8_t* dst, const int* v) {
    uint2 w;
    w.x = (v[0] & 0xFF) | ((v[1] & 0xFF) << 8) | ((v[2] & 0xFF) << 16) | ((v[3] & 0xFF) << 24);
    w.y = (v[4] & 0xFF) | ((v[5] & 0xFF) << 8) | ((v[6] & 0xFF) << 16) | ((v[7] & 0xFF) << 24);
    *reinterpret_cast<uint2*>(dst) = w;
  }
};
template <>
struct Store8<__half> {
  __device__ static void put(__half* dst, const int* v) {
    uint4 w;
    __half2 h0 = __halves2half2(__int2half_rn(v[0]), __int2half_rn(v[1]));
    __half2 h1 = __halves2half2(__int2half_rn(v[2]), __int2half_rn(v[3]));
    __half2 h2 = __halves2half2(__int2half_rn(v[4]), __int2half_rn(v[5]));
    __half2 h3 = __halves2half2(__int2half_rn(v[6]), __int2half_rn(v[7]));
    w.x = *reinterpret_cast<uint32_t*>(&h0);
    w.y = *reinterpret_cast<uint32_t*>(&h1);
    w.z = *reinterpret_cast<uint32_t*>(&h2);
    w.w = *reinterpret_cast<uint32_t*>(&h3);
    *reinterpret_cast<uint4*>(dst) = w;
  }
};

template <bool SINGLE, bool ROWS_CONTIG, typename T>
__global__ void __launch_bounds__(kThreads) split_kernel(const void* __restrict__ Xv, int64_t rows,
                                                         int64_t k, int64_t rs, int64_t hs,
                                                         bool conj, const int16_t* __restrict__ xexp,
                                                         const __grid_constant__ Plan pl,
                                                         int64_t kpad, T* __restrict__ planes) {
  // raw bits of the tile, [h][r] with one element of padding per h-row
  __shared__ uint64_t tre[kTileH][kTileR + 1];
  __shared__ uint64_t tim[kTileH][kTileR + 1];
  __shared__ uint8_t pow2s[kMaxModuli][kPow2Table];

  const int tid = threadIdx.x;
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * kTileR;
  const int64_t h0 = static_cast<int64_t>(blockIdx.y) * kTileH;

  for (int i = tid; i < pl.N * kPow2Table; i += kThreads)
    pow2s[i / kPow2Table][i % kPow2Table] = pl.pow2[i / kPow2Table][i % kPow2Table];

  // load phase: 2048 elements, 8 per thread, coalesced along the contiguous index
#pragma unroll
  for (int it = 0; it < (kTileR * kTileH) / kThreads; ++it) {
    int rr, hh;
    if (ROWS_CONTIG) {
      rr = tid & 31;
      hh = (tid >> 5) + 8 * it;
    } else {
      hh = tid & 63;
      rr = (tid >> 6) + 4 * it;
    }
    const int64_t r = r0 + rr, h = h0 + hh;
    uint64_t bre = 0, bim = 0;
    if (r < rows && h < k) {
      const int64_t off = r * rs + h * hs;
      if (SINGLE) {
        const float2 v = static_cast<const float2*>(Xv)[off];
        bre = __float_as_uint(v.x);
        bim = __float_as_uint(conj ? -v.y : v.y);
      } else {
        const double2 v = static_cast<const double2*>(Xv)[off];
        bre = static_cast<uint64_t>(__double_as_longlong(v.x));
        bim = static_cast<uint64_t>(__double_as_longlong(conj ? -v.y : v.y));
      }
    }
    tre[hh][rr] = bre;
    tim[hh][rr] = bim;
  }
  __syncthreads();

  const int rr = tid & 31;
  const int hb = (tid >> 5) * kPerThread;
  const int64_t r = r0 + rr;
  if (r >= rows) return;
  const int x = xexp[r];
  const bool flagged = (x == kExpNonfinite);

  Part pre[kPerThread], pim[kPerThread];
#pragma unroll
  for (int j = 0; j < kPerThread; ++j) {
    uint64_t br = tre[hb + j][rr], bi = tim[hb + j][rr];
    // a flagged row, or a non-finite entry, contributes zeros
    const bool bad = flagged ||
                     (SINGLE ? (((br >> 23) & 0xFF) == 0xFF || ((bi >> 23) & 0xFF) == 0xFF)
                             : (((br >> 52) & 0x7FF) == 0x7FF || ((bi >> 52) & 0x7FF) == 0x7FF));
    if (bad) br = bi = 0;
    pre[j] = decode<SINGLE>(br, flagged ? 0 : x);
    pim[j] = decode<SINGLE>(bi, flagged ? 0 : x);
  }
  const int64_t plane_stride = rows * kpad;
  T* base = planes + r * kpad + h0 + hb;
  for (int l = 0; l < pl.N; ++l) {
    const uint32_t p = static_cast<uint32_t>(pl.p[l]);
    const uint32_t bar = pl.barrett[l], two32 = pl.two32[l];
    const uint8_t* pw = pow2s[l];
    int vr[kPerThread], vi[kPerThread], vs[kPerThread];
#pragma unroll
    for (int j = 0; j < kPerThread; ++j) {
      vr[j] = residue(pre[j], p, bar, two32, pw);
      vi[j] = residue(pim[j], p, bar, two32, pw);
      vs[j] = sym_small(vr[j] + vi[j], static_cast<int>(p));
    }
    T* dst = base + static_cast<int64_t>(3 * l) * plane_stride;
    Store8<T>::put(dst, vr);
    Store8<T>::put(dst + plane_stride, vi);
    Store8<T>::put(dst + 2 * plane_stride, vs);
  }
}

template <bool SINGLE, typename T>
cudaError_t launch_t(bool conj, const void* X, int64_t rows, int64_t k, int64_t rs, int64_t hs,
                     const Plan& pl, const int16_t* xexp, int64_t kpad, void* planes,
                     cudaStream_t st) {
  dim3 grid(static_cast<unsigned int>((rows + kTileR - 1) / kTileR),
            static_cast<unsigned int>(kpad / kTileH));
  if (rs == 1)
    split_kernel<SINGLE, true, T><<<grid, kThreads, 0, st>>>(X, rows, k, rs, hs, conj, xexp, pl,
                                                             kpad, static_cast<T*>(planes));
  else
    split_kernel<SINGLE, false, T><<<grid, kThreads, 0, st>>>(X, rows, k, rs, hs, conj, xexp, pl,
                                                              kpad, static_cast<T*>(planes));
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_split(bool single, bool conj, const void* X, int64_t rows, int64_t k,
                         int64_t rs, int64_t hs, const Plan& pl, const int16_t* xexp, bool fp16,
                         int64_t kpad, void* planes, cudaStream_t st) {
  if (rows <= 0 || kpad <= 0) return cudaSuccess;
  if (kpad % kTileH) return cudaErrorInvalidValue;
  if (single)
    return fp16 ? launch_t<true, __half>(conj, X, rows, k, rs, hs, pl, xexp, kpad, planes, st)
                : launch_t<true, int8_t>(conj, X, rows, k, rs, hs, pl, xexp, kpad, planes, st);
  return fp16 ? launch_t<false, __half>(conj, X, rows, k, rs, hs, pl, xexp, kpad, planes, st)
              : launch_t<false, int8_t>(conj, X, rows, k, rs, hs, pl, xexp, kpad, planes, st);
}

}  // namespace emu
