// K2: truncation and residue split (Algorithm 1 Steps IV and V-i/ii, with the
// Karatsuba sum of Section III-A).
//
// For every entry v = X(r, h) (complex; conjugated for op C) of a row r with
// scaling exponent x_r:
//   a'_R = trunc(Re v 2^x_r),  a'_I = trunc(Im v 2^x_r)            (Step IV)
//   plane 3l+0 = mod(a'_R, p_l), plane 3l+1 = mod(a'_I, p_l),
//   plane 3l+2 = mod(plane 3l+0 + plane 3l+1, p_l)                 (Step V-i, eq. karatsuba)
// mod is the symmetric remainder of Section II with ties rounded up, so every
// residue fits int8 (and is exact in fp16).
//
// Arithmetic: a' (< 2^97) is formed exactly from the IEEE bits with integer
// shifts and cut once per entry into signed 13-bit chunks c_t (exact floats).
// Per modulus, a' == sum_t c_t w_t (mod p) with w_t = 2^(13t) mod p in
// [-128, 127]: every product is below 2^20 and the sum below 2^23, so the FP32
// sum is exact; one rint-based reduction and a symmetric fix-up give the
// residue.  The sums run as packed FP32 pairs (two entries of a row per
// instruction).
//
// Real input (DGEMM/SGEMM emulation) has one plane per modulus:
// plane l = mod(trunc(v 2^x_r), p_l).
//
// Output layout: planes[(3l+c) * rows * kpad + r * kpad + h] (real: plane l);
// h in [k, kpad) is zero.  A block handles 32 rows x 64 h: the tile goes through shared
// memory so global reads are coalesced whichever of r or h is contiguous;
// each thread then owns 4 consecutive h of one row, 16 threads per row, so a
// row of a block covers a whole 128-byte line of every fp16 plane.
#include <cuda_fp16.h>

#include <type_traits>

#include "emu_internal.h"

namespace emu {
namespace {

constexpr int kTileR = 32;
constexpr int kTileH = 32;     // accurate-mode bound planes
constexpr int kSplitH = 64;    // residue planes
constexpr int kThreads = 256;

template <int H>
struct TileSmem {
  uint64_t tre[kTileR][H + 1];     // raw bits of the tile, [r][h], one element of padding
  uint64_t tim[kTileR][H + 1];
};
using SplitSmem = TileSmem<kSplitH>;

// Signed 13-bit chunks of a' = trunc(v 2^x) (exact floats, least significant first).
template <bool SINGLE, int TC>
__device__ __forceinline__ void chunks(uint64_t bits, int x, int nchunk, float (&c)[TC]) {
  bool neg;
  int ex;
  uint64_t m;
  int elsb;
  if (SINGLE) {
    const uint32_t b = static_cast<uint32_t>(bits);
    neg = (b >> 31) != 0;
    ex = (b >> 23) & 0xFF;
    const uint32_t fr = b & 0x7FFFFFu;
    m = ex ? (fr | 0x800000u) : fr;
    elsb = ex ? ex - 150 : -149;
  } else {
    neg = (bits >> 63) != 0;
    ex = static_cast<int>((bits >> 52) & 0x7FF);
    const uint64_t fr = bits & 0xFFFFFFFFFFFFFull;
    m = ex ? (fr | (1ull << 52)) : fr;
    elsb = ex ? ex - 1075 : -1074;
  }
  const int s = elsb + x;                       // a' = m 2^s (s >= 0) or m >> -s
  uint64_t lo, hi;
  if (s >= 0) {
    // s < 44 whenever x comes from the exponent phase (|a'| < 2^(Emax+1) <= 2^97);
    // larger shifts only occur for caller-supplied exponents and saturate to zero
    lo = s < 64 ? (m << s) : 0ull;
    hi = s == 0 ? 0ull : (s < 64 ? (m >> (64 - s)) : (s < 128 ? (m << (s - 64)) : 0ull));
  } else {
    lo = (-s >= 64) ? 0ull : (m >> (-s));
    hi = 0ull;
  }
  const float sg = neg ? -1.0f : 1.0f;
#pragma unroll
  for (int t = 0; t < TC; ++t) {
    const int b = kChunkBits * t;
    uint32_t v;
    if (b + kChunkBits <= 64) v = static_cast<uint32_t>(lo >> b);
    else if (b >= 64) v = static_cast<uint32_t>(hi >> (b - 64));
    else v = static_cast<uint32_t>((lo >> b) | (hi << (64 - b)));
    v &= (1u << kChunkBits) - 1u;
    // exact int -> float for v < 2^23 through the bit pattern of 2^23 + v
    const float f = __int_as_float(static_cast<int>(0x4B000000u | v)) - 8388608.0f;
    c[t] = (t < nchunk) ? sg * f : 0.0f;
  }
}

// ---- packed FP32 pairs: one instruction for two lanes
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{.reg .b64 a2, b2, c2, d2;\n\tmov.b64 a2, {%2, %3};\n\tmov.b64 b2, {%4, %5};\n\t"
      "mov.b64 c2, {%6, %7};\n\tfma.rn.f32x2 d2, a2, b2, c2;\n\tmov.b64 {%0, %1}, d2;}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
  float2 d;
  asm("{.reg .b64 a2, b2, d2;\n\tmov.b64 a2, {%2, %3};\n\tmov.b64 b2, {%4, %5};\n\t"
      "mul.rn.f32x2 d2, a2, b2;\n\tmov.b64 {%0, %1}, d2;}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

// Symmetric residue (ties up) of the exact float integer z, |z| < 2^23;
// ph = p/2 (exact).
__device__ __forceinline__ float sym_mod_f(float z, float p, float ph, float inv_p) {
  float r = fmaf(-rintf(z * inv_p), p, z);      // exact; |r| <= p/2 + 1
  if (r >= ph) r -= p;
  if (r < -ph) r += p;
  return r;
}
__device__ __forceinline__ float sym_fix_f(float r, float p, float ph) {
  if (r >= ph) r -= p;
  if (r < -ph) r += p;
  return r;
}

// magic-number float -> int8 byte (|r| <= 128, exact integer r)
__device__ __forceinline__ uint32_t byte_of(float r) {
  return static_cast<uint32_t>(__float_as_int(r + 12582912.0f)) & 0xFFu;
}

// store E consecutive residues (exact small integers held as floats)
template <typename T, int E>
struct StoreE;
template <>
struct StoreE<int8_t, 4> {
  __device__ static void put(int8_t* dst, const float (&v)[4]) {
    *reinterpret_cast<uint32_t*>(dst) = byte_of(v[0]) | (byte_of(v[1]) << 8) | (byte_of(v[2]) << 16) |
                                        (byte_of(v[3]) << 24);
  }
};
template <>
struct StoreE<int8_t, 2> {
  __device__ static void put(int8_t* dst, const float (&v)[2]) {
    *reinterpret_cast<uint16_t*>(dst) = static_cast<uint16_t>(byte_of(v[0]) | (byte_of(v[1]) << 8));
  }
};
template <>
struct StoreE<__half, 4> {
  __device__ static void put(__half* dst, const float (&v)[4]) {
    __half2 a = __floats2half2_rn(v[0], v[1]);
    __half2 b = __floats2half2_rn(v[2], v[3]);
    *reinterpret_cast<uint2*>(dst) =
        make_uint2(*reinterpret_cast<uint32_t*>(&a), *reinterpret_cast<uint32_t*>(&b));
  }
};
template <>
struct StoreE<__half, 2> {
  __device__ static void put(__half* dst, const float (&v)[2]) {
    __half2 a = __floats2half2_rn(v[0], v[1]);
    *reinterpret_cast<uint32_t*>(dst) = *reinterpret_cast<uint32_t*>(&a);
  }
};

// NCH: the chunk count when known at compile time (0: pl.nchunk at run time).
template <bool SINGLE, bool ROWS_CONTIG, typename T, int kPerThread, bool R = false, int NCH = 0>
__device__ __forceinline__ void split_block(SplitSmem& sm, const void* __restrict__ Xv, int64_t rows, int64_t k,
                                            int64_t rs, int64_t hs, bool conj, const int16_t* __restrict__ xexp,
                                            const Plan& pl, int64_t kpad, T* __restrict__ planes, int64_t rtile,
                                            int64_t htile, int64_t prow) {
  // prow: rows between consecutive planes (a block of rows of a larger plane set)
  const int tid = threadIdx.x;
  const int64_t r0 = rtile * kTileR;
  const int64_t h0 = htile * kSplitH;

  // load phase: 2048 elements, 8 per thread, coalesced along the contiguous index
#pragma unroll
  for (int it = 0; it < (kTileR * kSplitH) / kThreads; ++it) {
    int rr, hh;
    if (ROWS_CONTIG) {
      rr = tid % kTileR;
      hh = tid / kTileR + (kThreads / kTileR) * it;
    } else {
      hh = tid % kSplitH;
      rr = tid / kSplitH + (kThreads / kSplitH) * it;
    }
    const int64_t r = r0 + rr, h = h0 + hh;
    uint64_t bre = 0, bim = 0;
    if (r < rows && h < k) {
      const int64_t off = r * rs + h * hs;
      if constexpr (R) {
        bre = SINGLE ? static_cast<uint64_t>(__float_as_uint(static_cast<const float*>(Xv)[off]))
                     : static_cast<uint64_t>(__double_as_longlong(static_cast<const double*>(Xv)[off]));
      } else if (SINGLE) {
        const float2 v = static_cast<const float2*>(Xv)[off];
        bre = __float_as_uint(v.x);
        bim = __float_as_uint(conj ? -v.y : v.y);
      } else {
        const double2 v = static_cast<const double2*>(Xv)[off];
        bre = static_cast<uint64_t>(__double_as_longlong(v.x));
        bim = static_cast<uint64_t>(__double_as_longlong(conj ? -v.y : v.y));
      }
    }
    sm.tre[rr][hh] = bre;
    sm.tim[rr][hh] = bim;
  }
  __syncthreads();

  // compute phase: each thread owns kPerThread consecutive h of one row; the
  // block covers kTileR rows x kSplitH h in 2048 / (256 kPerThread) passes
  constexpr int kThreadsPerRow = kSplitH / kPerThread;
  constexpr int kRowsPerPass = kThreads / kThreadsPerRow;
#pragma unroll 1
  for (int pass = 0; pass < kTileR / kRowsPerPass; ++pass) {
  const int rr = pass * kRowsPerPass + tid / kThreadsPerRow;
  const int hb = (tid % kThreadsPerRow) * kPerThread;
  const int64_t r = r0 + rr;
  if (r >= rows) continue;
  const int x = xexp[r];
  const bool flagged = (x == kExpNonfinite);
  const int nch = NCH ? NCH : pl.nchunk;
  constexpr int TC = NCH ? NCH : kMaxChunks;

  // chunks of entries 2i and 2i+1 side by side: the per-modulus steps run on pairs
  static_assert(kPerThread % 2 == 0, "entries are processed in pairs");
  constexpr int kPairs = kPerThread / 2;
  float2 cre[kPairs][TC], cim[kPairs][TC];
#pragma unroll
  for (int j = 0; j < kPerThread; ++j) {
    uint64_t br = sm.tre[rr][hb + j], bi = sm.tim[rr][hb + j];
    // a flagged row, or a non-finite entry, contributes zeros
    const bool bad = flagged ||
                     (SINGLE ? (((br >> 23) & 0xFF) == 0xFF || ((bi >> 23) & 0xFF) == 0xFF)
                             : (((br >> 52) & 0x7FF) == 0x7FF || ((bi >> 52) & 0x7FF) == 0x7FF));
    if (bad) br = bi = 0;
    float c[TC];
    chunks<SINGLE, TC>(br, flagged ? 0 : x, nch, c);
#pragma unroll
    for (int t = 0; t < TC; ++t) {
      if (j & 1) cre[j / 2][t].y = c[t];
      else cre[j / 2][t].x = c[t];
    }
    if constexpr (!R) {
      chunks<SINGLE, TC>(bi, flagged ? 0 : x, nch, c);
#pragma unroll
      for (int t = 0; t < TC; ++t) {
        if (j & 1) cim[j / 2][t].y = c[t];
        else cim[j / 2][t].x = c[t];
      }
    }
  }
  const int64_t plane_stride = prow * kpad;
  T* dst = planes + r * kpad + h0 + hb;
  for (int l = 0; l < pl.N; ++l) {
    const float p = static_cast<float>(pl.p[l]);
    const float ph = 0.5f * p;
    const float ip = pl.inv_p[l];
    float2 w[TC];
#pragma unroll
    for (int t = 0; t < TC; ++t) w[t] = make_float2(pl.w13[l][t], pl.w13[l][t]);
    // z = sum_t c_t w_t for one pair of entries (exact: |z| < 2^23)
    auto dot = [&](const float2 (&c)[TC]) {
      float2 z = mul2(c[0], w[0]);
#pragma unroll
      for (int t = 1; t < TC; ++t)
        if (NCH || t < nch) z = fma2(c[t], w[t], z);
      return z;
    };
    float vr[kPerThread];
    if constexpr (R) {
      // real input: one plane per modulus
#pragma unroll
      for (int i = 0; i < kPairs; ++i) {
        const float2 z = dot(cre[i]);
        vr[2 * i] = sym_mod_f(z.x, p, ph, ip);
        vr[2 * i + 1] = sym_mod_f(z.y, p, ph, ip);
      }
      StoreE<T, kPerThread>::put(dst, vr);
      dst += plane_stride;
    } else {
      float vi[kPerThread], vs[kPerThread];
#pragma unroll
      for (int i = 0; i < kPairs; ++i) {
        const float2 zr = dot(cre[i]), zi = dot(cim[i]);
        vr[2 * i] = sym_mod_f(zr.x, p, ph, ip);
        vr[2 * i + 1] = sym_mod_f(zr.y, p, ph, ip);
        vi[2 * i] = sym_mod_f(zi.x, p, ph, ip);
        vi[2 * i + 1] = sym_mod_f(zi.y, p, ph, ip);
        // Karatsuba sum plane: |vr + vi| <= p
        vs[2 * i] = sym_fix_f(vr[2 * i] + vi[2 * i], p, ph);
        vs[2 * i + 1] = sym_fix_f(vr[2 * i + 1] + vi[2 * i + 1], p, ph);
      }
      StoreE<T, kPerThread>::put(dst, vr);
      StoreE<T, kPerThread>::put(dst + plane_stride, vi);
      StoreE<T, kPerThread>::put(dst + 2 * plane_stride, vs);
      dst += 3 * plane_stride;
    }
  }
  }
}

// ---- accurate mode: the 7-bit ceiling planes of Section III-B.  For a row r
// with ilogb of its largest |entry| e_r, each entry becomes ceil(|v| 2^(5 - e_r))
// (an integer in [0, 64]; a nonzero entry too small to register has ceiling 1).
// Complex rows give plane 0 = ceil |Re|, plane 1 = ceil |Im|, plane 2 = their
// difference; real rows give plane 0.  Flagged rows and non-finite entries are 0.
template <bool SINGLE>
__device__ __forceinline__ float ceil_scaled(uint64_t bits, int e) {
  uint64_t m;
  int elsb;
  if (SINGLE) {
    const uint32_t b = static_cast<uint32_t>(bits) & 0x7FFFFFFFu;
    const int ex = static_cast<int>(b >> 23);
    m = ex ? ((b & 0x7FFFFFu) | 0x800000u) : b;
    elsb = ex ? ex - 150 : -149;
  } else {
    const uint64_t b = bits & 0x7FFFFFFFFFFFFFFFull;
    const int ex = static_cast<int>(b >> 52);
    m = ex ? ((b & 0xFFFFFFFFFFFFFull) | (1ull << 52)) : b;
    elsb = ex ? ex - 1075 : -1074;
  }
  if (m == 0) return 0.0f;
  const int s = elsb + kAccuPreBits - e;       // |v| 2^(5-e) = m 2^s < 2^6
  uint64_t q;
  if (s >= 0) q = m << s;                      // only for tiny m: the value stays below 64
  else if (-s >= 64) q = 1;
  else q = (m >> (-s)) + (((m & ((1ull << (-s)) - 1ull)) != 0ull) ? 1ull : 0ull);
  return static_cast<float>(q);
}

template <bool SINGLE, bool ROWS_CONTIG, bool R>
__global__ void __launch_bounds__(kThreads) bound_split_kernel(const void* __restrict__ Xv, int64_t rows, int64_t k,
                                                               int64_t rs, int64_t hs, const int* __restrict__ emax,
                                                               const unsigned int* __restrict__ flag, int64_t kpad,
                                                               __half* __restrict__ planes) {
  __shared__ TileSmem<kTileH> sm;
  const int tid = threadIdx.x;
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * kTileR;
  const int64_t h0 = static_cast<int64_t>(blockIdx.y) * kTileH;
#pragma unroll
  for (int it = 0; it < (kTileR * kTileH) / kThreads; ++it) {
    int rr, hh;
    if (ROWS_CONTIG) {
      rr = tid & 31;
      hh = (tid >> 5) + 8 * it;
    } else {
      hh = tid & 31;
      rr = (tid >> 5) + 8 * it;
    }
    const int64_t r = r0 + rr, h = h0 + hh;
    uint64_t bre = 0, bim = 0;
    if (r < rows && h < k) {
      const int64_t off = r * rs + h * hs;
      if constexpr (R) {
        bre = SINGLE ? static_cast<uint64_t>(__float_as_uint(static_cast<const float*>(Xv)[off]))
                     : static_cast<uint64_t>(__double_as_longlong(static_cast<const double*>(Xv)[off]));
      } else if (SINGLE) {
        const float2 v = static_cast<const float2*>(Xv)[off];
        bre = __float_as_uint(v.x);
        bim = __float_as_uint(v.y);
      } else {
        const double2 v = static_cast<const double2*>(Xv)[off];
        bre = static_cast<uint64_t>(__double_as_longlong(v.x));
        bim = static_cast<uint64_t>(__double_as_longlong(v.y));
      }
    }
    sm.tre[rr][hh] = bre;
    sm.tim[rr][hh] = bim;
  }
  __syncthreads();
  // each thread: 4 consecutive h of one row, 8 threads per row, 32 rows per pass
  const int rr = tid / 8;
  const int hb = (tid % 8) * 4;
  const int64_t r = r0 + rr;
  if (r >= rows) return;
  const bool zero = flag[r] != 0;
  const int e = emax[r] ? emax[r] - 2048 : 0;
  float vr[4], vi[4], vd[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    vr[j] = zero ? 0.0f : ceil_scaled<SINGLE>(sm.tre[rr][hb + j], e);
    vi[j] = (zero || R) ? 0.0f : ceil_scaled<SINGLE>(sm.tim[rr][hb + j], e);
    vd[j] = vr[j] - vi[j];
  }
  const int64_t plane = rows * kpad;
  __half* dst = planes + r * kpad + h0 + hb;
  StoreE<__half, 4>::put(dst, vr);
  if constexpr (!R) {
    StoreE<__half, 4>::put(dst + plane, vi);
    StoreE<__half, 4>::put(dst + 2 * plane, vd);
  }
}

template <bool SINGLE, bool ROWS_CONTIG, typename T, int E, bool R, int NCH = 0>
__global__ void __launch_bounds__(kThreads) split_kernel(const void* __restrict__ Xv, int64_t rows,
                                                         int64_t k, int64_t rs, int64_t hs,
                                                         bool conj, const int16_t* __restrict__ xexp,
                                                         const __grid_constant__ Plan pl,
                                                         int64_t kpad, T* __restrict__ planes, int64_t prow) {
  __shared__ SplitSmem sm;
  split_block<SINGLE, ROWS_CONTIG, T, E, R, NCH>(sm, Xv, rows, k, rs, hs, conj, xexp, pl, kpad, planes, blockIdx.x,
                                                 blockIdx.y, prow);
}

// one launch over every segment (rows of op(A) or columns of op(B) of each problem) of a grouped call
template <bool SINGLE, typename T, int NCH = 0>
__global__ void __launch_bounds__(kThreads) split_grouped(const SplitSeg* __restrict__ segs,
                                                          const int* __restrict__ block_seg,
                                                          const __grid_constant__ Plan pl) {
  __shared__ SplitSmem sm;
  const long long b = blockIdx.x;
  const SplitSeg& g = segs[block_seg[b]];
  const long long local = b - g.block_begin;
  const int64_t rt = local / g.htiles, ht = local % g.htiles;
  T* planes = static_cast<T*>(g.planes);
  if (g.rows_contig)
    split_block<SINGLE, true, T, 4, false, NCH>(sm, g.X, g.rows, g.k, g.rs, g.hs, g.conj != 0, g.xexp, pl, g.kpad,
                                                planes, rt, ht, g.rows);
  else
    split_block<SINGLE, false, T, 4, false, NCH>(sm, g.X, g.rows, g.k, g.rs, g.hs, g.conj != 0, g.xexp, pl, g.kpad,
                                                 planes, rt, ht, g.rows);
}

template <bool SINGLE, typename T, bool R>
cudaError_t launch_t(bool conj, const void* X, int64_t rows, int64_t k, int64_t rs, int64_t hs,
                     const Plan& pl, const int16_t* xexp, int64_t kpad, void* planes,
                     cudaStream_t st, int elems, int64_t prow) {
  if ((rows + kTileR - 1) / kTileR > 2147483647LL || kpad / kSplitH > 65535) return cudaErrorInvalidValue;
  dim3 grid(static_cast<unsigned int>((rows + kTileR - 1) / kTileR),
            static_cast<unsigned int>(kpad / kSplitH));
  T* P = static_cast<T*>(planes);
  // the common configuration (fp16 planes, 4 entries per thread) has the chunk count compiled in
  auto fixed = [&](auto nch_tag) {
    constexpr int NC = decltype(nch_tag)::value;
    if (rs == 1) {
      max_shared_carveout(split_kernel<SINGLE, true, T, 4, R, NC>);
      split_kernel<SINGLE, true, T, 4, R, NC><<<grid, kThreads, 0, st>>>(X, rows, k, rs, hs, conj, xexp, pl, kpad, P, prow);
    } else {
      max_shared_carveout(split_kernel<SINGLE, false, T, 4, R, NC>);
      split_kernel<SINGLE, false, T, 4, R, NC><<<grid, kThreads, 0, st>>>(X, rows, k, rs, hs, conj, xexp, pl, kpad, P, prow);
    }
  };
  bool done = false;
  if constexpr (std::is_same<T, __half>::value) {
    if (elems != 2) {
      done = true;
      switch (pl.nchunk) {
        case 3: fixed(std::integral_constant<int, 3>{}); break;
        case 4: fixed(std::integral_constant<int, 4>{}); break;
        case 5: fixed(std::integral_constant<int, 5>{}); break;
        case 6: fixed(std::integral_constant<int, 6>{}); break;
        case 7: fixed(std::integral_constant<int, 7>{}); break;
        case 8: fixed(std::integral_constant<int, 8>{}); break;
        default: done = false;
      }
    }
  }
  if (done) {
  } else if (elems == 2) {
    if (rs == 1) split_kernel<SINGLE, true, T, 2, R><<<grid, kThreads, 0, st>>>(X, rows, k, rs, hs, conj, xexp, pl, kpad, P, prow);
    else split_kernel<SINGLE, false, T, 2, R><<<grid, kThreads, 0, st>>>(X, rows, k, rs, hs, conj, xexp, pl, kpad, P, prow);
  } else {
    if (rs == 1) split_kernel<SINGLE, true, T, 4, R><<<grid, kThreads, 0, st>>>(X, rows, k, rs, hs, conj, xexp, pl, kpad, P, prow);
    else split_kernel<SINGLE, false, T, 4, R><<<grid, kThreads, 0, st>>>(X, rows, k, rs, hs, conj, xexp, pl, kpad, P, prow);
  }
  count_launches(1);
  return cudaGetLastError();
}

template <bool SINGLE, bool R>
cudaError_t launch_s(bool conj, const void* X, int64_t rows, int64_t k, int64_t rs, int64_t hs, const Plan& pl,
                     const int16_t* xexp, bool fp16, int64_t kpad, void* planes, cudaStream_t st, int elems,
                     int64_t prow) {
  return fp16 ? launch_t<SINGLE, __half, R>(conj, X, rows, k, rs, hs, pl, xexp, kpad, planes, st, elems, prow)
              : launch_t<SINGLE, int8_t, R>(conj, X, rows, k, rs, hs, pl, xexp, kpad, planes, st, elems, prow);
}

}  // namespace

long long split_seg_blocks(SplitSeg& g) {
  g.rows_contig = (g.rs == 1) ? 1 : 0;
  g.htiles = static_cast<int>(g.kpad / kSplitH);
  return ((g.rows + kTileR - 1) / kTileR) * g.htiles;
}

cudaError_t launch_split_grouped(bool single, bool fp16, const SplitSeg* segs_dev, const int* block_seg, int nseg,
                                 long long blocks, const Plan& pl, cudaStream_t st) {
  if (nseg <= 0 || blocks <= 0) return cudaSuccess;
  if (blocks > 2147483647LL) return cudaErrorInvalidValue;
  const unsigned int gb = static_cast<unsigned int>(blocks);
  // fp16 planes: the chunk count compiled in, as in the single-GEMM split
  auto fixed = [&](auto nch_tag) {
    constexpr int NC = decltype(nch_tag)::value;
    if (single) split_grouped<true, __half, NC><<<gb, kThreads, 0, st>>>(segs_dev, block_seg, pl);
    else split_grouped<false, __half, NC><<<gb, kThreads, 0, st>>>(segs_dev, block_seg, pl);
  };
  bool done = fp16;
  if (fp16) {
    switch (pl.nchunk) {
      case 3: fixed(std::integral_constant<int, 3>{}); break;
      case 4: fixed(std::integral_constant<int, 4>{}); break;
      case 5: fixed(std::integral_constant<int, 5>{}); break;
      case 6: fixed(std::integral_constant<int, 6>{}); break;
      case 7: fixed(std::integral_constant<int, 7>{}); break;
      case 8: fixed(std::integral_constant<int, 8>{}); break;
      default: done = false;
    }
  }
  if (!done) {
    if (single) {
      if (fp16) split_grouped<true, __half><<<gb, kThreads, 0, st>>>(segs_dev, block_seg, pl);
      else split_grouped<true, int8_t><<<gb, kThreads, 0, st>>>(segs_dev, block_seg, pl);
    } else {
      if (fp16) split_grouped<false, __half><<<gb, kThreads, 0, st>>>(segs_dev, block_seg, pl);
      else split_grouped<false, int8_t><<<gb, kThreads, 0, st>>>(segs_dev, block_seg, pl);
    }
  }
  count_launches(1);
  return cudaGetLastError();
}

template <bool S, bool R>
cudaError_t bound_t(const void* X, int64_t rows, int64_t k, int64_t rs, int64_t hs, const int* emax,
                    const unsigned int* flag, int64_t kpad, void* planes, cudaStream_t st) {
  dim3 grid(static_cast<unsigned int>((rows + kTileR - 1) / kTileR), static_cast<unsigned int>(kpad / kTileH));
  __half* P = static_cast<__half*>(planes);
  if (rs == 1) bound_split_kernel<S, true, R><<<grid, kThreads, 0, st>>>(X, rows, k, rs, hs, emax, flag, kpad, P);
  else bound_split_kernel<S, false, R><<<grid, kThreads, 0, st>>>(X, rows, k, rs, hs, emax, flag, kpad, P);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_bound_split(bool single, bool real, const void* X, int64_t rows, int64_t k, int64_t rs,
                               int64_t hs, const int* emax, const unsigned int* flag, int64_t kpad, void* planes,
                               cudaStream_t st) {
  if (rows <= 0 || kpad <= 0) return cudaSuccess;
  if (kpad % 64 || (rows + kTileR - 1) / kTileR > 2147483647LL || kpad / kTileH > 65535) return cudaErrorInvalidValue;
  if (real) return single ? bound_t<true, true>(X, rows, k, rs, hs, emax, flag, kpad, planes, st)
                          : bound_t<false, true>(X, rows, k, rs, hs, emax, flag, kpad, planes, st);
  return single ? bound_t<true, false>(X, rows, k, rs, hs, emax, flag, kpad, planes, st)
                : bound_t<false, false>(X, rows, k, rs, hs, emax, flag, kpad, planes, st);
}

cudaError_t launch_split(bool single, bool conj, const void* X, int64_t rows, int64_t k,
                         int64_t rs, int64_t hs, const Plan& pl, const int16_t* xexp, bool fp16,
                         int64_t kpad, void* planes, cudaStream_t st, int elems, bool real, int64_t plane_rows) {
  if (rows <= 0 || kpad <= 0) return cudaSuccess;
  if (kpad % 64) return cudaErrorInvalidValue;
  if (plane_rows == 0) plane_rows = rows;
  if (plane_rows < rows) return cudaErrorInvalidValue;
  if (real)
    return single ? launch_s<true, true>(false, X, rows, k, rs, hs, pl, xexp, fp16, kpad, planes, st, elems, plane_rows)
                  : launch_s<false, true>(false, X, rows, k, rs, hs, pl, xexp, fp16, kpad, planes, st, elems, plane_rows);
  return single ? launch_s<true, false>(conj, X, rows, k, rs, hs, pl, xexp, fp16, kpad, planes, st, elems, plane_rows)
                : launch_s<false, false>(conj, X, rows, k, rs, hs, pl, xexp, fp16, kpad, planes, st, elems, plane_rows);
}

}  // namespace emu
