// Integer pieces shared by the CRT kernels (k_crt.cu, k_crt_tc.cu): the
// multi-limb two's-complement value c' (exact, modulo 2^(32L)) rounded once to
// binary64, the accurate-mode range correction, and the 32 x 32 -> 64-bit
// multiply-add.
#pragma once

#include "emu_internal.h"

namespace emu {
namespace {

// Round the L-limb two's-complement integer c (exact c') times 2^e2 to the
// nearest binary64 (ties to even), by integer operations only: the magnitude's
// leading 64 bits (a window of the top nonzero limb and the two below it,
// shifted up to the leading one) give the 53 kept bits and the round bit, and
// everything below them only the sticky bit.
template <int L>
__device__ __forceinline__ double round_limbs(uint32_t (&c)[L], int e2) {
  const bool neg = (c[L - 1] >> 31) != 0;
  if (neg) {   // two's-complement negate
    uint32_t carry = 1;
#pragma unroll
    for (int t = 0; t < L; ++t) {
      const uint64_t v = static_cast<uint64_t>(~c[t]) + carry;
      c[t] = static_cast<uint32_t>(v);
      carry = static_cast<uint32_t>(v >> 32);
    }
  }
  // top nonzero limb and the two below it (no dynamic indexing)
  int top = -1;
  uint32_t w0 = 0, w1 = 0, w2 = 0;
#pragma unroll
  for (int t = 0; t < L; ++t)
    if (c[t]) {
      top = t;
      w0 = c[t];
      w1 = t >= 1 ? c[t >= 1 ? t - 1 : 0] : 0u;
      w2 = t >= 2 ? c[t >= 2 ? t - 2 : 0] : 0u;
    }
  if (top < 0) return 0.0;
  bool sticky = false;
#pragma unroll
  for (int t = 0; t + 3 < L; ++t) sticky |= (t + 3 <= top) && c[t] != 0u;
  const int lz = __clz(w0);
  uint64_t W = (static_cast<uint64_t>(w0) << 32) | w1;    // leading one moved to bit 63 below
  if (lz) {
    W = (W << lz) | (w2 >> (32 - lz));
    sticky |= (w2 << lz) != 0u;
  } else {
    sticky |= w2 != 0u;
  }
  const int lead = 32 * top + 31 - lz + e2;                // exponent of the leading bit
  const int lsb = max(lead - 52, -1074);                   // exponent of the result's LSB
  const int drop = 63 - (lead - lsb);                      // bits of W below it: >= 11
  uint64_t q;
  bool half;
  if (drop >= 65) {            // below half the smallest subnormal
    q = 0;
    half = false;
  } else if (drop == 64) {     // in [2^(lsb-1), 2^lsb): the round bit is the leading one
    q = 0;
    half = true;
    sticky |= (W << 1) != 0ull;
  } else {
    q = W >> drop;
    half = ((W >> (drop - 1)) & 1ull) != 0ull;
    sticky |= (W & ((1ull << (drop - 1)) - 1ull)) != 0ull;
  }
  if (half && (sticky || (q & 1ull))) ++q;
  uint64_t bits = (static_cast<uint64_t>(lsb + 1074) << 52) + q;
  if (bits >= 0x7FF0000000000000ull) bits = 0x7FF0000000000000ull;
  if (neg) bits |= 0x8000000000000000ull;
  return __longlong_as_double(static_cast<long long>(bits));
}

// The same rounding for L <= 4 (c' held in at most 128 bits), in 32-bit
// operations: the magnitude is formed by a conditional complement and one
// carry chain, the three words from the top nonzero one down are selected,
// two funnel shifts give the leading 64 bits and a third the sticky word.
// Results whose exponent leaves the normal range (subnormal, overflow) and
// zero take round_limbs, so every result is identical to it.
template <int L>
__device__ __forceinline__ double round_fast(uint32_t (&c)[L], int e2) {
  static_assert(L >= 1 && L <= 4, "at most four limbs");
  const uint32_t s = static_cast<uint32_t>(static_cast<int32_t>(c[L - 1]) >> 31);   // 0 or all ones
  uint32_t x0, x1 = s, x2 = s, x3 = s;                     // sign-extended to four words
  x0 = c[0];
  if constexpr (L >= 2) x1 = c[1];
  if constexpr (L >= 3) x2 = c[2];
  if constexpr (L >= 4) x3 = c[3];
  // |c| = (c ^ s) - s
  x0 ^= s; x1 ^= s; x2 ^= s; x3 ^= s;
  asm("sub.cc.u32 %0, %0, %4;\n\tsubc.cc.u32 %1, %1, %4;\n\tsubc.cc.u32 %2, %2, %4;\n\tsubc.u32 %3, %3, %4;"
      : "+r"(x0), "+r"(x1), "+r"(x2), "+r"(x3)
      : "r"(s));
  // top nonzero word t and the two below it
  uint32_t w0, w1, w2, below;
  int t;
  if (x3) { t = 3; w0 = x3; w1 = x2; w2 = x1; below = x0; }
  else if (x2) { t = 2; w0 = x2; w1 = x1; w2 = x0; below = 0u; }
  else if (x1) { t = 1; w0 = x1; w1 = x0; w2 = 0u; below = 0u; }
  else { t = 0; w0 = x0; w1 = 0u; w2 = 0u; below = 0u; }
  if (w0 == 0u) return round_limbs<L>(c, e2);             // zero
  const int lz = __clz(w0);
  const int elead = 32 * t + 31 - lz + e2;                 // exponent of the leading bit of c' 2^e2
  if (elead < -1022 || elead > 1023) return round_limbs<L>(c, e2);
  const uint32_t h = __funnelshift_l(w1, w0, lz);         // leading 64 bits: (h, l)
  const uint32_t l = __funnelshift_l(w2, w1, lz);
  const uint32_t st = (w2 << lz) | below;                  // bits below the window
  // 53 kept bits q = (h, l) >> 11, round bit = bit 10 of l, sticky = bits 0-9 and st
  uint32_t qh = h >> 11;
  uint32_t ql = __funnelshift_r(l, h, 11);
  const bool up = ((l >> 10) & 1u) && (((l & 0x3FFu) | st) != 0u || (ql & 1u));
  asm("add.cc.u32 %0, %0, %2;\n\taddc.u32 %1, %1, 0;" : "+r"(ql), "+r"(qh) : "r"(up ? 1u : 0u));
  // a carry out of 53 bits steps the exponent
  const uint32_t bh = qh + (static_cast<uint32_t>(elead + 1022) << 20) + (s & 0x80000000u);
  return __hiloint2double(static_cast<int>(bh), static_cast<int>(ql));
}

// round_fast where it applies, else round_limbs
template <int L>
__device__ __forceinline__ double round_exact(uint32_t (&c)[L], int e2) {
  if constexpr (L <= 4) return round_fast<L>(c, e2);
  else return round_limbs<L>(c, e2);
}

// Accurate-mode range fix: |c'| <= (P-1)/2 there, so the float quotient can be
// one off near the ends of the range and c holds c' - P or c' + P.  With H =
// (P-1)/2: c > H (H - c < 0) means c -= P; c < -H (c + H < 0) means c += P.
// The limbs hold these values without wrapping (2^(32L-1) > 2P).
template <int L>
__device__ __forceinline__ void fix_range(uint32_t (&c)[L], const Plan& pl) {
  uint32_t d[L];
  int64_t b = 0;
#pragma unroll
  for (int t = 0; t < L; ++t) {        // d = H - c
    const int64_t v = static_cast<int64_t>(pl.H[t]) - static_cast<int64_t>(c[t]) + b;
    d[t] = static_cast<uint32_t>(v);
    b = v >> 32;
  }
  if (d[L - 1] >> 31) {                // c > H: c -= P
    b = 0;
#pragma unroll
    for (int t = 0; t < L; ++t) {
      const int64_t v = static_cast<int64_t>(c[t]) - static_cast<int64_t>(pl.Pw[t]) + b;
      c[t] = static_cast<uint32_t>(v);
      b = v >> 32;
    }
    return;
  }
  uint64_t cy = 0;
#pragma unroll
  for (int t = 0; t < L; ++t) {        // d = c + H
    const uint64_t v = static_cast<uint64_t>(c[t]) + pl.H[t] + cy;
    d[t] = static_cast<uint32_t>(v);
    cy = v >> 32;
  }
  if (d[L - 1] >> 31) {                // c < -H: c += P
    cy = 0;
#pragma unroll
    for (int t = 0; t < L; ++t) {
      const uint64_t v = static_cast<uint64_t>(c[t]) + pl.Pw[t] + cy;
      c[t] = static_cast<uint32_t>(v);
      cy = v >> 32;
    }
  }
}

// a * b + c with a 32 x 32 -> 64-bit product
__device__ __forceinline__ uint64_t mad_wide(uint32_t a, uint32_t b, uint64_t c) {
  uint64_t r;
  asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(r) : "r"(a), "r"(b), "l"(c));
  return r;
}

// Host-computed alpha/beta case of a CRT launch (no floating-point compares per
// thread: FP64 instructions are scarce on GB300): bit 0 alpha = 1 and beta = 0,
// bit 1 beta != 0.
constexpr int kCrtPlain = 1, kCrtBeta = 2;
inline int crt_flags(double ar, double ai, double br, double bi) {
  return ((ar == 1.0 && ai == 0.0 && br == 0.0 && bi == 0.0) ? kCrtPlain : 0) |
         ((br != 0.0 || bi != 0.0) ? kCrtBeta : 0);
}

}  // namespace
}  // namespace emu
