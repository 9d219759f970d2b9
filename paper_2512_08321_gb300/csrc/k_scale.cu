// K1: fast-mode scaling exponents (Section III-B, eqs. mu-fast / nu-fast).
//
// For every row r of A-hat (2k real entries Re/Im of one row of op(A)) or
// column of B-hat (for real matrices: the k entries of the row or column):
//   e_r = max_h ilogb|v_rh|                                   (pass 1)
//   S_r = sum_h ceil(|v_rh| 2^(15 - e_r))^2   (exact uint64)  (pass 2)
//   E_r = max{E : 4^E max(2^32, S_r) <= (P-1) 2^27}           (finalize)
//   x_r = E_r - e_r  (int16), or EMU_EXP_NONFINITE if the row holds Inf/NaN.
// This is the paper's floor(P'_fast - max(1, log2 ||t_r||)) - e_r with
// P'_fast = log2(P-1)/2 - 1.5, decided exactly on the integer upper bound S_r
// of ||t_r||^2 2^30 (t = v 2^-e) instead of through __log2f; the sums are
// order independent, so the exponents are deterministic.
//
// Element (r, h) of the source is X[r*rs + h*hs] (complex, in elements);
// either rs == 1 (rows contiguous: one thread per row, coalesced along r) or
// hs == 1 (entries of a row contiguous: one warp per row).
#include <cuda.h>

#include <cmath>
#include <mutex>

#include "emu_internal.h"

namespace emu {
namespace {

constexpr int kChunkH = 512;      // h handled by one block (grouped forms; the most for single calls)
constexpr int kThreads = 256;

template <bool SINGLE>
struct Bits;
template <>
struct Bits<false> {
  using U = unsigned long long;
  using V = double2;
  static constexpr int kMant = 52, kExpMask = 0x7FF, kBias = 1023, kMinLsb = -1074;
  __device__ static U re(const V& v) { return __double_as_longlong(v.x) & 0x7FFFFFFFFFFFFFFFull; }
  __device__ static U im(const V& v) { return __double_as_longlong(v.y) & 0x7FFFFFFFFFFFFFFFull; }
};
template <>
struct Bits<true> {
  using U = unsigned int;
  using V = float2;
  static constexpr int kMant = 23, kExpMask = 0xFF, kBias = 127, kMinLsb = -149;
  __device__ static U re(const V& v) { return __float_as_uint(v.x) & 0x7FFFFFFFu; }
  __device__ static U im(const V& v) { return __float_as_uint(v.y) & 0x7FFFFFFFu; }
};

// Magnitude bits of the two real entries a complex element contributes to a
// row of A-hat (Re, Im), or of the one entry of a real element (b = 0).
template <bool S, bool R>
__device__ __forceinline__ void load_mag(const void* __restrict__ X, int64_t off, typename Bits<S>::U& a,
                                         typename Bits<S>::U& b) {
  using B = Bits<S>;
  if constexpr (R) {
    if constexpr (S) a = __float_as_uint(static_cast<const float*>(X)[off]) & 0x7FFFFFFFu;
    else a = __double_as_longlong(static_cast<const double*>(X)[off]) & 0x7FFFFFFFFFFFFFFFull;
    b = 0;
  } else {
    const typename B::V v = static_cast<const typename B::V*>(X)[off];
    a = B::re(v);
    b = B::im(v);
  }
}

// magnitude bits u (sign cleared): nonfinite?
template <bool S>
__device__ __forceinline__ bool nonfinite(typename Bits<S>::U u) {
  return static_cast<int>(u >> Bits<S>::kMant) == Bits<S>::kExpMask;
}

// ilogb of a finite nonzero magnitude, offset by +2048 (0 means "no entry")
template <bool S>
__device__ __forceinline__ int ilogb_off(typename Bits<S>::U u) {
  const int ex = static_cast<int>(u >> Bits<S>::kMant);
  if (ex) return ex - Bits<S>::kBias + 2048;
  // subnormal: u is the integer significand, value u * 2^kMinLsb
  const int lead = S ? (31 - __clz(static_cast<unsigned int>(u)))
                     : (63 - __clzll(static_cast<unsigned long long>(u)));
  return lead + Bits<S>::kMinLsb + 2048;
}

// ceil(|v| 2^(15 - e)) for a finite magnitude u (0 -> 0)
template <bool S>
__device__ __forceinline__ unsigned long long ceil_q(typename Bits<S>::U u, int e) {
  if (u == 0) return 0ull;
  const int ex = static_cast<int>(u >> Bits<S>::kMant);
  unsigned long long m;
  int elsb;
  if (ex) {
    m = (static_cast<unsigned long long>(u) & ((1ull << Bits<S>::kMant) - 1)) |
        (1ull << Bits<S>::kMant);
    elsb = ex - Bits<S>::kBias - Bits<S>::kMant;
  } else {
    m = static_cast<unsigned long long>(u);
    elsb = Bits<S>::kMinLsb;
  }
  const int s = e - kSumFracBits - elsb;   // value = m 2^-s
  if (s <= 0) return m << (-s);
  if (s >= 64) return 1ull;
  const unsigned long long q = m >> s;
  return q + ((m & ((1ull << s) - 1)) != 0ull ? 1ull : 0ull);
}

// Largest E with 4^E * M <= X = (P-1) 2^27 (M >= 1).
__device__ __forceinline__ int exponent_le(const Plan& pl, unsigned long long M) {
  const int bm = 64 - __clzll(M);
  const int bx = pl.sX + (64 - __clzll(pl.Xtop));
  auto fits = [&](int E) -> bool {
    const int sh = 2 * E - pl.sX;
    if (sh >= 64) return false;
    if (sh >= 0) return M <= (pl.Xtop >> sh);
    if (-sh >= 64) return true;
    const unsigned __int128 lhs = static_cast<unsigned __int128>(pl.Xtop) << (-sh);
    return static_cast<unsigned __int128>(M) <= lhs;
  };
  const int d = bx - bm;
  int E = d >= 0 ? d / 2 : -((-d + 1) / 2);
  while (!fits(E)) --E;
  while (fits(E + 1)) ++E;
  return E;
}

// Fast mode: 4^E max(2^32, S) <= (P-1) 2^27.
__device__ __forceinline__ int exponent_from_sum(const Plan& pl, unsigned long long S) {
  return exponent_le(pl, S > (1ull << 32) ? S : (1ull << 32));
}

// ---- pass 1: max exponent and non-finite flag (one block: row block rb, h chunk hc)
template <bool S, bool ROWS_CONTIG, bool R = false>
__device__ __forceinline__ void exp_max_block(const void* __restrict__ X, int64_t rows, int64_t k,
                                              int64_t rs, int64_t hs, int* __restrict__ emax,
                                              unsigned int* __restrict__ flag, int64_t rb, int64_t hc,
                                              int64_t chunk) {
  using B = Bits<S>;
  int best = 0;
  bool bad = false;
  int64_t r;
  if (ROWS_CONTIG) {
    r = rb * kThreads + threadIdx.x;
    if (r >= rows) return;
    const int64_t h0 = hc * chunk;
    const int64_t h1 = min(k, h0 + chunk);
    for (int64_t h = h0; h < h1; ++h) {
      typename B::U a, b;
      load_mag<S, R>(X, r + h * hs, a, b);
      bad |= nonfinite<S>(a) | nonfinite<S>(b);
      if (a && !nonfinite<S>(a)) best = max(best, ilogb_off<S>(a));
      if (b && !nonfinite<S>(b)) best = max(best, ilogb_off<S>(b));
    }
  } else {
    const int lane = threadIdx.x & 31;
    r = rb * (kThreads / 32) + (threadIdx.x >> 5);
    if (r >= rows) return;
    const int64_t h0 = hc * chunk;
    const int64_t h1 = min(k, h0 + chunk);
    for (int64_t h = h0 + lane; h < h1; h += 32) {
      typename B::U a, b;
      load_mag<S, R>(X, r * rs + h, a, b);
      bad |= nonfinite<S>(a) | nonfinite<S>(b);
      if (a && !nonfinite<S>(a)) best = max(best, ilogb_off<S>(a));
      if (b && !nonfinite<S>(b)) best = max(best, ilogb_off<S>(b));
    }
    for (int o = 16; o; o >>= 1) {
      best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
      bad |= __shfl_xor_sync(0xffffffffu, static_cast<int>(bad), o) != 0;
    }
    if (lane) return;
  }
  if (best) atomicMax(emax + r, best);
  if (bad) atomicOr(flag + r, 1u);
}

template <bool S, bool ROWS_CONTIG, bool R>
__global__ void __launch_bounds__(kThreads) exp_max_kernel(const void* __restrict__ X,
                                                           int64_t rows, int64_t k, int64_t rs,
                                                           int64_t hs, int* __restrict__ emax,
                                                           unsigned int* __restrict__ flag, int64_t chunk) {
  exp_max_block<S, ROWS_CONTIG, R>(X, rows, k, rs, hs, emax, flag, blockIdx.x, blockIdx.y, chunk);
}

// ---- pass 2: exact quantised sum of squares (one block)
template <bool S, bool ROWS_CONTIG, bool R = false>
__device__ __forceinline__ void exp_sum_block(const void* __restrict__ X, int64_t rows, int64_t k,
                                              int64_t rs, int64_t hs, const int* __restrict__ emax,
                                              const unsigned int* __restrict__ flag,
                                              unsigned long long* __restrict__ sum, int64_t rb, int64_t hc,
                                              int64_t chunk) {
  using B = Bits<S>;
  unsigned long long acc = 0;
  int64_t r;
  if (ROWS_CONTIG) {
    r = rb * kThreads + threadIdx.x;
    if (r >= rows || flag[r] || emax[r] == 0) return;
    const int e = emax[r] - 2048;
    const int64_t h0 = hc * chunk;
    const int64_t h1 = min(k, h0 + chunk);
    for (int64_t h = h0; h < h1; ++h) {
      typename B::U ua, ub;
      load_mag<S, R>(X, r + h * hs, ua, ub);
      const unsigned long long a = ceil_q<S>(ua, e), b = ceil_q<S>(ub, e);
      acc += a * a + b * b;
    }
  } else {
    const int lane = threadIdx.x & 31;
    r = rb * (kThreads / 32) + (threadIdx.x >> 5);
    if (r >= rows || flag[r] || emax[r] == 0) return;
    const int e = emax[r] - 2048;
    const int64_t h0 = hc * chunk;
    const int64_t h1 = min(k, h0 + chunk);
    for (int64_t h = h0 + lane; h < h1; h += 32) {
      typename B::U ua, ub;
      load_mag<S, R>(X, r * rs + h, ua, ub);
      const unsigned long long a = ceil_q<S>(ua, e), b = ceil_q<S>(ub, e);
      acc += a * a + b * b;
    }
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane) return;
  }
  if (acc) atomicAdd(sum + r, acc);
}

// ---- pass 2 for the moduli-selection features: the sums of exp_sum_block and,
// over every entry of every row (flagged and zero rows included), the 16-bin
// histogram of exponent spans d = e_r - ilogb|v| (zero and non-finite
// entries, and entries of zero rows: bin 15).  Each thread counts in two
// words, 8 bits a bin, emptied into 16 totals every 127 pairs of entries;
// warps and then the block add the totals before one global add per bin.
template <bool S>
__device__ __forceinline__ int span_bin(typename Bits<S>::U u, int eo) {
  return (u && !nonfinite<S>(u) && eo) ? min(eo - ilogb_off<S>(u), 15) : 15;
}

struct SpanCounts {
  unsigned long long lo = 0, hi = 0;   // bins 0..7 and 8..15, 8 bits each
  unsigned int tot[16] = {};
  __device__ __forceinline__ void add(int bin) {
    if (bin < 8) lo += 1ull << (8 * bin);
    else hi += 1ull << (8 * (bin - 8));
  }
  __device__ __forceinline__ void empty() {
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      tot[b] += static_cast<unsigned int>((lo >> (8 * b)) & 0xFFu);
      tot[b + 8] += static_cast<unsigned int>((hi >> (8 * b)) & 0xFFu);
    }
    lo = hi = 0;
  }
};

template <bool S, bool ROWS_CONTIG>
__global__ void __launch_bounds__(kThreads) exp_sum_hist_kernel(const void* __restrict__ X, int64_t rows, int64_t k,
                                                                int64_t rs, int64_t hs, const int* __restrict__ emax,
                                                                const unsigned int* __restrict__ flag,
                                                                unsigned long long* __restrict__ sum,
                                                                unsigned long long* __restrict__ hist, int64_t chunk) {
  using B = Bits<S>;
  __shared__ unsigned int block_hist[16];
  if (threadIdx.x < 16) block_hist[threadIdx.x] = 0;
  __syncthreads();
  SpanCounts cnt;
  unsigned long long acc = 0;
  const int lane = threadIdx.x & 31;
  const int64_t r = ROWS_CONTIG ? static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x
                                : static_cast<int64_t>(blockIdx.x) * (kThreads / 32) + (threadIdx.x >> 5);
  const bool valid = r < rows;
  const int eo = valid ? emax[r] : 0;
  const bool summing = valid && !flag[r] && eo != 0;
  const int e = eo - 2048;
  const int64_t h0 = static_cast<int64_t>(blockIdx.y) * chunk;
  const int64_t h1 = min(k, h0 + chunk);
  if (valid) {
    int since = 0;
    for (int64_t h = ROWS_CONTIG ? h0 : h0 + lane; h < h1; h += ROWS_CONTIG ? 1 : 32) {
      typename B::U ua, ub;
      load_mag<S, false>(X, ROWS_CONTIG ? r + h * hs : r * rs + h, ua, ub);
      if (summing) {
        const unsigned long long a = ceil_q<S>(ua, e), b = ceil_q<S>(ub, e);
        acc += a * a + b * b;
      }
      cnt.add(span_bin<S>(ua, eo));
      cnt.add(span_bin<S>(ub, eo));
      if (++since == 127) {
        cnt.empty();
        since = 0;
      }
    }
  }
  cnt.empty();
  if (!ROWS_CONTIG)
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (summing && acc && (ROWS_CONTIG || lane == 0)) atomicAdd(sum + r, acc);
#pragma unroll
  for (int b = 0; b < 16; ++b) {
    const unsigned int v = __reduce_add_sync(0xffffffffu, cnt.tot[b]);
    if (lane == 0 && v) atomicAdd(&block_hist[b], v);
  }
  __syncthreads();
  if (threadIdx.x < 16 && block_hist[threadIdx.x])
    atomicAdd(&hist[threadIdx.x], static_cast<unsigned long long>(block_hist[threadIdx.x]));
}

template <bool S, bool ROWS_CONTIG, bool R>
__global__ void __launch_bounds__(kThreads) exp_sum_kernel(const void* __restrict__ X,
                                                           int64_t rows, int64_t k, int64_t rs,
                                                           int64_t hs, const int* __restrict__ emax,
                                                           const unsigned int* __restrict__ flag,
                                                           unsigned long long* __restrict__ sum, int64_t chunk) {
  exp_sum_block<S, ROWS_CONTIG, R>(X, rows, k, rs, hs, emax, flag, sum, blockIdx.x, blockIdx.y, chunk);
}

__device__ __forceinline__ int16_t finalize_row(const Plan& pl, int em, unsigned int fl, unsigned long long S) {
  if (fl) return kExpNonfinite;
  const int e = em ? em - 2048 : 0;
  return static_cast<int16_t>(exponent_from_sum(pl, S) - e);
}

__global__ void exp_finalize_kernel(int64_t rows, const int* __restrict__ emax,
                                    const unsigned int* __restrict__ flag,
                                    const unsigned long long* __restrict__ sum,
                                    const __grid_constant__ Plan pl, int16_t* __restrict__ xout) {
  const int64_t r = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  xout[r] = finalize_row(pl, emax[r], flag[r], sum[r]);
}

// ---- grouped forms: one launch per pass over every segment of a grouped call
template <bool S>
__global__ void __launch_bounds__(kThreads) exp_max_grouped(const ExpSeg* __restrict__ segs,
                                                            const int* __restrict__ block_seg) {
  const ExpSeg& g = segs[block_seg[blockIdx.x]];
  const long long local = blockIdx.x - g.block_begin;
  const void* X = g.X;
  if (g.rows_contig)
    exp_max_block<S, true>(X, g.rows, g.k, g.rs, g.hs, g.emax, g.flag, local / g.hchunks, local % g.hchunks,
                          kChunkH);
  else
    exp_max_block<S, false>(X, g.rows, g.k, g.rs, g.hs, g.emax, g.flag, local / g.hchunks, local % g.hchunks,
                          kChunkH);
}

template <bool S>
__global__ void __launch_bounds__(kThreads) exp_sum_grouped(const ExpSeg* __restrict__ segs,
                                                            const int* __restrict__ block_seg) {
  const ExpSeg& g = segs[block_seg[blockIdx.x]];
  const long long local = blockIdx.x - g.block_begin;
  const void* X = g.X;
  if (g.rows_contig)
    exp_sum_block<S, true>(X, g.rows, g.k, g.rs, g.hs, g.emax, g.flag, g.sum, local / g.hchunks, local % g.hchunks,
                          kChunkH);
  else
    exp_sum_block<S, false>(X, g.rows, g.k, g.rs, g.hs, g.emax, g.flag, g.sum, local / g.hchunks, local % g.hchunks,
                          kChunkH);
}

// one thread per row of every segment; row_begin holds the prefix sums of rows
__global__ void exp_finalize_grouped(const ExpSeg* __restrict__ segs, int nseg,
                                     const long long* __restrict__ row_begin, long long total,
                                     const __grid_constant__ Plan pl) {
  const long long r = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= total) return;
  int lo = 0, hi = nseg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (row_begin[mid] <= r) lo = mid; else hi = mid - 1;
  }
  const ExpSeg& g = segs[lo];
  const long long i = r - row_begin[lo];
  g.xout[i] = finalize_row(pl, g.emax[i], g.flag[i], g.sum[i]);
}

// h per block for a single call: kChunkH, halved (down to 64) while the grid
// would hold fewer than 8 blocks per SM, so that short-and-wide operands (few
// row blocks) still keep every SM's loads in flight
int64_t num_sms() {
  static std::once_flag once;
  static int sms = 0;
  std::call_once(once, [] {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  });
  return sms > 0 ? sms : 1;
}

int64_t pick_chunk(int64_t rowblocks, int64_t k) {
  int64_t chunk = kChunkH;
  while (chunk > 64 && rowblocks * ((k + chunk - 1) / chunk) < 8 * num_sms()) chunk /= 2;
  return chunk;
}

// scratch of rows: emax (int), flag (uint) and sum (uint64) arrays, each padded to 64 rows
struct ExpScratch {
  int* emax;
  unsigned int* flag;
  unsigned long long* sum;
  ExpScratch(void* scratch, int64_t rows)
      : emax(static_cast<int*>(scratch)),
        flag(reinterpret_cast<unsigned int*>(emax + round_up(rows, 64))),
        sum(reinterpret_cast<unsigned long long*>(flag + round_up(rows, 64))) {}
};

// passes 1 and 2 (the N-independent part of the exponents), with the
// features' histogram when hist is given (complex input only)
template <bool S, bool R = false>
cudaError_t launch_sums_t(const void* X, int64_t rows, int64_t k, int64_t rs, int64_t hs, void* scratch,
                          unsigned long long* hist, cudaStream_t st) {
  const ExpScratch sc(scratch, rows);
  cudaError_t err = cudaMemsetAsync(scratch, 0, exponents_scratch_bytes(rows), st);
  if (err != cudaSuccess) return err;
  if (k > 0) {
    const bool rows_contig = (rs == 1);
    const int64_t rowblocks = rows_contig ? (rows + kThreads - 1) / kThreads : (rows + 7) / 8;
    const int64_t chunk = pick_chunk(rowblocks, k);
    const dim3 grid(static_cast<unsigned int>(rowblocks), static_cast<unsigned int>((k + chunk - 1) / chunk));
    if (rows_contig)
      exp_max_kernel<S, true, R><<<grid, kThreads, 0, st>>>(X, rows, k, rs, hs, sc.emax, sc.flag, chunk);
    else
      exp_max_kernel<S, false, R><<<grid, kThreads, 0, st>>>(X, rows, k, rs, hs, sc.emax, sc.flag, chunk);
    if constexpr (!R) {
      if (hist) {
        if (rows_contig)
          exp_sum_hist_kernel<S, true><<<grid, kThreads, 0, st>>>(X, rows, k, rs, hs, sc.emax, sc.flag, sc.sum, hist,
                                                                  chunk);
        else
          exp_sum_hist_kernel<S, false><<<grid, kThreads, 0, st>>>(X, rows, k, rs, hs, sc.emax, sc.flag, sc.sum, hist,
                                                                   chunk);
        count_launches(2);
        return cudaGetLastError();
      }
    }
    if (rows_contig)
      exp_sum_kernel<S, true, R><<<grid, kThreads, 0, st>>>(X, rows, k, rs, hs, sc.emax, sc.flag, sc.sum, chunk);
    else
      exp_sum_kernel<S, false, R><<<grid, kThreads, 0, st>>>(X, rows, k, rs, hs, sc.emax, sc.flag, sc.sum, chunk);
    count_launches(2);
  }
  return cudaGetLastError();
}

cudaError_t launch_finalize_t(int64_t rows, void* scratch, const Plan& pl, int16_t* xout, cudaStream_t st) {
  const ExpScratch sc(scratch, rows);
  exp_finalize_kernel<<<static_cast<unsigned int>((rows + 255) / 256), 256, 0, st>>>(rows, sc.emax, sc.flag, sc.sum,
                                                                                    pl, xout);
  count_launches(1);
  return cudaGetLastError();
}

template <bool S, bool R = false>
cudaError_t launch_t(const void* X, int64_t rows, int64_t k, int64_t rs, int64_t hs,
                     const Plan& pl, int16_t* xout, void* scratch, cudaStream_t st) {
  const cudaError_t err = launch_sums_t<S, R>(X, rows, k, rs, hs, scratch, nullptr, st);
  if (err != cudaSuccess) return err;
  return launch_finalize_t(rows, scratch, pl, xout, st);
}

// ---- accurate mode (Section III-B, eqs. mu-accu / nu-accu): x_r = 5 - e_r + E_r with
// E_r = max{E : 4^E max(M_r, 1) <= (P-1)/2}, M_r the row (column) maximum of the
// bound products, i.e. 4^E max(M_r, 1) 2^28 <= (P-1) 2^27.
__global__ void accu_finalize_kernel(int64_t rows, const int* __restrict__ emax, const unsigned int* __restrict__ flag,
                                     const unsigned int* __restrict__ Mb, const __grid_constant__ Plan pl,
                                     int16_t* __restrict__ xout) {
  const int64_t r = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  if (flag[r]) {
    xout[r] = kExpNonfinite;
    return;
  }
  const int e = emax[r] ? emax[r] - 2048 : 0;
  const unsigned long long M = Mb[r] > 1u ? Mb[r] : 1u;
  xout[r] = static_cast<int16_t>(kAccuPreBits - e + exponent_le(pl, M << 28));
}

template <bool S, bool R>
cudaError_t launch_max_t(const void* X, int64_t rows, int64_t k, int64_t rs, int64_t hs, int* emax,
                         unsigned int* flag, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(emax, 0, static_cast<size_t>(rows) * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, static_cast<size_t>(rows) * 4, st);
  if (e != cudaSuccess) return e;
  if (k <= 0) return cudaSuccess;
  const int64_t rowblocks = rs == 1 ? (rows + kThreads - 1) / kThreads : (rows + 7) / 8;
  const int64_t chunk = pick_chunk(rowblocks, k);
  const dim3 grid(static_cast<unsigned int>(rowblocks), static_cast<unsigned int>((k + chunk - 1) / chunk));
  if (rs == 1) exp_max_kernel<S, true, R><<<grid, kThreads, 0, st>>>(X, rows, k, rs, hs, emax, flag, chunk);
  else exp_max_kernel<S, false, R><<<grid, kThreads, 0, st>>>(X, rows, k, rs, hs, emax, flag, chunk);
  count_launches(1);
  return cudaGetLastError();
}

// ---- features of the moduli-selection network
// mean and max over rows of L = 0.5 log2(max(S, 1)) - 15
__global__ void __launch_bounds__(1024) feat_stats_kernel(const unsigned long long* __restrict__ sum, int64_t rows,
                                                          float* __restrict__ out) {
  __shared__ double ssum[32];
  __shared__ float smax[32];
  double acc = 0.0;
  float mx = -1e30f;
  for (int64_t r = threadIdx.x; r < rows; r += blockDim.x) {
    const unsigned long long S = sum[r] ? sum[r] : 1ull;
    const float L = 0.5f * log2f(static_cast<float>(S)) - 15.0f;
    acc += L;
    mx = fmaxf(mx, L);
  }
  for (int o = 16; o; o >>= 1) {
    acc += __shfl_xor_sync(0xffffffffu, acc, o);
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    ssum[w] = acc;
    smax[w] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    float b = -1e30f;
    for (int i = 0; i < static_cast<int>(blockDim.x >> 5); ++i) {
      a += ssum[i];
      b = fmaxf(b, smax[i]);
    }
    out[0] = static_cast<float>(a / static_cast<double>(rows > 0 ? rows : 1));
    out[1] = rows > 0 ? b : 0.0f;
  }
}

__global__ void feat_assemble_kernel(const unsigned long long* __restrict__ hist, const float* __restrict__ stats,
                                     double total_a, double total_b, float logk, float tgt, float single,
                                     float* __restrict__ f) {
  const int i = threadIdx.x;
  if (i < 16) f[i] = static_cast<float>(static_cast<double>(hist[i]) / total_a);
  else if (i < 32) f[i] = static_cast<float>(static_cast<double>(hist[i]) / total_b);
  else if (i < 36) f[i] = stats[i - 32];
  else if (i == 36) f[i] = logk;
  else if (i == 37) f[i] = tgt;
  else if (i == 38) f[i] = single;
}

}  // namespace

// Scratch of emu_moduli_features / the tolerance path: the exponent sums of A
// (m rows) and of B (n columns), then 32 histogram bins and 4 statistics.
size_t features_scratch_bytes(int64_t m, int64_t n) {
  return exponents_scratch_bytes(m) + exponents_scratch_bytes(n) + 32 * sizeof(unsigned long long) + 64;
}

cudaError_t launch_exponent_sums(bool single, bool real, const void* X, int64_t rows, int64_t k, int64_t rs,
                                 int64_t hs, void* scratch, unsigned long long* hist, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  if (real && hist) return cudaErrorInvalidValue;
  if (real)
    return single ? launch_sums_t<true, true>(X, rows, k, rs, hs, scratch, nullptr, st)
                  : launch_sums_t<false, true>(X, rows, k, rs, hs, scratch, nullptr, st);
  return single ? launch_sums_t<true>(X, rows, k, rs, hs, scratch, hist, st)
                : launch_sums_t<false>(X, rows, k, rs, hs, scratch, hist, st);
}

cudaError_t launch_exponent_finalize(int64_t rows, void* scratch, const Plan& pl, int16_t* xout, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  return launch_finalize_t(rows, scratch, pl, xout, st);
}

// Feature vector (39 floats) of op(A) (m x k) and op(B) (k x n) into feat.  The
// exponent sums of both operands stay in the scratch (features_scratch_bytes(m,
// n)), A's first, then B's, ready for launch_exponent_finalize.
cudaError_t launch_features(bool single, const void* A, int64_t m, int64_t rsa, int64_t hsa, const void* B,
                            int64_t n, int64_t rsb, int64_t hsb, int64_t k, double target, float* feat,
                            void* scratch, cudaStream_t st) {
  char* scr = static_cast<char*>(scratch);
  void* scrA = scr;
  void* scrB = scr + exponents_scratch_bytes(m);
  unsigned long long* hist =
      reinterpret_cast<unsigned long long*>(scr + exponents_scratch_bytes(m) + exponents_scratch_bytes(n));
  float* stats = reinterpret_cast<float*>(hist + 32);
  cudaError_t e = cudaMemsetAsync(hist, 0, 32 * sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = launch_exponent_sums(single, false, A, m, k, rsa, hsa, scrA, hist, st);
  if (e == cudaSuccess) e = launch_exponent_sums(single, false, B, n, k, rsb, hsb, scrB, hist + 16, st);
  if (e != cudaSuccess) return e;
  feat_stats_kernel<<<1, 1024, 0, st>>>(ExpScratch(scrA, m).sum, m, stats);
  feat_stats_kernel<<<1, 1024, 0, st>>>(ExpScratch(scrB, n).sum, n, stats + 2);
  const double ta = m > 0 && k > 0 ? 2.0 * m * k : 1.0, tb = n > 0 && k > 0 ? 2.0 * k * n : 1.0;
  const float logk = static_cast<float>(std::log2(static_cast<double>(k > 1 ? k : 1)) / 17.0);
  const float tgt = static_cast<float>(-std::log10(target) / 16.0);
  feat_assemble_kernel<<<1, 64, 0, st>>>(hist, stats, ta, tb, logk, tgt, single ? 1.0f : 0.0f, feat);
  count_launches(3);
  return cudaGetLastError();
}

long long exp_seg_blocks(ExpSeg& g) {
  g.rows_contig = (g.rs == 1) ? 1 : 0;
  g.hchunks = static_cast<int>(g.k > 0 ? (g.k + kChunkH - 1) / kChunkH : 0);
  const long long rb = g.rows_contig ? (g.rows + kThreads - 1) / kThreads : (g.rows + 7) / 8;
  return g.hchunks ? rb * g.hchunks : 0;
}

cudaError_t launch_exponents_grouped(bool single, const ExpSeg* segs_dev, const int* block_seg, int nseg, long long blocks,
                                     const long long* row_begin_dev, long long total_rows, const Plan& pl,
                                     cudaStream_t st) {
  if (nseg <= 0) return cudaSuccess;
  if (blocks > 0) {
    if (blocks > 2147483647LL) return cudaErrorInvalidValue;
    if (single) {
      exp_max_grouped<true><<<static_cast<unsigned int>(blocks), kThreads, 0, st>>>(segs_dev, block_seg);
      exp_sum_grouped<true><<<static_cast<unsigned int>(blocks), kThreads, 0, st>>>(segs_dev, block_seg);
    } else {
      exp_max_grouped<false><<<static_cast<unsigned int>(blocks), kThreads, 0, st>>>(segs_dev, block_seg);
      exp_sum_grouped<false><<<static_cast<unsigned int>(blocks), kThreads, 0, st>>>(segs_dev, block_seg);
    }
    count_launches(2);
  }
  if (total_rows > 0) {
    exp_finalize_grouped<<<static_cast<unsigned int>((total_rows + 255) / 256), 256, 0, st>>>(
        segs_dev, nseg, row_begin_dev, total_rows, pl);
    count_launches(1);
  }
  return cudaGetLastError();
}

// Row maxima of ilogb (offset 2048, 0 = zero row) and non-finite flags only (accurate mode).
cudaError_t launch_exp_max(bool single, bool real, const void* X, int64_t rows, int64_t k, int64_t rs, int64_t hs,
                           int* emax, unsigned int* flag, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  if (real)
    return single ? launch_max_t<true, true>(X, rows, k, rs, hs, emax, flag, st)
                  : launch_max_t<false, true>(X, rows, k, rs, hs, emax, flag, st);
  return single ? launch_max_t<true, false>(X, rows, k, rs, hs, emax, flag, st)
                : launch_max_t<false, false>(X, rows, k, rs, hs, emax, flag, st);
}

cudaError_t launch_accu_finalize(int64_t rows, const int* emax, const unsigned int* flag, const unsigned int* Mb,
                                 const Plan& pl, int16_t* xout, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  accu_finalize_kernel<<<static_cast<unsigned int>((rows + 255) / 256), 256, 0, st>>>(rows, emax, flag, Mb, pl, xout);
  count_launches(1);
  return cudaGetLastError();
}

size_t exponents_scratch_bytes(int64_t rows) {
  return static_cast<size_t>(round_up(rows, 64)) * (4 + 4 + 8);
}

cudaError_t launch_exponents(bool single, const void* X, int64_t rows, int64_t k, int64_t rs,
                             int64_t hs, const Plan& pl, int16_t* xout, void* scratch,
                             cudaStream_t st, bool real) {
  if (rows <= 0) return cudaSuccess;
  if (real)
    return single ? launch_t<true, true>(X, rows, k, rs, hs, pl, xout, scratch, st)
                  : launch_t<false, true>(X, rows, k, rs, hs, pl, xout, scratch, st);
  return single ? launch_t<true>(X, rows, k, rs, hs, pl, xout, scratch, st)
                : launch_t<false>(X, rows, k, rs, hs, pl, xout, scratch, st);
}

}  // namespace emu

// ---------------------------------------------------------------------------
// Allocation-free variant of the exponent phase.
//
// Some callers cannot let a library allocate device memory: applications whose
// device memory is owned by their own pool or caching allocator (a cudaMalloc
// from inside the library can fail, or fragment that pool, at a point the
// caller does not control), and latency-sensitive callers that cannot afford
// the implicit device-wide synchronisation of cudaMalloc/cudaFree.  For them,
// emu_stage_exponents_static computes the same per-row/per-column scaling
// exponents as emu_stage_exponents, but its per-row scratch (max exponent,
// non-finite flag, quantised sum: 16 bytes a row) lives in the fixed device
// array below instead of memory allocated per call.  The array holds up to
// kStaticExpMaxRows rows (1 MiB) and stays resident on every GPU that loads
// this library until the process exits.
namespace {

constexpr int64_t kStaticExpMaxRows = EMU_STATIC_EXP_MAX_ROWS;
constexpr int kStaticMaxDevices = 64;

// host code sees only a stand-in symbol: its device address comes from
// cudaGetSymbolAddress, taken per device (and per context) in static_scratch() below
static __device__ __align__(256) unsigned char g_exp_scratch[kStaticExpMaxRows * 16];

std::mutex g_static_mu;
void* g_static_ptr[kStaticMaxDevices] = {};
unsigned long long g_static_ctx[kStaticMaxDevices] = {};   // context id the address belongs to

// Unique id of the calling thread's current context (cuCtxGetId, found through
// the runtime's driver entry points); 0 when it cannot be had.  A device reset
// makes a new primary context with a new id, and the module (with the array)
// is loaded again at another address.
unsigned long long current_ctx_id() {
  using GetCur = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCur get_cur = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_cur = reinterpret_cast<GetCur>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(f);
  });
  if (!get_cur || !get_id) return 0;
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (get_cur(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of g_exp_scratch on the current device.  It is looked up on
// the first call made with that device current, and again whenever the
// device's context has changed since (a device reset), so a stale address is
// never used; without a context id it is looked up on every call.
cudaError_t static_scratch(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kStaticMaxDevices) return cudaErrorInvalidDevice;
  const unsigned long long ctx = current_ctx_id();   // 0 before the runtime has made a context current
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[dev] || ctx == 0 || g_static_ctx[dev] != ctx) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_exp_scratch);       // also makes the device's primary context current
    if (e != cudaSuccess) return e;
    g_static_ptr[dev] = p;
    g_static_ctx[dev] = current_ctx_id();
  }
  *out = g_static_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" emu_status_t emu_stage_exponents_static(int is_single, emu_op_t transa, emu_op_t transb,
                                                   int64_t m, int64_t n, int64_t k, const void* A,
                                                   int64_t lda, const void* B, int64_t ldb, int num_moduli,
                                                   int16_t* x, int16_t* y, void* stream) {
  // argument checks, and the bad-parameter index, as in emu_stage_exponents
  emu_status_t s = emu::check_stage_args(transa, transb, m, n, k, lda, ldb, num_moduli);
  if (s != EMU_OK) return s;
  if (m > kStaticExpMaxRows || n > kStaticExpMaxRows) return EMU_ERR_SIZE_LIMIT;
  if (k > 0 && m > 0 && !A) return emu::set_bad_param(7);
  if (k > 0 && n > 0 && !B) return emu::set_bad_param(9);
  if (m > 0 && !x) return emu::set_bad_param(12);
  if (n > 0 && !y) return emu::set_bad_param(13);
  void* scratch = nullptr;
  if (static_scratch(&scratch) != cudaSuccess) return EMU_ERR_CUDA;
  const emu::Plan* pl = emu::get_plan(num_moduli);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // op(A) rows (i, h) and op(B) columns (j, h): strides as in the allocating entry point
  const int64_t rsa = transa == EMU_OP_N ? 1 : lda, hsa = transa == EMU_OP_N ? lda : 1;
  const int64_t rsb = transb == EMU_OP_N ? ldb : 1, hsb = transb == EMU_OP_N ? 1 : ldb;
  // launch_exponents clears the part of the scratch it uses before each pass
  cudaError_t e = cudaSuccess;
  if (m > 0) e = emu::launch_exponents(is_single != 0, A, m, k, rsa, hsa, *pl, x, scratch, st);
  if (e == cudaSuccess && n > 0) e = emu::launch_exponents(is_single != 0, B, n, k, rsb, hsb, *pl, y, scratch, st);
  return e == cudaSuccess ? EMU_OK : EMU_ERR_CUDA;
}
