// K1 (accurate mode, Section III-B eqs. mu-accu / nu-accu): the exact bound
// products of the 7-bit ceiling planes on the 5th-generation tensor cores,
// reduced on the fly to the row and column maxima the exponent rule needs.
#include "tc_common.cuh"

namespace emu {
namespace {

// Exact non-negative bound products of
// the 7-bit ceiling planes (entries <= 64, products <= 2^12).  Planes of both
// operands: 0 = X_R (real input: X), 1 = X_I, 2 = X_R - X_I.
//   complex: product 0 = C-bar_I = A-bar_I B-bar_R + A-bar_R B-bar_I (2 nkb k-blocks),
//            product 1 = (A-bar_R - A-bar_I)(B-bar_R - B-bar_I) (nkb k-blocks),
//            C-bar_R = C-bar_I + product 1 (the identity of Section III-B);
//   real:    product 0 = C-bar = A-bar B-bar.
// FP32 accumulation is exact while partial sums stay below 2^24, so each
// accumulation restarts every kBoundChunk k-blocks: 4096 k of products of
// magnitude at most 64 x 64 = 2^12, so every partial sum is at most 2^24 in
// magnitude, an integer FP32 holds exactly.
// A tile is 256 output rows wide (MMA N = 256): an MMA of N = 128 reads a
// third more operand bytes per flop and ran at about 0.75 of the rate the
// 256-wide residue products reach.  TMEM holds the two FP32 accumulators (256
// columns each), which a tile's chunks take in turn, so the MMA runs the next
// chunk in one while the epilogue empties the other.  The int32 running sum of
// the product being accumulated lives in the epilogue's registers (16 warps,
// each thread one TMEM lane and 64 of the 256 columns); the products run one
// after the other, and the finished C-bar_I sum of a complex tile is parked in
// global scratch (128 KB per CTA, read back by the thread that wrote it) while
// product 1 accumulates.
// At the end of a tile each epilogue thread holds one output column (TMEM
// lane) and 64 output rows; the row maxima over columns (5-step butterflies
// across the warp) and the column maxima over rows of max(C-bar_R, C-bar_I) go
// to global memory by atomicMax.  Rows/columns beyond m/n read TMA's zero
// fill, so they add nothing.
constexpr int kBoundBN = 256;          // output rows per tile (MMA N)
constexpr int kBoundChunk = 64;
constexpr int kBoundTmemCols = 512;    // 2 FP32 accumulators, 256 columns each
constexpr int kBoundEpi = 16;          // epilogue warps: 4 on each TMEM lane quadrant
constexpr int kBoundThreads = 32 * (2 + kBoundEpi);
constexpr int kBoundSums = kBoundBN / (kBoundEpi / 4);                  // 64 columns per epilogue thread
constexpr size_t kBoundScratchPerCta = static_cast<size_t>(BM) * kBoundBN * 4;   // 128 KB
constexpr int kBoundMaxCtas = 256;     // scratch bound of bound_scratch_bytes (GB300: 152 SMs)

// One-SM tiles: 128 output columns x 256 rows, 4 stages of 48 KB.  SM pairs
// (cta_group::2, a cluster of two CTAs): 256 columns x 256 rows, each CTA
// holding 128 of the columns in its TMEM and loading 128 of the A-bar rows, so
// a stage is 32 KB and 6 of them fit; the even CTA issues the MMAs (M = 256).
// Measured at ZGEMM 16384^3, N = 15 in accurate mode: the exponent phase took
// 15.9 ms on pairs against 18.5 on one SM, so pairs are the default.
template <bool PAIR>
struct BoundCfg {
  static constexpr int kRowsB = PAIR ? kBoundBN / 2 : kBoundBN;      // A-bar rows per CTA and stage
  static constexpr int kStageBytes = kStageA + kRowsB * BK * 2;
  static constexpr int kStages = PAIR ? 6 : 4;
  static constexpr int kSmem = kStages * kStageBytes + 1024 + 256;
  static constexpr int kTileCols = PAIR ? 2 * BM : BM;
  static constexpr uint32_t kIdesc = (1u << 4) | (static_cast<uint32_t>(kBoundBN >> 3) << 17) |
                                     (static_cast<uint32_t>(kTileCols >> 4) << 24);
};

struct BoundSched {
  int TJ, TI, tiles, group, nkb, real;
};

// which operand planes and k-block of the planes feed k-block kb of a product
__device__ __forceinline__ void bound_src(int prod, int kb, int nkb, bool real, int& pa, int& pb, int& kc) {
  if (real) { pa = 0; pb = 0; kc = kb; return; }
  if (prod == 1) { pa = 2; pb = 2; kc = kb; return; }
  if (kb < nkb) { pa = 0; pb = 1; kc = kb; }        // B-bar_R (MMA A) x A-bar_I (MMA B)
  else { pa = 1; pb = 0; kc = kb - nkb; }           // B-bar_I x A-bar_R
}

template <bool PAIR>
__device__ __forceinline__ void bound_body(const CUtensorMap* mapA, const CUtensorMap* mapB, const BoundSched& s,
                                           unsigned int* __restrict__ Mrow, unsigned int* __restrict__ Ncol,
                                           int* __restrict__ scratch, int64_t m, int64_t n, unsigned int* status) {
  using BC = BoundCfg<PAIR>;
  constexpr int BN = kBoundBN;
  constexpr int S = BC::kStages;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (base - raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(gbase + S * BC::kStageBytes);
  const uint32_t bar0 = smem_u32(bars);
  auto full = [&](int i) { return bar0 + 8u * i; };
  auto empty = [&](int i) { return bar0 + 8u * (S + i); };
  auto tfull = [&](int i) { return bar0 + 8u * (2 * S + i); };
  auto tempty = [&](int i) { return bar0 + 8u * (2 * S + 2 + i); };
  const uint32_t done = bar0 + 8u * (2 * S + 4);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * S + 5);
  volatile int* abort_s = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  Ctl ctl{status, abort_s};
  const bool real = s.real != 0;
  const int len0 = real ? s.nkb : 2 * s.nkb, len1 = real ? 0 : s.nkb;   // k-blocks of products 0 and 1
  const long long nunits = s.tiles;
  const uint32_t rank = PAIR ? cluster_rank() : 0u;
  const bool leader = rank == 0;
  const long long first = PAIR ? (blockIdx.x >> 1) : blockIdx.x;
  const long long step = PAIR ? (gridDim.x >> 1) : gridDim.x;

  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(full(i), 1);
      mbar_init(empty(i), 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(tfull(i), 1);
      mbar_init(tempty(i), (PAIR ? 2 : 1) * 32 * kBoundEpi);
    }
    mbar_init(done, 1);
    *abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 1) {
    if constexpr (PAIR) {
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                   "r"(kBoundTmemCols));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;\n");
    } else {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                   "r"(kBoundTmemCols));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
  }
  tc_fence_before();
  if constexpr (PAIR) cluster_sync(); else __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // the even CTA's barriers (the pair's loads count on its full barriers, both epilogues free its accumulators)
  const uint32_t full_c0 = PAIR ? map_to_rank(full(0), 0) : full(0);
  const uint32_t tempty_c0 = PAIR ? map_to_rank(tempty(0), 0) : tempty(0);
  auto wait_x = [&](uint32_t bar, uint32_t parity) {     // waits on barriers the other CTA arrives on
    return PAIR ? mbar_wait_cluster(bar, parity, ctl) : mbar_wait(bar, parity, ctl);
  };

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      long long it = 0;
      bool ok = true;
      for (long long u = first; ok && u < nunits; u += step) {
        int tj, ti;
        tile_coords(static_cast<int>(u), s.TJ, s.TI, s.group, tj, ti);
        for (int prod = 0; ok && prod < 2; ++prod) {
          const int len = prod ? len1 : len0;
          for (int kb = 0; kb < len; ++kb, ++it) {
            const int st = static_cast<int>(it % S);
            const uint32_t ph = static_cast<uint32_t>((it / S) & 1);
            if (!mbar_wait(empty(st), ph ^ 1u, ctl)) { ok = false; break; }
            int pa, pb, kc;
            bound_src(prod, kb, s.nkb, real, pa, pb, kc);
            const uint32_t sa = base + st * BC::kStageBytes;
            if constexpr (PAIR) {
              if (leader) mbar_expect_tx(full(st), static_cast<uint32_t>(2 * BC::kStageBytes));
              const uint32_t fb = full_c0 + 8u * st;
              tma_load_3d_pair(sa, mapA, fb, kc * BK, tj * BC::kTileCols + static_cast<int>(rank) * BM, pa);
              tma_load_3d_pair(sa + kStageA, mapB, fb, kc * BK, ti * BN + static_cast<int>(rank) * BC::kRowsB, pb);
            } else {
              mbar_expect_tx(full(st), BC::kStageBytes);
              tma_load_3d(sa, mapA, full(st), kc * BK, tj * BM, pa);
              tma_load_3d(sa + kStageA, mapB, full(st), kc * BK, ti * BN, pb);
            }
          }
        }
      }
      // drain: every load issued has landed (for a pair, the even CTA's barriers count both CTAs' loads)
      if (leader) {
        for (int st = 0; st < S; ++st) {
          if (it <= st) continue;
          const long long last = st + ((it - 1 - st) / S) * S;
          const uint32_t ph = static_cast<uint32_t>((last / S) & 1);
          const long long t0 = clock64();
          while (!(PAIR ? mbar_try_cluster(full(st), ph) : mbar_try(full(st), ph)) && clock64() - t0 < kWaitLimit) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer (for a pair: the even CTA)
    if (lane == 0 && leader) {
      long long it = 0;
      uint32_t used = 0u;                           // bit a: parity of accumulator a's uses
      bool ok = true;
      int pos = 0;                                   // chunks so far: accumulator pos & 1
      for (long long u = first; ok && u < nunits; u += step) {
        for (int prod = 0; ok && prod < 2; ++prod) {
          const int len = prod ? len1 : len0;
          for (int kb0 = 0; ok && kb0 < len; kb0 += kBoundChunk) {
            const int acc = pos++ & 1;
            if (!wait_x(tempty(acc), ((used >> acc) & 1u) ^ 1u)) { ok = false; break; }
            tc_fence_after();
            const uint32_t td = tmem + static_cast<uint32_t>(acc * BN);
            const int kb1 = min(len, kb0 + kBoundChunk);
            for (int kb = kb0; kb < kb1; ++kb, ++it) {
              const int st = static_cast<int>(it % S);
              const uint32_t ph = static_cast<uint32_t>((it / S) & 1);
              if (!wait_x(full(st), ph)) { ok = false; break; }
              tc_fence_after();
              const uint32_t sa = base + st * BC::kStageBytes;
              const uint64_t da = smem_desc(sa), db = smem_desc(sa + kStageA);
#pragma unroll
              for (int kk = 0; kk < BK / UK; ++kk) {
                const uint64_t off = static_cast<uint64_t>((kk * UK * 2) >> 4);
                if constexpr (PAIR) mma_f16_pair(td, da + off, db + off, BC::kIdesc, !(kb == kb0 && kk == 0));
                else mma_f16(td, da + off, db + off, BC::kIdesc, !(kb == kb0 && kk == 0));   // fresh sum per chunk
              }
              if constexpr (PAIR) mma_commit_pair(empty(st)); else mma_commit(empty(st));
            }
            if (!ok) break;
            if constexpr (PAIR) mma_commit_pair(tfull(acc)); else mma_commit(tfull(acc));
            used ^= 1u << acc;
          }
        }
      }
      if constexpr (PAIR) mma_commit_pair(done); else mma_commit(done);
      const long long t0 = clock64();
      while (!mbar_try(done, 0u) && clock64() - t0 < kWaitLimit) {
      }
    } else if (PAIR && lane == 0) {
      // the odd CTA: the even CTA's last commit arrives here once every MMA touching this CTA is done
      const long long t0 = clock64();
      while (!mbar_try(done, 0u) && clock64() - t0 < kWaitLimit) {
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int ew = warp - 2;
    const int quad = warp & 3;                       // TMEM lanes [32 quad, 32 quad + 32)
    const int part = ew >> 2;                        // columns [64 part, 64 part + 64) of a tile
    const uint32_t lane_base = tmem + (static_cast<uint32_t>(quad * 32) << 16) + static_cast<uint32_t>(part * kBoundSums);
    // this CTA's scratch: (lane l, tile column c) at c * BM + l, so a warp's stores are 128 contiguous bytes
    int* park = real ? nullptr
                     : scratch + static_cast<int64_t>(blockIdx.x) * (BM * kBoundBN) + (part * kBoundSums) * BM + quad * 32 + lane;
    uint32_t used = 0u;                              // bit a: parity of accumulator a's uses
    int pos = 0;
    bool ok = true;
    for (long long u = first; ok && u < nunits; u += step) {
      int tj, ti;
      tile_coords(static_cast<int>(u), s.TJ, s.TI, s.group, tj, ti);
      int sum[kBoundSums];                           // running sum of the product in progress
      for (int prod = 0; ok && prod < 2; ++prod) {
        const int len = prod ? len1 : len0;
        if (len == 0) continue;
#pragma unroll
        for (int q = 0; q < kBoundSums; ++q) sum[q] = 0;
        for (int kb0 = 0; kb0 < len; kb0 += kBoundChunk) {
          const int acc = pos++ & 1;                  // the FP32 accumulator of this chunk
          if (!mbar_wait(tfull(acc), (used >> acc) & 1u, ctl)) { ok = false; break; }
          tc_fence_after();
#pragma unroll
          for (int piece = 0; piece < kBoundSums / 16; ++piece) {
            uint32_t v[16];
            tmem_ld16(lane_base + static_cast<uint32_t>(acc * BN + 16 * piece), v);
            tmem_wait_ld();
#pragma unroll
            for (int q = 0; q < 16; ++q) sum[16 * piece + q] += static_cast<int>(__uint_as_float(v[q]));   // exact integer
          }
          tc_fence_before();
          if constexpr (PAIR) mbar_arrive_cluster(tempty_c0 + 8u * acc); else mbar_arrive(tempty(acc));
          used ^= 1u << acc;
        }
        if (!ok) break;
        if (prod == 0 && len1 > 0) {                 // C-bar_I waits in scratch while product 1 accumulates
#pragma unroll
          for (int q = 0; q < kBoundSums; ++q) park[q * BM] = sum[q];
        }
      }
      if (!ok) break;
      // max(C-bar_R, C-bar_I) = C-bar_I + max(product 1, 0) per (row, this column)
      if (len1 > 0) {
#pragma unroll
        for (int q = 0; q < kBoundSums; ++q) {
          const int ci = park[q * BM];
          sum[q] = max(ci + sum[q], ci);
        }
      }
      const int64_t col = static_cast<int64_t>(tj) * BC::kTileCols + static_cast<int64_t>(rank) * BM + quad * 32 + lane;
      unsigned int colmax = 0u;
#pragma unroll
      for (int q = 0; q < kBoundSums; ++q) colmax = max(colmax, static_cast<unsigned int>(sum[q]));
      // butterflies: lane L ends with the maximum over the warp of row 32 piece + L of this part
#pragma unroll
      for (int piece = 0; piece < kBoundSums / 32; ++piece) {
#pragma unroll
        for (int d = 16; d >= 1; d >>= 1) {
          const bool up = (lane & d) != 0;
#pragma unroll
          for (int t = 0; t < d; ++t) {
            const int send = up ? sum[32 * piece + t] : sum[32 * piece + t + d];
            const int keep = up ? sum[32 * piece + t + d] : sum[32 * piece + t];
            sum[32 * piece + t] = max(keep, __shfl_xor_sync(0xffffffffu, send, d));
          }
        }
        const int64_t row = static_cast<int64_t>(ti) * BN + part * kBoundSums + 32 * piece + lane;
        if (row < m) atomicMax(Mrow + row, static_cast<unsigned int>(sum[32 * piece]));
      }
      if (col < n) atomicMax(Ncol + col, colmax);
    }
  }

  tc_fence_before();
  if constexpr (PAIR) cluster_sync(); else __syncthreads();   // a pair: no CTA leaves while the MMAs touch it
  tc_fence_after();
  if (warp == 1) {
    if constexpr (PAIR)
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kBoundTmemCols));
    else
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kBoundTmemCols));
  }
}

__global__ void __launch_bounds__(kBoundThreads, 1)
    gemm_bound_kernel(const __grid_constant__ CUtensorMap mapA,   // B-bar planes: MMA operand A
                      const __grid_constant__ CUtensorMap mapB,   // A-bar planes: MMA operand B
                      const BoundSched s, unsigned int* __restrict__ Mrow, unsigned int* __restrict__ Ncol,
                      int* __restrict__ scratch, int64_t m, int64_t n, unsigned int* status) {
  bound_body<false>(&mapA, &mapB, s, Mrow, Ncol, scratch, m, n, status);
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kBoundThreads, 1)
    gemm_bound_pair_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                           const BoundSched s, unsigned int* __restrict__ Mrow, unsigned int* __restrict__ Ncol,
                           int* __restrict__ scratch, int64_t m, int64_t n, unsigned int* status) {
  bound_body<true>(&mapA, &mapB, s, Mrow, Ncol, scratch, m, n, status);
}

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace

// Scratch of a complex launch: 128 KB for each CTA it can run, at most one per
// one-SM tile or two per pair tile, capped at kBoundMaxCtas (a launch with less
// scratch runs fewer CTAs).  Real input needs none.
size_t bound_scratch_bytes(int64_t m, int64_t n) {
  if (m <= 0 || n <= 0) return 0;
  const int64_t ti = cdiv(m, kBoundBN);
  const int64_t one = cdiv(n, BM) * ti, two = 2 * cdiv(n, BoundCfg<true>::kTileCols) * ti;
  int64_t ctas = one > two ? one : two;
  if (ctas > kBoundMaxCtas) ctas = kBoundMaxCtas;
  return static_cast<size_t>(ctas) * kBoundScratchPerCta;
}

cudaError_t launch_gemm_bound(int64_t m, int64_t n, int64_t kpad, bool real, const void* planesA,
                              const void* planesB, unsigned int* Mrow, unsigned int* Ncol, void* scratch,
                              size_t scratch_bytes, unsigned int* status, cudaStream_t st, bool pair) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  if (kpad % BK || ((reinterpret_cast<uintptr_t>(planesA) | reinterpret_cast<uintptr_t>(planesB)) & 15u))
    return cudaErrorInvalidValue;
  // complex input: room for at least one CTA (a pair: two), 4-byte aligned
  const long long scr_ctas = real ? (1ll << 30) : static_cast<long long>(scratch_bytes / kBoundScratchPerCta);
  if (!real && (!scratch || (reinterpret_cast<uintptr_t>(scratch) & 3u) || scr_ctas < 1)) return cudaErrorInvalidValue;
  if (!get_encoder()) return cudaErrorNotSupported;
  static const cudaError_t attr = [] {
    cudaError_t e = cudaFuncSetAttribute(gemm_bound_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         BoundCfg<false>::kSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(gemm_bound_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               BoundCfg<true>::kSmem);
    return e;
  }();
  if (attr != cudaSuccess) return attr;
  // SM pairs that can run a CTA pair of the pair kernel at once (0: none)
  static const int clusters = [] {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * 1024);
    cfg.blockDim = dim3(kBoundThreads);
    cfg.dynamicSmemBytes = BoundCfg<true>::kSmem;
    int v = 0;
    if (cudaOccupancyMaxActiveClusters(&v, gemm_bound_pair_kernel, &cfg) != cudaSuccess) {
      cudaGetLastError();
      v = 0;
    }
    return v;
  }();
  if (clusters <= 0 || scr_ctas < 2) pair = false;   // no room for a CTA pair: one-SM tiles
  const int planes = real ? 1 : 3;
  const int cols = pair ? BoundCfg<true>::kTileCols : BM;
  CUtensorMap mapA, mapB;
  if (!make_map(&mapA, planesB, n, kpad, planes, BM)) return cudaErrorInvalidValue;
  if (!make_map(&mapB, planesA, m, kpad, planes, pair ? BoundCfg<true>::kRowsB : kBoundBN)) return cudaErrorInvalidValue;
  BoundSched s;
  s.TJ = static_cast<int>(cdiv(n, cols));
  s.TI = static_cast<int>(cdiv(m, kBoundBN));
  s.tiles = s.TJ * s.TI;
  s.group = pair ? 8 : 16;                 // the same column span (2048) in a raster group
  s.nkb = static_cast<int>(kpad / BK);
  s.real = real ? 1 : 0;
  int* scr = static_cast<int*>(scratch);
  if (pair) {
    long long p = s.tiles < clusters ? s.tiles : clusters;
    if (p > scr_ctas / 2) p = scr_ctas / 2;
    gemm_bound_pair_kernel<<<static_cast<unsigned int>(2 * p), kBoundThreads, BoundCfg<true>::kSmem, st>>>(
        mapA, mapB, s, Mrow, Ncol, scr, m, n, status);
  } else {
    long long grid = s.tiles < g_sms ? s.tiles : g_sms;
    if (grid > scr_ctas) grid = scr_ctas;
    gemm_bound_kernel<<<static_cast<unsigned int>(grid), kBoundThreads, BoundCfg<false>::kSmem, st>>>(
        mapA, mapB, s, Mrow, Ncol, scr, m, n, status);
  }
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace emu
