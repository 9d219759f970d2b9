// K4 on the tensor cores: the CRT sum of Algorithm 1 Steps V-v/V-vi as an
// exact fp16 matrix product, then the same exact limb arithmetic and rounding
// as the integer CRT (k_crt.cu).
//
// For one output column j and 128 consecutive rows i, the residues of all
// J = 3N jobs (D_l, E_l, F_l of eq. karatsuba; J = N for real input) form a
// 128 x J matrix R of integers in [-128, 127].  Cut every CRT weight into
// balanced base-2^b digits, w_l = sum_c d_lc 2^(b c) with |d_lc| <= 2^(b-1).
// Then the real part's sum is
//   V_R = sum_l w_l (D_l - E_l) = sum_c 2^(b c) S_c,   S_c = sum_l d_lc (D_l - E_l),
// and likewise the imaginary part with F_l - D_l - E_l.  Every S_c is the
// product of R with a column of a constant J x 32 matrix W of digits (with the
// Karatsuba signs), so one tcgen05.mma kind::f16 (M = 128 rows, N = 32 or 64
// columns, K = J + 1 rounded up to 16) gives all of them.  The products and
// every partial sum are integers below 2^23 in magnitude (|R| <= 128, 3N
// terms, |d| <= 512 for N <= 16 and |d| <= 256 with b = 9 above), so the FP32
// accumulator holds them exactly.  One more K entry adds 1.5 * 2^23 to every
// digit column, so the FP32 bits of the result are 0x4B400000 + S_c: an
// integer that goes straight into the limb sums (the constant is taken back
// in the plan's K).  Two more columns per part hold sum_l (w_l / P) times the
// residues from fp16 hi/lo splits of w_l / P; their sum is the quotient
// estimate (error far below the 1/8 margin of condition (cond)).
//
// The epilogue (one thread per row, reading its TMEM lane) forms, modulo
// 2^(32L), c' = sum_c S_c 2^(b c) - r P with r = rint(estimate), carried
// once, range-fixed in accurate mode and rounded once to binary64 by the
// integer routine shared with k_crt.cu.  The result is bit-identical to the
// CUDA-core CRT.
//
// A persistent block of 128 threads owns 32 (64) TMEM columns and walks
// (column, 128-row block) items; the next item's residue bytes are copied into
// shared memory (cp.async, double-buffered) while the current one is
// converted to fp16, multiplied and finished.  The MMA completion wait is
// bounded: on expiry the block records EMU_ERR_TIMEOUT, drains and frees its
// TMEM and returns.
#include <cuda_fp16.h>

#include <climits>
#include <type_traits>

#include "crt_common.cuh"
#include "tc_common.cuh"

namespace emu {
namespace {

constexpr int kTcThreads = 128;          // one output row per thread: the MMA's M = 128 TMEM lanes
constexpr int kStageRow = 144;           // staging bytes per job (128 rows + 16: conflict-free reads)
constexpr uint32_t kMagicBits = 0x4B400000u;
constexpr float kMagic = 12582912.0f;    // 1.5 * 2^23

// Column layout of one kernel variant: parts (real 1, complex 2) of kSlot
// columns each, digits in the first kDig, the estimate's hi and lo in the last two.
template <bool REAL, bool WIDE>
struct TcLayout {
  static constexpr int kParts = REAL ? 1 : 2;
  static constexpr int kNC = (!REAL && WIDE) ? 64 : 32;
  static constexpr int kSlot = kNC / kParts;
  static constexpr int kDig = kSlot - 2;
  static constexpr int kB = (!REAL && WIDE) ? 9 : 10;
  static constexpr int kDigTable = kB == 10 ? 0 : 1;                 // Plan::tcdig / tcmul index
  static constexpr int kKTable = REAL ? 2 : (WIDE ? 1 : 0);          // Plan::tcK index
  // kind::f16, D = F32, A = B = F16, A MN-major (rows contiguous), B K-major, M = 128, N = kNC
  static constexpr uint32_t kIdesc = (1u << 4) | (1u << 15) | (static_cast<uint32_t>(kNC >> 3) << 17) |
                                     (static_cast<uint32_t>(128 >> 4) << 24);
  static constexpr int kBTileBytes = kNC * 32;                       // one K tile of 16: kNC x 16 fp16
};

// no-swizzle operand descriptor: core matrices of 8 x 16 bytes, `lbo` apart
// along K and `sbo` apart along M/N
__device__ __forceinline__ uint64_t plain_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = static_cast<uint64_t>((saddr >> 4) & 0x3FFFu);
  d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
  d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
  d |= static_cast<uint64_t>(1) << 46;
  return d;
}

// A operand (residues), MN-major: element (row m, job k) of K tile k / 16
__device__ __forceinline__ uint32_t a_off(int m, int k) {
  return static_cast<uint32_t>((k >> 4) * 4096 + (m >> 3) * 256 + ((k >> 3) & 1) * 128 + (k & 7) * 16 + (m & 7) * 2);
}
// B operand (digits), K-major: element (column n, job k)
template <int NC>
__device__ __forceinline__ uint32_t b_off(int n, int k) {
  return static_cast<uint32_t>((k >> 4) * (NC * 32) + (n >> 3) * 256 + ((k >> 3) & 1) * 128 + (n & 7) * 16 +
                               (k & 7) * 2);
}

// 4 residue bytes (two's complement) -> 4 fp16 values, two per word: the byte
// + 128 becomes the low mantissa bits of 1024 + (byte + 128), then 1152 is subtracted
__device__ __forceinline__ void bytes_to_half4(uint32_t w, uint32_t& h01, uint32_t& h23) {
  const uint32_t u = w ^ 0x80808080u;
  uint32_t a, b;
  asm("prmt.b32 %0, %1, %2, 0x5150;" : "=r"(a) : "r"(u), "r"(0x64646464u));
  asm("prmt.b32 %0, %1, %2, 0x5352;" : "=r"(b) : "r"(u), "r"(0x64646464u));
  const __half2 bias = __halves2half2(__ushort_as_half(0x6480u), __ushort_as_half(0x6480u));   // 1152
  const __half2 ha = __hsub2(*reinterpret_cast<const __half2*>(&a), bias);
  const __half2 hb = __hsub2(*reinterpret_cast<const __half2*>(&b), bias);
  h01 = *reinterpret_cast<const uint32_t*>(&ha);
  h23 = *reinterpret_cast<const uint32_t*>(&hb);
}

// Position of one item: problem p (grouped calls), output column j, rows
// [row0, row0 + 128); j < 0 marks the end.  Only this moves from item to
// item; the problem's pointers, sizes and alpha/beta are read through
// Work::prob(p).  Item counts stay below 2^31 (the launcher checks).
struct TcPos {
  int p, j, row0;
};

// One GEMM.  The block's items are first, first + stride, ...: the cursor
// (column, row block) advances by a fixed step, no division per item.
struct TcSingle {
  const int8_t* res;
  int64_t ldr, m, n, ldc;
  const int16_t* x;
  const int16_t* y;
  void* C;
  double ar, ai, br, bi;
  int flags;
  int iblocks, ncols;
  struct Cursor {
    int j, ib;
  };
  __device__ Cursor begin(int first) const { return Cursor{first / iblocks, first % iblocks}; }
  __device__ void steps(int stride, int& dj, int& dib) const {
    dj = stride / iblocks;
    dib = stride % iblocks;
  }
  __device__ void advance(Cursor& c, int dj, int dib) const {
    c.ib += dib;
    c.j += dj;
    if (c.ib >= iblocks) {
      c.ib -= iblocks;
      ++c.j;
    }
  }
  __device__ TcPos pos(const Cursor& c) const { return TcPos{0, c.j < ncols ? c.j : -1, c.ib * 128}; }
  __device__ const TcSingle& prob(int) const { return *this; }
};

// Many problems (a grouped call): CrtProb descriptors whose block_begin is the
// first item and iblocks the 128-row blocks of each problem.  A block's items
// only move forward, so the cursor keeps its problem and steps past the
// problems it has left (binary search only for the first item).
struct TcGrouped {
  const CrtProb* probs;
  int nprob;
  int total;
  struct Cursor {
    int it, p;
  };
  __device__ Cursor begin(int first) const {
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (probs[mid].block_begin <= first) lo = mid; else hi = mid - 1;
    }
    return Cursor{first, lo};
  }
  __device__ void steps(int stride, int& dj, int& dib) const {
    dj = stride;
    dib = 0;
  }
  __device__ void advance(Cursor& c, int dj, int) const {
    c.it += dj;
    while (c.p + 1 < nprob && probs[c.p + 1].block_begin <= c.it) ++c.p;
  }
  __device__ TcPos pos(const Cursor& cur) const {
    if (cur.it >= total) return TcPos{0, -1, 0};
    const unsigned local = static_cast<unsigned>(cur.it - probs[cur.p].block_begin);
    const unsigned ib = static_cast<unsigned>(probs[cur.p].iblocks);
    return TcPos{cur.p, static_cast<int>(local / ib), static_cast<int>(local % ib) * 128};
  }
  __device__ const CrtProb& prob(int p) const { return probs[p]; }
};

// A thread's share of an item's residue bytes: the 16-row chunk q0 of jobs
// k0, k0 + 16, k0 + 32, ... (k0 = 8 (tid / 64) + tid % 8, q0 = (tid / 8) % 8),
// so that the 8 threads of a quarter warp touch 8 different 16-byte bank
// groups both in the staging buffer (job stride 144 bytes) and in operand A.
constexpr int kMaxUnits = 5;                      // ceil(72 / 16): J <= 3 x 24
struct Units {
  int n;                    // jobs of this thread
  int k0;
  uint32_t s0;              // staging offset of job k0
  uint32_t a0;              // operand A offset of (row 16 q0, job k0)
  int q0;
};

__device__ __forceinline__ Units units_of(int J) {
  Units u;
  const int k0 = ((threadIdx.x >> 6) << 3) + (threadIdx.x & 7);
  u.q0 = (threadIdx.x >> 3) & 7;
  u.n = k0 < J ? (J - k0 + 15) >> 4 : 0;
  u.k0 = k0;
  u.s0 = static_cast<uint32_t>(k0 * kStageRow + 16 * u.q0);
  u.a0 = a_off(16 * u.q0, k0);
  return u;
}

// Stage the residue bytes of the item at `t` of problem q (rows from
// round_up(m, 16) on are not read).
template <class Q>
__device__ __forceinline__ void stage_item(const Q& q, const TcPos& t, const Units& u, uint32_t stage) {
  const int64_t rows_stored = (q.m + 15) / 16 * 16;
  if (t.row0 + 16 * u.q0 >= rows_stored) return;
  const int64_t plane = q.n * q.ldr;
  const int8_t* g = q.res + (static_cast<int64_t>(u.k0) * plane + 16 * u.q0 + static_cast<int64_t>(t.j) * q.ldr +
                             t.row0);
#pragma unroll
  for (int r = 0; r < kMaxUnits; ++r) {
    if (r >= u.n) break;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(stage + u.s0 + r * 16 * kStageRow),
                 "l"(g + r * 16 * plane)
                 : "memory");
  }
}

// fp16 operand A from the staged bytes of this thread's chunks
__device__ __forceinline__ void convert_item(const Units& u, const uint8_t* stage, uint8_t* sA) {
#pragma unroll
  for (int r = 0; r < kMaxUnits; ++r) {
    if (r >= u.n) break;
    const uint4 w = *reinterpret_cast<const uint4*>(stage + u.s0 + r * 16 * kStageRow);
    uint4 lo, hi;
    bytes_to_half4(w.x, lo.x, lo.y);
    bytes_to_half4(w.y, lo.z, lo.w);
    bytes_to_half4(w.z, hi.x, hi.y);
    bytes_to_half4(w.w, hi.z, hi.w);
    *reinterpret_cast<uint4*>(sA + u.a0 + r * 4096) = lo;
    *reinterpret_cast<uint4*>(sA + u.a0 + r * 4096 + 256) = hi;
  }
}

// One part's value from its TMEM columns v[0 .. kSlot): the digit sums (with
// the 1.5 * 2^23 bias in their bits) into L limbs starting at the plan's K,
// the quotient from the estimate columns, then c' carried, range-fixed and
// rounded.
template <class LY, int L, bool ROBUST>
__device__ __forceinline__ double tc_part(const uint32_t* v, const Plan& pl, int e2) {
  const float est = __uint_as_float(v[LY::kDig]) + __uint_as_float(v[LY::kDig + 1]);
  // r + R0 from the bits of est + 1.5 * 2^23 (|est| < 2^21)
  const uint32_t rq = __float_as_uint(est + kMagic) - (kMagicBits - static_cast<uint32_t>(pl.R0));
  uint64_t acc[L];
#pragma unroll
  for (int t = 0; t < L; ++t) acc[t] = pl.tcK[LY::kKTable][t];
#pragma unroll
  for (int c = 0; c < LY::kDig; ++c) {
    constexpr int kB = LY::kB;
    const int t = (kB * c) >> 5;
    if (t < L) acc[t] = mad_wide(v[c], pl.tcmul[LY::kDigTable][c], acc[t]);
  }
  uint32_t cl[L];
  uint64_t carry = 0;
#pragma unroll
  for (int t = 0; t < L; ++t) {
    const uint64_t s = mad_wide(rq, pl.negP[t], acc[t]) + carry;
    cl[t] = static_cast<uint32_t>(s);
    carry = s >> 32;
  }
  if constexpr (ROBUST) fix_range<L>(cl, pl);
  return round_exact<L>(cl, e2);
}

// Outputs of one item from its TMEM accumulator (columns tcol ..): thread = row.
template <bool SINGLE, bool REAL, bool WIDE, int L, bool ROBUST, class Q>
__device__ __forceinline__ void tc_epilogue(const Q& q, const TcPos& t, uint32_t tcol, const Plan& pl) {
  using LY = TcLayout<REAL, WIDE>;
  const int warp = threadIdx.x >> 5;
  const int64_t i = t.row0 + threadIdx.x;
  const uint32_t lane_base = tcol + (static_cast<uint32_t>(warp * 32) << 16);
  const bool active = i < q.m;
  const int xi = active ? q.x[i] : 0;
  const int yj = q.y[t.j];
  const bool nan = (xi == kExpNonfinite || yj == kExpNonfinite);
  const int e2 = -(xi + yj);
  double o[2] = {0.0, 0.0};
  if constexpr (WIDE) {
#pragma unroll
    for (int part = 0; part < 2; ++part) {
      uint32_t v[32];
      tmem_ld32(lane_base + static_cast<uint32_t>(part * 32), v);
      tmem_wait_ld();
      o[part] = tc_part<LY, L, ROBUST>(v, pl, e2);
    }
  } else {
    uint32_t v[32];
    tmem_ld32(lane_base, v);
    tmem_wait_ld();
    o[0] = tc_part<LY, L, ROBUST>(v, pl, e2);
    if constexpr (!REAL) o[1] = tc_part<LY, L, ROBUST>(v + LY::kSlot, pl, e2);
  }
  if (!active) return;
  const int64_t ci = static_cast<int64_t>(t.j) * q.ldc + i;
  const double qnan = __longlong_as_double(0x7FF8000000000000ll);
  if constexpr (REAL) {
    double val = nan ? qnan : o[0];
    if (!(q.flags & kCrtPlain)) {
      double u = __dmul_rn(q.ar, val);
      if (q.flags & kCrtBeta)
        u = __fma_rn(q.br, SINGLE ? static_cast<double>(static_cast<const float*>(q.C)[ci])
                                  : static_cast<const double*>(q.C)[ci], u);
      val = u;
    }
    if (SINGLE) static_cast<float*>(q.C)[ci] = __double2float_rn(val);
    else static_cast<double*>(q.C)[ci] = val;
  } else {
    double orr = nan ? qnan : o[0];
    double oi = nan ? qnan : o[1];
    if (!(q.flags & kCrtPlain)) {
      double tr = __fma_rn(q.ar, orr, -__dmul_rn(q.ai, oi));
      double ti = __fma_rn(q.ar, oi, __dmul_rn(q.ai, orr));
      if (q.flags & kCrtBeta) {
        double cr, cim;
        if (SINGLE) {
          const float2 cv = static_cast<const float2*>(q.C)[ci];
          cr = cv.x;
          cim = cv.y;
        } else {
          const double2 cv = static_cast<const double2*>(q.C)[ci];
          cr = cv.x;
          cim = cv.y;
        }
        tr = __fma_rn(q.br, cr, __fma_rn(-q.bi, cim, tr));
        ti = __fma_rn(q.br, cim, __fma_rn(q.bi, cr, ti));
      }
      orr = tr;
      oi = ti;
    }
    if (SINGLE) static_cast<float2*>(q.C)[ci] = make_float2(__double2float_rn(orr), __double2float_rn(oi));
    else static_cast<double2*>(q.C)[ci] = make_double2(orr, oi);
  }
}

// The block's items are pipelined two deep: item n is converted into an A
// buffer and its MMA issued into accumulator slot n & 1, then item n - 1's
// outputs are finished from the other slot while that MMA runs; item n + 1's
// bytes are copied in meanwhile (each thread stages and converts the same
// chunks, so one staging buffer suffices).  NBUF = 2: A buffer n & 1, and item
// n - 1's MMA is waited for after item n's is issued.  NBUF = 1: one A buffer,
// written once item n - 1's MMA has read it (issued a whole epilogue earlier,
// so this seldom waits); the smaller block fits as many blocks per SM as the
// TMEM columns allow.  Measured: single launches (ZGEMM 4096^3, N = 14) ran
// 5 % more instructions with one buffer at the same 6 blocks, and at ZGEMM
// 16384^3 (N = 15) took 5.47 ms with one buffer at 8 blocks against 5.36-5.39
// with two at 6; grouped launches (N = 16) gained from 5 to 8 blocks.  So
// single launches take 2, grouped 1.
template <bool SINGLE, bool REAL, bool WIDE, int L, bool ROBUST, int NBUF, class Work>
__device__ __forceinline__ void crt_tc_body(const Work& W, const Plan& pl, unsigned int* status) {
  using LY = TcLayout<REAL, WIDE>;
  constexpr int kNC = LY::kNC;
  const int J = (REAL ? 1 : 3) * pl.N;
  const int KT = (J + 1 + 15) >> 4;                      // K tiles: jobs, the bias entry, zero padding
  const int a_bytes = KT * 4096;
  extern __shared__ __align__(128) uint8_t tc_smem[];
  uint8_t* sB = tc_smem;                                  // KT x kBTileBytes
  uint8_t* sA = sB + KT * LY::kBTileBytes;                // NBUF x KT x 4096
  uint8_t* sS = sA + NBUF * a_bytes;                      // J x kStageRow
  const int stage_bytes = (J * kStageRow + 127) / 128 * 128;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sS + stage_bytes);   // MMA done, per slot
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2);
  volatile int* abort_s = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5;
  const uint32_t bar0 = smem_u32(bars);

  if (threadIdx.x == 0) {
    mbar_init(bar0, 1);
    mbar_init(bar0 + 8, 1);
    *abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"(2 * kNC));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  // constant operand B: digits (with the Karatsuba signs), the estimate's hi/lo, the bias entry
  for (int e = threadIdx.x; e < kNC * KT * 16; e += kTcThreads) {
    const int n = e % kNC, k = e / kNC;
    const int part = n / LY::kSlot, c = n % LY::kSlot;
    float val = 0.0f;
    if (k < J) {
      const int l = REAL ? k : k / 3, comp = REAL ? 0 : k % 3;
      // real part: D - E; imaginary part: F - D - E
      const int coef = REAL ? 1 : (part == 0 ? (comp == 0 ? 1 : (comp == 1 ? -1 : 0)) : (comp == 2 ? 1 : -1));
      if (coef != 0) {
        if (c < LY::kDig) val = static_cast<float>(coef * pl.tcdig[LY::kDigTable][l][c]);
        else val = static_cast<float>(coef) * __half2float(__ushort_as_half(pl.tcest[l][c - LY::kDig]));
      }
    } else if (k == J && c < LY::kDig) {
      val = 6144.0f;                                      // x 2048 in A: 1.5 * 2^23
    }
    *reinterpret_cast<__half*>(sB + b_off<kNC>(n, k)) = __float2half_rn(val);
  }
  // A's columns past the jobs, in every buffer: 2048 in the bias entry, zeros after it
  for (int e = threadIdx.x; e < NBUF * 128 * (KT * 16 - J); e += kTcThreads) {
    const int m = e & 127, k = J + ((e >> 7) % (KT * 16 - J)), b = (e >> 7) / (KT * 16 - J);
    *reinterpret_cast<__half*>(sA + b * a_bytes + a_off(m, k)) = __float2half_rn(k == J ? 2048.0f : 0.0f);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const Ctl ctl{status, abort_s};

  const Units U = units_of(J);
  const uint32_t sS_a = smem_u32(sS);
  const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
  int dj, dib;
  W.steps(static_cast<int>(gridDim.x), dj, dib);
  typename Work::Cursor cursor = W.begin(static_cast<int>(blockIdx.x));
  TcPos cur = W.pos(cursor);
  if (cur.j >= 0) stage_item(W.prob(cur.p), cur, U, sS_a);
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  uint32_t ph = 0u;                                       // bit s: parity of slot s's next completion
  uint32_t pending = 0u;                                  // bit s: a commit of slot s not yet waited for
  TcPos prev{0, -1, 0};
  // one pipeline step with accumulator slot SLOT for `cur` (SLOT ^ 1 for
  // `prev`); false when the block is done
  auto step = [&](auto slot_c) -> bool {
    constexpr int SLOT = decltype(slot_c)::value;
    constexpr int PS = SLOT ^ 1;
    constexpr int AB = NBUF == 1 ? 0 : SLOT;             // A buffer of `cur`
    TcPos next{0, -1, 0};
    // an expired wait sets the abort flag (seen by every thread after the next barrier);
    // the status word then reports the timeout
    auto wait_prev = [&]() {
      if (mbar_wait(bar0 + 8 * PS, (ph >> PS) & 1u, ctl)) {
        pending &= ~(1u << PS);
        ph ^= 1u << PS;
      }
    };
    if (NBUF == 1 && prev.j >= 0) wait_prev();             // prev's MMA has read the one A buffer
    if (cur.j >= 0) {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
      convert_item(U, sS, sA + AB * a_bytes);
      // the next item's bytes: this thread's chunks only, which it has just converted
      W.advance(cursor, dj, dib);
      next = W.pos(cursor);
      if (next.j >= 0) stage_item(W.prob(next.p), next, U, sS_a);
      asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    // A's generic-proxy writes become visible to the tensor core; earlier TMEM reads are done
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (*abort_s) return false;                           // read after the barrier: the same in every thread
    if (cur.j >= 0) {
      if (threadIdx.x == 0) {
        for (int kt = 0; kt < KT; ++kt)
          mma_f16(tmem + SLOT * kNC, plain_desc(a0 + AB * a_bytes + kt * 4096, 128, 256),
                  plain_desc(b0 + kt * LY::kBTileBytes, 128, 256), LY::kIdesc, kt > 0);
        mma_commit(bar0 + 8 * SLOT);
      }
      pending |= 1u << SLOT;
    }
    if (prev.j >= 0) {
      if (NBUF == 2) {
        wait_prev();
        tc_fence_after();
      }
      tc_epilogue<SINGLE, REAL, WIDE, L, ROBUST>(W.prob(prev.p), prev, tmem + PS * kNC, pl);
      tc_fence_before();
    }
    if (cur.j < 0) return false;
    prev = cur;
    cur = next;
    return true;
  };
  while (step(std::integral_constant<int, 0>()) && step(std::integral_constant<int, 1>())) {
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  // teardown: MMAs whose completion was not waited for (only after an expired wait) are drained
  if (threadIdx.x == 0) {
    for (int sl = 0; sl < 2; ++sl) {
      if (!((pending >> sl) & 1u)) continue;
      const long long t0 = clock64();
      while (!mbar_try(bar0 + 8 * sl, (ph >> sl) & 1u) && clock64() - t0 < kWaitLimit) {
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(2 * kNC));
}

// Minimum resident blocks (which caps registers per thread): 8 blocks of 64
// registers fill an SM (as many as its TMEM holds).  Single launches of four
// complex limbs (N >= 13: three or more K tiles, two A buffers) fit 6 blocks
// by shared memory, so they may use 80 registers, as may the ones that would
// spill at 64 (one limb; two or three real limbs); grouped launches of four
// limbs (one A buffer) fit 8; the 64-column ones (fewer blocks by TMEM) about 100.
template <bool REAL, bool WIDE, int L, bool GROUPED = false>
constexpr int tc_min_blocks() {
  return WIDE ? 5 : ((L == 1 || (REAL && (L == 2 || L == 3)) || (!GROUPED && !REAL && L == 4)) ? 6 : 8);
}

template <bool SINGLE, bool REAL, bool WIDE, int L, bool ROBUST>
__global__ void __launch_bounds__(kTcThreads, (tc_min_blocks<REAL, WIDE, L>())) crt_tc_kernel(const TcSingle W, const __grid_constant__ Plan pl,
                                                            unsigned int* status) {
  crt_tc_body<SINGLE, REAL, WIDE, L, ROBUST, 2>(W, pl, status);
}

template <bool SINGLE, bool WIDE, int L>
__global__ void __launch_bounds__(kTcThreads, (tc_min_blocks<false, WIDE, L, true>())) crt_tc_grouped_kernel(const TcGrouped W, const __grid_constant__ Plan pl,
                                                                    unsigned int* status) {
  crt_tc_body<SINGLE, false, WIDE, L, false, 1>(W, pl, status);
}

// Shared memory of one block: operand B, the A buffers (2 for single
// launches, 1 for grouped ones), the staging buffer, barriers; raised so that
// no more blocks fit on an SM than its 512 TMEM columns hold (2 x 32 or 2 x 64
// columns a block).  GB300: 228 KB per SM, 1 KB of it reserved per resident
// block.
constexpr int kSmemPerSM = 228 * 1024;

int tc_max_blocks(bool real, bool wide) { return 512 / (2 * ((!real && wide) ? 64 : 32)); }

size_t tc_smem_bytes(bool real, bool wide, int N, bool grouped) {
  const int J = (real ? 1 : 3) * N;
  const int KT = (J + 1 + 15) / 16;
  const int nc = (!real && wide) ? 64 : 32;
  const size_t stage = static_cast<size_t>((J * kStageRow + 127) / 128 * 128);
  const int nbuf = grouped ? 1 : 2;                       // A buffers (crt_tc_body's NBUF)
  size_t need = static_cast<size_t>(KT) * (nc * 32 + nbuf * 4096) + stage + 64;
  const int maxb = tc_max_blocks(real, wide);
  const size_t floor_bytes = static_cast<size_t>(kSmemPerSM / (maxb + 1) - 1024 + 128);   // maxb + 1 blocks do not fit
  if (need < floor_bytes) need = floor_bytes;
  return (need + 127) / 128 * 128;
}

template <class K>
cudaError_t prep(K* kern, size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void*>(kern), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(reinterpret_cast<const void*>(kern), cudaFuncAttributePreferredSharedMemoryCarveout,
                             static_cast<int>(cudaSharedmemCarveoutMaxShared));
  return e;
}

// persistent grid: the blocks that fit on every SM at once (by shared memory, which also bounds
// them by TMEM), or fewer when there are fewer items
int tc_grid(long long items, size_t smem) {
  get_encoder();                                             // sets g_sms
  int per_sm = static_cast<int>(kSmemPerSM / (smem + 1024));
  if (per_sm < 1) per_sm = 1;
  const long long g = static_cast<long long>(g_sms > 0 ? g_sms : 148) * per_sm;
  return static_cast<int>(items < g ? items : g);
}

template <bool SINGLE, bool REAL, bool WIDE, int L, bool ROBUST>
cudaError_t launch_tc_v(const TcSingle& W, long long items, const Plan& pl, unsigned int* status, cudaStream_t st) {
  const size_t smem = tc_smem_bytes(REAL, WIDE, pl.N, false);
  cudaError_t e = prep(crt_tc_kernel<SINGLE, REAL, WIDE, L, ROBUST>, smem);
  if (e != cudaSuccess) return e;
  const int grid = tc_grid(items, smem);
  crt_tc_kernel<SINGLE, REAL, WIDE, L, ROBUST><<<grid, kTcThreads, smem, st>>>(W, pl, status);
  count_launches(1);
  return cudaGetLastError();
}

template <bool SINGLE, bool REAL, int L>
cudaError_t launch_tc_r(const TcSingle& W, long long items, const Plan& pl, unsigned int* status, cudaStream_t st,
                        bool robust) {
  constexpr bool kWide = !REAL && L >= 5;
  return robust ? launch_tc_v<SINGLE, REAL, kWide, L, true>(W, items, pl, status, st)
                : launch_tc_v<SINGLE, REAL, kWide, L, false>(W, items, pl, status, st);
}

template <int L>
cudaError_t launch_tc_l(bool single, bool real, const TcSingle& W, long long items, const Plan& pl,
                        unsigned int* status, cudaStream_t st, bool robust) {
  if (real)
    return single ? launch_tc_r<true, true, L>(W, items, pl, status, st, robust)
                  : launch_tc_r<false, true, L>(W, items, pl, status, st, robust);
  return single ? launch_tc_r<true, false, L>(W, items, pl, status, st, robust)
                : launch_tc_r<false, false, L>(W, items, pl, status, st, robust);
}

template <bool SINGLE, int L>
cudaError_t launch_tc_grouped_l(const TcGrouped& W, const Plan& pl, unsigned int* status, cudaStream_t st,
                                bool prepare_only) {
  constexpr bool kWide = L >= 5;
  const size_t smem = tc_smem_bytes(false, kWide, pl.N, true);
  cudaError_t e = prep(crt_tc_grouped_kernel<SINGLE, kWide, L>, smem);
  if (e != cudaSuccess || prepare_only) return e;
  const int grid = tc_grid(W.total, smem);
  crt_tc_grouped_kernel<SINGLE, kWide, L><<<grid, kTcThreads, smem, st>>>(W, pl, status);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace

// One launch over every problem of a grouped call (complex; fast scaling).
// probs: device descriptors with block_begin = first 128-row item, iblocks =
// 128-row blocks of each problem (crt_tc_prob_items).  prepare_only sets the
// kernel's attributes without launching (before a stream capture).
cudaError_t launch_crt_tc_grouped(bool single, const CrtProb* probs_dev, int nprob, long long items, const Plan& pl,
                                  unsigned int* status, cudaStream_t st, bool prepare_only) {
  if (!prepare_only && (nprob <= 0 || items <= 0)) return cudaSuccess;
  if ((!status && !prepare_only) || items > INT_MAX) return cudaErrorInvalidValue;
  const TcGrouped W{probs_dev, nprob, static_cast<int>(items)};
  switch (pl.L) {
    case 1: return single ? launch_tc_grouped_l<true, 1>(W, pl, status, st, prepare_only)
                          : launch_tc_grouped_l<false, 1>(W, pl, status, st, prepare_only);
    case 2: return single ? launch_tc_grouped_l<true, 2>(W, pl, status, st, prepare_only)
                          : launch_tc_grouped_l<false, 2>(W, pl, status, st, prepare_only);
    case 3: return single ? launch_tc_grouped_l<true, 3>(W, pl, status, st, prepare_only)
                          : launch_tc_grouped_l<false, 3>(W, pl, status, st, prepare_only);
    case 4: return single ? launch_tc_grouped_l<true, 4>(W, pl, status, st, prepare_only)
                          : launch_tc_grouped_l<false, 4>(W, pl, status, st, prepare_only);
    case 5: return single ? launch_tc_grouped_l<true, 5>(W, pl, status, st, prepare_only)
                          : launch_tc_grouped_l<false, 5>(W, pl, status, st, prepare_only);
    case 6: return single ? launch_tc_grouped_l<true, 6>(W, pl, status, st, prepare_only)
                          : launch_tc_grouped_l<false, 6>(W, pl, status, st, prepare_only);
    default: return cudaErrorInvalidValue;
  }
}

// 128-row items of one problem of a grouped call (sets iblocks and flags).
long long crt_tc_prob_items(CrtProb& c) {
  c.iblocks = static_cast<int>((c.m + 127) / 128);
  c.flags = crt_flags(c.ar, c.ai, c.br, c.bi);
  return static_cast<long long>(c.n) * c.iblocks;
}

// The tensor-core CRT of one GEMM (same arguments and result as launch_crt).
cudaError_t launch_crt_tc(bool single, int64_t m, int64_t n, const Plan& pl, const int8_t* res, int64_t ldr,
                          const int16_t* x, const int16_t* y, double ar, double ai, double br, double bi, void* C,
                          int64_t ldc, cudaStream_t st, bool real, bool robust, unsigned int* status) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  if (ldr % 16 || m > ldr || (reinterpret_cast<uintptr_t>(res) & 15u) || !status) return cudaErrorInvalidValue;
  const int64_t iblocks = (m + 127) / 128;
  if (n * iblocks > INT_MAX)                                 // item positions are 32-bit: the CUDA-core kernel
    return launch_crt(single, m, n, pl, res, ldr, x, y, ar, ai, br, bi, C, ldc, st, 4, real, robust);
  TcSingle W{res, ldr, m, n, ldc, x, y, C, ar, ai, br, bi, crt_flags(ar, ai, br, bi), static_cast<int>(iblocks),
             static_cast<int>(n)};
  const long long items = n * iblocks;
  switch (pl.L) {
    case 1: return launch_tc_l<1>(single, real, W, items, pl, status, st, robust);
    case 2: return launch_tc_l<2>(single, real, W, items, pl, status, st, robust);
    case 3: return launch_tc_l<3>(single, real, W, items, pl, status, st, robust);
    case 4: return launch_tc_l<4>(single, real, W, items, pl, status, st, robust);
    case 5: return launch_tc_l<5>(single, real, W, items, pl, status, st, robust);
    case 6: return launch_tc_l<6>(single, real, W, items, pl, status, st, robust);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace emu
