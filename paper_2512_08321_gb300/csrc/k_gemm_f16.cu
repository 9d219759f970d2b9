// K3 (F16 engine): the residue products of Algorithm 1 Steps V-iii/iv on the
// 5th-generation tensor cores, tcgen05.mma kind::f16 with TMEM accumulators.
//
// sm_103a has no tcgen05 kind::i8, and its INT8 rate is a small fraction of
// its FP16 rate.  Symmetric residues |r| <= 128 are exact fp16 values and a
// product of two is at most 2^14, so an FP32 accumulator holds an exact
// integer as long as every partial sum stays below 2^24.  The kernel
// therefore splits k into chunks of `chunk_k` (<= 960): after each chunk the
// epilogue warps read the accumulator out of TMEM, reduce it modulo p_l
// (|v| <= p/2 + 2 afterwards) and write it back, and the next chunk
// accumulates on top.  The last chunk ends with the exact symmetric residue,
// written as int8.  The result is the exact mod(sum_h a_h b_h, p_l).
//
// Work: job j = 3l + c (c = D, E, F of eq. karatsuba), out[j][col][row] =
// mod(sum_h A_j[row][h] B_j[col][h], p_l).  The MMA's M dimension runs over
// 128 output columns (rows of the B planes) and its N dimension over 256
// output rows (rows of the A planes), so each TMEM lane holds one output
// column and the int8 result is stored with `row` contiguous.
//
// One persistent CTA per SM (192 KB of operand stages, all 512 TMEM
// columns).  A work unit is one 128 x 256 tile and a pair of jobs; the two
// jobs alternate chunk by chunk in two TMEM slots of 256 columns, so the
// epilogue reduces one slot while the tensor core fills the other.
// Warp roles: 0 = TMA producer, 1 = MMA issuer (and TMEM owner),
// 2..9 = epilogue (warp w reads TMEM lanes 32*(w%4).. and half of the columns).
// Every mbarrier wait is bounded; on expiry the kernel records
// EMU_ERR_TIMEOUT in the status word, drains its copies and MMAs in flight,
// frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

#include "emu_internal.h"

namespace emu {
namespace {

constexpr int BM = 128;                 // MMA M: output columns per tile
constexpr int BK = 64;                  // k per stage (128 bytes of fp16)
constexpr int UK = 16;                  // k per tcgen05.mma kind::f16
constexpr int kStages = 4;
constexpr int kStageA = BM * BK * 2;    // 16 KB: MMA operand A (B planes)
constexpr int kEpiWarps = 8;
constexpr int kThreads = 32 * (2 + kEpiWarps);
constexpr long long kWaitLimit = 1ll << 32;    // SM cycles (about 2 s) per wait

// Tile width BN (MMA N: output rows per tile) is a template parameter:
// 256 for large problems, 128 or 64 for small ones.
template <int BN>
struct Cfg {
  static constexpr int kStageB = BN * BK * 2;                 // MMA operand B (A planes)
  static constexpr int kStageBytes = kStageA + kStageB;
  static constexpr int kTmemCols = 2 * BN;                    // two accumulator slots
  static constexpr int kSmemBytes = kStages * kStageBytes + 1024 /*align*/ + 256 /*barriers*/;
  // kind::f16 instruction descriptor: fp16 A/B, fp32 D, both K-major, M = BM, N = BN
  static constexpr uint32_t kIdesc = (1u << 4) | (0u << 7) | (0u << 10) |
                                     (static_cast<uint32_t>(BN >> 3) << 17) |
                                     (static_cast<uint32_t>(BM >> 4) << 24);
  static_assert(BN == 64 || BN == 128 || BN == 256, "tile width");
};

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

struct Ctl {
  unsigned int* status;   // global status word
  volatile int* abort_s;  // shared abort flag
};

// Bounded wait for the phase of `parity` to complete.  false: expired/aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, const Ctl& c) {
  if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (mbar_try(bar, parity)) return true;
    if (*c.abort_s) return false;
    if (clock64() - t0 > kWaitLimit) {
      atomicCAS(c.status, 0u, static_cast<unsigned int>(EMU_ERR_TIMEOUT));
      *c.abort_s = 1;
      return false;
    }
  }
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1,
                                            int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%3, %4, %5}], [%2];\n" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// K-major operand tile, 128-byte rows, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = static_cast<uint64_t>((saddr >> 4) & 0x3FFFu);
  d |= static_cast<uint64_t>(1) << 16;                 // leading byte offset (unused here)
  d |= static_cast<uint64_t>(1024 >> 4) << 32;         // stride byte offset
  d |= static_cast<uint64_t>(1) << 46;                 // descriptor version
  d |= static_cast<uint64_t>(2) << 61;                 // 128-byte swizzle
  return d;
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        bool accumulate) {
  const uint32_t acc = accumulate ? 1u : 0u;
  asm volatile(
      "{\n.reg .pred p;\n"
      "setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
        "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
        "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
        "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
      "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};\n" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]),
      "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]),
      "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]),
      "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31]));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }

// ------------------------------------------------------------------ schedule
// One work unit: a BM x BN output tile of one problem and a pair of jobs
// (jb < 0 when the job count is odd and this is the last pair).
struct Unit {
  int ja, jb, tj, ti;
  int ppm;                          // planes (jobs) per modulus: 3 complex, 1 real
  int nkb, ck, nch;                 // k-blocks, k-blocks per chunk, chunks
  const CUtensorMap* mapA;          // B planes of the problem (MMA operand A)
  const CUtensorMap* mapB;          // A planes of the problem (MMA operand B)
  int8_t* res;
  int64_t ldr, n;
};

// Tile order inside one problem: column tiles in groups of `group`,
// column-fastest inside a group, so concurrently running CTAs share operands in L2.
__device__ __forceinline__ void tile_coords(int t, int TJ, int TI, int group, int& tj, int& ti) {
  const int per_group = group * TI;
  const int g = t / per_group;
  const int first = g * group;
  const int gsz = min(group, TJ - first);
  const int r = t - g * per_group;
  tj = first + r % gsz;
  ti = r / gsz;
}

struct Sched {
  int J;          // jobs = ppm N
  int ppm;        // jobs per modulus: 3 (D, E, F of eq. karatsuba) or 1 (real)
  int pairs;      // ceil(J / 2)
  int TJ, TI;     // tiles along output columns (BM) and rows (BN)
  int tiles;
  int group;      // tile rasterisation
  int nkb;        // k-blocks
  int ck;         // k-blocks per chunk
  int nch;        // chunks
  long long units;
};

// one GEMM: tensor maps are kernel parameters
struct SingleWork {
  const CUtensorMap* mapA;
  const CUtensorMap* mapB;
  Sched s;
  int8_t* res;
  int64_t ldr, n;
  __device__ long long units() const { return s.units; }
  __device__ Unit get(long long u) const {
    Unit w;
    const int pair = static_cast<int>(u / s.tiles);
    const int t = static_cast<int>(u % s.tiles);
    w.ja = 2 * pair;
    w.jb = (2 * pair + 1 < s.J) ? 2 * pair + 1 : -1;
    w.ppm = s.ppm;
    tile_coords(t, s.TJ, s.TI, s.group, w.tj, w.ti);
    w.nkb = s.nkb;
    w.ck = s.ck;
    w.nch = s.nch;
    w.mapA = mapA;
    w.mapB = mapB;
    w.res = res;
    w.ldr = ldr;
    w.n = n;
    return w;
  }
};

// many GEMMs sharing N: per-problem descriptors (with their tensor maps) in global memory
struct GroupProblem {  // CUtensorMap members give it 64-byte alignment
  CUtensorMap mapA;
  CUtensorMap mapB;
  int8_t* res;
  int64_t ldr, n;
  long long unit_begin;             // first unit of this problem
  int TJ, TI, tiles, group, nkb, ck, nch, J, ppm;
};

struct GroupWork {
  const GroupProblem* probs;
  int count;
  long long total;
  __device__ long long units() const { return total; }
  __device__ Unit get(long long u) const {
    int lo = 0, hi = count - 1;       // last problem with unit_begin <= u
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (probs[mid].unit_begin <= u) lo = mid; else hi = mid - 1;
    }
    const GroupProblem& P = probs[lo];
    const long long v = u - P.unit_begin;
    Unit w;
    const int pair = static_cast<int>(v / P.tiles);
    const int t = static_cast<int>(v % P.tiles);
    w.ja = 2 * pair;
    w.jb = (2 * pair + 1 < P.J) ? 2 * pair + 1 : -1;
    w.ppm = P.ppm;
    tile_coords(t, P.TJ, P.TI, P.group, w.tj, w.ti);
    w.nkb = P.nkb;
    w.ck = P.ck;
    w.nch = P.nch;
    w.mapA = &P.mapA;
    w.mapB = &P.mapB;
    w.res = P.res;
    w.ldr = P.ldr;
    w.n = P.n;
    return w;
  }
};

template <int BN, class Work>
__device__ __forceinline__ void gemm_body(const Work& W, const Plan& pl, unsigned int* status, bool fence_maps) {
  using C = Cfg<BN>;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;                 // 1024-aligned operand stages
  uint8_t* gbase = smem_raw + (base - raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(gbase + kStages * C::kStageBytes);
  // barrier layout: full[S], empty[S], tfull[2], tempty[2], done
  const uint32_t bar0 = smem_u32(bars);
  auto full = [&](int i) { return bar0 + 8u * i; };
  auto empty = [&](int i) { return bar0 + 8u * (kStages + i); };
  auto tfull = [&](int i) { return bar0 + 8u * (2 * kStages + i); };
  auto tempty = [&](int i) { return bar0 + 8u * (2 * kStages + 2 + i); };
  const uint32_t done = bar0 + 8u * (2 * kStages + 4);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kStages + 5);
  volatile int* abort_s = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  Ctl ctl{status, abort_s};
  const long long nunits = W.units();

  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(full(i), 1);
      mbar_init(empty(i), 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(tfull(i), 1);
      mbar_init(tempty(i), 32 * kEpiWarps);
    }
    mbar_init(done, 1);
    *abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"(C::kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      long long it = 0;
      bool ok = true;
      const CUtensorMap* fenced = nullptr;
      for (long long u = blockIdx.x; ok && u < nunits; u += gridDim.x) {
        const Unit U = W.get(u);
        if (fence_maps && U.mapA != fenced) {
          // descriptors written by the host into global memory: acquire them for the TMA unit
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;\n" ::"l"(U.mapA) : "memory");
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;\n" ::"l"(U.mapB) : "memory");
          fenced = U.mapA;
        }
        for (int c = 0; ok && c < U.nch; ++c) {
          for (int which = 0; ok && which < 2; ++which) {
            const int job = which ? U.jb : U.ja;
            if (job < 0) continue;
            const int kb1 = min(U.nkb, (c + 1) * U.ck);
            for (int kb = c * U.ck; kb < kb1; ++kb, ++it) {
              const int st = static_cast<int>(it % kStages);
              const uint32_t ph = static_cast<uint32_t>((it / kStages) & 1);
              if (!mbar_wait(empty(st), ph ^ 1u, ctl)) { ok = false; break; }
              const uint32_t sa = base + st * C::kStageBytes;
              mbar_expect_tx(full(st), C::kStageBytes);
              tma_load_3d(sa, U.mapA, full(st), kb * BK, U.tj * BM, job);
              tma_load_3d(sa + kStageA, U.mapB, full(st), kb * BK, U.ti * BN, job);
            }
          }
        }
      }
      // drain: every load issued has landed before the CTA may exit
      for (int st = 0; st < kStages; ++st) {
        if (it <= st) continue;                                    // stage never used
        const long long last = st + ((it - 1 - st) / kStages) * kStages;
        const uint32_t ph = static_cast<uint32_t>((last / kStages) & 1);
        const long long t0 = clock64();
        while (!mbar_try(full(st), ph) && clock64() - t0 < kWaitLimit) {
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      long long it = 0;
      int used[2] = {0, 0};
      bool ok = true;
      for (long long u = blockIdx.x; ok && u < nunits; u += gridDim.x) {
        const Unit U = W.get(u);
        for (int c = 0; ok && c < U.nch; ++c) {
          for (int which = 0; ok && which < 2; ++which) {
            const int job = which ? U.jb : U.ja;
            if (job < 0) continue;
            const int slot = which;
            if (!mbar_wait(tempty(slot), static_cast<uint32_t>(used[slot] & 1) ^ 1u, ctl)) { ok = false; break; }
            tc_fence_after();
            const uint32_t td = tmem + static_cast<uint32_t>(slot * BN);
            const int kb0 = c * U.ck, kb1 = min(U.nkb, (c + 1) * U.ck);
            for (int kb = kb0; kb < kb1; ++kb, ++it) {
              const int st = static_cast<int>(it % kStages);
              const uint32_t ph = static_cast<uint32_t>((it / kStages) & 1);
              if (!mbar_wait(full(st), ph, ctl)) { ok = false; break; }
              tc_fence_after();
              const uint32_t sa = base + st * C::kStageBytes;
              const uint64_t da = smem_desc(sa), db = smem_desc(sa + kStageA);
#pragma unroll
              for (int kk = 0; kk < BK / UK; ++kk) {
                // advance the start address by 32 bytes per 16 fp16 of k
                const uint64_t off = static_cast<uint64_t>((kk * UK * 2) >> 4);
                mma_f16(td, da + off, db + off, C::kIdesc, !(c == 0 && kb == kb0 && kk == 0));
              }
              mma_commit(empty(st));
            }
            if (!ok) break;
            mma_commit(tfull(slot));
            ++used[slot];
          }
        }
      }
      // all MMAs issued so far complete before TMEM is released
      mma_commit(done);
      const long long t0 = clock64();
      while (!mbar_try(done, 0u) && clock64() - t0 < kWaitLimit) {
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    constexpr int kHalf = BN / 2;                   // columns of a slot per epilogue warp
    const int ew = warp - 2;
    const int quad = warp & 3;                      // TMEM lanes 32*quad .. 32*quad+31
    const int half = ew >> 2;                       // columns [kHalf*half, kHalf*half + kHalf) of a slot
    const int row_in_tile = quad * 32 + lane;       // output column within the tile
    int used[2] = {0, 0};
    bool ok = true;
    for (long long u = blockIdx.x; ok && u < nunits; u += gridDim.x) {
      const Unit U = W.get(u);
      const int64_t col = static_cast<int64_t>(U.tj) * BM + row_in_tile;
      for (int c = 0; ok && c < U.nch; ++c) {
        const bool last = (c == U.nch - 1);
        for (int which = 0; ok && which < 2; ++which) {
          const int job = which ? U.jb : U.ja;
          if (job < 0) continue;
          const int slot = which;
          const int l = job / U.ppm;
          const float p = static_cast<float>(pl.p[l]);
          const float inv_p = 1.0f / p;
          const int pi = pl.p[l];
          if (!mbar_wait(tfull(slot), static_cast<uint32_t>(used[slot] & 1), ctl)) { ok = false; break; }
          tc_fence_after();
          const uint32_t ta = tmem + (static_cast<uint32_t>(quad * 32) << 16) +
                              static_cast<uint32_t>(slot * BN + half * kHalf);
          if (!last) {
            // in-place reduction: keeps every later partial sum below 2^24
#pragma unroll 1
            for (int cc = 0; cc < kHalf; cc += 32) {
              uint32_t v[32];
              tmem_ld32(ta + cc, v);
              tmem_wait_ld();
#pragma unroll
              for (int q = 0; q < 32; ++q) {
                const float x = __uint_as_float(v[q]);
                const float r = fmaf(-rintf(x * inv_p), p, x);
                v[q] = __float_as_uint(r);
              }
              tmem_st32(ta + cc, v);
            }
            tmem_wait_st();
            tc_fence_before();
            mbar_arrive(tempty(slot));
          } else {
            // final: exact symmetric residue, int8, row-contiguous
            const int64_t row0 = static_cast<int64_t>(U.ti) * BN + half * kHalf;
            int8_t* out = U.res + static_cast<int64_t>(job) * U.n * U.ldr + col * U.ldr + row0;
#pragma unroll 1
            for (int cc = 0; cc < kHalf; cc += 32) {
              uint32_t v[32];
              tmem_ld32(ta + cc, v);
              tmem_wait_ld();
              if (cc == kHalf - 32) {
                tc_fence_before();
                mbar_arrive(tempty(slot));          // TMEM slot may be refilled
              }
              uint32_t w[8];
#pragma unroll
              for (int q = 0; q < 8; ++q) {
                uint32_t packed = 0;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                  const float x = __uint_as_float(v[4 * q + b]);
                  int r = static_cast<int>(fmaf(-rintf(x * inv_p), p, x));
                  if (2 * r >= pi) r -= pi;
                  if (2 * r < -pi) r += pi;
                  packed |= (static_cast<uint32_t>(r) & 0xFFu) << (8 * b);
                }
                w[q] = packed;
              }
              if (col < U.n) {
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                  const int64_t r0 = row0 + cc + 16 * q;
                  if (r0 < U.ldr)
                    *reinterpret_cast<uint4*>(out + cc + 16 * q) =
                        make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
                }
              }
            }
          }
          ++used[slot];
        }
      }
    }
  }

  // ------------------------------------------------------------ teardown
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(C::kTmemCols));
}

template <int BN>
__global__ void __launch_bounds__(kThreads, 1)
    gemm_f16_kernel(const __grid_constant__ CUtensorMap mapA,   // B planes: MMA operand A
                    const __grid_constant__ CUtensorMap mapB,   // A planes: MMA operand B
                    const __grid_constant__ Plan pl, const Sched s, int8_t* __restrict__ res, int64_t ldr,
                    int64_t n, unsigned int* status) {
  const SingleWork W{&mapA, &mapB, s, res, ldr, n};
  gemm_body<BN>(W, pl, status, false);
}

template <int BN>
__global__ void __launch_bounds__(kThreads, 1)
    gemm_f16_grouped_kernel(const GroupProblem* __restrict__ probs, int count, long long total,
                            const __grid_constant__ Plan pl, unsigned int* status) {
  const GroupWork W{probs, count, total};
  gemm_body<BN>(W, pl, status, true);
}

// ------------------------------------------------------------------ bound products
// Accurate-mode scaling (Section III-B): exact non-negative bound products of
// the 7-bit ceiling planes (entries <= 64, products <= 2^12).  Planes of both
// operands: 0 = X_R (real input: X), 1 = X_I, 2 = X_R - X_I.
//   complex: slot 0 = C-bar_I = A-bar_I B-bar_R + A-bar_R B-bar_I (2 nkb k-blocks),
//            slot 1 = (A-bar_R - A-bar_I)(B-bar_R - B-bar_I) (nkb k-blocks),
//            C-bar_R = C-bar_I + slot 1 (the identity of Section III-B);
//   real:    slot 0 = C-bar = A-bar B-bar.
// FP32 accumulation is exact while partial sums stay below 2^24, so each
// accumulation restarts every kBoundChunk k-blocks (2048 k: sums <= 2^23) and
// the epilogue adds the chunk into int32 registers.  At the end of a tile each
// epilogue thread holds one output column (TMEM lane) and 32 output rows; the
// row maxima over columns (a 5-step butterfly across the warp) and the column
// maxima over rows of max(C-bar_R, C-bar_I) go to global memory by atomicMax.
// Output rows/columns beyond m/n read TMA's zero fill, so they add nothing.
constexpr int kBoundBN = 64;
constexpr int kBoundChunk = 32;

struct BoundSched {
  int TJ, TI, tiles, group, nkb, real;
};

// which operand planes and k-block of the planes feed k-block kb of a slot
__device__ __forceinline__ void bound_src(int slot, int kb, int nkb, bool real, int& pa, int& pb, int& kc) {
  if (real) { pa = 0; pb = 0; kc = kb; return; }
  if (slot == 1) { pa = 2; pb = 2; kc = kb; return; }
  if (kb < nkb) { pa = 0; pb = 1; kc = kb; }        // B-bar_R (MMA A) x A-bar_I (MMA B)
  else { pa = 1; pb = 0; kc = kb - nkb; }           // B-bar_I x A-bar_R
}

__global__ void __launch_bounds__(kThreads, 1)
    gemm_bound_kernel(const __grid_constant__ CUtensorMap mapA,   // B-bar planes: MMA operand A
                      const __grid_constant__ CUtensorMap mapB,   // A-bar planes: MMA operand B
                      const BoundSched s, unsigned int* __restrict__ Mrow, unsigned int* __restrict__ Ncol,
                      int64_t m, int64_t n, unsigned int* status) {
  constexpr int BN = kBoundBN;
  using C = Cfg<BN>;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (base - raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(gbase + kStages * C::kStageBytes);
  const uint32_t bar0 = smem_u32(bars);
  auto full = [&](int i) { return bar0 + 8u * i; };
  auto empty = [&](int i) { return bar0 + 8u * (kStages + i); };
  auto tfull = [&](int i) { return bar0 + 8u * (2 * kStages + i); };
  auto tempty = [&](int i) { return bar0 + 8u * (2 * kStages + 2 + i); };
  const uint32_t done = bar0 + 8u * (2 * kStages + 4);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kStages + 5);
  volatile int* abort_s = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  Ctl ctl{status, abort_s};
  const bool real = s.real != 0;
  const int len0 = real ? s.nkb : 2 * s.nkb, len1 = real ? 0 : s.nkb;
  const int nch0 = (len0 + kBoundChunk - 1) / kBoundChunk, nch1 = (len1 + kBoundChunk - 1) / kBoundChunk;
  const long long nunits = s.tiles;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(full(i), 1);
      mbar_init(empty(i), 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(tfull(i), 1);
      mbar_init(tempty(i), 32 * kEpiWarps);
    }
    mbar_init(done, 1);
    *abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"(C::kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      long long it = 0;
      bool ok = true;
      for (long long u = blockIdx.x; ok && u < nunits; u += gridDim.x) {
        int tj, ti;
        tile_coords(static_cast<int>(u), s.TJ, s.TI, s.group, tj, ti);
        for (int c = 0; ok && c < nch0; ++c) {
          for (int slot = 0; ok && slot < 2; ++slot) {
            const int len = slot ? len1 : len0;
            if (c * kBoundChunk >= len) continue;
            const int kb1 = min(len, (c + 1) * kBoundChunk);
            for (int kb = c * kBoundChunk; kb < kb1; ++kb, ++it) {
              const int st = static_cast<int>(it % kStages);
              const uint32_t ph = static_cast<uint32_t>((it / kStages) & 1);
              if (!mbar_wait(empty(st), ph ^ 1u, ctl)) { ok = false; break; }
              int pa, pb, kc;
              bound_src(slot, kb, s.nkb, real, pa, pb, kc);
              const uint32_t sa = base + st * C::kStageBytes;
              mbar_expect_tx(full(st), C::kStageBytes);
              tma_load_3d(sa, &mapA, full(st), kc * BK, tj * BM, pa);
              tma_load_3d(sa + kStageA, &mapB, full(st), kc * BK, ti * BN, pb);
            }
          }
        }
      }
      for (int st = 0; st < kStages; ++st) {
        if (it <= st) continue;
        const long long last = st + ((it - 1 - st) / kStages) * kStages;
        const uint32_t ph = static_cast<uint32_t>((last / kStages) & 1);
        const long long t0 = clock64();
        while (!mbar_try(full(st), ph) && clock64() - t0 < kWaitLimit) {
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      long long it = 0;
      int used[2] = {0, 0};
      bool ok = true;
      for (long long u = blockIdx.x; ok && u < nunits; u += gridDim.x) {
        for (int c = 0; ok && c < nch0; ++c) {
          for (int slot = 0; ok && slot < 2; ++slot) {
            const int len = slot ? len1 : len0;
            if (c * kBoundChunk >= len) continue;
            if (!mbar_wait(tempty(slot), static_cast<uint32_t>(used[slot] & 1) ^ 1u, ctl)) { ok = false; break; }
            tc_fence_after();
            const uint32_t td = tmem + static_cast<uint32_t>(slot * BN);
            const int kb0 = c * kBoundChunk, kb1 = min(len, (c + 1) * kBoundChunk);
            for (int kb = kb0; kb < kb1; ++kb, ++it) {
              const int st = static_cast<int>(it % kStages);
              const uint32_t ph = static_cast<uint32_t>((it / kStages) & 1);
              if (!mbar_wait(full(st), ph, ctl)) { ok = false; break; }
              tc_fence_after();
              const uint32_t sa = base + st * C::kStageBytes;
              const uint64_t da = smem_desc(sa), db = smem_desc(sa + kStageA);
#pragma unroll
              for (int kk = 0; kk < BK / UK; ++kk) {
                const uint64_t off = static_cast<uint64_t>((kk * UK * 2) >> 4);
                mma_f16(td, da + off, db + off, C::kIdesc, !(kb == kb0 && kk == 0));   // fresh sum per chunk
              }
              mma_commit(empty(st));
            }
            if (!ok) break;
            mma_commit(tfull(slot));
            ++used[slot];
          }
        }
      }
      mma_commit(done);
      const long long t0 = clock64();
      while (!mbar_try(done, 0u) && clock64() - t0 < kWaitLimit) {
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int ew = warp - 2;
    const int quad = warp & 3;
    const int half = ew >> 2;
    int used[2] = {0, 0};
    bool ok = true;
    for (long long u = blockIdx.x; ok && u < nunits; u += gridDim.x) {
      int tj, ti;
      tile_coords(static_cast<int>(u), s.TJ, s.TI, s.group, tj, ti);
      int acc0[32], acc1[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) acc0[q] = acc1[q] = 0;
      for (int c = 0; ok && c < nch0; ++c) {
        for (int slot = 0; ok && slot < 2; ++slot) {
          const int len = slot ? len1 : len0;
          if (c * kBoundChunk >= len) continue;
          if (!mbar_wait(tfull(slot), static_cast<uint32_t>(used[slot] & 1), ctl)) { ok = false; break; }
          tc_fence_after();
          const uint32_t ta = tmem + (static_cast<uint32_t>(quad * 32) << 16) +
                              static_cast<uint32_t>(slot * BN + half * 32);
          uint32_t v[32];
          tmem_ld32(ta, v);
          tmem_wait_ld();
          tc_fence_before();
          mbar_arrive(tempty(slot));
#pragma unroll
          for (int q = 0; q < 32; ++q) {
            const int x = static_cast<int>(__uint_as_float(v[q]));   // exact integer
            if (slot) acc1[q] += x; else acc0[q] += x;
          }
          ++used[slot];
        }
      }
      if (!ok) break;
      // max(C-bar_R, C-bar_I) per (row q, this column)
      unsigned int colmax = 0u;
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const int cr = real ? acc0[q] : acc0[q] + acc1[q];
        acc0[q] = max(cr, acc0[q]);
        colmax = max(colmax, static_cast<unsigned int>(acc0[q]));
      }
      const int64_t col = static_cast<int64_t>(tj) * BM + quad * 32 + lane;
      if (col < n) atomicMax(Ncol + col, colmax);
      // butterfly: after the step with distance d each lane keeps the maxima of half
      // of its rows; in the end lane L holds the maximum over the warp of row L
#pragma unroll
      for (int d = 16; d >= 1; d >>= 1) {
        const bool up = (lane & d) != 0;
#pragma unroll
        for (int t = 0; t < d; ++t) {
          const int send = up ? acc0[t] : acc0[t + d];
          const int keep = up ? acc0[t + d] : acc0[t];
          acc0[t] = max(keep, __shfl_xor_sync(0xffffffffu, send, d));
        }
      }
      const int64_t row = static_cast<int64_t>(ti) * BN + half * 32 + lane;
      if (row < m) atomicMax(Mrow + row, static_cast<unsigned int>(acc0[0]));
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(C::kTmemCols));
}

// ------------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;
int g_sms = 0;

bool get_encoder() {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
  });
  return g_encode != nullptr;
}

bool make_map(CUtensorMap* map, const void* planes, int64_t rows, int64_t kpad, int jobs, int box_rows) {
  const cuuint64_t dims[3] = {static_cast<cuuint64_t>(kpad), static_cast<cuuint64_t>(rows),
                              static_cast<cuuint64_t>(jobs)};
  const cuuint64_t strides[2] = {static_cast<cuuint64_t>(kpad) * 2, static_cast<cuuint64_t>(rows * kpad) * 2};
  const cuuint32_t box[3] = {static_cast<cuuint32_t>(BK), static_cast<cuuint32_t>(box_rows), 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, const_cast<void*>(planes), dims, strides,
                              box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int BN>
cudaError_t set_smem_attrs() {
  static cudaError_t err = [] {
    cudaError_t e = cudaFuncSetAttribute(gemm_f16_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         Cfg<BN>::kSmemBytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(gemm_f16_grouped_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               Cfg<BN>::kSmemBytes);
    return e;
  }();
  return err;
}

template <int BN>
cudaError_t launch_single(int64_t m, int64_t n, int64_t kpad, const Plan& pl, const void* planesA,
                          const void* planesB, int8_t* res, int64_t ldr, int chunk_k, int group,
                          unsigned int* status, cudaStream_t st, int ppm) {
  cudaError_t e = set_smem_attrs<BN>();
  if (e != cudaSuccess) return e;
  const int J = ppm * pl.N;
  CUtensorMap mapA, mapB;
  if (!make_map(&mapA, planesB, n, kpad, J, BM)) return cudaErrorInvalidValue;
  if (!make_map(&mapB, planesA, m, kpad, J, BN)) return cudaErrorInvalidValue;
  Sched s;
  s.J = J;
  s.ppm = ppm;
  s.pairs = (J + 1) / 2;
  s.TJ = static_cast<int>((n + BM - 1) / BM);
  s.TI = static_cast<int>((m + BN - 1) / BN);
  s.tiles = s.TJ * s.TI;
  s.group = group > 0 ? group : 16;
  s.nkb = static_cast<int>(kpad / BK);
  s.ck = chunk_k / BK;
  s.nch = (s.nkb + s.ck - 1) / s.ck;
  s.units = static_cast<long long>(s.pairs) * s.tiles;
  const long long grid = s.units < g_sms ? s.units : g_sms;
  gemm_f16_kernel<BN><<<static_cast<unsigned int>(grid), kThreads, Cfg<BN>::kSmemBytes, st>>>(
      mapA, mapB, pl, s, res, ldr, n, status);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace

int g_f16_group = 16;   // tile rasterisation group of grouped launches

cudaError_t launch_gemm_f16(int64_t m, int64_t n, int64_t kpad, const Plan& pl, const void* planesA,
                            const void* planesB, int8_t* res, int64_t ldr, int chunk_k, unsigned int* status,
                            cudaStream_t st, int tile_n, int group, int ppm) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  if (ppm != 1 && ppm != 3) return cudaErrorInvalidValue;
  if (kpad % BK || ldr % 16 || chunk_k % BK || chunk_k < BK || chunk_k > 960) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(planesA) | reinterpret_cast<uintptr_t>(planesB)) & 15u)
    return cudaErrorInvalidValue;
  if (!get_encoder()) return cudaErrorNotSupported;
  switch (tile_n) {
    case 64: return launch_single<64>(m, n, kpad, pl, planesA, planesB, res, ldr, chunk_k, group, status, st, ppm);
    case 128: return launch_single<128>(m, n, kpad, pl, planesA, planesB, res, ldr, chunk_k, group, status, st, ppm);
    default: return launch_single<256>(m, n, kpad, pl, planesA, planesB, res, ldr, chunk_k, group, status, st, ppm);
  }
}

cudaError_t launch_gemm_bound(int64_t m, int64_t n, int64_t kpad, bool real, const void* planesA,
                              const void* planesB, unsigned int* Mrow, unsigned int* Ncol, unsigned int* status,
                              cudaStream_t st) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  if (kpad % BK || ((reinterpret_cast<uintptr_t>(planesA) | reinterpret_cast<uintptr_t>(planesB)) & 15u))
    return cudaErrorInvalidValue;
  if (!get_encoder()) return cudaErrorNotSupported;
  static cudaError_t attr = cudaFuncSetAttribute(gemm_bound_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 Cfg<kBoundBN>::kSmemBytes);
  if (attr != cudaSuccess) return attr;
  const int planes = real ? 1 : 3;
  CUtensorMap mapA, mapB;
  if (!make_map(&mapA, planesB, n, kpad, planes, BM)) return cudaErrorInvalidValue;
  if (!make_map(&mapB, planesA, m, kpad, planes, kBoundBN)) return cudaErrorInvalidValue;
  BoundSched s;
  s.TJ = static_cast<int>((n + BM - 1) / BM);
  s.TI = static_cast<int>((m + kBoundBN - 1) / kBoundBN);
  s.tiles = s.TJ * s.TI;
  s.group = 16;
  s.nkb = static_cast<int>(kpad / BK);
  s.real = real ? 1 : 0;
  const int grid = s.tiles < g_sms ? s.tiles : g_sms;
  gemm_bound_kernel<<<grid, kThreads, Cfg<kBoundBN>::kSmemBytes, st>>>(mapA, mapB, s, Mrow, Ncol, m, n, status);
  count_launches(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- grouped
size_t group_problem_bytes() { return sizeof(GroupProblem); }

// Host set-up that must not happen inside a stream capture: the tensor-map
// encoder and the shared-memory attributes of every tile width.
cudaError_t prepare_gemm_f16() {
  if (!get_encoder()) return cudaErrorNotSupported;
  cudaError_t e = set_smem_attrs<64>();
  if (e == cudaSuccess) e = set_smem_attrs<128>();
  if (e == cudaSuccess) e = set_smem_attrs<256>();
  return e;
}

// Fill the host-side descriptor of problem p of a grouped launch (tensor maps,
// output, schedule); returns false on an invalid shape.  `unit_begin` is the
// running unit count, advanced past this problem's units.
bool fill_group_problem(void* desc, int64_t m, int64_t n, int64_t kpad, int N, const void* planesA,
                        const void* planesB, int8_t* res, int64_t ldr, int chunk_k, int group, int tile_n,
                        long long* unit_begin) {
  if (!get_encoder()) return false;
  GroupProblem& P = *static_cast<GroupProblem*>(desc);
  std::memset(&P, 0, sizeof(P));
  const int J = 3 * N;
  if (!make_map(&P.mapA, planesB, n, kpad, J, BM)) return false;
  if (!make_map(&P.mapB, planesA, m, kpad, J, tile_n)) return false;
  P.res = res;
  P.ldr = ldr;
  P.n = n;
  P.J = J;
  P.ppm = 3;
  P.TJ = static_cast<int>((n + BM - 1) / BM);
  P.TI = static_cast<int>((m + tile_n - 1) / tile_n);
  P.tiles = P.TJ * P.TI;
  P.group = group > 0 ? group : 16;
  P.nkb = static_cast<int>(kpad / BK);
  P.ck = chunk_k / BK;
  P.nch = (P.nkb + P.ck - 1) / P.ck;
  P.unit_begin = *unit_begin;
  *unit_begin += static_cast<long long>((J + 1) / 2) * P.tiles;
  return true;
}

cudaError_t launch_gemm_f16_grouped(const void* probs_dev, int count, long long total_units, const Plan& pl,
                                    int tile_n, unsigned int* status, cudaStream_t st) {
  if (count <= 0 || total_units <= 0) return cudaSuccess;
  if (!get_encoder()) return cudaErrorNotSupported;
  const GroupProblem* P = static_cast<const GroupProblem*>(probs_dev);
  const long long grid = total_units < g_sms ? total_units : g_sms;
  cudaError_t e;
  switch (tile_n) {
    case 64:
      if ((e = set_smem_attrs<64>()) != cudaSuccess) return e;
      gemm_f16_grouped_kernel<64><<<static_cast<unsigned int>(grid), kThreads, Cfg<64>::kSmemBytes, st>>>(
          P, count, total_units, pl, status);
      break;
    case 128:
      if ((e = set_smem_attrs<128>()) != cudaSuccess) return e;
      gemm_f16_grouped_kernel<128><<<static_cast<unsigned int>(grid), kThreads, Cfg<128>::kSmemBytes, st>>>(
          P, count, total_units, pl, status);
      break;
    default:
      if ((e = set_smem_attrs<256>()) != cudaSuccess) return e;
      gemm_f16_grouped_kernel<256><<<static_cast<unsigned int>(grid), kThreads, Cfg<256>::kSmemBytes, st>>>(
          P, count, total_units, pl, status);
  }
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace emu
