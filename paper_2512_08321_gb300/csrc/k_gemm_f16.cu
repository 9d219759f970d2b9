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

#include <mutex>

#include "emu_internal.h"

namespace emu {
namespace {

constexpr int BM = 128;                 // MMA M: output columns per tile
constexpr int BN = 256;                 // MMA N: output rows per tile
constexpr int BK = 64;                  // k per stage (128 bytes of fp16)
constexpr int UK = 16;                  // k per tcgen05.mma kind::f16
constexpr int kStages = 4;
constexpr int kStageA = BM * BK * 2;    // 16 KB: MMA operand A (B planes)
constexpr int kStageB = BN * BK * 2;    // 32 KB: MMA operand B (A planes)
constexpr int kStageBytes = kStageA + kStageB;
constexpr int kEpiWarps = 8;
constexpr int kThreads = 32 * (2 + kEpiWarps);
constexpr int kTmemCols = 512;
constexpr int kSmemBytes = kStages * kStageBytes + 1024 /*align*/ + 256 /*barriers*/;
constexpr long long kWaitLimit = 1ll << 32;    // SM cycles (about 2 s) per wait

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

// kind::f16 instruction descriptor: fp16 A/B, fp32 D, both K-major, M x N.
constexpr uint32_t kIdesc = (1u << 4) | (0u << 7) | (0u << 10) | (static_cast<uint32_t>(BN >> 3) << 17) |
                            (static_cast<uint32_t>(BM >> 4) << 24);

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, bool accumulate) {
  const uint32_t acc = accumulate ? 1u : 0u;
  asm volatile(
      "{\n.reg .pred p;\n"
      "setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(acc));
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
struct Sched {
  int J;          // jobs = 3N
  int pairs;      // ceil(J / 2)
  int TJ, TI;     // tiles along output columns (BM) and rows (BN)
  int tiles;
  int group;      // tile rasterisation: groups of `group` column tiles
  int nkb;        // k-blocks
  int ck;         // k-blocks per chunk
  int nch;        // chunks
  long long units;
};

__device__ __forceinline__ void unit_coords(const Sched& s, long long u, int& ja, int& jb, int& tj, int& ti) {
  const int pair = static_cast<int>(u / s.tiles);
  const int t = static_cast<int>(u % s.tiles);
  ja = 2 * pair;
  jb = (2 * pair + 1 < s.J) ? 2 * pair + 1 : -1;
  // column tiles in groups of s.group; inside a group, column-fastest
  const int per_group = s.group * s.TI;
  const int g = t / per_group;
  const int first = g * s.group;
  const int gsz = min(s.group, s.TJ - first);
  const int r = t - g * per_group;
  tj = first + r % gsz;
  ti = r / gsz;
}

__global__ void __launch_bounds__(kThreads, 1)
    gemm_f16_kernel(const __grid_constant__ CUtensorMap mapA,   // B planes: MMA operand A
                    const __grid_constant__ CUtensorMap mapB,   // A planes: MMA operand B
                    const __grid_constant__ Plan pl, const Sched s, int64_t m, int64_t n,
                    int8_t* __restrict__ res, int64_t ldr, unsigned int* status) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;                 // 1024-aligned operand stages
  uint8_t* gbase = smem_raw + (base - raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(gbase + kStages * kStageBytes);
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
                 "r"(kTmemCols));
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
      for (long long u = blockIdx.x; ok && u < s.units; u += gridDim.x) {
        int ja, jb, tj, ti;
        unit_coords(s, u, ja, jb, tj, ti);
        for (int c = 0; ok && c < s.nch; ++c) {
          for (int which = 0; ok && which < 2; ++which) {
            const int job = which ? jb : ja;
            if (job < 0) continue;
            const int kb1 = min(s.nkb, (c + 1) * s.ck);
            for (int kb = c * s.ck; kb < kb1; ++kb, ++it) {
              const int st = static_cast<int>(it % kStages);
              const uint32_t ph = static_cast<uint32_t>((it / kStages) & 1);
              if (!mbar_wait(empty(st), ph ^ 1u, ctl)) { ok = false; break; }
              const uint32_t sa = base + st * kStageBytes;
              mbar_expect_tx(full(st), kStageBytes);
              tma_load_3d(sa, &mapA, full(st), kb * BK, tj * BM, job);
              tma_load_3d(sa + kStageA, &mapB, full(st), kb * BK, ti * BN, job);
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
      for (long long u = blockIdx.x; ok && u < s.units; u += gridDim.x) {
        int ja, jb, tj, ti;
        unit_coords(s, u, ja, jb, tj, ti);
        for (int c = 0; ok && c < s.nch; ++c) {
          for (int which = 0; ok && which < 2; ++which) {
            const int job = which ? jb : ja;
            if (job < 0) continue;
            const int slot = which;
            if (!mbar_wait(tempty(slot), static_cast<uint32_t>(used[slot] & 1) ^ 1u, ctl)) { ok = false; break; }
            tc_fence_after();
            const uint32_t td = tmem + static_cast<uint32_t>(slot * BN);
            const int kb0 = c * s.ck, kb1 = min(s.nkb, (c + 1) * s.ck);
            for (int kb = kb0; kb < kb1; ++kb, ++it) {
              const int st = static_cast<int>(it % kStages);
              const uint32_t ph = static_cast<uint32_t>((it / kStages) & 1);
              if (!mbar_wait(full(st), ph, ctl)) { ok = false; break; }
              tc_fence_after();
              const uint32_t sa = base + st * kStageBytes;
              const uint64_t da = smem_desc(sa), db = smem_desc(sa + kStageA);
#pragma unroll
              for (int kk = 0; kk < BK / UK; ++kk) {
                // advance the start address by 32 bytes per 16 fp16 of k
                const uint64_t off = static_cast<uint64_t>((kk * UK * 2) >> 4);
                mma_f16(td, da + off, db + off, !(c == 0 && kb == kb0 && kk == 0));
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
    const int ew = warp - 2;
    const int quad = warp & 3;                      // TMEM lanes 32*quad .. 32*quad+31
    const int half = ew >> 2;                       // columns [128*half, 128*half+128) of a slot
    const int row_in_tile = quad * 32 + lane;       // output column within the tile
    int used[2] = {0, 0};
    bool ok = true;
    for (long long u = blockIdx.x; ok && u < s.units; u += gridDim.x) {
      int ja, jb, tj, ti;
      unit_coords(s, u, ja, jb, tj, ti);
      const int64_t col = static_cast<int64_t>(tj) * BM + row_in_tile;
      for (int c = 0; ok && c < s.nch; ++c) {
        const bool last = (c == s.nch - 1);
        for (int which = 0; ok && which < 2; ++which) {
          const int job = which ? jb : ja;
          if (job < 0) continue;
          const int slot = which;
          const int l = job / 3;
          const float p = static_cast<float>(pl.p[l]);
          const float inv_p = 1.0f / p;
          const int pi = pl.p[l];
          if (!mbar_wait(tfull(slot), static_cast<uint32_t>(used[slot] & 1), ctl)) { ok = false; break; }
          tc_fence_after();
          const uint32_t ta = tmem + (static_cast<uint32_t>(quad * 32) << 16) +
                              static_cast<uint32_t>(slot * BN + half * 128);
          if (!last) {
            // in-place reduction: keeps every later partial sum below 2^24
#pragma unroll 1
            for (int cc = 0; cc < 128; cc += 32) {
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
            int8_t* out = res + static_cast<int64_t>(job) * n * ldr + col * ldr + static_cast<int64_t>(ti) * BN +
                          half * 128;
            const int64_t row0 = static_cast<int64_t>(ti) * BN + half * 128;
#pragma unroll 1
            for (int cc = 0; cc < 128; cc += 32) {
              uint32_t v[32];
              tmem_ld32(ta + cc, v);
              tmem_wait_ld();
              if (cc == 96) {
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
              if (col < n) {
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                  const int64_t r0 = row0 + cc + 16 * q;
                  if (r0 < ldr)
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
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols));
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

}  // namespace

int g_f16_group = 16;   // tile rasterisation group (autotuned)

cudaError_t launch_gemm_f16(int64_t m, int64_t n, int64_t kpad, const Plan& pl, const void* planesA,
                            const void* planesB, int8_t* res, int64_t ldr, int chunk_k, unsigned int* status,
                            cudaStream_t st) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  if (kpad % BK || ldr % 16 || chunk_k % BK || chunk_k < BK || chunk_k > 960) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(planesA) | reinterpret_cast<uintptr_t>(planesB)) & 15u)
    return cudaErrorInvalidValue;
  if (!get_encoder()) return cudaErrorNotSupported;
  static std::once_flag attr_once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(attr_once, [] {
    attr_err = cudaFuncSetAttribute(gemm_f16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
  });
  if (attr_err != cudaSuccess) return attr_err;
  const int J = 3 * pl.N;
  CUtensorMap mapA, mapB;
  if (!make_map(&mapA, planesB, n, kpad, J, BM)) return cudaErrorInvalidValue;
  if (!make_map(&mapB, planesA, m, kpad, J, BN)) return cudaErrorInvalidValue;
  Sched s;
  s.J = J;
  s.pairs = (J + 1) / 2;
  s.TJ = static_cast<int>((n + BM - 1) / BM);
  s.TI = static_cast<int>((m + BN - 1) / BN);
  s.tiles = s.TJ * s.TI;
  s.group = g_f16_group > 0 ? g_f16_group : 16;
  s.nkb = static_cast<int>(kpad / BK);
  s.ck = chunk_k / BK;
  s.nch = (s.nkb + s.ck - 1) / s.ck;
  s.units = static_cast<long long>(s.pairs) * s.tiles;
  const long long grid = s.units < g_sms ? s.units : g_sms;
  gemm_f16_kernel<<<static_cast<unsigned int>(grid), kThreads, kSmemBytes, st>>>(mapA, mapB, pl, s, m, n, res, ldr,
                                                                                 status);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace emu
