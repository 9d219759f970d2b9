// K3 (F16 engine): the residue products of Algorithm 1 Steps V-iii/iv on the
// 5th-generation tensor cores, tcgen05.mma kind::f16 with TMEM accumulators.
//
// sm_103a has no tcgen05 kind::i8, and its INT8 rate is a small fraction of
// its FP16 rate.  Symmetric residues |r| <= 128 are exact fp16 values and a
// product of two is at most 2^14, so an FP32 accumulator holds an exact
// integer as long as every partial sum stays below 2^24.  The kernel
// therefore splits k into chunks of at most `chunk_k` (<= 960), as many as
// that needs and of nearly equal size: after each chunk the
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
//
// The modulus-loop schedule is a launch parameter (Sched, searched by the
// autotuner); every choice gives the same residues:
//   order    0  modulus outer: every tile of job pair 0, then of pair 1, ...
//            1  tile outer: every job pair of tile 0, then of tile 1, ...
//            2  column bands: the output columns in bands of `band` tiles
//               (the n-blocking of Section III-A), modulus outer inside a band
//   pairing  0  adjacent jobs (2p, 2p+1): D_l E_l, F_l D_l+1, ...
//            1  halves (p, p + ceil(J/2))
//            2  component-major job sequence D_0..D_N-1, E_0.., F_0.., adjacent pairs
//   kalt     1  a CTA runs the k chunks of its odd-numbered units in
//               descending order, so a unit starts on the operands the
//               previous wave read last (still in L2).  The reductions keep
//               every partial sum exact in any chunk order.
// Warp roles: 0 = TMA producer, 1 = MMA issuer (and TMEM owner),
// 2..9 = epilogue (warp w reads TMEM lanes 32*(w%4).. and half of the columns).
// Every mbarrier wait is bounded; on expiry the kernel records
// EMU_ERR_TIMEOUT in the status word, drains its copies and MMAs in flight,
// frees TMEM and returns.



#include "tc_common.cuh"

namespace emu {
namespace {

// ------------------------------------------------------------------ schedule
// One work unit: a BM x BN output tile of one problem and a pair of jobs
// (jb < 0 when the job count is odd and this is the last pair).
struct Unit {
  int ja, jb, tj, ti;
  int bn;                           // output rows of this tile (MMA N): the kernel's BN, or less (grouped)
  bool desc;                        // k chunks in descending order
  int ppm;                          // planes (jobs) per modulus: 3 complex, 1 real
  int nkb, ck, nch;                 // k-blocks, k-blocks per chunk, chunks
  const CUtensorMap* mapA;          // B planes of the problem (MMA operand A)
  const CUtensorMap* mapB;          // A planes of the problem (MMA operand B)
  int8_t* res;
  int64_t ldr, n;
  int64_t rcap;                     // residue rows stored per column: those below rcap
};

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
  int order;      // 0 modulus outer, 1 tile outer, 2 column bands
  int pairing;    // 0 adjacent, 1 halves, 2 component-major
  int kalt;       // 1: descending k chunks on a CTA's odd units
  int band;       // column tiles per band (order 2)
};

// unit index v of one problem -> (pair, tile coordinates) under the schedule
__device__ __forceinline__ void unit_coords(long long v, int pairs, int tiles, int TJ, int TI, int group, int order,
                                            int band, int& pair, int& tj, int& ti) {
  if (order == 1) {                          // tile outer
    pair = static_cast<int>(v % pairs);
    tile_coords(static_cast<int>(v / pairs), TJ, TI, group, tj, ti);
  } else if (order == 2) {                   // column bands, modulus outer inside
    const long long full = static_cast<long long>(pairs) * band * TI;
    const int b = static_cast<int>(v / full);
    const long long r = v - b * full;
    const int nbt = min(band, TJ - b * band);
    const int bt = nbt * TI;
    pair = static_cast<int>(r / bt);
    tile_coords(static_cast<int>(r - static_cast<long long>(pair) * bt), nbt, TI, group, tj, ti);
    tj += b * band;
  } else {                                   // modulus outer
    pair = static_cast<int>(v / tiles);
    tile_coords(static_cast<int>(v % tiles), TJ, TI, group, tj, ti);
  }
}

// jobs of pair p; J = ppm N
__device__ __forceinline__ void pair_jobs(int p, int J, int ppm, int pairing, int& ja, int& jb) {
  if (pairing == 1) {
    const int h = (J + 1) >> 1;
    ja = p;
    jb = p + h < J ? p + h : -1;
  } else if (pairing == 2 && ppm > 1) {      // sequence position s -> job 3 (s mod N) + s / N
    const int N = J / ppm;
    const int sa = 2 * p, sb = 2 * p + 1;
    ja = (sa % N) * ppm + sa / N;
    jb = sb < J ? (sb % N) * ppm + sb / N : -1;
  } else {
    ja = 2 * p;
    jb = 2 * p + 1 < J ? 2 * p + 1 : -1;
  }
}

// The epilogue's rounding stays on rintf and float-to-int conversion (the XU
// pipe, idle otherwise): the same steps on the FMA pipe with a magic constant
// were measured to slow the residue products beside them by 5-6 % (ZGEMM
// 16384^3: 246 against 233 ms, alternating builds on one GPU).

// Four exact symmetric residues (the accumulators v[0..3] are exact integers
// below 2^24 in magnitude) as the int8 bytes of one word, low byte first.
__device__ __forceinline__ uint32_t residue_word(const uint32_t* v, float p, float inv_p, int pi) {
  int r[4];
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const float x = __uint_as_float(v[b]);
    r[b] = static_cast<int>(fmaf(-rintf(x * inv_p), p, x));
    if (2 * r[b] >= pi) r[b] -= pi;
    if (2 * r[b] < -pi) r[b] += pi;
  }
  // low bytes of r0, r1 and of r2, r3 side by side, then the two halves
  const uint32_t lo = __byte_perm(static_cast<uint32_t>(r[0]), static_cast<uint32_t>(r[1]), 0x0040u);
  const uint32_t hi = __byte_perm(static_cast<uint32_t>(r[2]), static_cast<uint32_t>(r[3]), 0x0040u);
  return __byte_perm(lo, hi, 0x5410u);
}

// k-blocks of chunk a of a unit: the nkb k-blocks split into nch chunks of
// nearly equal size (at most ck each, as nch = ceil(nkb / ck)), so that the
// last chunk is not a sliver that cannot hide the other job's epilogue.
__device__ __forceinline__ int chunk_begin(int a, const Unit& U) { return (a * U.nkb) / U.nch; }
__device__ __forceinline__ int chunk_end(int a, const Unit& U) { return ((a + 1) * U.nkb) / U.nch; }

// In single launches a unit with one job (the last job pair when the job count
// is odd) and two or more chunks runs its chunks in the two accumulator slots in turn (slot
// c & 1), so the MMAs of one chunk overlap the in-place reduction of the one
// before; the final epilogue adds the two partial sums (one reduced, |v| <= p/2
// + 2, the other at most chunk_k products of 2^14: below 2^24, exact) before
// the last reduction.
__device__ __forceinline__ bool unit_split(const Unit& U) { return U.jb < 0 && U.nch >= 2; }

// job and accumulator slot of step (chunk c, which) of a unit; false: no such step
__device__ __forceinline__ bool unit_step(const Unit& U, bool split1, int c, int which, int& job, int& slot) {
  if (split1) {
    job = U.ja;
    slot = c & 1;
    return which == 0;
  }
  job = which ? U.jb : U.ja;
  slot = which;
  return job >= 0;
}

// descending k chunks on the odd units a CTA processes (its units are
// blockIdx.x, blockIdx.x + gridDim.x, ...)
__device__ __forceinline__ bool unit_desc(long long u, int kalt) {
  return kalt && (((u - blockIdx.x) / gridDim.x) & 1);
}

// one GEMM: tensor maps are kernel parameters; the tile width is the kernel's BN
template <int BN>
struct SingleWork {
  const CUtensorMap* mapA;
  const CUtensorMap* mapB;
  Sched s;
  int8_t* res;
  int64_t ldr, n, rcap;
  __device__ long long units() const { return s.units; }
  __device__ Unit get(long long u, int& /*hint*/) const {
    Unit w;
    int pair;
    unit_coords(u, s.pairs, s.tiles, s.TJ, s.TI, s.group, s.order, s.band, pair, w.tj, w.ti);
    pair_jobs(pair, s.J, s.ppm, s.pairing, w.ja, w.jb);
    w.desc = unit_desc(u, s.kalt);
    w.bn = BN;
    w.ppm = s.ppm;
    w.nkb = s.nkb;
    w.ck = s.ck;
    w.nch = s.nch;
    w.mapA = mapA;
    w.mapB = mapB;
    w.res = res;
    w.ldr = ldr;
    w.n = n;
    w.rcap = rcap;
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
  int order, pairing, kalt, band;   // schedule, as in Sched
  int bn;                           // this problem's tile width: 64, 128 or 256 (at most the kernel's BN)
};

struct GroupWork {
  const GroupProblem* probs;
  const long long* ubeg;            // first unit of each problem (compact copy of unit_begin)
  int count;
  long long total;
  __device__ long long units() const { return total; }
  // `hint`: the problem of the caller's previous unit.  Each role of a CTA
  // visits units in increasing order, so the problem index only moves forward
  // (usually by 0 or 1) and a short forward scan replaces a binary search.
  __device__ Unit get(long long u, int& hint) const {
    int lo = hint;
    while (lo + 1 < count && ubeg[lo + 1] <= u) ++lo;
    hint = lo;
    const GroupProblem& P = probs[lo];
    const long long v = u - P.unit_begin;
    Unit w;
    int pair;
    unit_coords(v, (P.J + 1) / 2, P.tiles, P.TJ, P.TI, P.group, P.order, P.band, pair, w.tj, w.ti);
    pair_jobs(pair, P.J, P.ppm, P.pairing, w.ja, w.jb);
    w.desc = unit_desc(u, P.kalt);
    w.bn = P.bn;
    w.ppm = P.ppm;
    w.nkb = P.nkb;
    w.ck = P.ck;
    w.nch = P.nch;
    w.mapA = &P.mapA;
    w.mapB = &P.mapB;
    w.res = P.res;
    w.ldr = P.ldr;
    w.n = P.n;
    w.rcap = P.ldr;
    return w;
  }
};

// BN: the largest tile width (shared-memory stages, TMEM slots); EPI: epilogue
// warps (8 or 16), EPI / 4 of them on each quarter of the TMEM lanes, each
// taking 4 / EPI of a tile's columns (at least 32: with 64-wide tiles and 16
// warps, half of them only wait and arrive).
template <int BN, int EPI, int RING, class Work>
__device__ __forceinline__ void gemm_body(const Work& W, const Plan& pl, unsigned int* status, bool fence_maps) {
  using C = Cfg<BN>;
  constexpr int kParts = EPI / 4;                 // column parts of a tile
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
  // unit ring (RING > 0): after the 256 bytes of barriers, ufull[RING], uempty[RING], then the units
  uint64_t* rbars = reinterpret_cast<uint64_t*>(gbase + kStages * C::kStageBytes + 256);
  const uint32_t rbar0 = smem_u32(rbars);
  auto ufull = [&](int i) { return rbar0 + 8u * i; };
  auto uempty = [&](int i) { return rbar0 + 8u * (RING + i); };
  Unit* ring = reinterpret_cast<Unit*>(rbars + 2 * RING);

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
      mbar_init(tempty(i), 32 * EPI);
    }
    mbar_init(done, 1);
    for (int i = 0; i < RING; ++i) {
      mbar_init(ufull(i), 1);
      mbar_init(uempty(i), 1 + EPI);                  // the MMA issuer and one lane per epilogue warp
    }
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
      int hint = 0;
      // the next unit's descriptor is fetched while this one's loads are issued
      Unit nxt;
      if (blockIdx.x < nunits) nxt = W.get(blockIdx.x, hint);
      long long t = 0;                                             // this CTA's unit count
      for (long long u = blockIdx.x; ok && u < nunits; u += gridDim.x, ++t) {
        const Unit U = nxt;
        if (u + gridDim.x < nunits) nxt = W.get(u + gridDim.x, hint);
        if constexpr (RING > 0) {
          // publish the unit to the MMA issuer and the epilogue warps
          const int rs = static_cast<int>(t % RING);
          if (!mbar_wait(uempty(rs), static_cast<uint32_t>((t / RING) & 1) ^ 1u, ctl)) { ok = false; break; }
          ring[rs] = U;
          mbar_arrive(ufull(rs));
        }
        if (fence_maps && U.mapA != fenced) {
          // descriptors written by the host into global memory: acquire them for the TMA unit
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;\n" ::"l"(U.mapA) : "memory");
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;\n" ::"l"(U.mapB) : "memory");
          fenced = U.mapA;
        }
        for (int c = 0; ok && c < U.nch; ++c) {
          const int a = U.desc ? U.nch - 1 - c : c;              // chunk of k processed c-th
          for (int which = 0; ok && which < 2; ++which) {
            const int job = which ? U.jb : U.ja;
            if (job < 0) continue;
            const int kb1 = chunk_end(a, U);
            for (int kb = chunk_begin(a, U); kb < kb1; ++kb, ++it) {
              const int st = static_cast<int>(it % kStages);
              const uint32_t ph = static_cast<uint32_t>((it / kStages) & 1);
              if (!mbar_wait(empty(st), ph ^ 1u, ctl)) { ok = false; break; }
              const uint32_t sa = base + st * C::kStageBytes;
              mbar_expect_tx(full(st), static_cast<uint32_t>(kStageA + U.bn * BK * 2));
              tma_load_3d(sa, U.mapA, full(st), kb * BK, U.tj * BM, job);
              tma_load_3d(sa + kStageA, U.mapB, full(st), kb * BK, U.ti * U.bn, job);
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
      uint32_t used = 0u;                           // bit s: parity of slot s's uses so far
      bool ok = true;
      int hint = 0;
      // the next unit's descriptor is fetched while this one's MMAs are issued (or read from the ring)
      Unit nxt;
      if (RING == 0 && blockIdx.x < nunits) nxt = W.get(blockIdx.x, hint);
      long long t = 0;
      for (long long u = blockIdx.x; ok && u < nunits; u += gridDim.x, ++t) {
        Unit U;
        if constexpr (RING > 0) {
          const int rs = static_cast<int>(t % RING);
          if (!mbar_wait(ufull(rs), static_cast<uint32_t>((t / RING) & 1), ctl)) { ok = false; break; }
          U = ring[rs];
          mbar_arrive(uempty(rs));
        } else {
          U = nxt;
          if (u + gridDim.x < nunits) nxt = W.get(u + gridDim.x, hint);
        }
        const bool split1 = RING == 0 && unit_split(U);   // single launches (the grouped kernel has no registers to spare)
        for (int c = 0; ok && c < U.nch; ++c) {
          for (int which = 0; ok && which < 2; ++which) {
            int job, slot;
            if (!unit_step(U, split1, c, which, job, slot)) continue;
            if (!mbar_wait(tempty(slot), ((used >> slot) & 1u) ^ 1u, ctl)) { ok = false; break; }
            tc_fence_after();
            const uint32_t td = tmem + static_cast<uint32_t>(slot * BN);
            const uint32_t idesc = C::kIdescNoN | (static_cast<uint32_t>(U.bn >> 3) << 17);
            const int a = U.desc ? U.nch - 1 - c : c;
            const int kb0 = chunk_begin(a, U), kb1 = chunk_end(a, U);
            const bool fresh = split1 ? c < 2 : c == 0;     // the slot's first chunk of this unit
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
                mma_f16(td, da + off, db + off, idesc, !(fresh && kb == kb0 && kk == 0));
              }
              mma_commit(empty(st));
            }
            if (!ok) break;
            mma_commit(tfull(slot));
            used ^= 1u << slot;
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
    const int part = ew >> 2;                       // column part of a tile
    const int row_in_tile = quad * 32 + lane;       // output column within the tile
    uint32_t used = 0u;                             // bit s: parity of slot s's uses so far
    bool ok = true;
    int hint = 0;
    long long t = 0;
    for (long long u = blockIdx.x; ok && u < nunits; u += gridDim.x, ++t) {
      Unit U;
      if constexpr (RING > 0) {
        const int rs = static_cast<int>(t % RING);
        if (!mbar_wait(ufull(rs), static_cast<uint32_t>((t / RING) & 1), ctl)) { ok = false; break; }
        U = ring[rs];
        __syncwarp();
        if (lane == 0) mbar_arrive(uempty(rs));
      } else {
        U = W.get(u, hint);
      }
      const int64_t col = static_cast<int64_t>(U.tj) * BM + row_in_tile;
      // columns of this warp: [part * pw, part * pw + pw), pw >= 32; parts past the tile only wait
      const int pw = (U.bn / kParts) < 32 ? 32 : (U.bn / kParts);
      const bool mine = part * pw < U.bn;
      const bool split1 = RING == 0 && unit_split(U);   // single launches (the grouped kernel has no registers to spare)
      for (int c = 0; ok && c < U.nch; ++c) {
        const bool last = (c == U.nch - 1);
        // one-job unit: the second-to-last chunk's slot is reduced and then held for the final
        const bool hold = split1 && c == U.nch - 2;
        for (int which = 0; ok && which < 2; ++which) {
          int job, slot;
          if (!unit_step(U, split1, c, which, job, slot)) continue;
          const int l = job / U.ppm;
          const float p = static_cast<float>(pl.p[l]);
          const float inv_p = 1.0f / p;
          const int pi = pl.p[l];
          if (!mbar_wait(tfull(slot), (used >> slot) & 1u, ctl)) { ok = false; break; }
          tc_fence_after();
          const uint32_t ta = tmem + (static_cast<uint32_t>(quad * 32) << 16) +
                              static_cast<uint32_t>(slot * BN + part * pw);
          if (!mine) {
            tc_fence_before();
            if (!hold) mbar_arrive(tempty(slot));
            if (split1 && last) mbar_arrive(tempty(slot ^ 1));   // the held slot
          } else if (!last) {
            // in-place reduction: keeps every later partial sum below 2^24
#pragma unroll 1
            for (int cc = 0; cc < pw; cc += 32) {
              uint32_t v[32];
              tmem_ld32(ta + cc, v);
              tmem_wait_ld();
#pragma unroll
              for (int q = 0; q < 32; ++q) {
                const float x = __uint_as_float(v[q]);
                v[q] = __float_as_uint(fmaf(-rintf(x * inv_p), p, x));
              }
              tmem_st32(ta + cc, v);
            }
            tmem_wait_st();
            tc_fence_before();
            if (!hold) mbar_arrive(tempty(slot));
          } else {
            // final: exact symmetric residue, int8, row-contiguous
            const int64_t row0 = static_cast<int64_t>(U.ti) * U.bn + part * pw;
            int8_t* out = U.res + static_cast<int64_t>(job) * U.n * U.ldr + col * U.ldr + row0;
            const uint32_t tb = ta + static_cast<uint32_t>(((slot ^ 1) - slot) * BN);   // the held slot
#pragma unroll 1
            for (int cc = 0; cc < pw; cc += 32) {
              uint32_t v[32];
              tmem_ld32(ta + cc, v);
              tmem_wait_ld();
              if (split1) {
                // add the held slot's partial sum, 16 columns at a time
#pragma unroll
                for (int h = 0; h < 32; h += 16) {
                  uint32_t o[16];
                  tmem_ld16(tb + cc + h, o);
                  tmem_wait_ld();
#pragma unroll
                  for (int q = 0; q < 16; ++q)
                    v[h + q] = __float_as_uint(__uint_as_float(v[h + q]) + __uint_as_float(o[q]));
                }
              }
              if (cc == pw - 32) {
                tc_fence_before();
                mbar_arrive(tempty(slot));          // TMEM slot may be refilled
                if (split1) mbar_arrive(tempty(slot ^ 1));
              }
              uint32_t w[8];
#pragma unroll
              for (int q = 0; q < 8; ++q) w[q] = residue_word(v + 4 * q, p, inv_p, pi);
              if (col < U.n) {
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                  const int64_t r0 = row0 + cc + 16 * q;
                  if (r0 < U.rcap)
                    *reinterpret_cast<uint4*>(out + cc + 16 * q) =
                        make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
                }
              }
            }
          }
          used ^= 1u << slot;
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
                    int64_t n, int64_t rcap, unsigned int* status) {
  const SingleWork<BN> W{&mapA, &mapB, s, res, ldr, n, rcap};
  gemm_body<BN, kEpiWarps, 0>(W, pl, status, false);
}

// ------------------------------------------------------------------ SM pairs
// cta_group::2: the two CTAs of a cluster share one 256 x 256 tile.  MMA M =
// 256 output columns, 128 in each CTA's TMEM lanes (CTA r holds the tile's
// columns 128 r .. 128 r + 127, from its own stage of B-plane rows); MMA N =
// 256 output rows, whose A-plane rows each CTA loads half of (rows 128 r ..).
// The even CTA issues the MMAs for both; its commits arrive on the barriers of
// both CTAs (multicast), and both CTAs' TMA loads count on its full barriers.
// Each SM stages 32 KB per k-block instead of the 48 KB of a 128 x 256 tile on
// one SM, for the same MMA work per SM.  The epilogue is the one-SM kernel's,
// each CTA on its own TMEM; its arrivals on `tempty` go to the even CTA.
// Measured at ZGEMM 16384^3, N = 15: 7 % fewer SM cycles than one-SM tiles,
// but the GPU then sits lower under its power cap (1515-1575 against
// 1826-1852 MHz), so the products took 255 ms against 231: an autotuner
// candidate, not the default.
constexpr int kPairStages = 6;
constexpr int kPairRows = 128;                                   // A-plane rows per CTA per stage
constexpr int kPairStageBytes = kStageA + kPairRows * BK * 2;    // 32 KB
constexpr int kPairBN = 256;                                     // MMA N: output rows per tile
constexpr int kPairBM = 2 * BM;                                  // output columns per tile
constexpr int kPairSmem = kPairStages * kPairStageBytes + 1024 + 256;
constexpr uint32_t kPairIdesc = (1u << 4) | (static_cast<uint32_t>(kPairBN >> 3) << 17) |
                                (static_cast<uint32_t>(kPairBM >> 4) << 24);

__device__ __forceinline__ void pair_body(const SingleWork<kPairBN>& W, const Plan& pl, unsigned int* status) {
  constexpr int EPI = kEpiWarps;
  constexpr int kParts = EPI / 4;
  constexpr int S = kPairStages;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;                 // the same offset in both CTAs
  uint8_t* gbase = smem_raw + (base - raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(gbase + S * kPairStageBytes);
  // barrier layout: full[S], empty[S], tfull[2], tempty[2], done
  const uint32_t bar0 = smem_u32(bars);
  auto full = [&](int i) { return bar0 + 8u * i; };
  auto empty = [&](int i) { return bar0 + 8u * (S + i); };
  auto tfull = [&](int i) { return bar0 + 8u * (2 * S + i); };
  auto tempty = [&](int i) { return bar0 + 8u * (2 * S + 2 + i); };
  const uint32_t done = bar0 + 8u * (2 * S + 4);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * S + 5);
  volatile int* abort_s = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const bool leader = rank == 0;
  Ctl ctl{status, abort_s};
  const long long nunits = W.units();
  const long long pid = blockIdx.x >> 1, npairs = gridDim.x >> 1;
  const int kalt = W.s.kalt;

  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(full(i), 1);
      mbar_init(empty(i), 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(tfull(i), 1);
      mbar_init(tempty(i), 2 * 32 * EPI);
    }
    mbar_init(done, 1);
    *abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 1) {   // one warp of each CTA: the same 512 columns in both
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"(2 * kPairBN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;\n");
  }
  tc_fence_before();
  cluster_sync();                    // both CTAs' barriers initialised and TMEM allocated
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t full_c0 = map_to_rank(full(0), 0);           // the even CTA's full barriers
  const uint32_t tempty_c0 = map_to_rank(tempty(0), 0);       // and tempty barriers

  auto get = [&](long long u, int& hint) {
    Unit U = W.get(u, hint);
    U.desc = kalt && ((((u - pid) / npairs) & 1) != 0);        // the same in both CTAs
    return U;
  };

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer (both CTAs)
    if (lane == 0) {
      long long it = 0;
      bool ok = true;
      int hint = 0;
      Unit nxt;
      if (pid < nunits) nxt = get(pid, hint);
      for (long long u = pid; ok && u < nunits; u += npairs) {
        const Unit U = nxt;
        if (u + npairs < nunits) nxt = get(u + npairs, hint);
        for (int c = 0; ok && c < U.nch; ++c) {
          const int a = U.desc ? U.nch - 1 - c : c;
          for (int which = 0; ok && which < 2; ++which) {
            const int job = which ? U.jb : U.ja;
            if (job < 0) continue;
            const int kb1 = chunk_end(a, U);
            for (int kb = chunk_begin(a, U); kb < kb1; ++kb, ++it) {
              const int st = static_cast<int>(it % S);
              const uint32_t ph = static_cast<uint32_t>((it / S) & 1);
              if (!mbar_wait(empty(st), ph ^ 1u, ctl)) { ok = false; break; }
              // the even CTA's full barrier counts the bytes of both CTAs' loads
              if (leader) mbar_expect_tx(full(st), static_cast<uint32_t>(2 * kPairStageBytes));
              const uint32_t sa = base + st * kPairStageBytes;
              const uint32_t fb = full_c0 + 8u * st;
              tma_load_3d_pair(sa, U.mapA, fb, kb * BK, U.tj * kPairBM + static_cast<int>(rank) * BM, job);
              tma_load_3d_pair(sa + kStageA, U.mapB, fb, kb * BK, U.ti * kPairBN + static_cast<int>(rank) * kPairRows,
                               job);
            }
          }
        }
      }
      // drain: every load issued has landed (the even CTA's barriers count both CTAs' bytes)
      if (leader) {
        for (int st = 0; st < S; ++st) {
          if (it <= st) continue;
          const long long last = st + ((it - 1 - st) / S) * S;
          const uint32_t ph = static_cast<uint32_t>((last / S) & 1);
          const long long t0 = clock64();
          while (!mbar_try_cluster(full(st), ph) && clock64() - t0 < kWaitLimit) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer (the even CTA)
    if (lane == 0 && leader) {
      long long it = 0;
      uint32_t used = 0u;
      bool ok = true;
      int hint = 0;
      Unit nxt;
      if (pid < nunits) nxt = get(pid, hint);
      for (long long u = pid; ok && u < nunits; u += npairs) {
        const Unit U = nxt;
        if (u + npairs < nunits) nxt = get(u + npairs, hint);
        for (int c = 0; ok && c < U.nch; ++c) {
          for (int which = 0; ok && which < 2; ++which) {
            const int job = which ? U.jb : U.ja;
            if (job < 0) continue;
            const int slot = which;
            // both CTAs' epilogues have emptied this slot
            if (!mbar_wait_cluster(tempty(slot), ((used >> slot) & 1u) ^ 1u, ctl)) { ok = false; break; }
            tc_fence_after();
            const uint32_t td = tmem + static_cast<uint32_t>(slot * kPairBN);
            const int a = U.desc ? U.nch - 1 - c : c;
            const int kb0 = chunk_begin(a, U), kb1 = chunk_end(a, U);
            for (int kb = kb0; kb < kb1; ++kb, ++it) {
              const int st = static_cast<int>(it % S);
              const uint32_t ph = static_cast<uint32_t>((it / S) & 1);
              if (!mbar_wait_cluster(full(st), ph, ctl)) { ok = false; break; }
              tc_fence_after();
              const uint32_t sa = base + st * kPairStageBytes;
              const uint64_t da = smem_desc(sa), db = smem_desc(sa + kStageA);
#pragma unroll
              for (int kk = 0; kk < BK / UK; ++kk) {
                const uint64_t off = static_cast<uint64_t>((kk * UK * 2) >> 4);
                mma_f16_pair(td, da + off, db + off, kPairIdesc, !(c == 0 && kb == kb0 && kk == 0));
              }
              mma_commit_pair(empty(st));             // the stage is free in both CTAs
            }
            if (!ok) break;
            mma_commit_pair(tfull(slot));
            used ^= 1u << slot;
          }
        }
      }
      mma_commit_pair(done);
      const long long t0 = clock64();
      while (!mbar_try(done, 0u) && clock64() - t0 < kWaitLimit) {
      }
    } else if (lane == 0) {
      // the odd CTA: the even CTA's last commit also arrives here once every MMA that
      // reads this CTA's shared memory or writes its TMEM is done
      const long long t0 = clock64();
      while (!mbar_try(done, 0u) && clock64() - t0 < kWaitLimit) {
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue (both CTAs)
    const int ew = warp - 2;
    const int quad = warp & 3;
    const int part = ew >> 2;
    const int row_in_tile = quad * 32 + lane;
    constexpr int pw = kPairBN / kParts;
    uint32_t used = 0u;
    bool ok = true;
    int hint = 0;
    for (long long u = pid; ok && u < nunits; u += npairs) {
      const Unit U = get(u, hint);
      const int64_t col = static_cast<int64_t>(U.tj) * kPairBM + static_cast<int64_t>(rank) * BM + row_in_tile;
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
          if (!mbar_wait(tfull(slot), (used >> slot) & 1u, ctl)) { ok = false; break; }
          tc_fence_after();
          const uint32_t ta = tmem + (static_cast<uint32_t>(quad * 32) << 16) +
                              static_cast<uint32_t>(slot * kPairBN + part * pw);
          if (!last) {
#pragma unroll 1
            for (int cc = 0; cc < pw; cc += 32) {
              uint32_t v[32];
              tmem_ld32(ta + cc, v);
              tmem_wait_ld();
#pragma unroll
              for (int q = 0; q < 32; ++q) {
                const float x = __uint_as_float(v[q]);
                v[q] = __float_as_uint(fmaf(-rintf(x * inv_p), p, x));
              }
              tmem_st32(ta + cc, v);
            }
            tmem_wait_st();
            tc_fence_before();
            mbar_arrive_cluster(tempty_c0 + 8u * slot);
          } else {
            const int64_t row0 = static_cast<int64_t>(U.ti) * kPairBN + part * pw;
            int8_t* out = U.res + static_cast<int64_t>(job) * U.n * U.ldr + col * U.ldr + row0;
#pragma unroll 1
            for (int cc = 0; cc < pw; cc += 32) {
              uint32_t v[32];
              tmem_ld32(ta + cc, v);
              tmem_wait_ld();
              if (cc == pw - 32) {
                tc_fence_before();
                mbar_arrive_cluster(tempty_c0 + 8u * slot);
              }
              uint32_t w[8];
#pragma unroll
              for (int q = 0; q < 8; ++q) w[q] = residue_word(v + 4 * q, p, inv_p, pi);
              if (col < U.n) {
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                  const int64_t r0 = row0 + cc + 16 * q;
                  if (r0 < U.rcap)
                    *reinterpret_cast<uint4*>(out + cc + 16 * q) =
                        make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
                }
              }
            }
          }
          used ^= 1u << slot;
        }
      }
    }
  }

  // ------------------------------------------------------------ teardown
  tc_fence_before();
  cluster_sync();                    // no CTA leaves while the pair's MMAs or loads may touch it
  tc_fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(2 * kPairBN));
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1)
    gemm_f16_pair_kernel(const __grid_constant__ CUtensorMap mapA,   // B planes: MMA operand A
                         const __grid_constant__ CUtensorMap mapB,   // A planes: MMA operand B
                         const __grid_constant__ Plan pl, const Sched s, int8_t* __restrict__ res, int64_t ldr,
                         int64_t n, int64_t rcap, unsigned int* status) {
  const SingleWork<kPairBN> W{&mapA, &mapB, s, res, ldr, n, rcap};
  pair_body(W, pl, status);
}

// Grouped launches: 256-row stages with each problem's own tile width, 16
// epilogue warps (short-k units are bound by their epilogue, not their MMAs),
// and a ring of unit descriptors in shared memory: the producer looks each
// unit up in the problem table once, the MMA issuer and the epilogue warps
// read it from the ring.
constexpr int kGroupedEpi = 16;
constexpr int kGroupedThreads = 32 * (2 + kGroupedEpi);
constexpr int kGroupedRing = 8;
static_assert(sizeof(Unit) % 8 == 0 && 2 * 8 * kGroupedRing + kGroupedRing * sizeof(Unit) <= 1024, "unit ring");
constexpr int kGroupedSmem = Cfg<256>::kSmemBytes + 1024;

__global__ void __launch_bounds__(kGroupedThreads, 1)
    gemm_f16_grouped_kernel(const GroupProblem* __restrict__ probs, int count, long long total,
                            const __grid_constant__ Plan pl, unsigned int* status) {
  const GroupWork W{probs, reinterpret_cast<const long long*>(probs + count), count, total};
  gemm_body<256, kGroupedEpi, kGroupedRing>(W, pl, status, true);
}

// The largest shared-memory carveout: an SM holding one block of this kernel
// then keeps the rest of its shared memory (about 34 KB at 256-wide tiles) for
// blocks of other kernels, instead of the smallest configuration that fits.
template <int BN>
cudaError_t set_smem_attrs() {
  static cudaError_t err = [] {
    cudaError_t e = cudaFuncSetAttribute(gemm_f16_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         Cfg<BN>::kSmemBytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(gemm_f16_kernel<BN>, cudaFuncAttributePreferredSharedMemoryCarveout,
                               static_cast<int>(cudaSharedmemCarveoutMaxShared));
    return e;
  }();
  return err;
}

cudaError_t set_grouped_attrs() {
  static cudaError_t err = [] {
    cudaError_t e = cudaFuncSetAttribute(gemm_f16_grouped_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kGroupedSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(gemm_f16_grouped_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                               static_cast<int>(cudaSharedmemCarveoutMaxShared));
    return e;
  }();
  return err;
}

template <int BN>
cudaError_t launch_single(int64_t m, int64_t n, int64_t kpad, const Plan& pl, const void* planesA,
                          const void* planesB, int8_t* res, int64_t ldr, int chunk_k, int group,
                          unsigned int* status, cudaStream_t st, int ppm, int64_t a_plane_rows, int64_t rcap,
                          const GemmSchedule& sc) {
  cudaError_t e = set_smem_attrs<BN>();
  if (e != cudaSuccess) return e;
  const int J = ppm * pl.N;
  CUtensorMap mapA, mapB;
  if (!make_map(&mapA, planesB, n, kpad, J, BM)) return cudaErrorInvalidValue;
  if (!make_map(&mapB, planesA, m, kpad, J, BN, a_plane_rows)) return cudaErrorInvalidValue;
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
  s.order = sc.order;
  s.pairing = sc.pairing;
  s.kalt = sc.kalt;
  s.band = sc.band_cols / BM;
  const long long grid = s.units < g_sms ? s.units : g_sms;
  gemm_f16_kernel<BN><<<static_cast<unsigned int>(grid), kThreads, Cfg<BN>::kSmemBytes, st>>>(
      mapA, mapB, pl, s, res, ldr, n, rcap, status);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t set_pair_attrs() {
  static cudaError_t err = [] {
    cudaError_t e = cudaFuncSetAttribute(gemm_f16_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kPairSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(gemm_f16_pair_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                               static_cast<int>(cudaSharedmemCarveoutMaxShared));
    return e;
  }();
  return err;
}

// SM pairs that can hold a CTA pair of the kernel at once (0 if none or on error)
int pair_clusters() {
  static int n = [] {
    if (set_pair_attrs() != cudaSuccess) return 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * 1024);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = kPairSmem;
    int v = 0;
    if (cudaOccupancyMaxActiveClusters(&v, gemm_f16_pair_kernel, &cfg) != cudaSuccess) {
      cudaGetLastError();
      v = 0;
    }
    return v;
  }();
  return n;
}

cudaError_t launch_pair(int64_t m, int64_t n, int64_t kpad, const Plan& pl, const void* planesA, const void* planesB,
                        int8_t* res, int64_t ldr, int chunk_k, int group, unsigned int* status, cudaStream_t st,
                        int ppm, int64_t a_plane_rows, int64_t rcap, const GemmSchedule& sc) {
  cudaError_t e = set_pair_attrs();
  if (e != cudaSuccess) return e;
  const int clusters = pair_clusters();
  if (clusters <= 0) return cudaErrorNotSupported;
  const int J = ppm * pl.N;
  CUtensorMap mapA, mapB;
  if (!make_map(&mapA, planesB, n, kpad, J, BM)) return cudaErrorInvalidValue;
  if (!make_map(&mapB, planesA, m, kpad, J, kPairRows, a_plane_rows)) return cudaErrorInvalidValue;
  Sched s;
  s.J = J;
  s.ppm = ppm;
  s.pairs = (J + 1) / 2;
  s.TJ = static_cast<int>((n + kPairBM - 1) / kPairBM);
  s.TI = static_cast<int>((m + kPairBN - 1) / kPairBN);
  s.tiles = s.TJ * s.TI;
  s.group = group > 0 ? group : 16;
  s.nkb = static_cast<int>(kpad / BK);
  s.ck = chunk_k / BK;
  s.nch = (s.nkb + s.ck - 1) / s.ck;
  s.units = static_cast<long long>(s.pairs) * s.tiles;
  s.order = sc.order;
  s.pairing = sc.pairing;
  s.kalt = sc.kalt;
  s.band = sc.band_cols / kPairBM > 0 ? sc.band_cols / kPairBM : 1;
  const long long pairs = s.units < clusters ? s.units : clusters;
  gemm_f16_pair_kernel<<<static_cast<unsigned int>(2 * pairs), kThreads, kPairSmem, st>>>(mapA, mapB, pl, s, res,
                                                                                          ldr, n, rcap, status);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace

int g_f16_group = 16;   // tile rasterisation group of grouped launches

bool gemm_pair_supported() { return get_encoder() && pair_clusters() > 0; }

// a_plane_rows: rows between consecutive planes of planesA (0: m), so that a
// block of rows of a larger plane set can be passed; rcap: residue rows stored
// per column (0: ldr), at most ldr and a multiple of 16.
cudaError_t launch_gemm_f16(int64_t m, int64_t n, int64_t kpad, const Plan& pl, const void* planesA,
                            const void* planesB, int8_t* res, int64_t ldr, int chunk_k, unsigned int* status,
                            cudaStream_t st, int tile_n, int group, int ppm, int64_t a_plane_rows, int64_t rcap,
                            const GemmSchedule& sc) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  if (!sc.valid()) return cudaErrorInvalidValue;
  if (ppm != 1 && ppm != 3) return cudaErrorInvalidValue;
  if (kpad % BK || ldr % 16 || chunk_k % BK || chunk_k < BK || chunk_k > 960) return cudaErrorInvalidValue;
  if (a_plane_rows == 0) a_plane_rows = m;
  if (rcap == 0) rcap = ldr;
  if (a_plane_rows < m || rcap % 16 || rcap > ldr || rcap < m || (reinterpret_cast<uintptr_t>(res) & 15u))
    return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(planesA) | reinterpret_cast<uintptr_t>(planesB)) & 15u)
    return cudaErrorInvalidValue;
  if (!get_encoder()) return cudaErrorNotSupported;
  if (sc.cta_pair)
    return launch_pair(m, n, kpad, pl, planesA, planesB, res, ldr, chunk_k, group, status, st, ppm, a_plane_rows,
                       rcap, sc);
  switch (tile_n) {
    case 64:
      return launch_single<64>(m, n, kpad, pl, planesA, planesB, res, ldr, chunk_k, group, status, st, ppm,
                               a_plane_rows, rcap, sc);
    case 128:
      return launch_single<128>(m, n, kpad, pl, planesA, planesB, res, ldr, chunk_k, group, status, st, ppm,
                                a_plane_rows, rcap, sc);
    default:
      return launch_single<256>(m, n, kpad, pl, planesA, planesB, res, ldr, chunk_k, group, status, st, ppm,
                                a_plane_rows, rcap, sc);
  }
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
  if (e == cudaSuccess) e = set_grouped_attrs();
  return e;
}

// Fill the host-side descriptor of problem p of a grouped launch (tensor maps,
// output, schedule); returns false on an invalid shape.  `unit_begin` is the
// running unit count, advanced past this problem's units.
bool fill_group_problem(void* desc, int64_t m, int64_t n, int64_t kpad, int N, const void* planesA,
                        const void* planesB, int8_t* res, int64_t ldr, int chunk_k, int group, int tile_n,
                        long long* unit_begin, const GemmSchedule& sc) {
  if (!get_encoder() || !sc.valid() || (tile_n != 64 && tile_n != 128 && tile_n != 256)) return false;
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
  P.order = sc.order;
  P.pairing = sc.pairing;
  P.kalt = sc.kalt;
  P.band = sc.band_cols / BM;
  P.bn = tile_n;
  P.unit_begin = *unit_begin;
  *unit_begin += static_cast<long long>((J + 1) / 2) * P.tiles;
  return true;
}

cudaError_t launch_gemm_f16_grouped(const void* probs_dev, int count, long long total_units, const Plan& pl,
                                    unsigned int* status, cudaStream_t st) {
  if (count <= 0 || total_units <= 0) return cudaSuccess;
  if (!get_encoder()) return cudaErrorNotSupported;
  const GroupProblem* P = static_cast<const GroupProblem*>(probs_dev);
  const long long grid = total_units < g_sms ? total_units : g_sms;
  const cudaError_t e = set_grouped_attrs();
  if (e != cudaSuccess) return e;
  gemm_f16_grouped_kernel<<<static_cast<unsigned int>(grid), kGroupedThreads, kGroupedSmem, st>>>(
      P, count, total_units, pl, status);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace emu
