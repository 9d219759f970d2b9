// Autotuner of the single-GEMM launch configuration.  For one problem shape it
// times, on synthetic data of that shape and with CUDA events, the candidates
// of each phase's knobs (the phases are independent, so each is timed on its
// own): the residue-product tile width, rasterisation group and reduction
// chunk, then the modulus-loop schedule of those products (unit order, among
// them the paper's n-blocked order of Section III-A; k direction; job
// pairing; tiles on SM pairs), searched one knob at a time from the best so
// far; the CRT engine and rows per thread; the split entries per thread.  A candidate replaces the incumbent
// only when it is at least 0.5 % faster, so timing noise does not move the
// choice.  The winners are kept per (dtype, N, ceil(log2) of m, n, k) and used
// by later calls in that bucket; EMU_AUTOTUNE_CACHE names a file that keeps
// the table across processes.
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "emu_internal.h"

namespace emu {
namespace {

using Key = std::tuple<int, int, int, int, int>;

// cache lines: tag, dtype, N, the three log2 buckets, then tile_n group chunk_k
// crt_rows split_elems order pairing kdir band crt_engine cta_pair
constexpr const char* kCacheTag = "gemm3";

std::mutex g_mu;
Tune g_default;
std::map<Key, Tune> g_table;
bool g_loaded = false;

int bucket(int64_t v) {
  int b = 0;
  while ((int64_t(1) << b) < v && b < 62) ++b;
  return b;
}

Key key_of(int dtype, int N, int64_t m, int64_t n, int64_t k) {
  return Key(dtype, N, bucket(m), bucket(n), bucket(k));
}

bool valid(int key, int v) {
  switch (key) {
    case EMU_TUNE_TILE_N: return v == 64 || v == 128 || v == 256;
    case EMU_TUNE_GROUP: return v >= 1 && v <= 64;
    case EMU_TUNE_CHUNK_K: return v >= 64 && v <= 960 && v % 64 == 0;
    case EMU_TUNE_CRT_ROWS: return v == 1 || v == 2 || v == 4;
    case EMU_TUNE_SPLIT_ELEMS: return v == 2 || v == 4;
    case EMU_TUNE_NBLOCK: return v == 0 || (v >= 128 && v % 128 == 0);
    case EMU_TUNE_OVERLAP: return v == -1 || v == 0 || v == 1;
    case EMU_TUNE_ORDER: return v >= 0 && v <= 2;
    case EMU_TUNE_PAIRING: return v >= 0 && v <= 2;
    case EMU_TUNE_KDIR: return v == 0 || v == 1;
    case EMU_TUNE_BAND: return v >= 128 && v <= 65536 && v % 128 == 0;
    case EMU_TUNE_CRT_ENGINE: return v == 0 || v == 1;
    case EMU_TUNE_CTA_PAIR: return v == 0 || v == 1;
    case EMU_TUNE_BOUND_PAIR: return v == 0 || v == 1;
    default: return false;
  }
}

void load_locked() {
  if (g_loaded) return;
  g_loaded = true;
  const char* path = std::getenv("EMU_AUTOTUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  char tag[64];
  int s, N, bm, bn, bk;
  Tune t;
  while (std::fscanf(f, "%63s", tag) == 1) {
    if (std::string(tag) != kCacheTag) {   // other tables (or older formats) share the file: skip the line
      int c;
      while ((c = std::fgetc(f)) != EOF && c != '\n') {
      }
      continue;
    }
    if (std::fscanf(f, "%d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d", &s, &N, &bm, &bn, &bk, &t.tile_n,
                    &t.group, &t.chunk_k, &t.crt_rows, &t.split_elems, &t.sched.order, &t.sched.pairing,
                    &t.sched.kalt, &t.sched.band_cols, &t.crt_engine, &t.sched.cta_pair) != 16)
      break;
    // a stale or hand-edited entry with a value the launchers would refuse is skipped,
    // so the defaults stay in force for its bucket
    if (valid(EMU_TUNE_TILE_N, t.tile_n) && valid(EMU_TUNE_GROUP, t.group) && valid(EMU_TUNE_CHUNK_K, t.chunk_k) &&
        valid(EMU_TUNE_CRT_ROWS, t.crt_rows) && valid(EMU_TUNE_SPLIT_ELEMS, t.split_elems) && t.sched.valid() &&
        valid(EMU_TUNE_CRT_ENGINE, t.crt_engine))
      g_table[Key(s, N, bm, bn, bk)] = t;
    else
      std::fprintf(stderr, "ozaki2emu: ignoring invalid autotune cache entry for dtype %d, N %d\n", s, N);
  }
  std::fclose(f);
}

void save_locked() {
  const char* path = std::getenv("EMU_AUTOTUNE_CACHE");
  if (!path) return;
  // keep lines of other tables that share the file
  std::vector<std::string> keep;
  if (FILE* f = std::fopen(path, "r")) {
    char line[4096];
    while (std::fgets(line, sizeof(line), f))
      if (std::string(line).rfind(std::string(kCacheTag) + " ", 0) != 0) keep.push_back(line);
    std::fclose(f);
  }
  FILE* f = std::fopen(path, "w");
  if (!f) return;
  for (const auto& l : keep) std::fputs(l.c_str(), f);
  for (const auto& kv : g_table) {
    const Key& k = kv.first;
    const Tune& t = kv.second;
    std::fprintf(f, "%s %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d\n", kCacheTag, std::get<0>(k),
                 std::get<1>(k), std::get<2>(k), std::get<3>(k), std::get<4>(k), t.tile_n, t.group, t.chunk_k,
                 t.crt_rows, t.split_elems, t.sched.order, t.sched.pairing, t.sched.kalt, t.sched.band_cols,
                 t.crt_engine, t.sched.cta_pair);
  }
  std::fclose(f);
}

void set(Tune& t, int key, int v) {
  switch (key) {
    case EMU_TUNE_TILE_N: t.tile_n = v; break;
    case EMU_TUNE_GROUP: t.group = v; break;
    case EMU_TUNE_CHUNK_K: t.chunk_k = v; break;
    case EMU_TUNE_CRT_ROWS: t.crt_rows = v; break;
    case EMU_TUNE_SPLIT_ELEMS: t.split_elems = v; break;
    case EMU_TUNE_NBLOCK: t.nblock = v; break;
    case EMU_TUNE_OVERLAP: t.overlap = v; break;
    case EMU_TUNE_ORDER: t.sched.order = v; break;
    case EMU_TUNE_PAIRING: t.sched.pairing = v; break;
    case EMU_TUNE_KDIR: t.sched.kalt = v; break;
    case EMU_TUNE_BAND: t.sched.band_cols = v; break;
    case EMU_TUNE_CRT_ENGINE: t.crt_engine = v; break;
    case EMU_TUNE_CTA_PAIR: t.sched.cta_pair = v; break;
    case EMU_TUNE_BOUND_PAIR: t.bound_pair = v; break;
    default: break;
  }
}

// synthetic inputs for timing: (u - 1/2) 2^(s) with u and s from a hash of the index
__global__ void fill_kernel(double* p, int64_t count) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= count) return;
  uint64_t h = static_cast<uint64_t>(i) * 0x9E3779B97F4A7C15ull;
  h ^= h >> 29;
  h *= 0xBF58476D1CE4E5B9ull;
  h ^= h >> 32;
  const double u = static_cast<double>(h & 0xFFFFFFull) * (1.0 / 16777216.0) - 0.5;
  const int s = static_cast<int>((h >> 24) & 7) - 3;
  p[i] = u * static_cast<double>(1 << (s + 3)) * 0.125;
}

__global__ void fill_kernel_f(float* p, int64_t count) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= count) return;
  uint64_t h = static_cast<uint64_t>(i) * 0x9E3779B97F4A7C15ull;
  h ^= h >> 29;
  h *= 0xBF58476D1CE4E5B9ull;
  h ^= h >> 32;
  p[i] = static_cast<float>(static_cast<double>(h & 0xFFFFFFull) * (1.0 / 16777216.0) - 0.5);
}

// Time fn() on st: one warm-up, then the minimum of `reps` runs (ms).
template <class F>
float time_min(cudaStream_t st, cudaEvent_t a, cudaEvent_t b, int reps, F fn) {
  fn();
  float best = 1e30f;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(a, st);
    fn();
    cudaEventRecord(b, st);
    if (cudaEventSynchronize(b) != cudaSuccess) return 1e30f;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, a, b);
    if (ms < best) best = ms;
  }
  return best;
}

size_t al(size_t v) { return (v + 255) / 256 * 256; }

constexpr float kKeep = 0.995f;   // a candidate must beat the incumbent by 0.5 %

}  // namespace

Tune tune_for(int dtype, int N, int64_t m, int64_t n, int64_t k) {
  std::lock_guard<std::mutex> lk(g_mu);
  load_locked();
  auto it = g_table.find(key_of(dtype, N, m, n, k));
  if (it == g_table.end()) return g_default;
  Tune t = it->second;
  t.nblock = g_default.nblock;          // column blocking, overlap and the bound products' tiles
  t.overlap = g_default.overlap;        // are process settings, not tuned
  t.bound_pair = g_default.bound_pair;
  return t;
}

void set_default_tuning(int key, int value) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (valid(key, value)) set(g_default, key, value);
}

}  // namespace emu

extern "C" {

emu_status_t emu_set_tuning(int key, int value) {
  if (!emu::valid(key, value)) return EMU_ERR_INVALID_ARG;
  emu::set_default_tuning(key, value);
  return EMU_OK;
}

int emu_get_tuning(int key) {
  std::lock_guard<std::mutex> lk(emu::g_mu);
  const emu::Tune& t = emu::g_default;
  switch (key) {
    case EMU_TUNE_TILE_N: return t.tile_n;
    case EMU_TUNE_GROUP: return t.group;
    case EMU_TUNE_CHUNK_K: return t.chunk_k;
    case EMU_TUNE_CRT_ROWS: return t.crt_rows;
    case EMU_TUNE_SPLIT_ELEMS: return t.split_elems;
    case EMU_TUNE_NBLOCK: return t.nblock;
    case EMU_TUNE_OVERLAP: return t.overlap;
    case EMU_TUNE_ORDER: return t.sched.order;
    case EMU_TUNE_PAIRING: return t.sched.pairing;
    case EMU_TUNE_KDIR: return t.sched.kalt;
    case EMU_TUNE_BAND: return t.sched.band_cols;
    case EMU_TUNE_CRT_ENGINE: return t.crt_engine;
    case EMU_TUNE_CTA_PAIR: return t.sched.cta_pair;
    case EMU_TUNE_BOUND_PAIR: return t.bound_pair;
    default: return -1;
  }
}

int emu_tuned_value(int dtype, int num_moduli, int64_t m, int64_t n, int64_t k, int key) {
  const emu::Tune t = emu::tune_for(dtype, num_moduli, m, n, k);
  switch (key) {
    case EMU_TUNE_TILE_N: return t.tile_n;
    case EMU_TUNE_GROUP: return t.group;
    case EMU_TUNE_CHUNK_K: return t.chunk_k;
    case EMU_TUNE_CRT_ROWS: return t.crt_rows;
    case EMU_TUNE_SPLIT_ELEMS: return t.split_elems;
    case EMU_TUNE_NBLOCK: return t.nblock;
    case EMU_TUNE_OVERLAP: return t.overlap;
    case EMU_TUNE_ORDER: return t.sched.order;
    case EMU_TUNE_PAIRING: return t.sched.pairing;
    case EMU_TUNE_KDIR: return t.sched.kalt;
    case EMU_TUNE_BAND: return t.sched.band_cols;
    case EMU_TUNE_CRT_ENGINE: return t.crt_engine;
    case EMU_TUNE_CTA_PAIR: return t.sched.cta_pair;
    case EMU_TUNE_BOUND_PAIR: return t.bound_pair;
    default: return -1;
  }
}

emu_status_t emu_autotune_clear(void) {
  std::lock_guard<std::mutex> lk(emu::g_mu);
  emu::g_table.clear();
  return EMU_OK;
}

emu_status_t emu_autotune_gemm(int dtype, int64_t m, int64_t n, int64_t k, int num_moduli, int* best) {
  using namespace emu;
  if (dtype < EMU_DTYPE_Z || dtype > EMU_DTYPE_S) return EMU_ERR_INVALID_ARG;
  if (m <= 0 || n <= 0 || k <= 0 || k > EMU_MAX_K) return EMU_ERR_INVALID_ARG;
  if (num_moduli < EMU_MIN_MODULI || num_moduli > EMU_MAX_MODULI) return EMU_ERR_MODULI_RANGE;
  unsigned int* status = device_status_ptr();
  if (!status) return EMU_ERR_UNSUPPORTED;
  const bool single = (dtype == EMU_DTYPE_C || dtype == EMU_DTYPE_S);
  const bool real = dtype >= EMU_DTYPE_D;
  const int ppm = real ? 1 : 3;
  const Plan* pl = get_plan(num_moduli);
  const int J = ppm * num_moduli;
  const int64_t kpad = round_up(k, 64), ldr = round_up(m, 16);
  const int parts = real ? 1 : 2;                     // real numbers per entry
  const size_t esz = static_cast<size_t>(parts) * (single ? 4 : 8);
  // one buffer: A, B, x, y, exponent scratch, fp16 planes, residues, C
  size_t o = 0;
  const size_t oA = o; o += al(esz * static_cast<size_t>(m) * k);
  const size_t oB = o; o += al(esz * static_cast<size_t>(k) * n);
  const size_t ox = o; o += al(2 * static_cast<size_t>(m));
  const size_t oy = o; o += al(2 * static_cast<size_t>(n));
  const size_t os = o; o += al(exponents_scratch_bytes(m > n ? m : n));
  const size_t opa = o; o += al(static_cast<size_t>(J) * m * kpad * 2);
  const size_t opb = o; o += al(static_cast<size_t>(J) * n * kpad * 2);
  const size_t ores = o; o += al(static_cast<size_t>(J) * n * ldr);
  const size_t oC = o; o += al(esz * static_cast<size_t>(m) * n);
  char* M = nullptr;
  if (cudaMalloc(&M, o) != cudaSuccess) {
    cudaGetLastError();
    return EMU_ERR_ALLOC;
  }
  cudaStream_t st = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  bool ok = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess;
  const int64_t cntA = parts * m * k, cntB = parts * k * n;   // real numbers in A and B
  if (ok && !single) {
    fill_kernel<<<static_cast<unsigned int>((cntA + 255) / 256), 256, 0, st>>>(reinterpret_cast<double*>(M + oA), cntA);
    fill_kernel<<<static_cast<unsigned int>((cntB + 255) / 256), 256, 0, st>>>(reinterpret_cast<double*>(M + oB), cntB);
  } else if (ok) {
    fill_kernel_f<<<static_cast<unsigned int>((cntA + 255) / 256), 256, 0, st>>>(reinterpret_cast<float*>(M + oA), cntA);
    fill_kernel_f<<<static_cast<unsigned int>((cntB + 255) / 256), 256, 0, st>>>(reinterpret_cast<float*>(M + oB), cntB);
  }
  int16_t* x = reinterpret_cast<int16_t*>(M + ox);
  int16_t* y = reinterpret_cast<int16_t*>(M + oy);
  Tune t = tune_for(dtype, num_moduli, m, n, k);
  if (ok) {
    ok = launch_exponents(single, M + oA, m, k, 1, m, *pl, x, M + os, st, real) == cudaSuccess &&
         launch_exponents(single, M + oB, n, k, k, 1, *pl, y, M + os, st, real) == cudaSuccess;
  }
  const int reps = (static_cast<double>(m) * n * k > 1e12) ? 2 : 3;
  if (ok) {
    // split: entries per thread
    float bt = 1e30f;
    for (int e : {4, 2}) {
      const float ms = time_min(st, a, b, reps, [&] {
        launch_split(single, false, M + oA, m, k, 1, m, *pl, x, true, kpad, M + opa, st, e, real);
        launch_split(single, false, M + oB, n, k, k, 1, *pl, y, true, kpad, M + opb, st, e, real);
      });
      if (ms < kKeep * bt) {
        bt = ms;
        t.split_elems = e;
      }
    }
    // residue products: tile width x group x chunk
    bt = 1e30f;
    const bool big = static_cast<double>(m) * n * k * num_moduli > 4e13;
    // the defaults first: a candidate must beat the incumbent by 0.5 % to replace it
    const std::vector<int> tiles = m <= 256 ? std::vector<int>{256, 128, 64} : std::vector<int>{256, 128};
    const std::vector<int> groups = big ? std::vector<int>{16, 32} : std::vector<int>{16, 8, 32};
    const std::vector<int> chunks = big ? std::vector<int>{960} : std::vector<int>{960, 512};
    if (prepare_gemm_f16() != cudaSuccess) ok = false;
    for (int tn : tiles)
      for (int g : groups)
        for (int c : chunks) {
          if (!ok) break;
          const float ms = time_min(st, a, b, reps, [&] {
            launch_gemm_f16(m, n, kpad, *pl, M + opa, M + opb, reinterpret_cast<int8_t*>(M + ores), ldr, c, status,
                            st, tn, g, ppm, 0, 0, GemmSchedule());
          });
          if (ms < kKeep * bt) {
            bt = ms;
            t.tile_n = tn;
            t.group = g;
            t.chunk_k = c;
          }
        }
    // modulus-loop schedule of the residue products, one knob at a time from the best so far:
    // unit order (modulus outer; tile outer; column bands of the paper's 8192 columns and of 2048),
    // then alternating k direction, then job pairing, then SM-pair tiles
    GemmSchedule sc;
    auto time_sched = [&](const GemmSchedule& cand) {
      return time_min(st, a, b, reps, [&] {
        launch_gemm_f16(m, n, kpad, *pl, M + opa, M + opb, reinterpret_cast<int8_t*>(M + ores), ldr, t.chunk_k,
                        status, st, t.tile_n, t.group, ppm, 0, 0, cand);
      });
    };
    std::vector<GemmSchedule> orders;
    {
      GemmSchedule c = sc;
      c.order = 1;
      orders.push_back(c);
      for (int bc : {8192, 2048}) {
        if (n <= bc) continue;                 // one band: the same order as modulus outer
        c.order = 2;
        c.band_cols = bc;
        orders.push_back(c);
      }
    }
    for (const GemmSchedule& c : orders) {
      if (!ok) break;
      const float ms = time_sched(c);
      if (ms < kKeep * bt) {
        bt = ms;
        sc = c;
      }
    }
    {
      GemmSchedule c = sc;
      c.kalt = 1;
      const float ms = time_sched(c);
      if (ms < kKeep * bt) {
        bt = ms;
        sc = c;
      }
    }
    for (int pr : {1, 2}) {
      if (real && pr == 2) continue;           // one job per modulus: the same as adjacent
      GemmSchedule c = sc;
      c.pairing = pr;
      const float ms = time_sched(c);
      if (ms < kKeep * bt) {
        bt = ms;
        sc = c;
      }
    }
    if (ok && gemm_pair_supported()) {          // 256 x 256 tiles on SM pairs
      GemmSchedule c = sc;
      c.cta_pair = 1;
      const float ms = time_sched(c);
      if (ms < kKeep * bt) {
        bt = ms;
        sc = c;
      }
    }
    t.sched = sc;
    // CRT: the tensor-core kernel, then the CUDA-core kernel's rows per thread
    bt = time_min(st, a, b, reps, [&] {
      launch_crt_tc(single, m, n, *pl, reinterpret_cast<int8_t*>(M + ores), ldr, x, y, 1.0, 0.0, 0.0, 0.0, M + oC, m,
                    st, real, false, status);
    });
    t.crt_engine = 1;
    for (int r : {4, 2, 1}) {
      const float ms = time_min(st, a, b, reps, [&] {
        launch_crt(single, m, n, *pl, reinterpret_cast<int8_t*>(M + ores), ldr, x, y, 1.0, 0.0, 0.0, 0.0, M + oC, m,
                   st, r, real);
      });
      if (ms < kKeep * bt) {
        bt = ms;
        t.crt_rows = r;
        t.crt_engine = 0;
      }
    }
    ok = cudaStreamSynchronize(st) == cudaSuccess;
  }
  if (b) cudaEventDestroy(b);
  if (a) cudaEventDestroy(a);
  if (st) cudaStreamDestroy(st);
  cudaFree(M);
  if (!ok) {
    cudaGetLastError();
    return EMU_ERR_CUDA;
  }
  {
    std::lock_guard<std::mutex> lk(g_mu);
    load_locked();
    t.nblock = 0;
    g_table[key_of(dtype, num_moduli, m, n, k)] = t;
    save_locked();
  }
  if (best) {
    best[0] = t.tile_n;
    best[1] = t.group;
    best[2] = t.chunk_k;
    best[3] = t.crt_rows;
    best[4] = t.split_elems;
  }
  return EMU_OK;
}

}  // extern "C"
