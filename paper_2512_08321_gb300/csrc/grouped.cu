// Grouped emulated GEMM: many complex GEMMs of uneven shapes sharing one
// moduli count, each phase of the method (Algorithm 1 Steps III to VI) run as
// ONE persistent launch over every problem, captured once in a CUDA graph and
// replayed.  The tile width of the residue-product launch is picked by timing
// the candidates on the problem set itself (autotuner), and remembered per
// problem-set signature (and optionally in a cache file).
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "emu_internal.h"

struct emu_grouped_s {
  int dev = -1;
  bool single = false;
  int N = 0;
  int count = 0;
  const emu::Plan* pl = nullptr;
  int tile_n = 256;
  int chunk_k = 960;                // k between in-TMEM reductions (the largest exact one)
  char* mem = nullptr;            // workspace + descriptor tables
  size_t mem_bytes = 0;
  size_t scratch_off = 0, scratch_bytes = 0;
  emu::ExpSeg* d_exp = nullptr;
  int* maps = nullptr;              // segment of every exponent block, then of every split block
  int* d_emap = nullptr;
  int* d_smap = nullptr;
  int nexp = 0;
  long long exp_blocks = 0;
  long long* d_rowbeg = nullptr;
  long long total_rows = 0;
  emu::SplitSeg* d_split = nullptr;
  int nsplit = 0;
  long long split_blocks = 0;
  void* d_gp = nullptr;
  int ngp = 0;
  long long total_units = 0;
  emu::CrtProb* d_crt = nullptr;
  int ncrt = 0;
  long long crt_blocks = 0;
  emu::CrtProb* d_crt_tc = nullptr;   // the same problems in 128-row items (tensor-core CRT)
  long long crt_tc_items = 0;
  int crt_engine = 1;               // EMU_TUNE_CRT_ENGINE at plan creation
  unsigned int* status = nullptr;
  int kernels = 0;                // kernel launches in one replay
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // host copies needed to rebuild the GEMM descriptors for another tile width
  struct Prob {
    int64_t m, n, kpad, ldr;
    void* pa;
    void* pb;
    int8_t* res;
  };
  std::vector<Prob> probs;
};

namespace emu {
namespace {

thread_local int t_bad = 0;

std::mutex g_tune_mu;
std::map<std::string, int> g_tune;     // signature -> tile width
bool g_tune_loaded = false;

size_t al(size_t v) { return (v + 255) / 256 * 256; }

const char* cache_path() { return std::getenv("EMU_AUTOTUNE_CACHE"); }

void load_cache() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = cache_path();
  if (!path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  char key[4096];
  int tn;
  while (std::fscanf(f, "%4095s %d", key, &tn) == 2) g_tune[key] = tn;
  std::fclose(f);
}

void save_cache() {
  const char* path = cache_path();
  if (!path) return;
  FILE* f = std::fopen(path, "w");
  if (!f) return;
  for (const auto& kv : g_tune) std::fprintf(f, "%s %d\n", kv.first.c_str(), kv.second);
  std::fclose(f);
}

// Signature of a problem set: dtype, N and the multiset of shapes (hashed).
std::string signature(bool single, int N, const std::vector<emu_grouped_s::Prob>& P, const int64_t* k) {
  unsigned long long h = 1469598103934665603ull;
  auto mix = [&](unsigned long long v) {
    h ^= v;
    h *= 1099511628211ull;
  };
  for (size_t i = 0; i < P.size(); ++i) {
    mix(static_cast<unsigned long long>(P[i].m));
    mix(static_cast<unsigned long long>(P[i].n));
    mix(static_cast<unsigned long long>(k[i]));
  }
  char buf[96];
  std::snprintf(buf, sizeof(buf), "grouped:%c:N%d:count%zu:%016llx", single ? 'c' : 'z', N, P.size(), h);
  return buf;
}

// Tile width of one problem under the per-problem rule: the width (64, 128,
// 256) with the fewest padded rows counting 64 rows of fixed cost per tile
// (its epilogue and pipeline fill), ties to the wider tile.
int problem_tile(int64_t m) {
  int best = 256;
  int64_t best_cost = -1;
  for (int tn : {256, 128, 64}) {
    const int64_t cost = (m + tn - 1) / tn * (tn + 64);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = tn;
    }
  }
  return best;
}

// Descriptors, then the first unit of every problem as a compact array the
// residue-product kernel scans (long long per problem).  tile_n: 64, 128 or
// 256 for every problem, EMU_GROUPED_TILE_PER_PROBLEM for problem_tile(m).
emu_status_t upload_gemm_descs(emu_grouped_s* g, int tile_n, void* d_dst, long long* total_units) {
  const size_t np = g->probs.size();
  std::vector<unsigned char> host(group_problem_bytes() * np + sizeof(long long) * np);
  long long* ubeg = reinterpret_cast<long long*>(host.data() + group_problem_bytes() * np);
  long long units = 0;
  for (size_t i = 0; i < np; ++i) {
    const auto& p = g->probs[i];
    ubeg[i] = units;
    const int tn = tile_n == EMU_GROUPED_TILE_PER_PROBLEM ? problem_tile(p.m) : tile_n;
    if (!fill_group_problem(host.data() + i * group_problem_bytes(), p.m, p.n, p.kpad, g->N, p.pa, p.pb, p.res, p.ldr,
                            g->chunk_k, g_f16_group, tn, &units))
      return EMU_ERR_CUDA;
  }
  if (cudaMemcpy(d_dst, host.data(), host.size(), cudaMemcpyHostToDevice) != cudaSuccess) return EMU_ERR_CUDA;
  *total_units = units;
  return EMU_OK;
}

// Phase 4: the CRT of every problem, on the tensor cores or the CUDA cores (the engine the
// process default named when the plan was created).
cudaError_t crt_phase(emu_grouped_s* g, cudaStream_t st) {
  if (g->crt_engine == 1)
    return launch_crt_tc_grouped(g->single, g->d_crt_tc, g->ncrt, g->crt_tc_items, *g->pl, g->status, st);
  return launch_crt_grouped(g->single, g->d_crt, g->ncrt, g->crt_blocks, *g->pl, st);
}

// Phases 1-2 (exponents, split) and 4 (CRT) around a given residue-product launch.
cudaError_t enqueue(emu_grouped_s* g, cudaStream_t st, bool with_gemm) {
  cudaError_t e = cudaMemsetAsync(g->mem + g->scratch_off, 0, g->scratch_bytes, st);
  if (e != cudaSuccess) return e;
  if ((e = launch_exponents_grouped(g->single, g->d_exp, g->d_emap, g->nexp, g->exp_blocks, g->d_rowbeg,
                                    g->total_rows, *g->pl, st)) != cudaSuccess)
    return e;
  if ((e = launch_split_grouped(g->single, true, g->d_split, g->d_smap, g->nsplit, g->split_blocks, *g->pl, st)) !=
      cudaSuccess)
    return e;
  if (!with_gemm) return cudaSuccess;
  if ((e = launch_gemm_f16_grouped(g->d_gp, g->ngp, g->total_units, *g->pl, g->status, st)) !=
      cudaSuccess)
    return e;
  return crt_phase(g, st);
}

// Time the residue-product launch for the per-problem widths and each uniform
// tile width on this problem set.
int autotune(emu_grouped_s* g, cudaStream_t st) {
  const int cands[4] = {EMU_GROUPED_TILE_PER_PROBLEM, 256, 128, 64};
  int best = EMU_GROUPED_TILE_PER_PROBLEM;
  float best_ms = 1e30f;
  if (enqueue(g, st, false) != cudaSuccess) return best;      // planes for the timing runs
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  for (int tn : cands) {
    long long units = 0;
    if (upload_gemm_descs(g, tn, g->d_gp, &units) != EMU_OK) continue;
    float ms_min = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
      cudaEventRecord(a, st);
      launch_gemm_f16_grouped(g->d_gp, g->ngp, units, *g->pl, g->status, st);
      cudaEventRecord(b, st);
      if (cudaEventSynchronize(b) != cudaSuccess) break;
      float ms = 0;
      cudaEventElapsedTime(&ms, a, b);
      if (rep > 0) ms_min = std::min(ms_min, ms);            // first run is warm-up
    }
    if (ms_min < best_ms) {
      best_ms = ms_min;
      best = tn;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return best;
}

}  // namespace
}  // namespace emu

extern "C" {

emu_status_t emu_grouped_create(int is_single, int count, const emu_op_t* transa, const emu_op_t* transb,
                                const int64_t* m, const int64_t* n, const int64_t* k, const double* alpha,
                                const void* const* A, const int64_t* lda, const void* const* B,
                                const int64_t* ldb, const double* beta, void* const* C, const int64_t* ldc,
                                int num_moduli, int tile_n, emu_grouped_t* out) {
  using namespace emu;
  t_bad = 0;
  if (!out) return EMU_ERR_INVALID_ARG;
  *out = nullptr;
  if (count < 0) return EMU_ERR_INVALID_ARG;
  if (num_moduli < EMU_MIN_MODULI || num_moduli > EMU_MAX_MODULI) return EMU_ERR_MODULI_RANGE;
  if (tile_n != 0 && tile_n != EMU_GROUPED_TILE_PER_PROBLEM && tile_n != 64 && tile_n != 128 && tile_n != 256)
    return EMU_ERR_INVALID_ARG;
  if (count > 0 && (!transa || !transb || !m || !n || !k || !alpha || !A || !lda || !B || !ldb || !beta || !C || !ldc))
    return EMU_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i) {
    const bool okop = (transa[i] >= EMU_OP_N && transa[i] <= EMU_OP_C) && (transb[i] >= EMU_OP_N && transb[i] <= EMU_OP_C);
    if (!okop || m[i] < 0 || n[i] < 0 || k[i] < 0) return EMU_ERR_INVALID_ARG;
    const int64_t ra = transa[i] == EMU_OP_N ? m[i] : k[i];
    const int64_t rb = transb[i] == EMU_OP_N ? k[i] : n[i];
    if (lda[i] < std::max<int64_t>(1, ra) || ldb[i] < std::max<int64_t>(1, rb) || ldc[i] < std::max<int64_t>(1, m[i]))
      return EMU_ERR_INVALID_ARG;
    if (k[i] > EMU_MAX_K) return EMU_ERR_K_TOO_LARGE;
    if (m[i] > (int64_t(1) << 31) || n[i] > (int64_t(1) << 31)) return EMU_ERR_INVALID_ARG;
    if (m[i] > 0 && n[i] > 0 && (!C[i] || (k[i] > 0 && (!A[i] || !B[i])))) return EMU_ERR_INVALID_ARG;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return EMU_ERR_CUDA;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return EMU_ERR_CUDA;
  if (!(prop.major == 10 && prop.minor == 3)) return EMU_ERR_UNSUPPORTED;
  unsigned int* status = device_status_ptr();
  if (!status) return EMU_ERR_CUDA;

  emu_grouped_s* g = new emu_grouped_s();
  g->dev = dev;
  g->single = is_single != 0;
  g->N = num_moduli;
  g->count = count;
  g->pl = get_plan(num_moduli);
  g->status = status;
  const int J = 3 * num_moduli;
  const size_t esz = 2;  // fp16 planes

  // workspace layout per problem (problems with an empty output are skipped)
  struct Off {
    size_t x, y, scr_a, scr_b, pa, pb, res;
    int64_t kpad, ldr;
  };
  std::vector<Off> off(count);
  std::vector<int> live;
  size_t o = 0, scr = 0;
  for (int i = 0; i < count; ++i) {
    if (m[i] == 0 || n[i] == 0) continue;
    live.push_back(i);
    Off& f = off[i];
    f.kpad = round_up(k[i] > 0 ? k[i] : 1, 64);
    f.ldr = round_up(m[i], 16);
    f.scr_a = scr;
    scr += al(exponents_scratch_bytes(m[i]));
    f.scr_b = scr;
    scr += al(exponents_scratch_bytes(n[i]));
  }
  g->scratch_off = 0;
  g->scratch_bytes = scr;
  o = scr;
  for (int i : live) {
    Off& f = off[i];
    f.x = o;   o += al(static_cast<size_t>(m[i]) * 2);
    f.y = o;   o += al(static_cast<size_t>(n[i]) * 2);
    f.pa = o;  o += al(static_cast<size_t>(J) * m[i] * f.kpad * esz);
    f.pb = o;  o += al(static_cast<size_t>(J) * n[i] * f.kpad * esz);
    f.res = o; o += al(static_cast<size_t>(J) * n[i] * f.ldr);
  }
  const size_t nl = live.size();
  const size_t off_exp = o;     o += al(sizeof(ExpSeg) * 2 * nl + 1);
  const size_t off_rowb = o;    o += al(sizeof(long long) * (2 * nl + 1));
  const size_t off_split = o;   o += al(sizeof(SplitSeg) * 2 * nl + 1);
  const size_t off_gp = o;      o += al((group_problem_bytes() + sizeof(long long)) * nl + 1);
  const size_t off_crt = o;     o += al(sizeof(CrtProb) * nl + 1);
  const size_t off_crt_tc = o;  o += al(sizeof(CrtProb) * nl + 1);
  g->mem_bytes = o;
  if (cudaMalloc(&g->mem, o) != cudaSuccess) {
    cudaGetLastError();
    delete g;
    return EMU_ERR_ALLOC;
  }
  char* M = g->mem;
  std::vector<ExpSeg> es;
  std::vector<long long> rowb;
  std::vector<SplitSeg> ss;
  std::vector<CrtProb> cp, cpt;
  long long eb = 0, sb = 0, cb = 0, ct = 0, rows = 0;
  for (int i : live) {
    const Off& f = off[i];
    int16_t* x = reinterpret_cast<int16_t*>(M + f.x);
    int16_t* y = reinterpret_cast<int16_t*>(M + f.y);
    // op(A) rows (i, h) and op(B) columns (j, h), as in the single-GEMM path
    const int64_t rsa = transa[i] == EMU_OP_N ? 1 : lda[i], hsa = transa[i] == EMU_OP_N ? lda[i] : 1;
    const int64_t rsb = transb[i] == EMU_OP_N ? ldb[i] : 1, hsb = transb[i] == EMU_OP_N ? 1 : ldb[i];
    for (int side = 0; side < 2; ++side) {
      ExpSeg e{};
      e.X = side ? B[i] : A[i];
      e.rows = side ? n[i] : m[i];
      e.k = k[i];
      e.rs = side ? rsb : rsa;
      e.hs = side ? hsb : hsa;
      e.xout = side ? y : x;
      char* sp = M + (side ? f.scr_b : f.scr_a);
      const int64_t rr = round_up(e.rows, 64);
      e.emax = reinterpret_cast<int*>(sp);
      e.flag = reinterpret_cast<unsigned int*>(sp + 4 * rr);
      e.sum = reinterpret_cast<unsigned long long*>(sp + 8 * rr);
      e.block_begin = eb;
      eb += exp_seg_blocks(e);
      es.push_back(e);
      rowb.push_back(rows);
      rows += e.rows;
      SplitSeg s{};
      s.X = e.X;
      s.rows = e.rows;
      s.k = k[i];
      s.rs = e.rs;
      s.hs = e.hs;
      s.xexp = e.xout;
      s.planes = M + (side ? f.pb : f.pa);
      s.kpad = f.kpad;
      s.conj = (side ? transb[i] : transa[i]) == EMU_OP_C;
      s.block_begin = sb;
      sb += split_seg_blocks(s);
      ss.push_back(s);
    }
    CrtProb c{};
    c.res = reinterpret_cast<int8_t*>(M + f.res);
    c.ldr = f.ldr;
    c.m = m[i];
    c.n = n[i];
    c.ldc = ldc[i];
    c.x = x;
    c.y = y;
    c.C = C[i];
    c.ar = alpha[2 * i];
    c.ai = alpha[2 * i + 1];
    c.br = beta[2 * i];
    c.bi = beta[2 * i + 1];
    CrtProb t = c;
    c.block_begin = cb;
    cb += crt_prob_blocks(c);
    cp.push_back(c);
    t.block_begin = ct;
    ct += crt_tc_prob_items(t);
    cpt.push_back(t);
    g->probs.push_back({m[i], n[i], f.kpad, f.ldr, M + f.pa, M + f.pb, reinterpret_cast<int8_t*>(M + f.res)});
  }
  rowb.push_back(rows);
  g->d_exp = reinterpret_cast<ExpSeg*>(M + off_exp);
  g->d_rowbeg = reinterpret_cast<long long*>(M + off_rowb);
  g->d_split = reinterpret_cast<SplitSeg*>(M + off_split);
  g->d_gp = M + off_gp;
  g->d_crt = reinterpret_cast<CrtProb*>(M + off_crt);
  g->d_crt_tc = reinterpret_cast<CrtProb*>(M + off_crt_tc);
  g->crt_tc_items = ct;
  g->crt_engine = emu_get_tuning(EMU_TUNE_CRT_ENGINE) == 1 ? 1 : 0;
  g->nexp = g->nsplit = static_cast<int>(es.size());
  g->ngp = g->ncrt = static_cast<int>(cp.size());
  g->exp_blocks = eb;
  g->split_blocks = sb;
  g->crt_blocks = cb;
  g->total_rows = rows;
  bool ok = true;
  {
    // segment of every block of the exponent and split launches
    std::vector<int> maps(static_cast<size_t>(eb + sb) + 1, 0);
    for (size_t q = 0; q < es.size(); ++q) {
      const long long b1 = q + 1 < es.size() ? es[q + 1].block_begin : eb;
      for (long long b = es[q].block_begin; b < b1; ++b) maps[b] = static_cast<int>(q);
    }
    for (size_t q = 0; q < ss.size(); ++q) {
      const long long b1 = q + 1 < ss.size() ? ss[q + 1].block_begin : sb;
      for (long long b = ss[q].block_begin; b < b1; ++b) maps[eb + b] = static_cast<int>(q);
    }
    if (cudaMalloc(&g->maps, sizeof(int) * maps.size()) == cudaSuccess) {
      ok &= cudaMemcpy(g->maps, maps.data(), sizeof(int) * maps.size(), cudaMemcpyHostToDevice) == cudaSuccess;
      g->d_emap = g->maps;
      g->d_smap = g->maps + eb;
    } else {
      g->maps = nullptr;
      cudaGetLastError();
      ok = false;
    }
  }
  if (!es.empty()) {
    ok &= cudaMemcpy(g->d_exp, es.data(), sizeof(ExpSeg) * es.size(), cudaMemcpyHostToDevice) == cudaSuccess;
    ok &= cudaMemcpy(g->d_rowbeg, rowb.data(), sizeof(long long) * rowb.size(), cudaMemcpyHostToDevice) == cudaSuccess;
    ok &= cudaMemcpy(g->d_split, ss.data(), sizeof(SplitSeg) * ss.size(), cudaMemcpyHostToDevice) == cudaSuccess;
    ok &= cudaMemcpy(g->d_crt, cp.data(), sizeof(CrtProb) * cp.size(), cudaMemcpyHostToDevice) == cudaSuccess;
    ok &= cudaMemcpy(g->d_crt_tc, cpt.data(), sizeof(CrtProb) * cpt.size(), cudaMemcpyHostToDevice) == cudaSuccess;
  }
  cudaStream_t st = nullptr;
  ok &= cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
  ok &= prepare_gemm_f16() == cudaSuccess;
  if (g->crt_engine == 1)
    ok &= launch_crt_tc_grouped(g->single, nullptr, 0, 0, *g->pl, nullptr, nullptr, true) == cudaSuccess;
  if (ok && !cp.empty()) {
    int tn = tile_n;
    if (tn == 0) {
      const std::string sig = signature(g->single, g->N, g->probs, k);
      std::lock_guard<std::mutex> lk(g_tune_mu);
      load_cache();
      auto it = g_tune.find(sig);
      if (it != g_tune.end()) {
        tn = it->second;
      } else {
        tn = autotune(g, st);
        g_tune[sig] = tn;
        save_cache();
      }
    }
    g->tile_n = tn;
    ok &= upload_gemm_descs(g, tn, g->d_gp, &g->total_units) == EMU_OK;
  }
  // capture the four phases once; emu_grouped_run replays them
  if (ok) {
    ok &= cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      const uint64_t before = emu_kernel_launches();
      const bool enq = cp.empty() || enqueue(g, st, true) == cudaSuccess;
      g->kernels = static_cast<int>(emu_kernel_launches() - before);
      const bool end = cudaStreamEndCapture(st, &g->graph) == cudaSuccess;
      ok = enq && end;
    }
    if (ok) ok &= cudaGraphInstantiate(&g->exec, g->graph, 0) == cudaSuccess;
  }
  if (st) cudaStreamDestroy(st);
  if (!ok) {
    cudaGetLastError();
    emu_grouped_destroy(g);
    return EMU_ERR_CUDA;
  }
  *out = g;
  return EMU_OK;
}

emu_status_t emu_grouped_run(emu_grouped_t g, void* stream) {
  if (!g || !g->exec) return EMU_ERR_INVALID_ARG;
  return cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream)) == cudaSuccess ? EMU_OK : EMU_ERR_CUDA;
}

int emu_grouped_tile(emu_grouped_t g) { return g ? g->tile_n : 0; }

emu_status_t emu_grouped_phase_times(emu_grouped_t g, float* ms, void* stream) {
  using namespace emu;
  if (!g || !ms) return EMU_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t ev[5];
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) return EMU_ERR_CUDA;
  bool ok = cudaEventRecord(ev[0], st) == cudaSuccess;
  ok = ok && cudaMemsetAsync(g->mem + g->scratch_off, 0, g->scratch_bytes, st) == cudaSuccess;
  ok = ok && launch_exponents_grouped(g->single, g->d_exp, g->d_emap, g->nexp, g->exp_blocks, g->d_rowbeg,
                                      g->total_rows, *g->pl, st) == cudaSuccess;
  ok = ok && cudaEventRecord(ev[1], st) == cudaSuccess;
  ok = ok && launch_split_grouped(g->single, true, g->d_split, g->d_smap, g->nsplit, g->split_blocks, *g->pl,
                                  st) == cudaSuccess;
  ok = ok && cudaEventRecord(ev[2], st) == cudaSuccess;
  ok = ok && launch_gemm_f16_grouped(g->d_gp, g->ngp, g->total_units, *g->pl, g->status, st) ==
                 cudaSuccess;
  ok = ok && cudaEventRecord(ev[3], st) == cudaSuccess;
  ok = ok && crt_phase(g, st) == cudaSuccess;
  ok = ok && cudaEventRecord(ev[4], st) == cudaSuccess;
  ok = ok && cudaEventSynchronize(ev[4]) == cudaSuccess;
  for (int i = 0; ok && i < 4; ++i) ok = cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]) == cudaSuccess;
  for (auto& e : ev) cudaEventDestroy(e);
  return ok ? EMU_OK : EMU_ERR_CUDA;
}

int emu_grouped_kernels(emu_grouped_t g) { return g ? g->kernels : 0; }

emu_status_t emu_grouped_destroy(emu_grouped_t g) {
  if (!g) return EMU_OK;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  if (g->mem) cudaFree(g->mem);   // waits for work that still uses it
  if (g->maps) cudaFree(g->maps);
  delete g;
  return EMU_OK;
}

static emu_status_t grouped_once(int single, int count, const emu_op_t* ta, const emu_op_t* tb, const int64_t* m,
                                 const int64_t* n, const int64_t* k, const double* alpha, const void* const* A,
                                 const int64_t* lda, const void* const* B, const int64_t* ldb, const double* beta,
                                 void* const* C, const int64_t* ldc, int num_moduli, void* stream) {
  emu_grouped_t g = nullptr;
  emu_status_t s = emu_grouped_create(single, count, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc,
                                      num_moduli, 0, &g);
  if (s != EMU_OK) return s;
  s = emu_grouped_run(g, stream);
  if (s == EMU_OK && cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) s = EMU_ERR_CUDA;
  emu_grouped_destroy(g);
  return s;
}

emu_status_t emu_zgemm_grouped(int count, const emu_op_t* transa, const emu_op_t* transb, const int64_t* m,
                               const int64_t* n, const int64_t* k, const double* alpha, const void* const* A,
                               const int64_t* lda, const void* const* B, const int64_t* ldb, const double* beta,
                               void* const* C, const int64_t* ldc, int num_moduli, void* stream) {
  return grouped_once(0, count, transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, num_moduli, stream);
}

emu_status_t emu_cgemm_grouped(int count, const emu_op_t* transa, const emu_op_t* transb, const int64_t* m,
                               const int64_t* n, const int64_t* k, const double* alpha, const void* const* A,
                               const int64_t* lda, const void* const* B, const int64_t* ldb, const double* beta,
                               void* const* C, const int64_t* ldc, int num_moduli, void* stream) {
  return grouped_once(1, count, transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, num_moduli, stream);
}

}  // extern "C"
