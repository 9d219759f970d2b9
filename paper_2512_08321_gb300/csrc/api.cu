// C ABI entry points: argument checks, workspace, the four phases in order.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "emu_internal.h"

namespace emu {

// Device status word: first device-side error recorded (0 = none).
__device__ unsigned int g_device_status;

int g_scaling = EMU_SCALING_FAST;

namespace {

constexpr int kMaxDevices = 64;

thread_local int t_bad_param = 0;

struct DeviceState {
  bool init = false;
  unsigned int* status = nullptr;
  void* own = nullptr;         // library-managed workspace
  size_t own_bytes = 0;
  void* user = nullptr;        // caller workspace (emu_set_workspace)
  size_t user_bytes = 0;
  float* mlp = nullptr;        // moduli-selection weights (emu_mlp_set_weights)
  bool mlp_loaded = false;
  float* feat = nullptr;       // 39 features + chosen N (pinned host mirror below)
  int* chosen_host = nullptr;
  void* stage = nullptr;       // staging of the host-buffer entry points
  size_t stage_bytes = 0;
  void* tol_scr = nullptr;     // exponent sums and features of the tolerance path
  size_t tol_scr_bytes = 0;
  // overlapped column blocks: the library's second stream and its events
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_start = nullptr, ev_done = nullptr, ev_split[2] = {}, ev_gemm[2] = {}, ev_crt[2] = {};
};

cudaError_t aux_stream(DeviceState* ds) {
  if (ds->aux) return cudaSuccess;
  cudaError_t e = cudaStreamCreateWithFlags(&ds->aux, cudaStreamNonBlocking);
  cudaEvent_t* evs[] = {&ds->ev_start, &ds->ev_done, &ds->ev_split[0], &ds->ev_split[1], &ds->ev_gemm[0],
                        &ds->ev_gemm[1], &ds->ev_crt[0], &ds->ev_crt[1]};
  for (cudaEvent_t* ev : evs)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  return e;
}

// Columns per block of an overlapped GEMM: about eight blocks of a multiple of
// 256 (the residue GEMM's tile width), at least 1024.
int64_t overlap_block(int64_t n) {
  const int64_t nb = round_up((n + 7) / 8, 256);
  return nb < 1024 ? 1024 : nb;
}

std::mutex g_mu;
DeviceState g_dev[kMaxDevices];
std::atomic<uint64_t> g_launches{0};
cudaEvent_t g_phase_ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
bool g_phase_on = false;

void phase(int i, cudaStream_t st) {
  if (g_phase_on) cudaEventRecord(g_phase_ev[i], st);
}
emu_engine_t g_engine = EMU_ENGINE_AUTO;

emu_status_t bad(int idx) {
  t_bad_param = idx;
  return EMU_ERR_INVALID_ARG;
}

int current_device() {
  int d = -1;
  if (cudaGetDevice(&d) != cudaSuccess) return -1;
  return d;
}

// Per-device set-up: sm_103 check and the address of the status word.
emu_status_t device_init(int dev, DeviceState*& ds) {
  if (dev < 0 || dev >= kMaxDevices) return EMU_ERR_UNSUPPORTED;
  ds = &g_dev[dev];
  if (ds->init) return EMU_OK;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return EMU_ERR_CUDA;
  if (!(prop.major == 10 && prop.minor == 3)) return EMU_ERR_UNSUPPORTED;
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_device_status) != cudaSuccess) return EMU_ERR_CUDA;
  ds->status = static_cast<unsigned int*>(p);
  ds->init = true;
  return EMU_OK;
}

// Workspace layout of one GEMM whose output columns are processed nb at a time
// (nb == n: one pass).  ppm = residue planes per modulus (3 complex, 1 real).
// bufs = 2: two sets of B planes and residues (column blocks overlapped).
struct Layout {
  int64_t kpad, ldr;
  size_t off_x, off_y, off_scr, off_acc, off_bnd, off_pa, off_pb, off_res, total;
  size_t bnd_bytes;             // accurate mode, complex input: bound-product scratch
  size_t pb_bytes, res_bytes;   // one set
};

size_t al(size_t v) { return (v + 255) / 256 * 256; }

Layout layout(int64_t m, int64_t n, int64_t k, int N, bool fp16, int ppm = 3, int64_t nb = -1, int bufs = 1) {
  if (nb < 0 || nb > n) nb = n;
  Layout L;
  L.kpad = round_up(k > 0 ? k : 1, 64);
  L.ldr = round_up(m, 16);
  const size_t esz = fp16 ? 2 : 1;
  size_t o = 0;
  L.off_x = o;   o += al(static_cast<size_t>(m) * 2);
  L.off_y = o;   o += al(static_cast<size_t>(n) * 2);
  L.off_scr = o; o += al(exponents_scratch_bytes(m > nb ? m : nb));
  L.off_acc = o; o += al(static_cast<size_t>(12) * (m + n));   // accurate mode: e, flag, bound maxima
  L.bnd_bytes = ppm == 3 ? al(bound_scratch_bytes(m, nb)) : 0;
  L.off_bnd = o; o += L.bnd_bytes;
  L.off_pa = o;  o += al(static_cast<size_t>(ppm * N) * m * L.kpad * esz);
  L.pb_bytes = al(static_cast<size_t>(ppm * N) * nb * L.kpad * esz);
  L.res_bytes = al(static_cast<size_t>(ppm * N) * nb * L.ldr);
  L.off_pb = o;  o += bufs * L.pb_bytes;
  L.off_res = o; o += bufs * L.res_bytes;
  L.total = o;
  return L;
}

emu_engine_t resolve(emu_engine_t e) { return e == EMU_ENGINE_AUTO ? EMU_ENGINE_F16 : e; }

emu_status_t get_workspace(DeviceState* ds, size_t need, char** out) {
  if (ds->user) {
    if (ds->user_bytes < need) return EMU_ERR_WORKSPACE;
    *out = static_cast<char*>(ds->user);
    return EMU_OK;
  }
  if (ds->own_bytes < need) {
    if (ds->own) {
      cudaFree(ds->own);   // implicitly waits for work that used it
      ds->own = nullptr;
      ds->own_bytes = 0;
    }
    if (cudaMalloc(&ds->own, need) != cudaSuccess) {
      cudaGetLastError();
      return EMU_ERR_ALLOC;
    }
    ds->own_bytes = need;
  }
  *out = static_cast<char*>(ds->own);
  return EMU_OK;
}

// Strides of op(A) rows (i, h) and of op(B) columns seen as rows (j, h).
void strides_a(emu_op_t ta, int64_t lda, int64_t& rs, int64_t& hs) {
  if (ta == EMU_OP_N) { rs = 1; hs = lda; } else { rs = lda; hs = 1; }
}
void strides_b(emu_op_t tb, int64_t ldb, int64_t& rs, int64_t& hs) {
  if (tb == EMU_OP_N) { rs = ldb; hs = 1; } else { rs = 1; hs = ldb; }
}

bool valid_op(emu_op_t t) { return t == EMU_OP_N || t == EMU_OP_T || t == EMU_OP_C; }

emu_status_t check_common(emu_op_t ta, emu_op_t tb, int64_t m, int64_t n, int64_t k, int64_t lda,
                          int64_t ldb, int64_t ldc, int N, bool need_c) {
  t_bad_param = 0;
  if (!valid_op(ta)) return bad(1);
  if (!valid_op(tb)) return bad(2);
  if (m < 0) return bad(3);
  if (n < 0) return bad(4);
  if (k < 0) return bad(5);
  const int64_t rows_a = ta == EMU_OP_N ? m : k;
  const int64_t rows_b = tb == EMU_OP_N ? k : n;
  if (lda < (rows_a > 1 ? rows_a : 1)) return bad(8);
  if (ldb < (rows_b > 1 ? rows_b : 1)) return bad(10);
  if (need_c && ldc < (m > 1 ? m : 1)) return bad(13);
  if (N < EMU_MIN_MODULI || N > EMU_MAX_MODULI) return EMU_ERR_MODULI_RANGE;
  if (k > EMU_MAX_K) return EMU_ERR_K_TOO_LARGE;
  if (m > (int64_t(1) << 31) || n > (int64_t(1) << 31)) return bad(m > n ? 3 : 4);
  return EMU_OK;
}

emu_status_t cuda_status(cudaError_t e) { return e == cudaSuccess ? EMU_OK : EMU_ERR_CUDA; }


// a_plane_rows / rcap (tcgen05 engine only): pa is a block of rows of planes
// a_plane_rows rows tall, and residues are stored for rows below rcap.
emu_status_t run_residue_gemm(emu_engine_t eng, int64_t m, int64_t n, int64_t kpad, const Plan& pl,
                              const void* pa, const void* pb, int8_t* res, int64_t ldr,
                              DeviceState* ds, cudaStream_t st, const Tune& t, int ppm, int64_t a_plane_rows = 0,
                              int64_t rcap = 0) {
  if (eng == EMU_ENGINE_I8) {
    if (a_plane_rows || rcap) return EMU_ERR_UNSUPPORTED;
    return cuda_status(launch_gemm_i8(m, n, kpad, pl, static_cast<const int8_t*>(pa),
                                      static_cast<const int8_t*>(pb), res, ldr, st, ppm));
  }
  const cudaError_t e = launch_gemm_f16(m, n, kpad, pl, pa, pb, res, ldr, t.chunk_k, ds->status, st, t.tile_n,
                                        t.group, ppm, a_plane_rows, rcap, t.sched);
  if (e == cudaErrorNotSupported) return EMU_ERR_UNSUPPORTED;
  return cuda_status(e);
}

// Element type of a GEMM: complex128 (Z), complex64 (C), float64 (D), float32 (S).
struct Dt {
  bool single, real;
  int ppm() const { return real ? 1 : 3; }
  int code() const { return (real ? 2 : 0) + (single ? 1 : 0); }
};

constexpr size_t kFreeMargin = size_t(256) << 20;   // device memory left to others when blocking

// Output columns per block.  The knob (if set) wins; otherwise `want` columns
// (0: all n) when that workspace fits (the caller's buffer, or the library's
// plus free device memory), else the widest multiple of 128 columns that fits.
int64_t choose_nblock(const DeviceState* ds, int64_t m, int64_t n, int64_t k, int N, bool fp16, int ppm,
                      const Tune& t, int64_t want = 0, int bufs = 1) {
  if (t.nblock > 0) return t.nblock < n ? t.nblock : n;
  if (want <= 0 || want > n) want = n;
  const size_t full = layout(m, n, k, N, fp16, ppm, want, bufs).total;
  size_t limit;
  if (ds->user) {
    limit = ds->user_bytes;
  } else {
    if (full <= ds->own_bytes) return want;
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      cudaGetLastError();
      return want;
    }
    limit = fr + ds->own_bytes;
    limit = limit > kFreeMargin ? limit - kFreeMargin : 0;
  }
  if (full <= limit || want <= 128) return want;
  int64_t lo = 0, hi = (want - 1) / 128;  // widths 128 * [1, hi] are candidates
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) / 2;
    if (layout(m, n, k, N, fp16, ppm, 128 * mid, bufs).total <= limit) lo = mid; else hi = mid - 1;
  }
  return lo > 0 ? 128 * lo : want;         // nothing fits: one block, and the workspace check reports it
}

// hooks (host-buffer calls): the operands move in blocks on another stream and
// each step waits for the blocks it reads (BlockHooks).  presums (fast scaling):
// the exponent sums of op(A)'s rows and op(B)'s columns already formed
// (launch_exponent_sums), so only the N-dependent last step of the exponent
// rule runs here.
emu_status_t gemm(Dt dt, emu_op_t ta, emu_op_t tb, int64_t m, int64_t n, int64_t k, double ar, double ai,
                  const void* A, int64_t lda, const void* B, int64_t ldb, double br, double bi,
                  void* C, int64_t ldc, int N, void* stream, const BlockHooks* hooks = nullptr,
                  void* const* presums = nullptr) {
  emu_status_t s = check_common(ta, tb, m, n, k, lda, ldb, ldc, N, true);
  if (s != EMU_OK) return s;
  if (m == 0 || n == 0) return EMU_OK;
  if (!C) return bad(12);
  if (k > 0 && !A) return bad(7);
  if (k > 0 && !B) return bad(9);
  DeviceState* ds = nullptr;
  s = device_init(current_device(), ds);
  if (s != EMU_OK) return s;
  const Plan* pl = get_plan(N);
  const emu_engine_t eng = resolve(g_engine);
  const bool fp16 = (eng == EMU_ENGINE_F16);
  const int ppm = dt.ppm();
  const Tune tn = tune_for(dt.code(), N, m, n, k);
  char* ws = nullptr;
  int64_t nb;
  Layout L;
  const bool accurate = (g_scaling == EMU_SCALING_ACCURATE);
  const bool presummed = presums && !accurate && k > 0;
  // overlapped column blocks: device-buffer calls on the tcgen05 engine (accurate mode: once the
  // bound products have given every exponent)
  bool overlap = !hooks && (tn.overlap == 1 || (tn.overlap < 0 && dt.real)) && k > 0 && fp16 && n >= 2048;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (overlap) {
      nb = choose_nblock(ds, m, n, k, N, fp16, ppm, tn, overlap_block(n), 2);
      overlap = nb < n && aux_stream(ds) == cudaSuccess;
    }
    if (!overlap) {
      nb = choose_nblock(ds, m, n, k, N, fp16, ppm, tn);
      if (hooks && hooks->nb > 0 && hooks->nb < nb) nb = hooks->nb;
    }
    L = layout(m, n, k, N, fp16, ppm, nb, overlap ? 2 : 1);
    s = get_workspace(ds, L.total, &ws);
  }
  if (s != EMU_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int16_t* x = reinterpret_cast<int16_t*>(ws + L.off_x);
  int16_t* y = reinterpret_cast<int16_t*>(ws + L.off_y);
  void* scr = ws + L.off_scr;
  void* pa = ws + L.off_pa;
  void* pb = ws + L.off_pb;
  int8_t* res = reinterpret_cast<int8_t*>(ws + L.off_res);
  int64_t rsa, hsa, rsb, hsb;
  strides_a(ta, lda, rsa, hsa);
  strides_b(tb, ldb, rsb, hsb);
  // element sizes of B and C, to step to a column block
  const size_t in_esz = (dt.real ? 1 : 2) * (dt.single ? 4 : 8);
  const bool conj_a = !dt.real && ta == EMU_OP_C, conj_b = !dt.real && tb == EMU_OP_C;
  // accurate-mode exponents reach 7 bits further: the split covers them with more chunks
  Plan pls = *pl;
  if (accurate) pls.nchunk = pl->nchunk_accu;
  auto block_ptr = [&](int64_t j0) {
    return k > 0 ? static_cast<const void*>(static_cast<const char*>(B) + static_cast<size_t>(j0) * rsb * in_esz)
                 : B;
  };
  // beside_products: the CRT runs on the library's stream next to residue products, which hold all
  // of an SM's TMEM, so it takes the CUDA-core kernel (the tensor-core one would wait for TMEM)
  auto crt_on = [&](cudaStream_t cs, int64_t mi, int64_t nj, const int8_t* r, const int16_t* xi,
                    const int16_t* yj, void* Ci, bool beside_products) {
    if (g_crt_mode == 1)
      return cuda_status(launch_crt_fp(dt.single, mi, nj, *pl, r, L.ldr, xi, yj, ar, ai, br, bi, Ci, ldc, cs,
                                       dt.real));
    if (tn.crt_engine == 1 && !beside_products)
      return cuda_status(launch_crt_tc(dt.single, mi, nj, *pl, r, L.ldr, xi, yj, ar, ai, br, bi, Ci, ldc, cs,
                                       dt.real, accurate, ds->status));
    return cuda_status(launch_crt(dt.single, mi, nj, *pl, r, L.ldr, xi, yj, ar, ai, br, bi, Ci, ldc, cs,
                                  tn.crt_rows, dt.real, accurate));
  };
  auto crt = [&](int64_t mi, int64_t nj, const int8_t* r, const int16_t* xi, const int16_t* yj, void* Ci) {
    return crt_on(st, mi, nj, r, xi, yj, Ci, false);
  };
  cudaError_t e;
  // Section III-B accurate mode on the caller's stream: pre-scaling, 7-bit ceiling planes, bound
  // products (B's planes column block by column block, in the first set of B planes), exponents
  auto accurate_exponents = [&]() -> emu_status_t {
    int* emA = reinterpret_cast<int*>(ws + L.off_acc);
    unsigned int* fA = reinterpret_cast<unsigned int*>(emA + m);
    unsigned int* MA = fA + m;
    int* emB = reinterpret_cast<int*>(MA + m);
    unsigned int* fB = reinterpret_cast<unsigned int*>(emB + n);
    unsigned int* NB = fB + n;
    if (cudaMemsetAsync(MA, 0, static_cast<size_t>(m) * 4, st) != cudaSuccess ||
        cudaMemsetAsync(NB, 0, static_cast<size_t>(n) * 4, st) != cudaSuccess ||
        launch_exp_max(dt.single, dt.real, A, m, k, rsa, hsa, emA, fA, st) != cudaSuccess ||
        launch_bound_split(dt.single, dt.real, A, m, k, rsa, hsa, emA, fA, L.kpad, pa, st) != cudaSuccess)
      return EMU_ERR_CUDA;
    for (int64_t j0 = 0; j0 < n; j0 += nb) {
      const int64_t nj = (n - j0) < nb ? (n - j0) : nb;
      const void* Bj = block_ptr(j0);
      emu_status_t r;
      if (hooks && (r = hooks->wait_inputs(hooks->ctx, j0, nj, st)) != EMU_OK) return r;
      if (launch_exp_max(dt.single, dt.real, Bj, nj, k, rsb, hsb, emB + j0, fB + j0, st) != cudaSuccess ||
          launch_bound_split(dt.single, dt.real, Bj, nj, k, rsb, hsb, emB + j0, fB + j0, L.kpad, pb, st) !=
              cudaSuccess)
        return EMU_ERR_CUDA;
      const cudaError_t be = launch_gemm_bound(m, nj, L.kpad, dt.real, pa, pb, MA, NB + j0, ws + L.off_bnd,
                                               L.bnd_bytes, ds->status, st, tn.bound_pair == 1);
      if (be == cudaErrorNotSupported) return EMU_ERR_UNSUPPORTED;
      if (be != cudaSuccess) return EMU_ERR_CUDA;
    }
    if (launch_accu_finalize(m, emA, fA, MA, *pl, x, st) != cudaSuccess ||
        launch_accu_finalize(n, emB, fB, NB, *pl, y, st) != cudaSuccess)
      return EMU_ERR_CUDA;
    return EMU_OK;
  };
  phase(0, st);
  if (overlap) {
    // Column block b's residue products on the caller's stream; beside them,
    // on the library's stream, block b+1's exponents and planes (into the
    // other set of B planes, free once block b-1's products are done) and
    // block b-1's CRT (from the other set of residues, which block b+1's
    // products then overwrite).  Phase events: 1 and 2 when A's and the first
    // block's planes are ready, 3 after the last products, 4 at the end.
    cudaStream_t ax = ds->aux;
    const int64_t nblk = (n + nb - 1) / nb;
    auto pbuf = [&](int64_t b) { return static_cast<char*>(pb) + (b & 1) * L.pb_bytes; };
    auto rbuf = [&](int64_t b) { return res + (b & 1) * L.res_bytes; };
    auto width = [&](int64_t b) { return (n - b * nb) < nb ? (n - b * nb) : nb; };
    const bool have_xy = presummed || accurate;     // every exponent known before the pipeline starts
    auto prepare = [&](int64_t b) -> cudaError_t {   // exponents and planes of block b's columns of B
      const int64_t j0 = b * nb, nj = width(b);
      cudaError_t err = have_xy ? cudaSuccess
                                  : launch_exponents(dt.single, block_ptr(j0), nj, k, rsb, hsb, *pl, y + j0, scr, ax,
                                                     dt.real);
      if (err == cudaSuccess)
        err = launch_split(dt.single, conj_b, block_ptr(j0), nj, k, rsb, hsb, pls, y + j0, fp16, L.kpad, pbuf(b), ax,
                           tn.split_elems, dt.real);
      if (err == cudaSuccess) err = cudaEventRecord(ds->ev_split[b & 1], ax);
      return err;
    };
    auto finish_block = [&](int64_t b) -> emu_status_t {   // CRT of block b, once its products are done
      if (cudaStreamWaitEvent(ax, ds->ev_gemm[b & 1], 0) != cudaSuccess) return EMU_ERR_CUDA;
      const int64_t j0 = b * nb;
      void* Cj = static_cast<char*>(C) + static_cast<size_t>(j0) * ldc * in_esz;
      const emu_status_t r = crt_on(ax, m, width(b), rbuf(b), x, y + j0, Cj, true);
      if (r != EMU_OK) return r;
      return cuda_status(cudaEventRecord(ds->ev_crt[b & 1], ax));
    };
    if (accurate && (s = accurate_exponents()) != EMU_OK) return s;
    if ((presummed && (launch_exponent_finalize(m, presums[0], *pl, x, st) != cudaSuccess ||
                       launch_exponent_finalize(n, presums[1], *pl, y, st) != cudaSuccess)) ||
        cudaEventRecord(ds->ev_start, st) != cudaSuccess || cudaStreamWaitEvent(ax, ds->ev_start, 0) != cudaSuccess ||
        (!have_xy && launch_exponents(dt.single, A, m, k, rsa, hsa, *pl, x, scr, ax, dt.real) != cudaSuccess) ||
        launch_split(dt.single, conj_a, A, m, k, rsa, hsa, pls, x, fp16, L.kpad, pa, ax, tn.split_elems, dt.real) !=
            cudaSuccess ||
        prepare(0) != cudaSuccess)
      return EMU_ERR_CUDA;
    for (int64_t b = 0; b < nblk; ++b) {
      if (cudaStreamWaitEvent(st, ds->ev_split[b & 1], 0) != cudaSuccess ||
          (b >= 2 && cudaStreamWaitEvent(st, ds->ev_crt[b & 1], 0) != cudaSuccess))
        return EMU_ERR_CUDA;
      if (b == 0) {
        phase(1, st);
        phase(2, st);
      }
      if ((s = run_residue_gemm(eng, m, width(b), L.kpad, *pl, pa, pbuf(b), rbuf(b), L.ldr, ds, st, tn, ppm)) !=
          EMU_OK)
        return s;
      if (cudaEventRecord(ds->ev_gemm[b & 1], st) != cudaSuccess) return EMU_ERR_CUDA;
      if (b + 1 < nblk) {
        if ((b >= 1 && cudaStreamWaitEvent(ax, ds->ev_gemm[(b + 1) & 1], 0) != cudaSuccess) ||
            prepare(b + 1) != cudaSuccess)
          return EMU_ERR_CUDA;
      }
      if (b >= 1 && (s = finish_block(b - 1)) != EMU_OK) return s;
    }
    phase(3, st);
    if ((s = finish_block(nblk - 1)) != EMU_OK) return s;
    if (cudaEventRecord(ds->ev_done, ax) != cudaSuccess || cudaStreamWaitEvent(st, ds->ev_done, 0) != cudaSuccess)
      return EMU_ERR_CUDA;
    phase(4, st);
    return EMU_OK;
  }
  // rows_piped: the first column block row block by row block as A arrives
  const bool rows_piped = hooks && hooks->mb > 0 && hooks->mb % 16 == 0 && k > 0 && !accurate && fp16;
  if (hooks && !rows_piped && (s = hooks->wait_rows(hooks->ctx, 0, m, st)) != EMU_OK) return s;
  const bool a_first = hooks && !rows_piped;
  if (k == 0) {
    // empty inner dimension: the product is zero
    if ((e = cudaMemsetAsync(x, 0, static_cast<size_t>(m) * 2, st)) != cudaSuccess) return EMU_ERR_CUDA;
    if ((e = cudaMemsetAsync(y, 0, static_cast<size_t>(n) * 2, st)) != cudaSuccess) return EMU_ERR_CUDA;
  } else if (accurate) {
    if ((s = accurate_exponents()) != EMU_OK) return s;
  } else if (presummed) {
    if (launch_exponent_finalize(m, presums[0], *pl, x, st) != cudaSuccess ||
        launch_exponent_finalize(n, presums[1], *pl, y, st) != cudaSuccess)
      return EMU_ERR_CUDA;
  } else if (!rows_piped) {
    if ((e = launch_exponents(dt.single, A, m, k, rsa, hsa, *pl, x, scr, st, dt.real)) != cudaSuccess)
      return EMU_ERR_CUDA;
    // A's planes while B is in flight
    if (a_first && (e = launch_split(dt.single, conj_a, A, m, k, rsa, hsa, pls, x, fp16, L.kpad, pa, st,
                                     tn.split_elems, dt.real)) != cudaSuccess)
      return EMU_ERR_CUDA;
  }
  for (int64_t j0 = 0, nj = 0; j0 < n; j0 += nj) {
    const int64_t w = (hooks && j0 == 0 && hooks->nb0 > 0 && hooks->nb0 < nb) ? hooks->nb0 : nb;
    nj = (n - j0) < w ? (n - j0) : w;
    const void* Bj = block_ptr(j0);
    void* Cbase = (hooks && hooks->c_dev && j0 < hooks->c_dev_end) ? hooks->c_dev : C;
    void* Cj = static_cast<char*>(Cbase) + static_cast<size_t>(j0) * ldc * in_esz;
    int16_t* yj = y + j0;
    if (hooks && (s = hooks->wait_inputs(hooks->ctx, j0, nj, st)) != EMU_OK) return s;
    if (k == 0) {
      if ((e = cudaMemsetAsync(res, 0, static_cast<size_t>(ppm * N) * nj * L.ldr, st)) != cudaSuccess)
        return EMU_ERR_CUDA;
    } else {
      if (!accurate && !presummed &&
          (e = launch_exponents(dt.single, Bj, nj, k, rsb, hsb, *pl, yj, scr, st, dt.real)) != cudaSuccess)
        return EMU_ERR_CUDA;
      phase(1, st);
      if (rows_piped && j0 == 0) {
        // B's planes, then per block of rows of op(A): exponents, planes, residue products, CRT
        if (launch_split(dt.single, conj_b, Bj, nj, k, rsb, hsb, pls, yj, fp16, L.kpad, pb, st, tn.split_elems,
                         dt.real) != cudaSuccess)
          return EMU_ERR_CUDA;
        for (int64_t i0 = 0; i0 < m; i0 += hooks->mb) {
          const int64_t mi = (m - i0) < hooks->mb ? (m - i0) : hooks->mb;
          const void* Ai = static_cast<const char*>(A) + static_cast<size_t>(i0) * rsa * in_esz;
          void* pai = static_cast<char*>(pa) + static_cast<size_t>(i0) * L.kpad * 2;
          if ((s = hooks->wait_rows(hooks->ctx, i0, mi, st)) != EMU_OK) return s;
          if (launch_exponents(dt.single, Ai, mi, k, rsa, hsa, *pl, x + i0, scr, st, dt.real) != cudaSuccess ||
              launch_split(dt.single, conj_a, Ai, mi, k, rsa, hsa, pls, x + i0, fp16, L.kpad, pai, st,
                           tn.split_elems, dt.real, m) != cudaSuccess)
            return EMU_ERR_CUDA;
          const int64_t rcap = (L.ldr - i0) < round_up(mi, 16) ? (L.ldr - i0) : round_up(mi, 16);
          if ((s = hooks->products_start(hooks->ctx, st)) != EMU_OK ||
              (s = run_residue_gemm(eng, mi, nj, L.kpad, *pl, pai, pb, res + i0, L.ldr, ds, st, tn, ppm, m, rcap)) !=
                  EMU_OK ||
              (s = crt(mi, nj, res + i0, x + i0, yj, static_cast<char*>(Cj) + static_cast<size_t>(i0) * in_esz)) !=
                  EMU_OK)
            return s;
        }
        if ((s = hooks->output_done(hooks->ctx, j0, nj, st)) != EMU_OK) return s;
        continue;
      }
      if (j0 == 0 && !(a_first && !accurate) &&
          (e = launch_split(dt.single, conj_a, A, m, k, rsa, hsa, pls, x, fp16, L.kpad, pa, st, tn.split_elems,
                            dt.real)) != cudaSuccess)
        return EMU_ERR_CUDA;
      if ((e = launch_split(dt.single, conj_b, Bj, nj, k, rsb, hsb, pls, yj, fp16, L.kpad, pb, st, tn.split_elems,
                            dt.real)) != cudaSuccess)
        return EMU_ERR_CUDA;
      phase(2, st);
      if (hooks && (s = hooks->products_start(hooks->ctx, st)) != EMU_OK) return s;
      s = run_residue_gemm(eng, m, nj, L.kpad, *pl, pa, pb, res, L.ldr, ds, st, tn, ppm);
      if (s != EMU_OK) return s;
      phase(3, st);
    }
    if ((s = crt(m, nj, res, x, yj, Cj)) != EMU_OK) return s;
    if (hooks && (s = hooks->output_done(hooks->ctx, j0, nj, st)) != EMU_OK) return s;
  }
  phase(4, st);
  return EMU_OK;
}

}  // namespace

emu_status_t run_gemm(bool single, bool real, emu_op_t ta, emu_op_t tb, int64_t m, int64_t n, int64_t k, double ar,
                      double ai, const void* A, int64_t lda, const void* B, int64_t ldb, double br, double bi, void* C,
                      int64_t ldc, int N, void* stream, const BlockHooks* hooks) {
  return gemm(Dt{single != 0, real != 0}, ta, tb, m, n, k, ar, ai, A, lda, B, ldb, br, bi, C, ldc, N, stream, hooks);
}

emu_status_t check_gemm_args(emu_op_t ta, emu_op_t tb, int64_t m, int64_t n, int64_t k, int64_t lda, int64_t ldb,
                             int64_t ldc, int N) {
  return check_common(ta, tb, m, n, k, lda, ldb, ldc, N, true);
}

emu_status_t set_bad_param(int idx) { return bad(idx); }

emu_status_t check_stage_args(emu_op_t ta, emu_op_t tb, int64_t m, int64_t n, int64_t k, int64_t lda, int64_t ldb,
                              int N) {
  return check_common(ta, tb, m, n, k, lda, ldb, 1, N, false);
}

// Per-device staging buffer of the host-buffer entry points (grown on demand).
emu_status_t get_staging(size_t need, char** out) {
  DeviceState* ds = nullptr;
  emu_status_t s = device_init(current_device(), ds);
  if (s != EMU_OK) return s;
  std::lock_guard<std::mutex> lk(g_mu);
  if (ds->stage_bytes < need) {
    if (ds->stage) {
      cudaFree(ds->stage);
      ds->stage = nullptr;
      ds->stage_bytes = 0;
    }
    if (cudaMalloc(&ds->stage, need) != cudaSuccess) {
      cudaGetLastError();
      return EMU_ERR_ALLOC;
    }
    ds->stage_bytes = need;
  }
  *out = static_cast<char*>(ds->stage);
  return EMU_OK;
}

void count_launches(int n) { g_launches.fetch_add(static_cast<uint64_t>(n), std::memory_order_relaxed); }

unsigned int* device_status_ptr() {
  DeviceState* ds = nullptr;
  if (device_init(current_device(), ds) != EMU_OK) return nullptr;
  return ds->status;
}

__global__ void bounded_wait_kernel(const volatile unsigned int* flag, long long limit,
                                    unsigned int* status) {
  const long long t0 = clock64();
  while (*flag == 0u) {
    if (clock64() - t0 > limit) {
      atomicCAS(status, 0u, static_cast<unsigned int>(EMU_ERR_TIMEOUT));
      return;
    }
    __nanosleep(1000);
  }
}

// A flag no code ever sets: the self-test's wait on it can only expire.
__device__ unsigned int g_never_set = 0u;

cudaError_t launch_bounded_wait_selftest(int64_t limit_cycles, unsigned int* status, cudaStream_t st) {
  void* f = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&f, g_never_set);
  if (e != cudaSuccess) return e;
  bounded_wait_kernel<<<1, 1, 0, st>>>(static_cast<const unsigned int*>(f), limit_cycles, status);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace emu

extern "C" {

emu_status_t emu_zgemm(emu_op_t transa, emu_op_t transb, int64_t m, int64_t n, int64_t k,
                       const double* alpha, const void* A, int64_t lda, const void* B, int64_t ldb,
                       const double* beta, void* C, int64_t ldc, int num_moduli, void* stream) {
  if (!alpha) return emu::bad(6);
  if (!beta) return emu::bad(11);
  return emu::gemm(emu::Dt{false, false}, transa, transb, m, n, k, alpha[0], alpha[1], A, lda, B, ldb, beta[0],
                          beta[1], C, ldc, num_moduli, stream);
}

emu_status_t emu_cgemm(emu_op_t transa, emu_op_t transb, int64_t m, int64_t n, int64_t k,
                       const float* alpha, const void* A, int64_t lda, const void* B, int64_t ldb,
                       const float* beta, void* C, int64_t ldc, int num_moduli, void* stream) {
  if (!alpha) return emu::bad(6);
  if (!beta) return emu::bad(11);
  return emu::gemm(emu::Dt{true, false}, transa, transb, m, n, k, alpha[0], alpha[1], A, lda, B, ldb, beta[0],
                   beta[1], C, ldc, num_moduli, stream);
}

emu_status_t emu_dgemm(emu_op_t transa, emu_op_t transb, int64_t m, int64_t n, int64_t k, const double* alpha,
                       const double* A, int64_t lda, const double* B, int64_t ldb, const double* beta, double* C,
                       int64_t ldc, int num_moduli, void* stream) {
  if (!alpha) return emu::bad(6);
  if (!beta) return emu::bad(11);
  return emu::gemm(emu::Dt{false, true}, transa, transb, m, n, k, *alpha, 0.0, A, lda, B, ldb, *beta, 0.0, C, ldc,
                   num_moduli, stream);
}

emu_status_t emu_sgemm(emu_op_t transa, emu_op_t transb, int64_t m, int64_t n, int64_t k, const float* alpha,
                       const float* A, int64_t lda, const float* B, int64_t ldb, const float* beta, float* C,
                       int64_t ldc, int num_moduli, void* stream) {
  if (!alpha) return emu::bad(6);
  if (!beta) return emu::bad(11);
  return emu::gemm(emu::Dt{true, true}, transa, transb, m, n, k, *alpha, 0.0, A, lda, B, ldb, *beta, 0.0, C, ldc,
                   num_moduli, stream);
}

size_t emu_workspace_bytes(int dtype, int64_t m, int64_t n, int64_t k, int num_moduli) {
  if (m < 0 || n < 0 || k < 0 || num_moduli < EMU_MIN_MODULI || num_moduli > EMU_MAX_MODULI) return 0;
  if (dtype < EMU_DTYPE_Z || dtype > EMU_DTYPE_S) return 0;
  const int ppm = dtype >= EMU_DTYPE_D ? 1 : 3;
  return emu::layout(m, n, k, num_moduli, emu::resolve(emu::g_engine) == EMU_ENGINE_F16, ppm).total;
}

emu_status_t emu_set_workspace(void* ptr, size_t bytes) {
  emu::DeviceState* ds = nullptr;
  const int dev = emu::current_device();
  if (dev < 0 || dev >= emu::kMaxDevices) return EMU_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(emu::g_mu);
  ds = &emu::g_dev[dev];
  ds->user = bytes ? ptr : nullptr;
  ds->user_bytes = ptr ? bytes : 0;
  return EMU_OK;
}

emu_status_t emu_set_engine(emu_engine_t engine, int chunk_k) {
  if (engine != EMU_ENGINE_AUTO && engine != EMU_ENGINE_F16 && engine != EMU_ENGINE_I8) return emu::bad(1);
  if (chunk_k != 0 && (chunk_k < 64 || chunk_k > 960 || chunk_k % 64)) return emu::bad(2);
  emu::g_engine = engine;
  if (chunk_k) emu::set_default_tuning(EMU_TUNE_CHUNK_K, chunk_k);
  return EMU_OK;
}

emu_status_t emu_stage_exponents(int is_single, emu_op_t transa, emu_op_t transb, int64_t m,
                                 int64_t n, int64_t k, const void* A, int64_t lda, const void* B,
                                 int64_t ldb, int num_moduli, int16_t* x, int16_t* y, void* stream) {
  emu_status_t s = emu::check_common(transa, transb, m, n, k, lda, ldb, 1, num_moduli, false);
  if (s != EMU_OK) return s;
  emu::DeviceState* ds = nullptr;
  s = emu::device_init(emu::current_device(), ds);
  if (s != EMU_OK) return s;
  const emu::Plan* pl = emu::get_plan(num_moduli);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  void* scr = nullptr;
  const size_t sb = emu::exponents_scratch_bytes(m > n ? m : n);
  if (cudaMallocAsync(&scr, sb, st) != cudaSuccess) return EMU_ERR_ALLOC;
  int64_t rs, hs;
  cudaError_t e = cudaSuccess;
  emu::strides_a(transa, lda, rs, hs);
  if (m > 0) e = emu::launch_exponents(is_single != 0, A, m, k, rs, hs, *pl, x, scr, st);
  emu::strides_b(transb, ldb, rs, hs);
  if (e == cudaSuccess && n > 0) e = emu::launch_exponents(is_single != 0, B, n, k, rs, hs, *pl, y, scr, st);
  cudaFreeAsync(scr, st);
  return emu::cuda_status(e);
}

emu_status_t emu_stage_split(int is_single, emu_op_t transa, emu_op_t transb, int64_t m, int64_t n,
                             int64_t k, const void* A, int64_t lda, const void* B, int64_t ldb,
                             int num_moduli, const int16_t* x, const int16_t* y, int plane_fp16,
                             int64_t kpad, void* planesA, void* planesB, void* stream) {
  emu_status_t s = emu::check_common(transa, transb, m, n, k, lda, ldb, 1, num_moduli, false);
  if (s != EMU_OK) return s;
  if (kpad < k || kpad % 64) return emu::bad(15);
  emu::DeviceState* ds = nullptr;
  s = emu::device_init(emu::current_device(), ds);
  if (s != EMU_OK) return s;
  const emu::Plan* pl = emu::get_plan(num_moduli);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int64_t rs, hs;
  cudaError_t e = cudaSuccess;
  emu::strides_a(transa, lda, rs, hs);
  e = emu::launch_split(is_single != 0, transa == EMU_OP_C, A, m, k, rs, hs, *pl, x, plane_fp16 != 0,
                        kpad, planesA, st);
  emu::strides_b(transb, ldb, rs, hs);
  if (e == cudaSuccess)
    e = emu::launch_split(is_single != 0, transb == EMU_OP_C, B, n, k, rs, hs, *pl, y, plane_fp16 != 0,
                          kpad, planesB, st);
  return emu::cuda_status(e);
}

emu_status_t emu_stage_residue_gemm(emu_engine_t engine, int64_t m, int64_t n, int64_t kpad,
                                    int num_moduli, const void* planesA, const void* planesB,
                                    int8_t* residues, int64_t ldr, void* stream) {
  emu::t_bad_param = 0;
  if (engine != EMU_ENGINE_AUTO && engine != EMU_ENGINE_F16 && engine != EMU_ENGINE_I8) return emu::bad(1);
  if (m < 0) return emu::bad(2);
  if (n < 0) return emu::bad(3);
  if (kpad < 0 || kpad % 64) return emu::bad(4);
  if (num_moduli < EMU_MIN_MODULI || num_moduli > EMU_MAX_MODULI) return EMU_ERR_MODULI_RANGE;
  if (ldr < m || ldr % 16) return emu::bad(9);
  emu::DeviceState* ds = nullptr;
  emu_status_t s = emu::device_init(emu::current_device(), ds);
  if (s != EMU_OK) return s;
  const emu::Plan* pl = emu::get_plan(num_moduli);
  return emu::run_residue_gemm(emu::resolve(engine), m, n, kpad, *pl, planesA, planesB, residues, ldr, ds,
                               static_cast<cudaStream_t>(stream), emu::tune_for(0, num_moduli, m, n, kpad), 3);
}

emu_status_t emu_stage_crt(int is_single, int64_t m, int64_t n, int num_moduli, const int8_t* residues,
                           int64_t ldr, const int16_t* x, const int16_t* y, const void* alpha,
                           const void* beta, void* C, int64_t ldc, void* stream) {
  emu::t_bad_param = 0;
  if (m < 0) return emu::bad(2);
  if (n < 0) return emu::bad(3);
  if (num_moduli < EMU_MIN_MODULI || num_moduli > EMU_MAX_MODULI) return EMU_ERR_MODULI_RANGE;
  if (ldr < m || ldr % 16) return emu::bad(6);
  if (!alpha) return emu::bad(9);
  if (!beta) return emu::bad(10);
  if (ldc < (m > 1 ? m : 1)) return emu::bad(12);
  emu::DeviceState* ds = nullptr;
  emu_status_t s = emu::device_init(emu::current_device(), ds);
  if (s != EMU_OK) return s;
  const emu::Plan* pl = emu::get_plan(num_moduli);
  double ar, ai, br, bi;
  if (is_single) {
    const float* a = static_cast<const float*>(alpha);
    const float* b = static_cast<const float*>(beta);
    ar = a[0]; ai = a[1]; br = b[0]; bi = b[1];
  } else {
    const double* a = static_cast<const double*>(alpha);
    const double* b = static_cast<const double*>(beta);
    ar = a[0]; ai = a[1]; br = b[0]; bi = b[1];
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (emu::g_crt_mode == 1)
    return emu::cuda_status(emu::launch_crt_fp(is_single != 0, m, n, *pl, residues, ldr, x, y, ar, ai, br, bi, C,
                                               ldc, st));
  if (emu_get_tuning(EMU_TUNE_CRT_ENGINE) == 1)
    return emu::cuda_status(emu::launch_crt_tc(is_single != 0, m, n, *pl, residues, ldr, x, y, ar, ai, br, bi, C,
                                               ldc, st, false, false, ds->status));
  return emu::cuda_status(emu::launch_crt(is_single != 0, m, n, *pl, residues, ldr, x, y, ar, ai, br, bi, C,
                                          ldc, st));
}

emu_status_t emu_set_scaling(int mode) {
  if (mode != EMU_SCALING_FAST && mode != EMU_SCALING_ACCURATE) return emu::bad(1);
  emu::g_scaling = mode;
  return EMU_OK;
}

int emu_get_scaling(void) { return emu::g_scaling; }

emu_status_t emu_set_crt_mode(int mode) {
  if (mode != EMU_CRT_EXACT && mode != EMU_CRT_PAPER_FP64) return emu::bad(1);
  emu::g_crt_mode = mode;
  return EMU_OK;
}

int emu_last_bad_param(void) { return emu::t_bad_param; }

emu_status_t emu_stream_status(void* stream) {
  emu::DeviceState* ds = nullptr;
  emu_status_t s = emu::device_init(emu::current_device(), ds);
  if (s != EMU_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(st) != cudaSuccess) return EMU_ERR_CUDA;
  unsigned int v = 0;
  if (cudaMemcpy(&v, ds->status, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) return EMU_ERR_CUDA;
  if (v) {
    const unsigned int zero = 0;
    if (cudaMemcpy(ds->status, &zero, sizeof(zero), cudaMemcpyHostToDevice) != cudaSuccess)
      return EMU_ERR_CUDA;
  }
  return static_cast<emu_status_t>(v);
}

emu_status_t emu_selftest_bounded_wait(int64_t limit_cycles, void* stream) {
  if (limit_cycles <= 0 || limit_cycles > (int64_t(1) << 36)) return emu::bad(1);
  emu::DeviceState* ds = nullptr;
  emu_status_t s = emu::device_init(emu::current_device(), ds);
  if (s != EMU_OK) return s;
  return emu::cuda_status(
      emu::launch_bounded_wait_selftest(limit_cycles, ds->status, static_cast<cudaStream_t>(stream)));
}

emu_status_t emu_set_phase_events(void* const* events, int count) {
  if (count == 0) {
    emu::g_phase_on = false;
    return EMU_OK;
  }
  if (count != 5 || !events) return emu::bad(2);
  for (int i = 0; i < 5; ++i) {
    if (!events[i]) return emu::bad(1);
    emu::g_phase_ev[i] = static_cast<cudaEvent_t>(events[i]);
  }
  emu::g_phase_on = true;
  return EMU_OK;
}

uint64_t emu_kernel_launches(void) { return emu::g_launches.load(); }

// ------------------------------------------------------- moduli selection
int emu_mlp_param_count(void) { return emu::kMlpParams; }

int emu_moduli_apriori(int is_single, int64_t k, double target) {
  (void)is_single;
  if (!(target > 0.0) || k < 0) return EMU_MAX_MODULI;
  // smallest N with 2^(1 - (P'_fast(N) - 0.5 log2(8k))) <= target,
  // P'_fast = log2(P - 1)/2 - 1.5 (uniform-row Cauchy-Schwarz estimate)
  const double need = 1.0 - std::log2(target);
  const double lk = 0.5 * std::log2(8.0 * static_cast<double>(k > 1 ? k : 1));
  for (int N = EMU_MIN_MODULI; N <= EMU_MAX_MODULI; ++N) {
    const emu::Plan* pl = emu::get_plan(N);
    double log2P = 0.0;
    for (int l = 0; l < pl->N; ++l) log2P += std::log2(static_cast<double>(pl->p[l]));
    const double Pf = log2P / 2.0 - 1.5;
    if (Pf - lk >= need) return N;
  }
  return EMU_MAX_MODULI;
}

emu_status_t emu_mlp_set_weights(const float* params, int count) {
  emu::DeviceState* ds = nullptr;
  emu_status_t s = emu::device_init(emu::current_device(), ds);
  if (s != EMU_OK) return s;
  std::lock_guard<std::mutex> lk(emu::g_mu);
  if (!params) {
    ds->mlp_loaded = false;
    return EMU_OK;
  }
  if (count != emu::kMlpParams) return emu::bad(2);
  if (!ds->mlp && cudaMalloc(&ds->mlp, sizeof(float) * emu::kMlpParams) != cudaSuccess) return EMU_ERR_ALLOC;
  if (cudaMemcpy(ds->mlp, params, sizeof(float) * count, cudaMemcpyHostToDevice) != cudaSuccess) return EMU_ERR_CUDA;
  ds->mlp_loaded = true;
  return EMU_OK;
}

emu_status_t emu_mlp_forward(const float* theta, const float* X, int batch, float* logits, void* stream) {
  if (!theta || !X || !logits || batch < 0) return emu::bad(batch < 0 ? 3 : 1);
  return emu::cuda_status(emu::launch_mlp_forward(theta, X, batch, logits, static_cast<cudaStream_t>(stream)));
}

emu_status_t emu_mlp_backward(const float* theta, const float* X, const float* Y, int batch, float* grad, float* loss,
                              void* stream) {
  if (!theta || !X || !Y || !grad || !loss || batch < 0) return emu::bad(batch < 0 ? 4 : 1);
  return emu::cuda_status(emu::launch_mlp_backward(theta, X, Y, batch, grad, loss, static_cast<cudaStream_t>(stream)));
}

emu_status_t emu_mlp_adam(float* theta, const float* grad, float* m, float* v, int step, float lr, void* stream) {
  if (!theta || !grad || !m || !v || step < 1) return emu::bad(step < 1 ? 5 : 1);
  return emu::cuda_status(emu::launch_mlp_adam(theta, grad, m, v, step, lr, static_cast<cudaStream_t>(stream)));
}

emu_status_t emu_mlp_choose(const float* theta, const float* features, float threshold, int* n_out, void* stream) {
  if (!theta || !features || !n_out) return emu::bad(1);
  return emu::cuda_status(emu::launch_mlp_choose(theta, features, threshold, n_out, static_cast<cudaStream_t>(stream)));
}

emu_status_t emu_moduli_features(int is_single, emu_op_t transa, emu_op_t transb, int64_t m, int64_t n, int64_t k,
                                 const void* A, int64_t lda, const void* B, int64_t ldb, double target, float* features,
                                 void* stream) {
  emu_status_t s = emu::check_common(transa, transb, m, n, k, lda, ldb, 1, EMU_MIN_MODULI, false);
  if (s != EMU_OK) return s;
  if (!(target > 0.0) || !features) return emu::bad(!features ? 12 : 11);
  emu::DeviceState* ds = nullptr;
  s = emu::device_init(emu::current_device(), ds);
  if (s != EMU_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  void* scr = nullptr;
  if (cudaMallocAsync(&scr, emu::features_scratch_bytes(m, n), st) != cudaSuccess) return EMU_ERR_ALLOC;
  int64_t rsa, hsa, rsb, hsb;
  emu::strides_a(transa, lda, rsa, hsa);
  emu::strides_b(transb, ldb, rsb, hsb);
  const cudaError_t e =
      emu::launch_features(is_single != 0, A, m, rsa, hsa, B, n, rsb, hsb, k, target, features, scr, st);
  cudaFreeAsync(scr, st);
  return emu::cuda_status(e);
}

static emu_status_t gemm_tol(int single, emu_op_t ta, emu_op_t tb, int64_t m, int64_t n, int64_t k, double ar,
                             double ai, const void* A, int64_t lda, const void* B, int64_t ldb, double br, double bi,
                             void* C, int64_t ldc, double target, int* n_used, void* stream) {
  emu_status_t s = emu::check_common(ta, tb, m, n, k, lda, ldb, ldc, EMU_MIN_MODULI, true);
  if (s != EMU_OK) return s;
  if (!(target > 0.0)) return emu::bad(14);
  int N = emu_moduli_apriori(single, k, target);
  if (m > 0 && n > 0 && k > 0) {
    emu::DeviceState* ds = nullptr;
    s = emu::device_init(emu::current_device(), ds);
    if (s != EMU_OK) return s;
    if (ds->mlp_loaded) {
      // The features come from the exponent passes the GEMM needs anyway (their
      // row maxima and sums do not depend on N): formed once here, with the
      // histograms, and handed to the GEMM, which adds only the N-dependent step.
      cudaStream_t st = static_cast<cudaStream_t>(stream);
      const size_t need = emu::features_scratch_bytes(m, n);
      {
        std::lock_guard<std::mutex> lk(emu::g_mu);
        if (!ds->feat && cudaMalloc(&ds->feat, 64 * sizeof(float)) != cudaSuccess) return EMU_ERR_ALLOC;
        if (!ds->chosen_host && cudaMallocHost(&ds->chosen_host, sizeof(int)) != cudaSuccess) return EMU_ERR_ALLOC;
        if (ds->tol_scr_bytes < need) {
          if (ds->tol_scr) cudaFree(ds->tol_scr);
          ds->tol_scr = nullptr;
          ds->tol_scr_bytes = 0;
          if (cudaMalloc(&ds->tol_scr, need) != cudaSuccess) {
            cudaGetLastError();
            return EMU_ERR_ALLOC;
          }
          ds->tol_scr_bytes = need;
        }
      }
      int64_t rsa, hsa, rsb, hsb;
      emu::strides_a(ta, lda, rsa, hsa);
      emu::strides_b(tb, ldb, rsb, hsb);
      if (emu::launch_features(single != 0, A, m, rsa, hsa, B, n, rsb, hsb, k, target, ds->feat, ds->tol_scr, st) !=
          cudaSuccess)
        return EMU_ERR_CUDA;
      int* dn = reinterpret_cast<int*>(ds->feat + 48);
      if (emu::launch_mlp_choose(ds->mlp, ds->feat, 0.99f, dn, st) != cudaSuccess) return EMU_ERR_CUDA;
      if (cudaMemcpyAsync(ds->chosen_host, dn, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        return EMU_ERR_CUDA;
      const int Nm = *ds->chosen_host;
      if (Nm >= EMU_MIN_MODULI && Nm <= EMU_MAX_MODULI) N = Nm;   // else: the a priori rule
      if (n_used) *n_used = N;
      void* const presums[2] = {ds->tol_scr, static_cast<char*>(ds->tol_scr) + emu::exponents_scratch_bytes(m)};
      return emu::gemm(emu::Dt{single != 0, false}, ta, tb, m, n, k, ar, ai, A, lda, B, ldb, br, bi, C, ldc, N,
                       stream, nullptr, presums);
    }
  }
  if (n_used) *n_used = N;
  return emu::gemm(emu::Dt{single != 0, false}, ta, tb, m, n, k, ar, ai, A, lda, B, ldb, br, bi, C, ldc, N, stream);
}

emu_status_t emu_zgemm_tol(emu_op_t transa, emu_op_t transb, int64_t m, int64_t n, int64_t k, const double* alpha,
                           const void* A, int64_t lda, const void* B, int64_t ldb, const double* beta, void* C,
                           int64_t ldc, double target_err, int* n_used, void* stream) {
  if (!alpha) return emu::bad(6);
  if (!beta) return emu::bad(11);
  return gemm_tol(0, transa, transb, m, n, k, alpha[0], alpha[1], A, lda, B, ldb, beta[0], beta[1], C, ldc,
                  target_err, n_used, stream);
}

emu_status_t emu_cgemm_tol(emu_op_t transa, emu_op_t transb, int64_t m, int64_t n, int64_t k, const float* alpha,
                           const void* A, int64_t lda, const void* B, int64_t ldb, const float* beta, void* C,
                           int64_t ldc, double target_err, int* n_used, void* stream) {
  if (!alpha) return emu::bad(6);
  if (!beta) return emu::bad(11);
  return gemm_tol(1, transa, transb, m, n, k, alpha[0], alpha[1], A, lda, B, ldb, beta[0], beta[1], C, ldc,
                  target_err, n_used, stream);
}

const char* emu_version(void) { return "ozaki2-emu 0.1 (sm_103a)"; }

}  // extern "C"
