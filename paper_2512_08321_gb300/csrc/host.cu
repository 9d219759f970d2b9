// Host-buffer GEMMs: A, B and C live in host memory.
//
// On GB300 the GPU reaches host memory over the chip-to-chip link.  The inputs
// go through a device staging buffer in blocks (the column blocking of Section
// III-A, and blocks of rows of op(A)), moved on a side stream in the order the
// computation needs them: the first column block of B, A block of rows by block
// of rows, then the other column blocks of B.  The first column block of C is
// computed one block of rows at a time as A arrives, the others as their
// columns of B arrive, so the residue products start after one block of A and
// one of B instead of after all of A.  Contiguous inputs move by the DMA
// engines, strided ones by a copy kernel through the device address of pinned
// memory; the CRT writes pinned C in place (see the shapes below for why).
// Pageable memory always goes through cudaMemcpy2DAsync, and pageable C goes
// back in one piece at the end.
#include <algorithm>
#include <mutex>

#include "emu_internal.h"

namespace emu {
namespace {

// rows segments of w words of type W; segment r at s + r * sp and d + r * dp (in
// words).  Each thread keeps four loads in flight; at most 32 registers.
template <typename W, int T>
__global__ void __launch_bounds__(T, 2048 / T)
    copy2d_kernel(const W* __restrict__ s, size_t sp, W* __restrict__ d, size_t dp, size_t w, size_t rows) {
  constexpr int U = 4;
  const size_t step = static_cast<size_t>(gridDim.x) * T;
  for (size_t r = blockIdx.y; r < rows; r += gridDim.y) {
    const W* sr = s + r * sp;
    W* dr = d + r * dp;
    size_t c = static_cast<size_t>(blockIdx.x) * T + threadIdx.x;
    for (; c + (U - 1) * step < w; c += U * step) {
      W v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) v[u] = sr[c + u * step];
#pragma unroll
      for (int u = 0; u < U; ++u) dr[c + u * step] = v[u];
    }
    for (; c < w; c += step) dr[c] = sr[c];
  }
}

// How a copy moves.  kDma: the DMA engines, which leave the SMs alone;
// measured here, they kept the link's 211 GB/s for contiguous host-to-device
// copies, but beside the residue products a copy of k segments of 32 KB (a
// block of rows of a column-major A) ran at 12-100 GB/s and device-to-host
// copies at 12-190 GB/s.  kNarrow: a copy kernel of one block of 128 threads
// per SM (1.25 MB of loads in flight, 4096 registers, which three resident
// split blocks of 256 threads x 80 registers leave free), for strided inputs:
// it keeps 211 GB/s, at the price of slowing the kernels beside it by about
// 40 % of its own duration.  C is not copied back beside the computation at
// all: stores to host memory from SMs held up the residue products beside
// them (a column block took 37.5 ms instead of 31), so the CRT writes pinned
// C in place, link-bound (2.8 ms per 2048 columns instead of 1.4).
enum class Shape { kNarrow, kDma };

template <typename W>
cudaError_t copy_words(void* dst, size_t dpitch, const void* src, size_t spitch, size_t width, size_t rows,
                       cudaStream_t st) {
  constexpr int kT = 128;
  constexpr size_t kCap = 152;
  const size_t w = width / sizeof(W);
  const size_t gx = std::min<size_t>((w + 4 * kT - 1) / (4 * kT), kCap);
  const size_t gy = std::min<size_t>(std::min<size_t>(rows, std::max<size_t>(kCap / gx, 1)), 65535);
  copy2d_kernel<W, kT><<<dim3(static_cast<unsigned int>(gx), static_cast<unsigned int>(gy)), kT, 0, st>>>(
      static_cast<const W*>(src), spitch / sizeof(W), static_cast<W*>(dst), dpitch / sizeof(W), w, rows);
  count_launches(1);
  return cudaGetLastError();
}

// rows segments of `width` bytes (pitches in bytes), both sides device-accessible;
// moved in the widest words (16, 8, 4 or 1 bytes) that the addresses, width and
// pitches allow.
cudaError_t copy_2d(void* dst, size_t dpitch, const void* src, size_t spitch, size_t width, size_t rows,
                    cudaStream_t st) {
  if (width == 0 || rows == 0) return cudaSuccess;
  if (rows > 1 && dpitch == width && spitch == width) {   // contiguous: one segment
    width *= rows;
    dpitch = spitch = width;
    rows = 1;
  }
  const uintptr_t base = reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src);
  if (rows == 1 && (base & 15u) == 0 && (width & 15u) != 0 && width >= 16) {
    // one segment with a ragged end: 16-byte words, then the tail bytes
    const size_t head = width / 16 * 16;
    cudaError_t e = copy_words<uint4>(dst, head, src, head, head, 1, st);
    if (e != cudaSuccess) return e;
    return copy_words<unsigned char>(static_cast<char*>(dst) + head, width - head,
                                     static_cast<const char*>(src) + head, width - head, width - head, 1, st);
  }
  const uintptr_t a = base | width | (rows > 1 ? (dpitch | spitch) : 0);
  if ((a & 15u) == 0) return copy_words<uint4>(dst, dpitch, src, spitch, width, rows, st);
  if ((a & 7u) == 0) return copy_words<unsigned long long>(dst, dpitch, src, spitch, width, rows, st);
  if ((a & 3u) == 0) return copy_words<unsigned int>(dst, dpitch, src, spitch, width, rows, st);
  return copy_words<unsigned char>(dst, dpitch, src, spitch, width, rows, st);
}

// Address under which kernels reach memory p (pinned or registered host memory,
// or device / managed memory), or nullptr for pageable host memory.
const void* device_view(const void* p) {
  if (!p) return nullptr;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type == cudaMemoryTypeHost) return a.devicePointer ? a.devicePointer : p;
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return p;
  return nullptr;
}

// Bytes of a stored column-major matrix of `rows` x `cols` with leading dimension ld.
size_t stored_bytes(int64_t rows, int64_t cols, int64_t ld, size_t esz) {
  if (rows <= 0 || cols <= 0) return 0;
  return (static_cast<size_t>(cols - 1) * static_cast<size_t>(ld) + static_cast<size_t>(rows)) * esz;
}

size_t al(size_t v) { return (v + 255) / 256 * 256; }

// A 2-D copy between the staging buffer (dev) and caller memory (host, with
// device address view; nullptr when pageable): the copy kernel through the
// view, or the DMA engines (cudaMemcpy2DAsync) for pageable memory and for
// shape kDma.
cudaError_t transfer(bool to_host, void* dev, size_t dpitch, const void* host, const void* view, size_t hpitch,
                     size_t width, size_t rows, Shape shape, cudaStream_t st) {
  if (width == 0 || rows == 0) return cudaSuccess;
  if (view && shape != Shape::kDma)
    return to_host ? copy_2d(const_cast<void*>(view), hpitch, dev, dpitch, width, rows, st)
                   : copy_2d(dev, dpitch, view, hpitch, width, rows, st);
  return to_host ? cudaMemcpy2DAsync(const_cast<void*>(host), hpitch, dev, dpitch, width, rows, cudaMemcpyDeviceToHost, st)
                 : cudaMemcpy2DAsync(dev, dpitch, host, hpitch, width, rows, cudaMemcpyHostToDevice, st);
}

constexpr int kMaxHostBlocks = 16;           // events of column blocks (at most 9 are used) and row blocks
constexpr int kTargetBlocks = 8;
constexpr int64_t kHostBlockMin = 2048;

// Columns of C (rows of op(A)) per block of a host-buffer call: about eight
// blocks of a multiple of 256 (the residue GEMM's tile width), at least 2048
// (narrower blocks cost more in per-block overhead than they hide: CGEMM
// 8192^3 from pinned buffers ran at 165 TFLOPS with 1024, 182 with 2048).
int64_t host_block(int64_t len) {
  if (len <= kHostBlockMin) return len;
  int64_t cb = round_up((len + kTargetBlocks - 1) / kTargetBlocks, 256);
  return cb < kHostBlockMin ? kHostBlockMin : cb;
}

// Width of the first column block when there are several: half a block
// (a multiple of 256).  While A arrives block of rows by block of rows, the
// first column block's products are all the GPU can do, and the copy of A
// slows them; a narrower first block keeps that work close to the pace A
// arrives at, and the wider blocks after it run at full speed.
int64_t first_block(int64_t n, int64_t cb) {
  if (n <= cb) return n;
  const int64_t h = round_up(cb / 2, 256);
  return h < cb ? h : cb;
}

// Per-device side stream and events.  Host-buffer calls on one device are
// serialised (they share the staging buffers): each waits for the previous
// one's `last` event.
struct Side {
  std::mutex mu;
  cudaStream_t s = nullptr;
  cudaEvent_t start = nullptr, done = nullptr, out = nullptr, last = nullptr;
  cudaEvent_t in[kMaxHostBlocks] = {};    // columns of B (and C) of a column block
  cudaEvent_t in_a[kMaxHostBlocks] = {};  // rows of op(A) of a row block
  bool used = false;
};
std::mutex g_side_mu;
Side g_side[64];

cudaError_t side_for_device(Side** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_side_mu);
  Side& sd = g_side[dev];
  if (!sd.s) {
    if ((e = cudaStreamCreateWithFlags(&sd.s, cudaStreamNonBlocking)) != cudaSuccess) return e;
    cudaEvent_t* evs[] = {&sd.start, &sd.done, &sd.out, &sd.last};
    for (cudaEvent_t* ev : evs)
      if ((e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming)) != cudaSuccess) return e;
    for (cudaEvent_t& ev : sd.in)
      if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return e;
    for (cudaEvent_t& ev : sd.in_a)
      if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return e;
  }
  *out = &sd;
  return cudaSuccess;
}

// Trace of the latest host-buffer call (emu_host_trace_*): timing events at
// each step of the pipeline, on the stream where the step happens.
struct Trace {
  std::mutex mu;
  bool on = false;
  int n = 0;
  int label[EMU_TRACE_MAX];
  cudaEvent_t ev[EMU_TRACE_MAX] = {};
};
Trace g_trace;

void trace(int label, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_trace.mu);
  if (!g_trace.on || g_trace.n >= EMU_TRACE_MAX) return;
  const int i = g_trace.n;
  if (!g_trace.ev[i] && cudaEventCreate(&g_trace.ev[i]) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  if (cudaEventRecord(g_trace.ev[i], s) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  g_trace.label[i] = label;
  g_trace.n = i + 1;
}

void trace_reset() {
  std::lock_guard<std::mutex> lk(g_trace.mu);
  g_trace.n = 0;
}

// State of one host-buffer call, seen by the block hooks.  Column block 0
// covers [0, nb0), block c > 0 covers [nb0 + (c - 1) cb, ...).
struct HostCall {
  Side* sd;
  int64_t n;
  int64_t cb, mb;             // columns per column block (after the first), rows per row block
  int64_t nb0;                // columns of the first column block
  char* dC;                   // device copy of C (leading dimension ldc)
  void* C;                    // caller's C
  const void* Cv;             // its device view, or nullptr (pageable)
  size_t pitch, width;        // ldc and m in bytes
  int64_t c_dev_end;          // pinned C: columns below this go through dC and back by DMA
  int64_t block_of(int64_t j) const { return j < nb0 ? 0 : 1 + (j - nb0) / cb; }
  int64_t block_begin(int64_t c) const { return c == 0 ? 0 : nb0 + (c - 1) * cb; }
  int64_t block_cols(int64_t c) const {
    const int64_t b = block_begin(c), w = c == 0 ? nb0 : cb;
    return std::min(w, n - b);
  }
};

emu_status_t wait_inputs(void* ctx, int64_t j0, int64_t nj, cudaStream_t st) {
  const HostCall* hc = static_cast<const HostCall*>(ctx);
  for (int64_t c = hc->block_of(j0); c <= hc->block_of(j0 + nj - 1); ++c)
    if (cudaStreamWaitEvent(st, hc->sd->in[c], 0) != cudaSuccess) return EMU_ERR_CUDA;
  trace(EMU_TRACE_BLOCK_START, st);
  return EMU_OK;
}

emu_status_t wait_rows(void* ctx, int64_t i0, int64_t mi, cudaStream_t st) {
  const HostCall* hc = static_cast<const HostCall*>(ctx);
  for (int64_t r = i0 / hc->mb; r <= (i0 + mi - 1) / hc->mb; ++r)
    if (cudaStreamWaitEvent(st, hc->sd->in_a[r], 0) != cudaSuccess) return EMU_ERR_CUDA;
  return EMU_OK;
}

// A column block of C is final once its CRT is done.  Pinned C, last two
// blocks (or beta != 0): the CRT wrote it straight into host memory.  Pinned C,
// earlier blocks: the CRT wrote the device copy, and the DMA engines bring it
// back on the side stream while the next blocks compute (stores from SMs into
// host memory slowed the residue products beside them; the DMA engines do not).
// Pageable C: it goes back in one piece after the last block (a copy into
// pageable memory holds the calling thread).
emu_status_t output_done(void* ctx, int64_t j0, int64_t nj, cudaStream_t st) {
  const HostCall* hc = static_cast<const HostCall*>(ctx);
  trace(EMU_TRACE_BLOCK_CRT, st);
  if (hc->Cv && j0 < hc->c_dev_end) {
    const size_t off = static_cast<size_t>(j0) * hc->pitch;
    if (cudaEventRecord(hc->sd->out, st) != cudaSuccess || cudaStreamWaitEvent(hc->sd->s, hc->sd->out, 0) != cudaSuccess ||
        cudaMemcpy2DAsync(static_cast<char*>(hc->C) + off, hc->pitch, hc->dC + off, hc->pitch, hc->width,
                          static_cast<size_t>(nj), cudaMemcpyDeviceToHost, hc->sd->s) != cudaSuccess)
      return EMU_ERR_CUDA;
    trace(EMU_TRACE_C_OUT, hc->sd->s);
  }
  return EMU_OK;
}

emu_status_t products_start(void* /*ctx*/, cudaStream_t /*st*/) { return EMU_OK; }

emu_status_t gemm_host(bool single, bool real, emu_op_t ta, emu_op_t tb, int64_t m, int64_t n, int64_t k,
                       double ar, double ai, const void* A, int64_t lda, const void* B, int64_t ldb, double br,
                       double bi, void* C, int64_t ldc, int N, void* stream) {
  emu_status_t s = check_gemm_args(ta, tb, m, n, k, lda, ldb, ldc, N);
  if (s != EMU_OK) return s;
  if (m == 0 || n == 0) return EMU_OK;
  if (!C) return set_bad_param(12);
  if (k > 0 && !A) return set_bad_param(7);
  if (k > 0 && !B) return set_bad_param(9);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t esz = static_cast<size_t>(real ? 1 : 2) * (single ? 4 : 8);
  const size_t bA = stored_bytes(ta == EMU_OP_N ? m : k, ta == EMU_OP_N ? k : m, lda, esz);
  const size_t bB = stored_bytes(tb == EMU_OP_N ? k : n, tb == EMU_OP_N ? n : k, ldb, esz);
  const size_t bC = stored_bytes(m, n, ldc, esz);
  const bool use_beta = !(br == 0.0 && bi == 0.0);
  Side* sd = nullptr;
  if (side_for_device(&sd) != cudaSuccess) return EMU_ERR_CUDA;
  std::lock_guard<std::mutex> lk(sd->mu);
  char* stg = nullptr;
  const void* Cv = device_view(C);
  const int64_t cb_all = host_block(n);
  const int64_t nb0 = first_block(n, cb_all);
  const int64_t cb = n > nb0 ? host_block(n - nb0) : n;
  const int64_t nblk = n > nb0 ? 1 + (n - nb0 + cb - 1) / cb : 1;
  // pinned C with beta = 0: the blocks before the last two go through the device copy and back by
  // DMA, each copy hidden behind at least two blocks of computation (beside the residue products
  // those copies ran at 12-190 GB/s, too slow to hide behind the last block alone); the last two
  // blocks' CRTs write host memory in place
  const int64_t c_dev_end = (Cv && !use_beta && nblk > 2) ? nb0 + (nblk - 3) * cb : 0;
  s = get_staging(al(bA) + al(bB) + ((!Cv || c_dev_end > 0) ? al(bC) : 0), &stg);
  if (s != EMU_OK) return s;
  char* dA = stg;
  char* dB = stg + al(bA);
  char* dC = dB + al(bB);
  HostCall hc{sd, n, cb, host_block(m), nb0, dC, C, Cv, static_cast<size_t>(ldc) * esz,
              static_cast<size_t>(m) * esz, c_dev_end};
  const int64_t mblk = (m + hc.mb - 1) / hc.mb;
  if (nblk > kMaxHostBlocks || mblk > kMaxHostBlocks) return EMU_ERR_UNSUPPORTED;
  const size_t lda_b = static_cast<size_t>(lda) * esz, ldb_b = static_cast<size_t>(ldb) * esz;
  const void* Av = device_view(A);
  const void* Bv = device_view(B);
  // once the previous host-buffer call is done, the inputs move on the side
  // stream in the order the caller's stream needs them; contiguous copies by
  // the DMA engines, strided ones (from pinned memory) by the narrow copy kernel
  trace_reset();
  if (sd->used && cudaStreamWaitEvent(st, sd->last, 0) != cudaSuccess) return EMU_ERR_CUDA;
  trace(EMU_TRACE_START, st);
  if (cudaEventRecord(sd->start, st) != cudaSuccess || cudaStreamWaitEvent(sd->s, sd->start, 0) != cudaSuccess)
    return EMU_ERR_CUDA;
  sd->used = true;
  auto bring = [&](char* dst, const void* src, const void* view, size_t off, size_t pitch, size_t width,
                   size_t rows) -> cudaError_t {
    const bool contiguous = rows == 1 || pitch == width;
    return transfer(false, dst + off, pitch, static_cast<const char*>(src) + off,
                    view ? static_cast<const char*>(view) + off : nullptr, pitch, width, rows,
                    contiguous || !view ? Shape::kDma : Shape::kNarrow, sd->s);
  };
  auto bring_cols = [&](int64_t c) -> cudaError_t {   // columns c0.. of op(B) (and of C)
    const int64_t c0 = hc.block_begin(c), cn = hc.block_cols(c);
    cudaError_t e = cudaSuccess;
    if (bB)   // columns c0.. of the stored k x n matrix, or rows c0.. of the stored n x k matrix
      e = tb == EMU_OP_N ? bring(dB, B, Bv, c0 * ldb_b, ldb_b, static_cast<size_t>(k) * esz, static_cast<size_t>(cn))
                         : bring(dB, B, Bv, c0 * esz, ldb_b, static_cast<size_t>(cn) * esz, static_cast<size_t>(k));
    if (e == cudaSuccess && use_beta && !Cv)   // pageable C: its columns into the device copy
      e = bring(dC, C, nullptr, static_cast<size_t>(c0) * hc.pitch, hc.pitch, hc.width, static_cast<size_t>(cn));
    if (e == cudaSuccess) e = cudaEventRecord(sd->in[c], sd->s);
    trace(EMU_TRACE_B_IN, sd->s);
    return e;
  };
  auto bring_rows = [&](int64_t r) -> cudaError_t {   // rows r0.. of op(A)
    const int64_t r0 = r * hc.mb, rn = std::min(hc.mb, m - r0);
    cudaError_t e = cudaSuccess;
    if (bA)   // rows r0.. of the stored m x k matrix, or columns r0.. of the stored k x m matrix
      e = ta == EMU_OP_N ? bring(dA, A, Av, r0 * esz, lda_b, static_cast<size_t>(rn) * esz, static_cast<size_t>(k))
                         : bring(dA, A, Av, r0 * lda_b, lda_b, static_cast<size_t>(k) * esz, static_cast<size_t>(rn));
    if (e == cudaSuccess) e = cudaEventRecord(sd->in_a[r], sd->s);
    trace(EMU_TRACE_A_IN, sd->s);
    return e;
  };
  emu_status_t res = EMU_OK;
  if (bring_cols(0) != cudaSuccess) res = EMU_ERR_CUDA;
  for (int64_t r = 0; r < mblk && res == EMU_OK; ++r)
    if (bring_rows(r) != cudaSuccess) res = EMU_ERR_CUDA;
  for (int64_t c = 1; c < nblk && res == EMU_OK; ++c)
    if (bring_cols(c) != cudaSuccess) res = EMU_ERR_CUDA;
  if (res == EMU_OK) {
    const BlockHooks hooks{hc.cb, hc.mb, hc.nb0, c_dev_end > 0 ? static_cast<void*>(dC) : nullptr, c_dev_end, &hc,
                           wait_inputs, wait_rows, output_done, products_start};
    res = run_gemm(single, real, ta, tb, m, n, k, ar, ai, bA ? dA : nullptr, lda, bB ? dB : nullptr, ldb, br, bi,
                   Cv ? const_cast<void*>(Cv) : static_cast<void*>(dC),
                   ldc, N, stream, &hooks);
  }
  if (res == EMU_OK && !hc.Cv) {   // pageable C: all of it once the last block is done
    if (cudaEventRecord(sd->out, st) != cudaSuccess || cudaStreamWaitEvent(sd->s, sd->out, 0) != cudaSuccess ||
        transfer(true, dC, hc.pitch, C, nullptr, hc.pitch, hc.width, static_cast<size_t>(n), Shape::kDma, sd->s) !=
            cudaSuccess)
      res = EMU_ERR_CUDA;
    trace(EMU_TRACE_C_OUT, sd->s);
  }
  // the caller's stream completes only after the last block of C has arrived
  if (cudaEventRecord(sd->done, sd->s) != cudaSuccess || cudaStreamWaitEvent(st, sd->done, 0) != cudaSuccess ||
      cudaEventRecord(sd->last, st) != cudaSuccess)
    return res == EMU_OK ? EMU_ERR_CUDA : res;
  trace(EMU_TRACE_END, st);
  return res;
}

}  // namespace
}  // namespace emu

extern "C" {

emu_status_t emu_host_trace_enable(int on) {
  std::lock_guard<std::mutex> lk(emu::g_trace.mu);
  emu::g_trace.on = (on != 0);
  emu::g_trace.n = 0;
  return EMU_OK;
}

int emu_host_trace_read(int* labels, float* ms, int cap) {
  std::lock_guard<std::mutex> lk(emu::g_trace.mu);
  const int n = emu::g_trace.n;
  if (n == 0 || cap <= 0 || !labels || !ms) return 0;
  const int cnt = n < cap ? n : cap;
  for (int i = 0; i < cnt; ++i) {
    if (cudaEventSynchronize(emu::g_trace.ev[i]) != cudaSuccess ||
        cudaEventElapsedTime(&ms[i], emu::g_trace.ev[0], emu::g_trace.ev[i]) != cudaSuccess) {
      cudaGetLastError();
      return -1;
    }
    labels[i] = emu::g_trace.label[i];
  }
  return cnt;
}

emu_status_t emu_zgemm_host(emu_op_t transa, emu_op_t transb, int64_t m, int64_t n, int64_t k, const double* alpha,
                            const void* A, int64_t lda, const void* B, int64_t ldb, const double* beta, void* C,
                            int64_t ldc, int num_moduli, void* stream) {
  if (!alpha) return emu::set_bad_param(6);
  if (!beta) return emu::set_bad_param(11);
  return emu::gemm_host(false, false, transa, transb, m, n, k, alpha[0], alpha[1], A, lda, B, ldb, beta[0], beta[1],
                        C, ldc, num_moduli, stream);
}

emu_status_t emu_cgemm_host(emu_op_t transa, emu_op_t transb, int64_t m, int64_t n, int64_t k, const float* alpha,
                            const void* A, int64_t lda, const void* B, int64_t ldb, const float* beta, void* C,
                            int64_t ldc, int num_moduli, void* stream) {
  if (!alpha) return emu::set_bad_param(6);
  if (!beta) return emu::set_bad_param(11);
  return emu::gemm_host(true, false, transa, transb, m, n, k, alpha[0], alpha[1], A, lda, B, ldb, beta[0], beta[1],
                        C, ldc, num_moduli, stream);
}

emu_status_t emu_dgemm_host(emu_op_t transa, emu_op_t transb, int64_t m, int64_t n, int64_t k, const double* alpha,
                            const double* A, int64_t lda, const double* B, int64_t ldb, const double* beta,
                            double* C, int64_t ldc, int num_moduli, void* stream) {
  if (!alpha) return emu::set_bad_param(6);
  if (!beta) return emu::set_bad_param(11);
  return emu::gemm_host(false, true, transa, transb, m, n, k, *alpha, 0.0, A, lda, B, ldb, *beta, 0.0, C, ldc,
                        num_moduli, stream);
}

emu_status_t emu_sgemm_host(emu_op_t transa, emu_op_t transb, int64_t m, int64_t n, int64_t k, const float* alpha,
                            const float* A, int64_t lda, const float* B, int64_t ldb, const float* beta, float* C,
                            int64_t ldc, int num_moduli, void* stream) {
  if (!alpha) return emu::set_bad_param(6);
  if (!beta) return emu::set_bad_param(11);
  return emu::gemm_host(true, true, transa, transb, m, n, k, *alpha, 0.0, A, lda, B, ldb, *beta, 0.0, C, ldc,
                        num_moduli, stream);
}

}  // extern "C"
