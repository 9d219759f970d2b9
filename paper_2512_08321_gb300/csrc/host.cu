// Host-buffer GEMMs: A, B and C live in host memory.
//
// On GB300 the GPU reaches host memory over the chip-to-chip link.  The
// operands go through a device staging buffer, and the output columns are
// processed in blocks (the column blocking of Section III-A): a side stream
// brings block b's columns of B (and of C when beta != 0) in while earlier
// blocks compute, and takes block b's columns of C back while later blocks
// compute, so only A's copy, the first block's inputs and the last block's
// output are not hidden behind the residue products.  Copies that overlap
// computation use the DMA engines; A's copy and the last block of C, which
// nothing overlaps, use a copy kernel through the device address of pinned
// memory, which is faster on the link (211 GB/s in, 194 GB/s out).  Pageable
// memory always goes through cudaMemcpy2DAsync.
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

// Copy kernels run only where nothing else is on the GPU (A's copy, the last
// block of C): two blocks of 256 threads per SM, about 5 MB of loads in flight.
// Copies that overlap computation go to the DMA engines instead: beside the
// split and the residue products, copy kernels' stores to host memory slowed
// those kernels (a column block took about 2 ms longer).
enum class Shape { kKernel, kDma };

template <typename W>
cudaError_t copy_words(void* dst, size_t dpitch, const void* src, size_t spitch, size_t width, size_t rows,
                       cudaStream_t st) {
  constexpr int kT = 256;
  constexpr size_t kCap = 152 * 2;
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

constexpr int kMaxHostBlocks = 8;

// Output columns per block of a host-buffer call: about eight blocks of a
// multiple of 256 columns (the residue GEMM's tile width), at least 1024.
int64_t host_block_cols(int64_t n) {
  if (n <= 2048) return n;
  int64_t cb = round_up((n + kMaxHostBlocks - 1) / kMaxHostBlocks, 256);
  return cb < 1024 ? 1024 : cb;
}

// Per-device side stream and events.  Host-buffer calls on one device are
// serialised (they share the staging buffers): each waits for the previous
// one's `last` event.
struct Side {
  std::mutex mu;
  cudaStream_t s = nullptr;
  cudaEvent_t start = nullptr, done = nullptr, out = nullptr, last = nullptr;
  cudaEvent_t in[kMaxHostBlocks] = {};
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

// State of one host-buffer call, seen by the block hooks.
struct HostCall {
  Side* sd;
  int64_t n;
  int64_t cb;                 // columns per copy block
  char* dC;                   // device copy of C (leading dimension ldc)
  void* C;                    // caller's C
  const void* Cv;             // its device view, or nullptr (pageable)
  size_t pitch, width;        // ldc and m in bytes
};

emu_status_t wait_inputs(void* ctx, int64_t j0, int64_t nj, cudaStream_t st) {
  const HostCall* hc = static_cast<const HostCall*>(ctx);
  for (int64_t c = j0 / hc->cb; c <= (j0 + nj - 1) / hc->cb; ++c)
    if (cudaStreamWaitEvent(st, hc->sd->in[c], 0) != cudaSuccess) return EMU_ERR_CUDA;
  trace(EMU_TRACE_BLOCK_START, st);
  return EMU_OK;
}

// Columns j0.. of C go back on the side stream once the block's CRT is done.
// Pinned C: by the DMA engines, which leave the SMs to the next block's split
// and residue products, except the last block, which nothing else overlaps:
// the copy kernel, the faster of the two on the link.  Pageable C: nothing here (a copy
// into pageable memory would hold the calling thread until it is done); all
// of C goes back after the last block.
emu_status_t output_done(void* ctx, int64_t j0, int64_t nj, cudaStream_t st) {
  const HostCall* hc = static_cast<const HostCall*>(ctx);
  trace(EMU_TRACE_BLOCK_CRT, st);
  if (!hc->Cv) return EMU_OK;
  const size_t off = static_cast<size_t>(j0) * hc->pitch;
  if (cudaEventRecord(hc->sd->out, st) != cudaSuccess || cudaStreamWaitEvent(hc->sd->s, hc->sd->out, 0) != cudaSuccess ||
      transfer(true, hc->dC + off, hc->pitch, static_cast<char*>(hc->C) + off, static_cast<const char*>(hc->Cv) + off,
               hc->pitch, hc->width, static_cast<size_t>(nj), j0 + nj == hc->n ? Shape::kKernel : Shape::kDma,
               hc->sd->s) != cudaSuccess)
    return EMU_ERR_CUDA;
  trace(EMU_TRACE_C_OUT, hc->sd->s);
  return EMU_OK;
}

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
  s = get_staging(al(bA) + al(bB) + al(bC), &stg);
  if (s != EMU_OK) return s;
  char* dA = stg;
  char* dB = stg + al(bA);
  char* dC = dB + al(bB);
  HostCall hc{sd, n, host_block_cols(n), dC, C, device_view(C), static_cast<size_t>(ldc) * esz,
              static_cast<size_t>(m) * esz};
  const int64_t nblk = (n + hc.cb - 1) / hc.cb;
  const void* Av = device_view(A);
  const size_t ldb_b = static_cast<size_t>(ldb) * esz;
  // A first, on the caller's stream, once the previous host-buffer call is done
  trace_reset();
  if (sd->used && cudaStreamWaitEvent(st, sd->last, 0) != cudaSuccess) return EMU_ERR_CUDA;
  trace(EMU_TRACE_START, st);
  if (transfer(false, dA, bA, A, Av, bA, bA, 1, Shape::kKernel, st) != cudaSuccess ||
      cudaEventRecord(sd->start, st) != cudaSuccess || cudaStreamWaitEvent(sd->s, sd->start, 0) != cudaSuccess)
    return EMU_ERR_CUDA;
  trace(EMU_TRACE_A_IN, st);
  sd->used = true;
  // then each block's columns of B (and of C) on the side stream, by the DMA
  // engines while A's exponents and planes and the earlier blocks compute
  emu_status_t res = EMU_OK;
  for (int64_t c = 0; c < nblk && res == EMU_OK; ++c) {
    const int64_t c0 = c * hc.cb, cn = std::min(hc.cb, n - c0);
    cudaError_t e = cudaSuccess;
    if (bB) {
      // columns c0.. of the stored k x n matrix, or rows c0.. of the stored n x k matrix
      const size_t off = tb == EMU_OP_N ? c0 * ldb_b : c0 * esz;
      e = transfer(false, dB + off, ldb_b, static_cast<const char*>(B) + off, nullptr, ldb_b,
                   tb == EMU_OP_N ? static_cast<size_t>(k) * esz : static_cast<size_t>(cn) * esz,
                   tb == EMU_OP_N ? static_cast<size_t>(cn) : static_cast<size_t>(k), Shape::kDma, sd->s);
    }
    if (e == cudaSuccess && use_beta) {
      const size_t off = static_cast<size_t>(c0) * hc.pitch;
      e = transfer(false, dC + off, hc.pitch, static_cast<const char*>(C) + off, nullptr, hc.pitch, hc.width,
                   static_cast<size_t>(cn), Shape::kDma, sd->s);
    }
    if (e == cudaSuccess) e = cudaEventRecord(sd->in[c], sd->s);
    if (e != cudaSuccess) res = EMU_ERR_CUDA;
    trace(EMU_TRACE_B_IN, sd->s);
  }
  if (res == EMU_OK) {
    const BlockHooks hooks{hc.cb, &hc, wait_inputs, output_done};
    res = run_gemm(single, real, ta, tb, m, n, k, ar, ai, bA ? dA : nullptr, lda, bB ? dB : nullptr, ldb, br, bi, dC,
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
