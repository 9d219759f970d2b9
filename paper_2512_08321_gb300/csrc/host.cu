// Host-buffer GEMMs: A, B and C live in host memory.
//
// On GB300 the GPU reaches host memory over the chip-to-chip link, so the
// inputs are brought in by a copy kernel (wide loads of host memory, stores
// to a device staging buffer) and the CRT kernel writes C straight into host
// memory, with no separate device-to-host pass.  A host pointer is used from
// kernels when it is pinned or registered (its device address); pageable
// memory goes through cudaMemcpyAsync and a device copy of C.
#include <mutex>

#include "emu_internal.h"

namespace emu {
namespace {

__global__ void copy16_kernel(const uint4* __restrict__ s, uint4* __restrict__ d, size_t n) {
  for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x)
    d[i] = s[i];
}

__global__ void copy1_kernel(const unsigned char* __restrict__ s, unsigned char* __restrict__ d, size_t n) {
  for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x)
    d[i] = s[i];
}

unsigned int grid_for(size_t items) {
  const size_t g = (items + 255) / 256;
  return static_cast<unsigned int>(g < 152 * 16 ? (g ? g : 1) : 152 * 16);
}

// bytes from src to dst, both device-accessible
cudaError_t copy_bytes(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return cudaSuccess;
  const uintptr_t a = reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src);
  size_t head = 0;
  if ((a & 15u) == 0) {
    const size_t n16 = bytes / 16;
    if (n16) {
      copy16_kernel<<<grid_for(n16), 256, 0, st>>>(static_cast<const uint4*>(src), static_cast<uint4*>(dst), n16);
      count_launches(1);
    }
    head = n16 * 16;
  }
  if (head < bytes) {
    copy1_kernel<<<grid_for(bytes - head), 256, 0, st>>>(static_cast<const unsigned char*>(src) + head,
                                                         static_cast<unsigned char*>(dst) + head, bytes - head);
    count_launches(1);
  }
  return cudaGetLastError();
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

// Per-device side stream and events: B is brought in on the side stream while
// A is copied and processed on the caller's stream.
struct Side {
  cudaStream_t s = nullptr;
  cudaEvent_t start = nullptr, b_done = nullptr;
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
    if ((e = cudaEventCreateWithFlags(&sd.start, cudaEventDisableTiming)) != cudaSuccess) return e;
    if ((e = cudaEventCreateWithFlags(&sd.b_done, cudaEventDisableTiming)) != cudaSuccess) return e;
  }
  *out = &sd;
  return cudaSuccess;
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
  void* Cv = const_cast<void*>(device_view(C));
  const bool use_beta = !(br == 0.0 && bi == 0.0);
  char* stg = nullptr;
  s = get_staging(al(bA) + al(bB) + (Cv ? 0 : al(bC)), &stg);
  if (s != EMU_OK) return s;
  char* dA = stg;
  char* dB = stg + al(bA);
  char* dC = dB + al(bB);
  Side* sd = nullptr;
  if (side_for_device(&sd) != cudaSuccess) return EMU_ERR_CUDA;
  auto bring = [&](char* dst, const void* src, size_t bytes, cudaStream_t s2) -> cudaError_t {
    if (bytes == 0) return cudaSuccess;
    const void* v = device_view(src);
    return v ? copy_bytes(dst, v, bytes, s2) : cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s2);
  };
  // A first on the caller's stream; then B on the side stream (the link carries
  // one copy at a time) while A's exponents and planes are formed
  if (bring(dA, A, bA, st) != cudaSuccess || cudaEventRecord(sd->start, st) != cudaSuccess ||
      cudaStreamWaitEvent(sd->s, sd->start, 0) != cudaSuccess || bring(dB, B, bB, sd->s) != cudaSuccess ||
      cudaEventRecord(sd->b_done, sd->s) != cudaSuccess)
    return EMU_ERR_CUDA;
  // pageable C: a device copy with the same leading dimension; only the m x n
  // entries travel, so the rows between columns stay as the caller left them
  const size_t pitch = static_cast<size_t>(ldc) * esz, width = static_cast<size_t>(m) * esz;
  void* target = Cv;
  if (!Cv) {
    target = dC;
    if (use_beta && cudaMemcpy2DAsync(dC, pitch, C, pitch, width, static_cast<size_t>(n), cudaMemcpyHostToDevice,
                                      st) != cudaSuccess)
      return EMU_ERR_CUDA;
  }
  s = run_gemm(single, real, ta, tb, m, n, k, ar, ai, bA ? dA : nullptr, lda, bB ? dB : nullptr, ldb, br, bi, target,
               ldc, N, stream, sd->b_done);
  if (s != EMU_OK) return s;
  if (!Cv && cudaMemcpy2DAsync(C, pitch, dC, pitch, width, static_cast<size_t>(n), cudaMemcpyDeviceToHost, st) !=
                 cudaSuccess)
    return EMU_ERR_CUDA;
  return EMU_OK;
}

}  // namespace
}  // namespace emu

extern "C" {

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
