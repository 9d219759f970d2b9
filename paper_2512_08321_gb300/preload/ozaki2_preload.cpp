// LD_PRELOAD interposer: redirects an application's cuBLAS GEMM calls to the
// Ozaki-II emulation (the paper's Section III-D: the library is activated by
// adding it to LD_PRELOAD, and the cuBLAS S/D/C/Z GEMM routines, their _v2
// forms and cublasGemmEx are redirected without changing the application).
//
// Interposed: cublas{S,D,C,Z}gemm_v2, their _64 forms, cublasGemmEx (when A, B
// and C share one of CUDA_R_32F / CUDA_R_64F / CUDA_C_32F / CUDA_C_64F and the
// compute type is the matching 32F / 64F one, default or pedantic), and the
// legacy cublas{S,D,C,Z}gemm with cublasSetKernelStream.  Every other call,
// and every call the emulation does not take, goes to the real cuBLAS routine
// (looked up with dlsym(RTLD_NEXT)):
//   - transa/transb other than N, T, C; k > 2^17; a negative size;
//   - min(m, n, k) below OZAKI2_EMU_MIN_DIM (default 1: everything non-empty);
//   - OZAKI2_EMU_DISABLE set to a non-empty value other than "0";
//   - any error status from the emulation (argument, workspace, launch).
// Scalars in device pointer mode are read with a copy on the handle's stream
// followed by a synchronisation of that stream.
//
// Number of moduli per element type: OZAKI2_EMU_MODULI_Z (default 15),
// _C (8), _D (16), _S (8); or, for ZGEMM and CGEMM, OZAKI2_EMU_TOL = a
// normalised accuracy target, which selects N per call (emu_zgemm_tol).
// OZAKI2_EMU_VERBOSE=1 prints one line on the first call of each routine.
#include <dlfcn.h>

#include <atomic>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "ozaki2_emu.h"
#include "ozaki2_preload.h"

namespace {

// cuBLAS ABI types and values (cublas_api.h, library_types.h)
typedef void* Handle;
typedef int Status;          // cublasStatus_t, CUBLAS_STATUS_SUCCESS = 0
typedef int Op;              // cublasOperation_t: N 0, T 1, C 2, CONJG 3
typedef int DataType;        // cudaDataType
typedef int ComputeType;     // cublasComputeType_t
typedef int GemmAlgo;
struct alignas(8) f2 { float x, y; };     // layout and alignment of float2 / cuComplex
struct alignas(16) d2 { double x, y; };   // of double2 / cuDoubleComplex
constexpr Status kSuccess = 0;
constexpr int kPointerModeDevice = 1;
constexpr DataType R_32F = 0, R_64F = 1, C_32F = 4, C_64F = 5;
constexpr ComputeType COMPUTE_32F = 68, COMPUTE_32F_PEDANTIC = 69, COMPUTE_64F = 70, COMPUTE_64F_PEDANTIC = 71;

enum Routine { kS = 0, kD, kC, kZ, kGemmEx, kLegacy, kRoutines };
const char* kNames[kRoutines] = {"cublasSgemm", "cublasDgemm", "cublasCgemm", "cublasZgemm", "cublasGemmEx",
                                 "legacy cublas?gemm"};

std::atomic<uint64_t> g_emulated[kRoutines];
std::atomic<uint64_t> g_forwarded[kRoutines];
std::atomic<bool> g_announced[kRoutines];

void* real_sym(const char* name) {
  void* p = dlsym(RTLD_NEXT, name);
  if (!p) std::fprintf(stderr, "ozaki2_preload: %s not found in the libraries after the interposer\n", name);
  return p;
}

template <class F>
F* real(const char* name, F*& cache) {
  if (!cache) cache = reinterpret_cast<F*>(real_sym(name));
  return cache;
}

int env_int(const char* name, int dflt) {
  const char* v = std::getenv(name);
  if (!v || !*v) return dflt;
  return std::atoi(v);
}

bool disabled() {
  const char* v = std::getenv("OZAKI2_EMU_DISABLE");
  return v && *v && std::strcmp(v, "0") != 0;
}

double tolerance() {
  const char* v = std::getenv("OZAKI2_EMU_TOL");
  return (v && *v) ? std::atof(v) : 0.0;
}

int moduli(Routine r) {
  switch (r) {
    case kZ: return env_int("OZAKI2_EMU_MODULI_Z", 15);
    case kC: return env_int("OZAKI2_EMU_MODULI_C", 8);
    case kD: return env_int("OZAKI2_EMU_MODULI_D", 16);
    default: return env_int("OZAKI2_EMU_MODULI_S", 8);
  }
}

void announce(Routine r, int N) {
  if (env_int("OZAKI2_EMU_VERBOSE", 0) && !g_announced[r].exchange(true))
    std::fprintf(stderr, "ozaki2_preload: %s -> Ozaki-II emulation (N = %d)\n", kNames[r], N);
}

// Take the call?  (the forwarded cases of the header comment, before any GPU work)
bool takes(Op ta, Op tb, int64_t m, int64_t n, int64_t k) {
  if (disabled()) return false;
  if (ta < 0 || ta > 2 || tb < 0 || tb > 2) return false;
  if (m < 0 || n < 0 || k < 0 || k > EMU_MAX_K) return false;
  const int64_t mn = m < n ? m : n;
  const int64_t mnk = mn < k ? mn : k;
  return mnk >= env_int("OZAKI2_EMU_MIN_DIM", 1);
}

// Handle queries through the real cuBLAS.
typedef Status GetStreamFn(Handle, cudaStream_t*);
typedef Status GetPtrModeFn(Handle, int*);
GetStreamFn* p_get_stream = nullptr;
GetPtrModeFn* p_get_ptr_mode = nullptr;

bool handle_state(Handle h, cudaStream_t* st, bool* device_scalars) {
  GetStreamFn* gs = real("cublasGetStream_v2", p_get_stream);
  GetPtrModeFn* gp = real("cublasGetPointerMode_v2", p_get_ptr_mode);
  if (!gs || !gp) return false;
  int mode = 0;
  if (gs(h, st) != kSuccess || gp(h, &mode) != kSuccess) return false;
  *device_scalars = (mode == kPointerModeDevice);
  return true;
}

// Host copies of alpha and beta (each `bytes` long).
bool scalars(const void* alpha, const void* beta, size_t bytes, bool on_device, cudaStream_t st, void* ha,
             void* hb) {
  if (!alpha || !beta) return false;
  if (!on_device) {
    std::memcpy(ha, alpha, bytes);
    std::memcpy(hb, beta, bytes);
    return true;
  }
  return cudaMemcpyAsync(ha, alpha, bytes, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
         cudaMemcpyAsync(hb, beta, bytes, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
         cudaStreamSynchronize(st) == cudaSuccess;
}

// The emulated call for each element type; returns true when it was enqueued.
bool run_z(Op ta, Op tb, int64_t m, int64_t n, int64_t k, const d2& a, const void* A, int64_t lda, const void* B,
           int64_t ldb, const d2& b, void* C, int64_t ldc, cudaStream_t st) {
  const double al[2] = {a.x, a.y}, be[2] = {b.x, b.y};
  const double tol = tolerance();
  emu_status_t s;
  int N = moduli(kZ);
  if (tol > 0.0)
    s = emu_zgemm_tol(static_cast<emu_op_t>(ta), static_cast<emu_op_t>(tb), m, n, k, al, A, lda, B, ldb, be, C, ldc,
                      tol, &N, st);
  else
    s = emu_zgemm(static_cast<emu_op_t>(ta), static_cast<emu_op_t>(tb), m, n, k, al, A, lda, B, ldb, be, C, ldc, N,
                  st);
  if (s == EMU_OK) announce(kZ, N);
  return s == EMU_OK;
}

bool run_c(Op ta, Op tb, int64_t m, int64_t n, int64_t k, const f2& a, const void* A, int64_t lda, const void* B,
           int64_t ldb, const f2& b, void* C, int64_t ldc, cudaStream_t st) {
  const float al[2] = {a.x, a.y}, be[2] = {b.x, b.y};
  const double tol = tolerance();
  emu_status_t s;
  int N = moduli(kC);
  if (tol > 0.0)
    s = emu_cgemm_tol(static_cast<emu_op_t>(ta), static_cast<emu_op_t>(tb), m, n, k, al, A, lda, B, ldb, be, C, ldc,
                      tol, &N, st);
  else
    s = emu_cgemm(static_cast<emu_op_t>(ta), static_cast<emu_op_t>(tb), m, n, k, al, A, lda, B, ldb, be, C, ldc, N,
                  st);
  if (s == EMU_OK) announce(kC, N);
  return s == EMU_OK;
}

bool run_d(Op ta, Op tb, int64_t m, int64_t n, int64_t k, double a, const double* A, int64_t lda, const double* B,
           int64_t ldb, double b, double* C, int64_t ldc, cudaStream_t st) {
  const int N = moduli(kD);
  const emu_status_t s = emu_dgemm(static_cast<emu_op_t>(ta), static_cast<emu_op_t>(tb), m, n, k, &a, A, lda, B, ldb,
                                   &b, C, ldc, N, st);
  if (s == EMU_OK) announce(kD, N);
  return s == EMU_OK;
}

bool run_s(Op ta, Op tb, int64_t m, int64_t n, int64_t k, float a, const float* A, int64_t lda, const float* B,
           int64_t ldb, float b, float* C, int64_t ldc, cudaStream_t st) {
  const int N = moduli(kS);
  const emu_status_t s = emu_sgemm(static_cast<emu_op_t>(ta), static_cast<emu_op_t>(tb), m, n, k, &a, A, lda, B, ldb,
                                   &b, C, ldc, N, st);
  if (s == EMU_OK) announce(kS, N);
  return s == EMU_OK;
}

// Handle-based entry: emulate if possible, else forward.
template <class T, class Run, class Fwd>
Status handle_gemm(Routine r, Handle h, Op ta, Op tb, int64_t m, int64_t n, int64_t k, const T* alpha, const void* A,
                   int64_t lda, const void* B, int64_t ldb, const T* beta, void* C, int64_t ldc, Run run, Fwd fwd) {
  if (takes(ta, tb, m, n, k)) {
    cudaStream_t st = nullptr;
    bool dev = false;
    T a, b;
    if (handle_state(h, &st, &dev) && scalars(alpha, beta, sizeof(T), dev, st, &a, &b) &&
        run(ta, tb, m, n, k, a, A, lda, B, ldb, b, C, ldc, st)) {
      g_emulated[r].fetch_add(1);
      return kSuccess;
    }
  }
  g_forwarded[r].fetch_add(1);
  return fwd();
}

cudaStream_t g_legacy_stream = nullptr;   // set by cublasSetKernelStream
std::mutex g_legacy_mu;

cudaStream_t legacy_stream() {
  std::lock_guard<std::mutex> lk(g_legacy_mu);
  return g_legacy_stream;
}

}  // namespace

extern "C" {

// ------------------------------------------------------------------ v2 API
#define OZ_V2(NAME, IDX, T, ELEM, RUN)                                                                        \
  Status NAME(Handle h, Op ta, Op tb, int m, int n, int k, const T* alpha, const ELEM* A, int lda,           \
              const ELEM* B, int ldb, const T* beta, ELEM* C, int ldc) {                                     \
    typedef Status Fn(Handle, Op, Op, int, int, int, const T*, const ELEM*, int, const ELEM*, int, const T*, \
                      ELEM*, int);                                                                           \
    static Fn* fn = nullptr;                                                                                 \
    return handle_gemm<T>(                                                                                   \
        IDX, h, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc,                                        \
        [](Op a1, Op a2, int64_t a3, int64_t a4, int64_t a5, const T& a6, const void* a7, int64_t a8,          \
           const void* a9, int64_t a10, const T& a11, void* a12, int64_t a13, cudaStream_t a14) {            \
          return RUN(a1, a2, a3, a4, a5, a6, static_cast<const ELEM*>(a7), a8, static_cast<const ELEM*>(a9),  \
                     a10, a11, static_cast<ELEM*>(a12), a13, a14);                                           \
        },                                                                                                   \
        [&]() {                                                                                              \
          Fn* f = real(#NAME, fn);                                                                           \
          return f ? f(h, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc) : 13; /* EXECUTION_FAILED */ \
        });                                                                                                  \
  }

#define OZ_V2_64(NAME, IDX, T, ELEM, RUN)                                                                     \
  Status NAME(Handle h, Op ta, Op tb, int64_t m, int64_t n, int64_t k, const T* alpha, const ELEM* A,        \
              int64_t lda, const ELEM* B, int64_t ldb, const T* beta, ELEM* C, int64_t ldc) {                \
    typedef Status Fn(Handle, Op, Op, int64_t, int64_t, int64_t, const T*, const ELEM*, int64_t, const ELEM*, \
                      int64_t, const T*, ELEM*, int64_t);                                                    \
    static Fn* fn = nullptr;                                                                                 \
    return handle_gemm<T>(                                                                                   \
        IDX, h, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc,                                        \
        [](Op a1, Op a2, int64_t a3, int64_t a4, int64_t a5, const T& a6, const void* a7, int64_t a8,          \
           const void* a9, int64_t a10, const T& a11, void* a12, int64_t a13, cudaStream_t a14) {            \
          return RUN(a1, a2, a3, a4, a5, a6, static_cast<const ELEM*>(a7), a8, static_cast<const ELEM*>(a9),  \
                     a10, a11, static_cast<ELEM*>(a12), a13, a14);                                           \
        },                                                                                                   \
        [&]() {                                                                                              \
          Fn* f = real(#NAME, fn);                                                                           \
          return f ? f(h, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc) : 13;                        \
        });                                                                                                  \
  }

OZ_V2(cublasSgemm_v2, kS, float, float, run_s)
OZ_V2(cublasDgemm_v2, kD, double, double, run_d)
OZ_V2(cublasCgemm_v2, kC, f2, f2, run_c)
OZ_V2(cublasZgemm_v2, kZ, d2, d2, run_z)
OZ_V2_64(cublasSgemm_v2_64, kS, float, float, run_s)
OZ_V2_64(cublasDgemm_v2_64, kD, double, double, run_d)
OZ_V2_64(cublasCgemm_v2_64, kC, f2, f2, run_c)
OZ_V2_64(cublasZgemm_v2_64, kZ, d2, d2, run_z)

// --------------------------------------------------------------- GemmEx
Status cublasGemmEx(Handle h, Op ta, Op tb, int m, int n, int k, const void* alpha, const void* A, DataType Atype,
                    int lda, const void* B, DataType Btype, int ldb, const void* beta, void* C, DataType Ctype,
                    int ldc, ComputeType ct, GemmAlgo algo) {
  typedef Status Fn(Handle, Op, Op, int, int, int, const void*, const void*, DataType, int, const void*, DataType,
                    int, const void*, void*, DataType, int, ComputeType, GemmAlgo);
  static Fn* fn = nullptr;
  auto fwd = [&]() {
    g_forwarded[kGemmEx].fetch_add(1);
    Fn* f = real("cublasGemmEx", fn);
    return f ? f(h, ta, tb, m, n, k, alpha, A, Atype, lda, B, Btype, ldb, beta, C, Ctype, ldc, ct, algo) : 13;
  };
  if (Atype != Btype || Atype != Ctype || !takes(ta, tb, m, n, k)) return fwd();
  const bool c32 = (ct == COMPUTE_32F || ct == COMPUTE_32F_PEDANTIC);
  const bool c64 = (ct == COMPUTE_64F || ct == COMPUTE_64F_PEDANTIC);
  cudaStream_t st = nullptr;
  bool dev = false;
  if (!handle_state(h, &st, &dev)) return fwd();
  bool ok = false;
  if (Atype == R_32F && c32) {
    float a, b;
    ok = scalars(alpha, beta, sizeof(float), dev, st, &a, &b) &&
         run_s(ta, tb, m, n, k, a, static_cast<const float*>(A), lda, static_cast<const float*>(B), ldb, b,
               static_cast<float*>(C), ldc, st);
  } else if (Atype == R_64F && c64) {
    double a, b;
    ok = scalars(alpha, beta, sizeof(double), dev, st, &a, &b) &&
         run_d(ta, tb, m, n, k, a, static_cast<const double*>(A), lda, static_cast<const double*>(B), ldb, b,
               static_cast<double*>(C), ldc, st);
  } else if (Atype == C_32F && c32) {
    f2 a, b;
    ok = scalars(alpha, beta, sizeof(f2), dev, st, &a, &b) && run_c(ta, tb, m, n, k, a, A, lda, B, ldb, b, C, ldc, st);
  } else if (Atype == C_64F && c64) {
    d2 a, b;
    ok = scalars(alpha, beta, sizeof(d2), dev, st, &a, &b) && run_z(ta, tb, m, n, k, a, A, lda, B, ldb, b, C, ldc, st);
  }
  if (!ok) return fwd();
  g_emulated[kGemmEx].fetch_add(1);
  return kSuccess;
}

// ------------------------------------------------------------- legacy API
Status cublasSetKernelStream(cudaStream_t stream) {
  typedef Status Fn(cudaStream_t);
  static Fn* fn = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_legacy_mu);
    g_legacy_stream = stream;
  }
  Fn* f = real("cublasSetKernelStream", fn);
  return f ? f(stream) : kSuccess;
}

static Op legacy_op(char c) {
  switch (c) {
    case 'N': case 'n': return 0;
    case 'T': case 't': return 1;
    case 'C': case 'c': return 2;
    default: return -1;
  }
}

#define OZ_LEGACY(NAME, T, RUN, CALL_A, CALL_B)                                                            \
  void NAME(char transa, char transb, int m, int n, int k, T alpha, const T* A, int lda, const T* B, int ldb, \
            T beta, T* C, int ldc) {                                                                       \
    typedef void Fn(char, char, int, int, int, T, const T*, int, const T*, int, T, T*, int);                \
    static Fn* fn = nullptr;                                                                               \
    const Op ta = legacy_op(transa), tb = legacy_op(transb);                                               \
    if (takes(ta, tb, m, n, k) && RUN(ta, tb, m, n, k, CALL_A, A, lda, B, ldb, CALL_B, C, ldc, legacy_stream())) { \
      g_emulated[kLegacy].fetch_add(1);                                                                    \
      return;                                                                                              \
    }                                                                                                      \
    g_forwarded[kLegacy].fetch_add(1);                                                                     \
    if (Fn* f = real(#NAME, fn)) f(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);          \
  }

OZ_LEGACY(cublasSgemm, float, run_s, alpha, beta)
OZ_LEGACY(cublasDgemm, double, run_d, alpha, beta)
OZ_LEGACY(cublasCgemm, f2, run_c, alpha, beta)
OZ_LEGACY(cublasZgemm, d2, run_z, alpha, beta)

// ------------------------------------------------------------- counters
// Calls of routine r (0 S, 1 D, 2 C, 3 Z, 4 GemmEx, 5 legacy) that the
// emulation took (emulated != 0) or that went to cuBLAS.
uint64_t ozaki2_preload_calls(int r, int emulated) {
  if (r < 0 || r >= kRoutines) return 0;
  return emulated ? g_emulated[r].load() : g_forwarded[r].load();
}

}  // extern "C"
