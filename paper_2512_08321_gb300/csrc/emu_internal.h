// Internal definitions shared by the library's translation units.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/ozaki2_emu.h"

namespace emu {

constexpr int kMaxModuli = EMU_MAX_MODULI;
constexpr int kMaxLimbs = 6;        // 32-bit limbs of the CRT accumulator (P < 2^191)
constexpr int kPow2Table = 128;     // 2^s mod p for s in [0, 128)
constexpr int kChunkBits = 13;      // residue split: a' in signed 13-bit chunks
constexpr int kMaxChunks = 8;       // 8 x 13 = 104 bits > every |a'| (< 2^97)
constexpr int kSumFracBits = 15;    // row sums use ceil(|t| 2^15), Section III-B reading
constexpr int kAccuPreBits = 5;     // accurate mode: pre-scaling 2^(5 - e), magnitudes below 2^6
constexpr int16_t kExpNonfinite = EMU_EXP_NONFINITE;
// moduli-selection network
constexpr int kMlpIn = 39, kMlpHidden = 64, kMlpOut = 21, kMlpNmin = 4;
constexpr int kTcDigits = 30;       // tensor-core CRT: digit slots per part (the largest layout)
constexpr int kMlpParams = kMlpHidden * kMlpIn + kMlpHidden + kMlpHidden * kMlpHidden + kMlpHidden +
                           kMlpOut * kMlpHidden + kMlpOut;

// Per-N constants of Algorithm 1 Steps I-II and of the exact CRT, computed on
// the host (plan.cpp) and passed to kernels by value.
struct Plan {
  int N;                                  // number of moduli
  int L;                                  // 32-bit limbs of the CRT accumulator
  int R0;                                 // offset making the CRT quotient non-negative
  int sX;                                 // X = (P-1) 2^27 ~= Xtop * 2^sX (floor)
  uint64_t Xtop;
  int p[kMaxModuli];                      // moduli
  uint32_t barrett[kMaxModuli];           // floor(2^32 / p)
  uint32_t two32[kMaxModuli];             // 2^32 mod p
  float qinv[kMaxLimbs];                  // 2^(32 t) / P rounded to float (0 below the float range)
  float off128, off255, off382;           // 128, 255, 382 times sum_l q_l / p_l, rounded to float
  uint32_t w[kMaxModuli][kMaxLimbs];      // w_l = (P/p_l) q_l, little endian
  uint32_t negP[kMaxLimbs];               // 2^(32L) - P
  uint32_t K[kMaxLimbs];                  // R0*P - 128*sum_l w_l  (mod 2^(32L)), real input
  uint32_t KR[kMaxLimbs];                 // R0*P - 255*sum_l w_l (mod 2^(32L)), complex real part (D - E)
  uint32_t KI[kMaxLimbs];                 // R0*P - 382*sum_l w_l (mod 2^(32L)), complex imaginary part
  uint32_t Pw[kMaxLimbs];                 // P
  uint32_t H[kMaxLimbs];                  // (P - 1) / 2
  uint8_t pow2[kMaxModuli][kPow2Table];   // 2^s mod p_l
  int nchunk;                             // 13-bit chunks covering every |a'| (< 2^(Emax+1))
  int nchunk_accu;                        // the same for accurate-mode exponents
  float w13[kMaxModuli][kMaxChunks];      // 2^(13 t) mod p_l, symmetric, as float
  float inv_p[kMaxModuli];                // 1 / p_l rounded to float
  // tensor-core CRT (k_crt_tc.cu): the sum over moduli as an exact fp16 product of
  // the residues with balanced digits of the weights, w_l = sum_c dig[c] 2^(b c),
  // |dig| <= 2^(b-1); [0]: b = 10, [1]: b = 9
  int16_t tcdig[2][kMaxModuli][kTcDigits];
  uint16_t tcest[kMaxModuli][2];          // fp16 bits of hi, lo with hi + lo ~= w_l / P
  uint32_t tcmul[2][kTcDigits];           // 2^((b c) mod 32): digit c's shift inside its limb
  // R0 P - (bits of 1.5 * 2^23) * sum_c 2^(b c) over the digit slots of a layout
  // (mod 2^(32L)): [0] complex 14 slots b = 10, [1] complex 30 slots b = 9, [2] real 30 slots b = 10
  uint32_t tcK[3][kMaxLimbs];
  // the paper's floating-point CRT (Section II, eq. CRTaccumulation)
  double s1[kMaxModuli];                  // upper bits of w_l on the common grid 2^g
  double s2[kMaxModuli];                  // RN(w_l - s1_l)
  double wd[kMaxModuli];                  // RN(w_l)
  double Ph, Pl;                          // P = Ph + Pl, Ph = RN(P), Pl = RN(P - Ph)
};

// Host: build (and cache) the plan of N moduli; nullptr when N is out of range.
const Plan* get_plan(int N);
int plan_exponent(const Plan& pl, uint64_t S);
int plan_exponent_accu(const Plan& pl, uint64_t M);

// Device status word helpers (api.cu).
unsigned int* device_status_ptr();

// Launchers (one per translation unit).
cudaError_t launch_exponents(bool single, const void* X, int64_t rows, int64_t k,
                             int64_t rs, int64_t hs, const Plan& pl, int16_t* xout,
                             void* scratch, cudaStream_t st, bool real = false);
size_t exponents_scratch_bytes(int64_t rows);

// Accurate-mode scaling (Section III-B, eqs. mu-accu / nu-accu):
//   launch_exp_max        row maxima of ilogb (offset 2048; 0 = zero row) and Inf/NaN flags
//   launch_bound_split    7-bit ceiling planes ceil(|v| 2^(5-e)) as fp16, [planes][rows][kpad]:
//                         complex 3 planes (Re, Im, Re - Im), real 1; flagged rows are zero
//   launch_gemm_bound     exact bound products on tcgen05; atomicMax of the row maxima into
//                         Mrow[m] and of the column maxima into Ncol[n] (both zeroed by the caller);
//                         complex input parks one running sum per tile in `scratch`
//                         (bound_scratch_bytes(m, n) bytes, fewer CTAs when it is smaller)
//   launch_accu_finalize  x_r = 5 - e_r + max{E : 4^E max(M_r,1) <= (P-1)/2}
cudaError_t launch_exp_max(bool single, bool real, const void* X, int64_t rows, int64_t k, int64_t rs, int64_t hs,
                           int* emax, unsigned int* flag, cudaStream_t st);
cudaError_t launch_bound_split(bool single, bool real, const void* X, int64_t rows, int64_t k, int64_t rs,
                               int64_t hs, const int* emax, const unsigned int* flag, int64_t kpad, void* planes,
                               cudaStream_t st);
cudaError_t launch_gemm_bound(int64_t m, int64_t n, int64_t kpad, bool real, const void* planesA,
                              const void* planesB, unsigned int* Mrow, unsigned int* Ncol, void* scratch,
                              size_t scratch_bytes, unsigned int* status, cudaStream_t st, bool pair = false);
size_t bound_scratch_bytes(int64_t m, int64_t n);
cudaError_t launch_accu_finalize(int64_t rows, const int* emax, const unsigned int* flag, const unsigned int* Mb,
                                 const Plan& pl, int16_t* xout, cudaStream_t st);

// Modulus-loop schedule of the residue-product kernel (k_gemm_f16.cu): the
// order of its (tile, job pair) units, which jobs share a unit, and the k
// direction.  None of it changes a result.
struct GemmSchedule {
  int order = 0;          // 0 modulus outer, 1 tile outer, 2 column bands (modulus outer inside a band)
  int pairing = 0;        // 0 adjacent jobs, 1 halves (p, p + ceil(J/2)), 2 component-major (all D, E, F)
  int kalt = 0;           // 1: a CTA's odd units run their k chunks in descending order
  int band_cols = 8192;   // columns per band for order 2 (the paper's n-block), a multiple of 128
  int cta_pair = 0;       // 1: 256 x 256 tiles on SM pairs (cta_group::2); 0: 128 x tile_n tiles on one SM
  bool valid() const {
    return order >= 0 && order <= 2 && pairing >= 0 && pairing <= 2 && (kalt == 0 || kalt == 1) &&
           band_cols >= 128 && band_cols <= 65536 && band_cols % 128 == 0 && (cta_pair == 0 || cta_pair == 1);
  }
};

// Launch-configuration knobs of one GEMM (process defaults, autotuned per shape bucket).
struct Tune {
  int tile_n = 256;      // residue products: output rows per tile (64, 128, 256)
  int group = 16;        // residue products: tile rasterisation group
  int chunk_k = 960;     // residue products: k between in-TMEM reductions (64..960; 960 the largest
                         // exact one: 960 products of at most 2^14 plus a residue stay below 2^24)
  int crt_rows = 4;      // CRT: rows per thread (1, 2, 4) of the CUDA-core kernel
  int crt_engine = 1;    // CRT: 1 the sum over moduli on the tensor cores, 0 on the CUDA cores
  int split_elems = 4;   // split: entries per thread (2, 4)
  int nblock = 0;        // output columns per block (0: automatic, by workspace size)
  int overlap = -1;      // split and CRT of neighbouring column blocks beside the residue products:
                         // 1 on, 0 off, -1 (default) on for the real GEMMs only
  GemmSchedule sched;    // residue products: modulus-loop schedule
  int bound_pair = 1;    // accurate-mode bound products: 1 on SM pairs (cta_group::2) where the device
                         // can run them, 0 on one SM
};

// Tuning of a call of this shape: the autotuned entry of its (dtype, N, shape
// bucket) if one exists, else the process defaults (tune.cu).  dtype is an
// EMU_DTYPE_* code.
Tune tune_for(int dtype, int N, int64_t m, int64_t n, int64_t k);
void set_default_tuning(int key, int value);

cudaError_t launch_split(bool single, bool conj, const void* X, int64_t rows, int64_t k,
                         int64_t rs, int64_t hs, const Plan& pl, const int16_t* xexp,
                         bool fp16, int64_t kpad, void* planes, cudaStream_t st, int elems = 4,
                         bool real = false, int64_t plane_rows = 0);

cudaError_t launch_gemm_i8(int64_t m, int64_t n, int64_t kpad, const Plan& pl,
                           const int8_t* planesA, const int8_t* planesB, int8_t* res,
                           int64_t ldr, cudaStream_t st, int ppm = 3);

// true when the SM-pair residue-product kernel (GemmSchedule::cta_pair) can run on this device
bool gemm_pair_supported();

cudaError_t launch_gemm_f16(int64_t m, int64_t n, int64_t kpad, const Plan& pl,
                            const void* planesA, const void* planesB, int8_t* res,
                            int64_t ldr, int chunk_k, unsigned int* status, cudaStream_t st,
                            int tile_n = 256, int group = 16, int ppm = 3, int64_t a_plane_rows = 0,
                            int64_t rcap = 0, const GemmSchedule& sched = GemmSchedule());

cudaError_t launch_crt(bool single, int64_t m, int64_t n, const Plan& pl,
                       const int8_t* res, int64_t ldr, const int16_t* x, const int16_t* y,
                       double ar, double ai, double br, double bi,
                       void* C, int64_t ldc, cudaStream_t st, int rows_per_thread = 4, bool real = false,
                       bool robust = false);

// The same CRT with its sum over moduli on the tensor cores (k_crt_tc.cu): bit-identical
// results.  Each block holds TMEM for its whole run, so it must not run beside the residue
// products (which take all of an SM's TMEM); status receives EMU_ERR_TIMEOUT if a wait expires.
cudaError_t launch_crt_tc(bool single, int64_t m, int64_t n, const Plan& pl, const int8_t* res, int64_t ldr,
                          const int16_t* x, const int16_t* y, double ar, double ai, double br, double bi, void* C,
                          int64_t ldc, cudaStream_t st, bool real, bool robust, unsigned int* status);

cudaError_t launch_crt_fp(bool single, int64_t m, int64_t n, const Plan& pl, const int8_t* res, int64_t ldr,
                          const int16_t* x, const int16_t* y, double ar, double ai, double br, double bi, void* C,
                          int64_t ldc, cudaStream_t st, bool real = false);
extern int g_crt_mode;   // 0: exact integer CRT, 1: the paper's floating-point CRT
extern int g_scaling;    // EMU_SCALING_FAST or EMU_SCALING_ACCURATE

cudaError_t launch_bounded_wait_selftest(int64_t limit_cycles, unsigned int* status,
                                         cudaStream_t st);

// ------------------------------------------------------------- grouped launches
// A segment is the rows of op(A) (or the columns of op(B)) of one problem of a
// grouped call; a block of a grouped launch finds its segment by binary search
// on block_begin.
struct ExpSeg {
  const void* X;
  int64_t rows, k, rs, hs;
  int16_t* xout;
  int* emax;
  unsigned int* flag;
  unsigned long long* sum;
  long long block_begin;     // first block of this segment in the flattened grid
  int hchunks;               // blocks along h per row block
  int rows_contig;
};
struct SplitSeg {
  const void* X;
  int64_t rows, k, rs, hs;
  const int16_t* xexp;
  void* planes;
  int64_t kpad;
  long long block_begin;
  int htiles;
  int conj;
  int rows_contig;
};
struct CrtProb {
  const int8_t* res;
  int64_t ldr, m, n, ldc;
  const int16_t* x;
  const int16_t* y;
  void* C;
  double ar, ai, br, bi;
  long long block_begin;
  int iblocks;
  int flags;                // alpha/beta case (crt_common.cuh: kCrtPlain, kCrtBeta), set by crt_prob_blocks
};
// block counts of one segment/problem in the grouped launches
long long exp_seg_blocks(ExpSeg& s);       // sets hchunks, rows_contig; returns blocks
long long split_seg_blocks(SplitSeg& s);   // sets htiles, rows_contig
long long crt_prob_blocks(CrtProb& c);     // sets iblocks
// block_seg: the segment of every block of the flattened grid (no search per block)
cudaError_t launch_exponents_grouped(bool single, const ExpSeg* segs_dev, const int* block_seg, int nseg, long long blocks,
                                     const long long* row_begin_dev, long long total_rows, const Plan& pl,
                                     cudaStream_t st);
cudaError_t launch_split_grouped(bool single, bool fp16, const SplitSeg* segs_dev, const int* block_seg, int nseg,
                                 long long blocks,
                                 const Plan& pl, cudaStream_t st);
cudaError_t launch_crt_grouped(bool single, const CrtProb* probs_dev, int nprob, long long blocks, const Plan& pl,
                               cudaStream_t st);
// the grouped CRT on the tensor cores (k_crt_tc.cu): items of 128 rows
long long crt_tc_prob_items(CrtProb& c);   // sets iblocks (128-row blocks) and flags; returns items
cudaError_t launch_crt_tc_grouped(bool single, const CrtProb* probs_dev, int nprob, long long items, const Plan& pl,
                                  unsigned int* status, cudaStream_t st, bool prepare_only = false);
size_t group_problem_bytes();
bool fill_group_problem(void* desc, int64_t m, int64_t n, int64_t kpad, int N, const void* planesA,
                        const void* planesB, int8_t* res, int64_t ldr, int chunk_k, int group, int tile_n,
                        long long* unit_begin, const GemmSchedule& sched = GemmSchedule());
cudaError_t launch_gemm_f16_grouped(const void* probs_dev, int count, long long total_units, const Plan& pl,
                                    unsigned int* status, cudaStream_t st);
cudaError_t prepare_gemm_f16();
// moduli-selection network (mlp.cu) and its features (k_scale.cu)
cudaError_t launch_mlp_forward(const float* th, const float* X, int batch, float* Z, cudaStream_t st);
cudaError_t launch_mlp_backward(const float* th, const float* X, const float* Y, int batch, float* grad,
                                float* loss, cudaStream_t st);
cudaError_t launch_mlp_adam(float* th, const float* g, float* m, float* v, int step, float lr, cudaStream_t st);
cudaError_t launch_mlp_choose(const float* th, const float* x, float threshold, int* out, cudaStream_t st);
// The N-independent part of the exponents (passes 1 and 2: row maxima, flags,
// quantised sums of squares) into a scratch of exponents_scratch_bytes(rows),
// with the moduli-selection histogram when hist is given (complex only); the
// exponents of a plan then need only launch_exponent_finalize.
cudaError_t launch_exponent_sums(bool single, bool real, const void* X, int64_t rows, int64_t k, int64_t rs,
                                 int64_t hs, void* scratch, unsigned long long* hist, cudaStream_t st);
cudaError_t launch_exponent_finalize(int64_t rows, void* scratch, const Plan& pl, int16_t* xout, cudaStream_t st);
// features of the moduli-selection network; the scratch (features_scratch_bytes(m, n))
// keeps A's exponent sums and then B's
size_t features_scratch_bytes(int64_t m, int64_t n);
cudaError_t launch_features(bool single, const void* A, int64_t m, int64_t rsa, int64_t hsa, const void* B,
                            int64_t n, int64_t rsb, int64_t hsb, int64_t k, double target, float* feat,
                            void* scratch, cudaStream_t st);
extern int g_f16_group;

// Block hooks of a host-buffer call (host.cu).  The output columns are
// processed in blocks of at most `nb` (0: the library's choice), the first of
// `nb0` (when nonzero); before a
// block's columns of B (and of C, when beta != 0) are touched the caller's
// stream is made to wait for them (`wait_inputs`); once the block's CRT is
// enqueued `output_done` is told its columns of C are final, and
// `products_start` is called just before each launch of residue products (so
// that copies can be placed beside those).  A arrives in blocks of `mb` rows
// (a multiple of 16; 0: all of A before the call): `wait_rows` makes the
// stream wait for rows i0.. of op(A).  In fast mode on the tcgen05 engine the
// first column block is computed one block of rows at a time as A arrives;
// otherwise all of A is waited for first.
struct BlockHooks {
  int64_t nb, mb;
  int64_t nb0;              // width of the first column block (0: nb)
  void* c_dev;              // columns below c_dev_end are written here (same ldc) instead of into C
  int64_t c_dev_end;
  void* ctx;
  emu_status_t (*wait_inputs)(void* ctx, int64_t j0, int64_t nj, cudaStream_t st);
  emu_status_t (*wait_rows)(void* ctx, int64_t i0, int64_t mi, cudaStream_t st);
  emu_status_t (*output_done)(void* ctx, int64_t j0, int64_t nj, cudaStream_t st);
  emu_status_t (*products_start)(void* ctx, cudaStream_t st);
};

// GEMM entry shared by the device- and host-buffer calls (api.cu).
emu_status_t run_gemm(bool single, bool real, emu_op_t ta, emu_op_t tb, int64_t m, int64_t n, int64_t k, double ar,
                      double ai, const void* A, int64_t lda, const void* B, int64_t ldb, double br, double bi, void* C,
                      int64_t ldc, int N, void* stream, const BlockHooks* hooks = nullptr);
emu_status_t check_gemm_args(emu_op_t ta, emu_op_t tb, int64_t m, int64_t n, int64_t k, int64_t lda, int64_t ldb,
                             int64_t ldc, int N);
emu_status_t set_bad_param(int idx);
// the checks of the stage entry points (operands, sizes, leading dimensions, N, k; no C)
emu_status_t check_stage_args(emu_op_t ta, emu_op_t tb, int64_t m, int64_t n, int64_t k, int64_t lda, int64_t ldb,
                              int N);
emu_status_t get_staging(size_t need, char** out);

// Launch accounting (api.cu): launchers report each kernel they enqueue.
void count_launches(int n);

inline int64_t round_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

// Kernels that may run beside the residue GEMM ask for the largest shared-memory
// carveout, the configuration an SM holding a residue-GEMM block already has.
template <typename K>
inline void max_shared_carveout(K* kern) {
  if (cudaFuncSetAttribute(reinterpret_cast<const void*>(kern), cudaFuncAttributePreferredSharedMemoryCarveout,
                           static_cast<int>(cudaSharedmemCarveoutMaxShared)) != cudaSuccess)
    cudaGetLastError();
}

}  // namespace emu
