/*
 * ozaki2_emu.h -- C ABI of the GB300 (sm_103a) Ozaki-II emulation of complex
 * matrix multiplication (ZGEMM / CGEMM) through the Chinese Remainder Theorem,
 * with the real analogues (DGEMM / SGEMM) of the paper's supplemental study.
 *
 * Method (arXiv 2512.08321): Algorithm 1 (Ozaki-II outline, Section II) with
 * the Karatsuba complex product (Section III-A, eq. karatsuba) and fast-mode
 * scaling vectors (Section III-B, eqs. mu-fast / nu-fast):
 *   1. per-row / per-column power-of-two scaling exponents          (Step III)
 *   2. truncation to integers and split into symmetric residues
 *      modulo N pairwise-coprime moduli p_l <= 256                  (Steps IV, V-i, V-ii)
 *   3. three residue products D, E, F per modulus, reduced mod p_l  (Steps V-iii, V-iv)
 *   4. CRT reconstruction, inverse scaling, alpha/beta              (Steps V-v, V-vi, VI)
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Matrices are column-major, as in BLAS.  op(X) is X (EMU_OP_N), X^T
 *   (EMU_OP_T) or X^H (EMU_OP_C).  op(A) is m x k, op(B) is k x n, C is m x n.
 * - A, B, C and every buffer argument named "device" are device pointers the
 *   caller owns; the library never frees them.  alpha and beta point to host
 *   memory holding {re, im}.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   All work is enqueued on it; calls return without synchronising.  Argument
 *   errors are returned synchronously and nothing is enqueued.  Launch
 *   failures return EMU_ERR_CUDA.  Errors detected on the device (a bounded
 *   wait that expired) are recorded in a device status word that
 *   emu_stream_status() reads.
 * - beta == 0 means C is not read.  m, n or k == 0 is a quick return (with
 *   k == 0, C becomes beta*C, or 0 when beta == 0).
 * - num_moduli N lies in [EMU_MIN_MODULI, EMU_MAX_MODULI]; k <= 2^17 (Section
 *   II: the bound under which INT8 products accumulate without error).
 * - The result equals, bit for bit, the round-to-nearest-even binary64 value
 *   of the exact CRT reconstruction c'_ij scaled by 2^-(x_i + y_j) (then
 *   alpha/beta in a fixed fma sequence; complex64 output rounds that binary64
 *   value once more).  Rows of op(A) / columns of op(B) holding Inf or NaN
 *   produce NaN in the matching row / column of the result.
 */
#ifndef OZAKI2_EMU_H
#define OZAKI2_EMU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  EMU_OK = 0,
  EMU_ERR_INVALID_ARG = 1,   /* emu_last_bad_param() gives the 1-based position */
  EMU_ERR_K_TOO_LARGE = 2,   /* k > 2^17 (Section II) */
  EMU_ERR_MODULI_RANGE = 3,  /* num_moduli outside [EMU_MIN_MODULI, EMU_MAX_MODULI] */
  EMU_ERR_ALLOC = 4,         /* workspace allocation failed */
  EMU_ERR_CUDA = 5,          /* a CUDA runtime call or launch failed */
  EMU_ERR_TIMEOUT = 6,       /* a bounded device-side wait expired */
  EMU_ERR_UNSUPPORTED = 7,   /* no GPU / not an sm_103 device / feature not built */
  EMU_ERR_WORKSPACE = 8,     /* caller workspace smaller than emu_workspace_bytes() */
  EMU_ERR_SIZE_LIMIT = 9     /* m or n above EMU_STATIC_EXP_MAX_ROWS (allocation-free entry point) */
} emu_status_t;

typedef enum { EMU_OP_N = 0, EMU_OP_T = 1, EMU_OP_C = 2 } emu_op_t;

/* Engine of the residue products (Step V-iii).  Both are exact and give
 * identical results:
 *   EMU_ENGINE_F16: tcgen05.mma kind::f16 with TMEM accumulators.  Residues
 *     |r| <= 128 are exact in fp16; the FP32 accumulator is reduced modulo p
 *     in TMEM every `chunk` k so every partial sum stays an integer < 2^24.
 *   EMU_ENGINE_I8: warp-level mma.sync s8 x s8 -> s32 (the INT8 path sm_103a
 *     offers; tcgen05 kind::i8 is not available on this target). */
typedef enum { EMU_ENGINE_AUTO = 0, EMU_ENGINE_F16 = 1, EMU_ENGINE_I8 = 2 } emu_engine_t;

#define EMU_MIN_MODULI 2
#define EMU_MAX_MODULI 24
#define EMU_MAX_K (1 << 17)
#define EMU_EXP_NONFINITE (-32768) /* int16 scaling exponent of a flagged row/column */

/* ---------------------------------------------------------------- GEMMs --- */

/* C = alpha * op(A) op(B) + beta * C, complex128 (double2 interleaved {re,im}).
 * A: device, lda >= max(1, rows of stored A); B: device, ldb likewise;
 * C: device, ldc >= max(1, m).  alpha, beta: host double[2]. */
emu_status_t emu_zgemm(emu_op_t transa, emu_op_t transb, int64_t m, int64_t n, int64_t k,
                       const double* alpha, const void* A, int64_t lda,
                       const void* B, int64_t ldb, const double* beta,
                       void* C, int64_t ldc, int num_moduli, void* stream);

/* complex64 analogue (float2 data, host float[2] alpha/beta); the CRT is the
 * same exact integer reconstruction, the output is rounded to binary32. */
emu_status_t emu_cgemm(emu_op_t transa, emu_op_t transb, int64_t m, int64_t n, int64_t k,
                       const float* alpha, const void* A, int64_t lda,
                       const void* B, int64_t ldb, const float* beta,
                       void* C, int64_t ldc, int num_moduli, void* stream);

/* Real analogues: Algorithm 1 as Section II states it for real matrices (the
 * scheme of the real-valued comparison of Section IV-C), one residue product per modulus
 * (E'_l = mod(A'_l B'_l, p_l)), fast-mode scaling on the k entries of each
 * row of op(A) / column of op(B), the same exact CRT.  C = alpha op(A) op(B)
 * + beta C with host scalars alpha and beta; with (alpha, beta) != (1, 0) the
 * result is fma(beta, C, RN(alpha o)) in binary64 (beta = 0: RN(alpha o)),
 * then rounded once to binary32 for emu_sgemm.  EMU_OP_C equals EMU_OP_T. */
emu_status_t emu_dgemm(emu_op_t transa, emu_op_t transb, int64_t m, int64_t n, int64_t k,
                       const double* alpha, const double* A, int64_t lda,
                       const double* B, int64_t ldb, const double* beta,
                       double* C, int64_t ldc, int num_moduli, void* stream);
emu_status_t emu_sgemm(emu_op_t transa, emu_op_t transb, int64_t m, int64_t n, int64_t k,
                       const float* alpha, const float* A, int64_t lda,
                       const float* B, int64_t ldb, const float* beta,
                       float* C, int64_t ldc, int num_moduli, void* stream);

/* Host-buffer forms of the four GEMMs: A, B and C are in host memory (same
 * arguments, layouts and results as the device forms; alpha/beta as there).
 * The inputs go through a library-owned device staging buffer in blocks: the
 * output columns in blocks, and the rows of op(A) in blocks (each about an
 * eighth, a multiple of 256 and at least 2048; one block when the dimension is
 * at most 2048; narrower column blocks when column blocking below asks for
 * them).  A library-owned side stream brings op(B)'s (and, for pageable C with
 * beta != 0, C's) first column block, then op(A) block of rows by block of
 * rows, then the other column blocks -- contiguous blocks by the DMA engines,
 * strided ones from pinned memory by a copy kernel -- while the caller's
 * stream computes the first column block one block of rows at a time (fast
 * scaling, tcgen05 engine; otherwise after all of A) and the other column
 * blocks as their columns arrive.  Pinned or registered C is read (beta != 0)
 * and written in place by the CRT kernel through its device address; pageable
 * C goes through a device copy and comes back after the last block.  Only the
 * m x n entries of C are written (rows beyond m of a column are left as they
 * are).  Asynchronous on `stream` like the device forms: the host buffers must
 * stay valid and untouched until the stream reaches the end of the call.
 * Calls on one device share the staging buffer, so each host-buffer call waits
 * on the device for the previous one to finish, whatever stream it was issued
 * on. */
emu_status_t emu_zgemm_host(emu_op_t transa, emu_op_t transb, int64_t m, int64_t n, int64_t k,
                            const double* alpha, const void* A, int64_t lda, const void* B, int64_t ldb,
                            const double* beta, void* C, int64_t ldc, int num_moduli, void* stream);
emu_status_t emu_cgemm_host(emu_op_t transa, emu_op_t transb, int64_t m, int64_t n, int64_t k,
                            const float* alpha, const void* A, int64_t lda, const void* B, int64_t ldb,
                            const float* beta, void* C, int64_t ldc, int num_moduli, void* stream);
emu_status_t emu_dgemm_host(emu_op_t transa, emu_op_t transb, int64_t m, int64_t n, int64_t k,
                            const double* alpha, const double* A, int64_t lda, const double* B, int64_t ldb,
                            const double* beta, double* C, int64_t ldc, int num_moduli, void* stream);
emu_status_t emu_sgemm_host(emu_op_t transa, emu_op_t transb, int64_t m, int64_t n, int64_t k,
                            const float* alpha, const float* A, int64_t lda, const float* B, int64_t ldb,
                            const float* beta, float* C, int64_t ldc, int num_moduli, void* stream);

/* Trace of host-buffer calls (for profiling the pipeline above).  While
 * enabled, each host-buffer call records timing events at its steps, on the
 * caller's stream (EMU_TRACE_START; EMU_TRACE_BLOCK_START: a column block's
 * inputs are in and its computation starts; EMU_TRACE_BLOCK_CRT: its CRT is
 * done; EMU_TRACE_END) and on the side stream (EMU_TRACE_A_IN: a block of rows
 * of op(A) has arrived; EMU_TRACE_B_IN: a column block's columns of B and C
 * have arrived; EMU_TRACE_C_OUT: pageable C is back), up to
 * EMU_TRACE_MAX
 * events of the latest call; enabling clears the record.
 * emu_host_trace_read waits for those events, writes up to `cap` pairs
 * (label, milliseconds after EMU_TRACE_START) in recording order and returns
 * how many it wrote, or -1 on a CUDA error. */
#define EMU_TRACE_START 0
#define EMU_TRACE_A_IN 1
#define EMU_TRACE_B_IN 2
#define EMU_TRACE_BLOCK_START 3
#define EMU_TRACE_BLOCK_CRT 4
#define EMU_TRACE_C_OUT 5
#define EMU_TRACE_END 6
#define EMU_TRACE_MAX 64
emu_status_t emu_host_trace_enable(int on);
int emu_host_trace_read(int* labels, float* ms, int cap);

/* Element-type codes of emu_workspace_bytes and emu_autotune_gemm. */
#define EMU_DTYPE_Z 0   /* complex128 */
#define EMU_DTYPE_C 1   /* complex64 */
#define EMU_DTYPE_D 2   /* float64 */
#define EMU_DTYPE_S 3   /* float32 */

/* Column blocking (all four GEMMs).  The output columns can be processed in
 * blocks of nb: the exponents and residue planes of op(A) are formed once,
 * those of op(B), the residue products and the CRT once per block of nb
 * columns of op(B) and C (the paper's n-blocking, Section III-A).  Results
 * are bit-identical for every nb, since each scaling exponent depends on one
 * row or one column only.  nb is the EMU_TUNE_NBLOCK setting when nonzero;
 * otherwise n when the whole workspace (emu_workspace_bytes) fits -- in the
 * caller's workspace if one is set, else in the library's workspace plus the
 * device's free memory less 256 MiB -- and else the widest multiple of 128
 * columns that fits. */

/* --------------------------------------------------------- grouped GEMMs ---
 * Many complex GEMMs of uneven shapes on one moduli count.  Every phase of
 * the method (Algorithm 1 Steps III-VI, Karatsuba of Section III-A) runs as
 * ONE persistent launch over all problems; the sequence is captured once in
 * a CUDA graph.  Problem i: C_i = alpha_i op(A_i) op(B_i) + beta_i C_i with the
 * per-problem arguments of emu_zgemm taken from the arrays (host arrays of
 * length count; alpha and beta hold 2*count doubles {re, im}, also for
 * complex64).  Problems with m_i = 0 or n_i = 0 are skipped.  The results are
 * bit-identical to count separate emu_zgemm/emu_cgemm calls. */
typedef struct emu_grouped_s* emu_grouped_t;

/* Build a grouped plan: workspace (cudaMalloc, owned by the plan), device
 * descriptor tables and the CUDA graph.  tile_n: rows of op(A) per tile of the
 * residue-product launch (64, 128 or 256 for every problem), or
 * EMU_GROUPED_TILE_PER_PROBLEM for each problem's own width from its row
 * count (the one launch mixes them), or 0 to let the autotuner time these four
 * choices on this problem set (the choice is remembered per problem-set
 * signature, and kept in the file named by EMU_AUTOTUNE_CACHE if set).  The
 * CRT phase uses the engine EMU_TUNE_CRT_ENGINE names at creation.
 * Synchronous; returns EMU_ERR_INVALID_ARG / EMU_ERR_K_TOO_LARGE /
 * EMU_ERR_MODULI_RANGE as emu_zgemm would for any problem. */
#define EMU_GROUPED_TILE_PER_PROBLEM (-1)
emu_status_t emu_grouped_create(int is_single, int count, const emu_op_t* transa, const emu_op_t* transb,
                                const int64_t* m, const int64_t* n, const int64_t* k, const double* alpha,
                                const void* const* A, const int64_t* lda, const void* const* B,
                                const int64_t* ldb, const double* beta, void* const* C, const int64_t* ldc,
                                int num_moduli, int tile_n, emu_grouped_t* plan);
/* Replay the plan's graph on `stream` (asynchronous).  The matrices are read
 * and written at the addresses given at creation. */
emu_status_t emu_grouped_run(emu_grouped_t plan, void* stream);
/* Tile width the plan uses (EMU_GROUPED_TILE_PER_PROBLEM for per-problem
 * widths), and the number of kernels one replay launches. */
int emu_grouped_tile(emu_grouped_t plan);
int emu_grouped_kernels(emu_grouped_t plan);
/* Diagnostic: run the plan's four phases once on `stream` outside the graph,
 * with events between them, synchronise, and store the milliseconds of the
 * exponent, split, residue-product and CRT launches in ms[0..3]. */
emu_status_t emu_grouped_phase_times(emu_grouped_t plan, float* ms, void* stream);
/* Free the plan (waits for its work to finish). */
emu_status_t emu_grouped_destroy(emu_grouped_t plan);

/* One-shot grouped ZGEMM / CGEMM: create (autotuned), run on `stream`,
 * synchronise, destroy. */
emu_status_t emu_zgemm_grouped(int count, const emu_op_t* transa, const emu_op_t* transb,
                               const int64_t* m, const int64_t* n, const int64_t* k, const double* alpha,
                               const void* const* A, const int64_t* lda, const void* const* B,
                               const int64_t* ldb, const double* beta, void* const* C, const int64_t* ldc,
                               int num_moduli, void* stream);
emu_status_t emu_cgemm_grouped(int count, const emu_op_t* transa, const emu_op_t* transb,
                               const int64_t* m, const int64_t* n, const int64_t* k, const double* alpha,
                               const void* const* A, const int64_t* lda, const void* const* B,
                               const int64_t* ldb, const double* beta, void* const* C, const int64_t* ldc,
                               int num_moduli, void* stream);

/* ----------------------------------------------------- moduli selection ---
 * The paper chooses N from measured accuracy bands (Section IV-A).  This
 * library adds (1) an a priori rule and (2) a small learned network that
 * predicts, from features of A and B and the requested accuracy, the fewest
 * moduli that meet it; the network's weights are loaded by the caller. */

/* C = alpha op(A) op(B) + beta C with N chosen for the normalised accuracy
 * target_err (max_ij |error| / ((|A_R|+|A_I|)(|B_R|+|B_I|))_ij): the loaded
 * network's choice, else emu_moduli_apriori.  With a network loaded this
 * synchronises `stream` once (the chosen N decides the launch configuration).
 * *n_used (may be NULL) receives N. */
emu_status_t emu_zgemm_tol(emu_op_t transa, emu_op_t transb, int64_t m, int64_t n, int64_t k,
                           const double* alpha, const void* A, int64_t lda, const void* B, int64_t ldb,
                           const double* beta, void* C, int64_t ldc, double target_err, int* n_used,
                           void* stream);
emu_status_t emu_cgemm_tol(emu_op_t transa, emu_op_t transb, int64_t m, int64_t n, int64_t k,
                           const float* alpha, const void* A, int64_t lda, const void* B, int64_t ldb,
                           const float* beta, void* C, int64_t ldc, double target_err, int* n_used,
                           void* stream);

/* A priori rule: the smallest N in [EMU_MIN_MODULI, EMU_MAX_MODULI] with
 * 2^(1 - (P'_fast(N) - log2(8k)/2)) <= target, P'_fast = log2(P-1)/2 - 1.5
 * (the fast-mode bound of Section III-B for rows of equal magnitude); host only. */
int emu_moduli_apriori(int is_single, int64_t k, double target);

/* Network: 39 features -> 64 -> 64 -> 21 logits (ReLU), logit t for N = 4 + t.
 * Parameter vector (float): W1 (64x39 row major), b1, W2 (64x64), b2, W3 (21x64), b3. */
int emu_mlp_param_count(void);
/* Load (host pointer, count = emu_mlp_param_count()) or unload (NULL) the weights
 * emu_zgemm_tol uses on the current device. */
emu_status_t emu_mlp_set_weights(const float* params, int count);
/* Features (39 floats, device) of op(A), op(B) and the target: 16-bin
 * histograms of exponent spans of A-hat rows and B-hat columns, mean/max of
 * 0.5 log2 of the quantised row sums, log2(k)/17, -log10(target)/16, dtype. */
emu_status_t emu_moduli_features(int is_single, emu_op_t transa, emu_op_t transb, int64_t m, int64_t n,
                                 int64_t k, const void* A, int64_t lda, const void* B, int64_t ldb,
                                 double target, float* features, void* stream);
/* Training and inference kernels (all pointers device):
 * forward: logits[batch][21] of X[batch][39];
 * backward: grad (parameter-sized) and *loss of the mean binary cross-entropy
 *   against Y[batch][21] (zeroed first, then accumulated);
 * adam: one Adam step (beta 0.9/0.999, eps 1e-8, bias-corrected; step >= 1);
 * choose: smallest N whose probability, and that of every larger N, is >=
 *   threshold, or -1, into *n_out. */
emu_status_t emu_mlp_forward(const float* theta, const float* X, int batch, float* logits, void* stream);
emu_status_t emu_mlp_backward(const float* theta, const float* X, const float* Y, int batch, float* grad,
                              float* loss, void* stream);
emu_status_t emu_mlp_adam(float* theta, const float* grad, float* m, float* v, int step, float lr, void* stream);
emu_status_t emu_mlp_choose(const float* theta, const float* features, float threshold, int* n_out,
                            void* stream);

/* ------------------------------------------------------------ workspace --- */

/* Bytes of device workspace one unblocked call of the given shape needs
 * (dtype: an EMU_DTYPE_* code; 0 and 1 keep their old meaning of ZGEMM and
 * CGEMM).  Column blocking needs less.  0 on invalid arguments. */
size_t emu_workspace_bytes(int dtype, int64_t m, int64_t n, int64_t k, int num_moduli);

/* Use caller-owned device memory [ptr, ptr+bytes) as the workspace of this
 * device (the current device) for subsequent calls; NULL/0 returns to the
 * library-managed workspace (cudaMalloc'd, grown on demand, freed at exit).
 * Calls sharing one workspace must be ordered on one stream. */
emu_status_t emu_set_workspace(void* ptr, size_t bytes);

/* Select the residue-product engine (default EMU_ENGINE_AUTO = F16) and the
 * k chunk after which the F16 engine reduces its accumulator (multiple of 64,
 * 64..960; 0 keeps the default 960, the largest that keeps the FP32 sums
 * exact). */
emu_status_t emu_set_engine(emu_engine_t engine, int chunk_k);

/* Launch-configuration knobs of emu_zgemm/cgemm/dgemm/sgemm (no effect on results):
 *   EMU_TUNE_TILE_N      residue products: rows of op(A) per tile, 64/128/256
 *   EMU_TUNE_GROUP       residue products: tile rasterisation group, 1..64
 *   EMU_TUNE_CHUNK_K     residue products: k between in-TMEM reductions, 64..960, multiple of 64
 *   EMU_TUNE_CRT_ROWS    CRT: rows per thread, 1/2/4
 *   EMU_TUNE_SPLIT_ELEMS residue split: entries per thread, 2/4
 *   EMU_TUNE_NBLOCK      output columns per block, 0 (automatic) or a multiple of 128;
 *                        a process setting only, never autotuned
 *   EMU_TUNE_OVERLAP     1: device-buffer GEMMs on the tcgen05 engine with
 *                        n >= 2048 run in column blocks (the
 *                        EMU_TUNE_NBLOCK width, else about eight blocks of a
 *                        multiple of 256 columns, at least 1024), and a
 *                        library-owned stream forms the next block's exponents
 *                        and planes and the previous block's CRT beside each
 *                        block's residue products (planes of B and residues
 *                        double-buffered; in accurate scaling the bound
 *                        products give every exponent first); 0: one phase
 *                        after another; -1
 *                        (default): 1 for emu_dgemm/emu_sgemm, 0 for the complex
 *                        GEMMs.  On a power-capped GB300 the residue products
 *                        slow down beside the other phases: for the complex
 *                        GEMMs by about what the overlap hides, for the real
 *                        ones (a third of the products per output) by less.  A
 *                        process setting only, never autotuned
 *   EMU_TUNE_ORDER       residue products, modulus-loop schedule: order of the
 *                        (tile, job pair) units.  0 modulus outer (every tile of
 *                        one job pair before the next pair), 1 tile outer (every
 *                        job pair of one tile before the next tile), 2 column
 *                        bands of EMU_TUNE_BAND columns, modulus outer inside a
 *                        band (the n-blocking of Section III-A)
 *   EMU_TUNE_PAIRING     residue products: the two jobs that share a unit (and
 *                        alternate in its two accumulators).  0 adjacent jobs of
 *                        the sequence D_0 E_0 F_0 D_1 ..., 1 job p with job
 *                        p + ceil(J/2), 2 adjacent jobs of the component-major
 *                        sequence D_0 .. D_N-1 E_0 .. F_N-1 (J = 3N complex, N real)
 *   EMU_TUNE_KDIR        residue products: 0 k chunks ascending, 1 descending on
 *                        every other unit of a persistent block
 *   EMU_TUNE_BAND        columns per band for EMU_TUNE_ORDER 2, a multiple of
 *                        128 (default 8192, the paper's block)
 *   EMU_TUNE_CRT_ENGINE  CRT: 1 (default) the sum over moduli as an exact fp16
 *                        product with digits of the CRT weights on the tensor
 *                        cores, 0 limb products on the CUDA cores (also used,
 *                        whatever the setting, for a CRT running beside residue
 *                        products on the library's second stream)
 *   EMU_TUNE_CTA_PAIR    residue products: 1 tiles of 256 output columns x 256
 *                        rows on pairs of SMs (a cluster of two CTAs sharing
 *                        each MMA, cta_group::2; EMU_TUNE_TILE_N then has no
 *                        effect), 0 (default) 128-column tiles on one SM; a
 *                        device without cluster launch support refuses 1 at
 *                        call time (EMU_ERR_CUDA).  Grouped calls always use
 *                        one-SM tiles
 *   EMU_TUNE_BOUND_PAIR  accurate-mode bound products: 1 (default) tiles of 256
 *                        output columns x 256 rows on pairs of SMs
 *                        (cta_group::2; one-SM tiles on a device that cannot
 *                        run them), 0 128 x 256 tiles on one SM; a process
 *                        setting only, never autotuned
 * emu_set_tuning sets the process default; emu_autotune_gemm times the
 * candidates of every knob for one shape on synthetic data (phases timed
 * separately), and later calls whose (dtype, N, ceil(log2) of m, n, k) match
 * use the winners.  The table is kept in the file EMU_AUTOTUNE_CACHE names, if
 * set.  Tuning state is per process; emu_autotune_gemm allocates its own
 * temporary buffers (inputs, planes, residues of the shape), synchronises, and
 * frees them.  dtype is an EMU_DTYPE_* code.  best (may be NULL) receives the
 * first 5 knobs' chosen values in key order; emu_tuned_value gives any knob's
 * value that a call of the given dtype, N and shape will use (the autotuned
 * entry of its bucket, else the process default; -1 for an unknown key).
 * The autotuner searches the tile width, group and chunk, then the schedule
 * knobs 8-11 and 13 one at a time, then the CRT engine (and the CUDA-core
 * kernel's rows) and the split entries. */
#define EMU_TUNE_TILE_N 1
#define EMU_TUNE_GROUP 2
#define EMU_TUNE_CHUNK_K 3
#define EMU_TUNE_CRT_ROWS 4
#define EMU_TUNE_SPLIT_ELEMS 5
#define EMU_TUNE_NBLOCK 6
#define EMU_TUNE_OVERLAP 7
#define EMU_TUNE_ORDER 8
#define EMU_TUNE_PAIRING 9
#define EMU_TUNE_KDIR 10
#define EMU_TUNE_BAND 11
#define EMU_TUNE_CRT_ENGINE 12
#define EMU_TUNE_CTA_PAIR 13
#define EMU_TUNE_BOUND_PAIR 14
emu_status_t emu_set_tuning(int key, int value);
int emu_get_tuning(int key);
int emu_tuned_value(int dtype, int num_moduli, int64_t m, int64_t n, int64_t k, int key);
emu_status_t emu_autotune_gemm(int dtype, int64_t m, int64_t n, int64_t k, int num_moduli, int* best);
/* Forget the autotuned entries (the defaults stay). */
emu_status_t emu_autotune_clear(void);

/* CRT reconstruction used by emu_zgemm/cgemm/dgemm/sgemm and emu_stage_crt
 * (the grouped path always uses the exact one):
 *   EMU_CRT_EXACT (default): exact multi-limb integer reconstruction, result
 *     RN(c' 2^-(x+y)) with c' = A'B' exactly;
 *   EMU_CRT_PAPER_FP64: the paper's floating-point reconstruction (Section II,
 *     eq. CRTaccumulation): S1 = sum s_l1 E'_l exact, S2 = sum s_l2 E'_l, then
 *     mod(S1 + S2, P) in double-double (complex128, float64) or one double
 *     sum (complex64, float32). */
#define EMU_CRT_EXACT 0
#define EMU_CRT_PAPER_FP64 1
emu_status_t emu_set_crt_mode(int mode);

/* Scaling vectors (Algorithm 1 Step III) of emu_zgemm/cgemm/dgemm/sgemm (the
 * grouped path always uses fast mode):
 *   EMU_SCALING_FAST (default): fast mode, Section III-B eqs. mu-fast/nu-fast,
 *     the Cauchy-Schwarz bound decided exactly on quantised row sums;
 *   EMU_SCALING_ACCURATE: accurate mode, Section III-B eqs. mu-accu/nu-accu:
 *     rows of op(A) and columns of op(B) pre-scaled by 2^(5 - e) (e = ilogb of
 *     the largest |entry|), their magnitudes rounded up to integers <= 64, the
 *     bound product C-bar (complex: C-bar_I = A-bar_I B-bar_R + A-bar_R B-bar_I,
 *     C-bar_R = C-bar_I + (A-bar_R - A-bar_I)(B-bar_R - B-bar_I)) formed exactly
 *     on the tensor cores, and x_i = 5 - e_i + max{E : 4^E max(M_i, 1) <= (P-1)/2}
 *     with M_i = max_j max(C-bar_R, C-bar_I)_ij (y_j likewise over i).  The exact
 *     CRT then corrects its quotient so that |c'| up to (P-1)/2 is recovered.
 * A process setting, not per thread. */
#define EMU_SCALING_FAST 0
#define EMU_SCALING_ACCURATE 1
emu_status_t emu_set_scaling(int mode);
int emu_get_scaling(void);

/* ----------------------------------------------------- stage entry points --
 * The four phases of one emulated GEMM on caller buffers, for stage-wise
 * checking and for composing other pipelines.  is_single selects complex64
 * (1) or complex128 (0) inputs/outputs. */

/* Step III (Section III-B): int16 exponents x (m, of mu) and y (n, of nu);
 * EMU_EXP_NONFINITE marks a row/column holding Inf or NaN. */
emu_status_t emu_stage_exponents(int is_single, emu_op_t transa, emu_op_t transb,
                                 int64_t m, int64_t n, int64_t k,
                                 const void* A, int64_t lda, const void* B, int64_t ldb,
                                 int num_moduli, int16_t* x, int16_t* y, void* stream);

/* Steps IV and V-i/ii: residue planes.  planesA holds 3N planes of m rows,
 * planesB 3N planes of n rows, each row kpad elements (kpad >= k, multiple of
 * 64, zero padded); plane 3l+0 / 3l+1 / 3l+2 holds mod(a'_R), mod(a'_I) and
 * mod(mod(a'_R)+mod(a'_I)) for modulus l.  Elements are int8 (plane_fp16 = 0)
 * or the same integers as fp16 (plane_fp16 = 1). */
emu_status_t emu_stage_split(int is_single, emu_op_t transa, emu_op_t transb,
                             int64_t m, int64_t n, int64_t k,
                             const void* A, int64_t lda, const void* B, int64_t ldb,
                             int num_moduli, const int16_t* x, const int16_t* y,
                             int plane_fp16, int64_t kpad, void* planesA, void* planesB,
                             void* stream);

/* Steps V-iii/iv: for job j = 3l + c (c = 0: D, 1: E, 2: F of eq. karatsuba)
 * residues[j*n*ldr + col*ldr + row] = mod(sum_h planesA[j][row][h] *
 * planesB[j][col][h], p_l) as int8; ldr >= m, multiple of 16.  The engine
 * must match the plane element type (F16 <-> fp16 planes, I8 <-> int8). */
emu_status_t emu_stage_residue_gemm(emu_engine_t engine, int64_t m, int64_t n, int64_t kpad,
                                    int num_moduli, const void* planesA, const void* planesB,
                                    int8_t* residues, int64_t ldr, void* stream);

/* Steps V-v, V-vi, VI: C = alpha * 2^-(x_i+y_j) c'_ij + beta * C from the
 * D/E/F residues (E'_R = mod(D-E), E'_I = mod(F-D-E), then exact CRT). */
emu_status_t emu_stage_crt(int is_single, int64_t m, int64_t n, int num_moduli,
                           const int8_t* residues, int64_t ldr,
                           const int16_t* x, const int16_t* y,
                           const void* alpha, const void* beta,
                           void* C, int64_t ldc, void* stream);

/* Allocation-free variant of emu_stage_exponents (the paper has no counterpart:
 * this is a service to callers that cannot let the library allocate).
 * Callers whose device memory belongs to their own pool or caching allocator,
 * or that cannot accept the device-wide synchronisation of cudaMalloc/cudaFree,
 * get the same x and y as emu_stage_exponents, with the per-row scratch (16
 * bytes a row) taken from a fixed device array compiled into the library
 * instead of memory allocated per call.  Nothing is allocated: no cudaMalloc,
 * cudaFree or allocating library routine is called.
 * - m and n are limited to EMU_STATIC_EXP_MAX_ROWS; larger sizes return
 *   EMU_ERR_SIZE_LIMIT before any GPU work.
 * - The array (1 MiB) stays resident on every GPU that loads the library
 *   until the process exits.
 * - The first call made with a device current looks up the array's device
 *   address (cudaGetSymbolAddress) for that device; make that first call
 *   before any stream capture.  The address is kept per device together with
 *   the id of the context it belongs to; after a device reset (a new primary
 *   context, the library's module loaded again) the next call looks it up
 *   again, and that call too belongs outside any stream capture.
 * - Argument errors as in emu_stage_exponents (the same checks, the same
 *   emu_last_bad_param() positions); a NULL A, B, x or y that would be used
 *   is EMU_ERR_INVALID_ARG with position 7, 9, 12 or 13.
 * - Every call on a device shares the one array, which keeps the last call's
 *   contents; each call clears the part it uses before using it.  Calls that
 *   can overlap on the GPU (different streams, no ordering between them)
 *   race on the array and must not be issued that way. */
#define EMU_STATIC_EXP_MAX_ROWS 65536
emu_status_t emu_stage_exponents_static(int is_single, emu_op_t transa, emu_op_t transb,
                                        int64_t m, int64_t n, int64_t k,
                                        const void* A, int64_t lda, const void* B, int64_t ldb,
                                        int num_moduli, int16_t* x, int16_t* y, void* stream);

/* ------------------------------------------------------ host-side queries -- */

/* Algorithm 1 Steps I-II as computed by the library: the N moduli (greedy
 * descending pairwise coprime from 256), q_l = (P/p_l)^-1 mod p_l, P as
 * little-endian 32-bit limbs (p_limbs capacity >= 8) and the limb count L the
 * CRT uses.  Host only; no GPU needed.  Any output pointer may be NULL. */
emu_status_t emu_plan_info(int num_moduli, int32_t* moduli, int32_t* q,
                           uint32_t* p_limbs, int32_t* crt_limbs);

/* Fast-mode scaling exponent E of the library for a quantised row sum S
 * (sum of ceil(|t| 2^15)^2), i.e. the largest E with 4^E max(2^32,S) <=
 * (P-1) 2^27.  Host only. */
int emu_plan_exponent(int num_moduli, uint64_t S);

/* Accurate-mode exponent of the library for a bound-product maximum M (< 2^35):
 * the largest E with 4^E max(M, 1) <= (P-1)/2.  Host only. */
int emu_plan_exponent_accu(int num_moduli, uint64_t M);

/* 1-based index of the offending argument of the last EMU_ERR_INVALID_ARG
 * returned on this thread (0 if none). */
int emu_last_bad_param(void);

/* Reads and clears the device status word of the current device after
 * synchronising `stream`: EMU_OK or the first device-side error recorded. */
emu_status_t emu_stream_status(void* stream);

/* Launches one kernel that waits, with a bounded spin of about
 * `limit_cycles` SM cycles, on a device flag that nothing sets; the wait
 * expires and records EMU_ERR_TIMEOUT in the status word.  Exercises the
 * bounded-wait path without faulting or hanging the GPU. */
emu_status_t emu_selftest_bounded_wait(int64_t limit_cycles, void* stream);

/* Phase timing: when set, every following emu_zgemm/cgemm/dgemm/sgemm records
 * events[0..4] (cudaEvent_t passed as void*) on its stream at the start of
 * the call and after the exponent, split, residue-product and CRT phases.
 * With column blocking, events 1-3 mark the phases of the last block.
 * count must be 5, or 0 with events NULL to stop.  The caller owns the events.
 * Host state of the calling process, not per thread. */
emu_status_t emu_set_phase_events(void* const* events, int count);

/* Number of kernels this library has launched in this process so far. */
uint64_t emu_kernel_launches(void);

/* Library version string (static storage). */
const char* emu_version(void);

#ifdef __cplusplus
}
#endif

#endif /* OZAKI2_EMU_H */
