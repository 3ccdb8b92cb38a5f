/*
 * lsk.h -- C ABI of the GB300 sketching library (liblsk.so).
 *
 * Randomised sketching kernels for tall-and-skinny matrices after
 * Sobczyk & Gallopoulos, "pylspack: Parallel algorithms and data structures
 * for sketching, column subset selection, regression and leverage scores"
 * (arXiv 2203.02798).  Section, definition and algorithm numbers below refer
 * to that paper.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Every call returns LSK_OK (0) or a negative LSK_ERR_* code; on error
 *    lsk_error_string(ctx) holds a one-line description.  Argument errors are
 *    detected on the host before anything is launched.
 *  - Calls are asynchronous on the context's CUDA stream (lsk_set_stream).
 *    Errors found on the device (a rank-deficient sketch, an out-of-range
 *    CSR index, a wait that timed out) set a device flag; lsk_sync()
 *    synchronises the stream and returns that error (and clears the flag).
 *    lsk_sketch_precondition_lsq is the exception: it synchronises itself.
 *  - All matrix and vector pointers are DEVICE pointers owned by the caller.
 *    The library never frees them and keeps no reference after the call
 *    returns.  Inputs are const; outputs have the documented sizes.
 *  - Scratch memory comes from a workspace owned by the context, grown on
 *    demand (stream-ordered cudaMallocAsync) and freed by lsk_destroy.
 *  - Dense matrices are row-major (C_CONTIGUOUS, Sec. 2.1 and Sec. 5) with a
 *    row stride ld >= d (in elements).  CSR matrices (Sec. 1.3: V, J, I) are
 *    0-based with int64 row pointers and int32 column indices; column
 *    indices must lie in [0, d).  Values are float32.
 *  - Random draws are a pure function of (seed, index) through
 *    Philox-4x32-10 (Salmon et al., SC'11), so results do not depend on the
 *    launch configuration:
 *      CountSketch (Def. 3): w = Philox(ctr=(i_lo, i_hi, 0, 0), key=seed),
 *        h(i) = (w0 * r) >> 32,  sigma_i = (w1 >> 31) ? -1 : +1.
 *      Gaussian G (Alg. 3, csrcgs scaling 1/sqrt(k)): column c, row j:
 *        w = Philox(ctr=(c_lo, c_hi, 1, j >> 2), key=seed), the pair
 *        (a, b) = (w_{2p} >> 8, w_{2p+1} >> 8) with p = (j >> 1) & 1 feeds
 *        Box-Muller, u1 = (a + 1) 2^-24, u2 = b 2^-24 (exact in float32),
 *        z = sqrt(-2 ln u1) cos(2 pi u2)
 *        for even j, sin(...) for odd j;  G[j, c] = z / sqrt(k)
 *        (rounded to bfloat16, nearest-even, in LSK_PREC_BF16).
 */
#ifndef LSK_H
#define LSK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define LSK_OK                   0
#define LSK_ERR_INVALID_ARG     -1  /* bad size, null pointer, bad enum      */
#define LSK_ERR_BAD_CSR         -2  /* rowptr not monotone / colidx >= d     */
#define LSK_ERR_UNSUPPORTED     -3  /* dtype or size this build does not run */
#define LSK_ERR_RANK_DEFICIENT  -4  /* sketch R has a (near-)zero pivot      */
#define LSK_ERR_NOT_CONVERGED   -5  /* least squares did not reach its tol   */
#define LSK_ERR_OOM             -6  /* workspace allocation failed           */
#define LSK_ERR_TIMEOUT         -7  /* a bounded device-side wait gave up    */
#define LSK_ERR_CUDA            -8  /* a CUDA runtime call failed            */

/* ---- matrix descriptor ------------------------------------------------- */
#define LSK_DENSE 0
#define LSK_CSR   1
#define LSK_F32   0

typedef struct lsk_mat {
    int32_t kind;           /* LSK_DENSE or LSK_CSR                         */
    int32_t dtype;          /* LSK_F32 (the only value type of this build)  */
    int64_t n;              /* rows    (tall dimension)                     */
    int64_t d;              /* columns (skinny dimension)                   */
    int64_t ld;             /* dense: row stride in elements, >= d          */
    const void* values;     /* dense: n*ld floats; CSR: nnz floats (V)      */
    const int64_t* rowptr;  /* CSR: n+1 entries (I), rowptr[0] == 0         */
    const int32_t* colidx;  /* CSR: nnz entries (J), each in [0, d)         */
    int64_t nnz;            /* CSR: number of stored entries                */
} lsk_mat;

/* precision of the contractions (Gaussian stage, row-norm GEMM) */
#define LSK_PREC_FP32 0     /* FP32 accuracy: CUDA cores, or (the Gaussian  */
                            /* stage of a sketch with r >= 8192) the BF16   */
                            /* tensor pipe on three-term bf16 splits of G   */
                            /* and SA with FP32 accumulation                */
#define LSK_PREC_TF32 1     /* LSK_PREC_BF16 with the row-norm GEMM A B in  */
                            /* TF32: one product of A and B each rounded to */
                            /* the nearest TF32 (10 mantissa bits), FP32    */
                            /* accumulation; every other stage as BF16      */
#define LSK_PREC_BF16 2     /* tensor cores: BF16 G, split-BF16 operands,   */
                            /* FP32 accumulation                            */

typedef struct lsk_ctx lsk_ctx;

/* ---- context ----------------------------------------------------------- */
/* Create a context on CUDA device `device`, launching on `stream` (a
 * cudaStream_t; NULL = the legacy default stream).  *ctx receives the
 * handle, owned by the caller until lsk_destroy. */
int lsk_create(lsk_ctx** ctx, int device, void* stream);
/* Free the context and its workspace (synchronises its stream first). */
int lsk_destroy(lsk_ctx* ctx);
/* Change the stream later calls launch on. */
int lsk_set_stream(lsk_ctx* ctx, void* stream);
/* Synchronise the stream; return (and clear) any deferred device error. */
int lsk_sync(lsk_ctx* ctx);
/* Detail of the last error on this context (never NULL). */
const char* lsk_error_string(const lsk_ctx* ctx);
/* Bytes currently held by the context's workspace. */
size_t lsk_workspace_bytes(const lsk_ctx* ctx);
/* Grow the workspace to at least `bytes` now (so later calls allocate
 * nothing, e.g. before stream capture). */
int lsk_reserve(lsk_ctx* ctx, size_t bytes);

/* ---- the sketching path ------------------------------------------------ */

/* CountSketch S*A (Def. 3, Alg. 2; the library call csrcgs / rmcgs with
 * m = 0, Sec. 5).  S is r x n with one +-1 per column (hash and signs from
 * `seed`, see the header comment).  A: dense or CSR, n x d.  SA: device,
 * r*d floats, row-major, fully overwritten (rows no row of A hashes to are
 * zero).  Requires 1 <= r < 2^31, n < 2^31. */
int lsk_cs_sketch(lsk_ctx* ctx, const lsk_mat* A, int64_t r, uint64_t seed,
                  float* SA);

/* Gaussian stage of CountGauss (Alg. 3; csrcgs / rmcgs with m = k, Sec. 5):
 * GSA = G * SA with G k x r, N(0,1) entries scaled by 1/sqrt(k) (header
 * comment).  SA: device r*d floats row-major; GSA: device k*d floats
 * row-major, overwritten.  prec: LSK_PREC_FP32 or LSK_PREC_BF16 (G exact in
 * bfloat16, SA split into two bfloat16 terms, FP32 accumulation;
 * LSK_PREC_TF32 runs this stage as LSK_PREC_BF16).  In the
 * FP32 mode a sketch with r >= 8192 runs on the tensor cores with G and SA
 * each split into three bfloat16 terms (24 significant bits, exact) and the
 * six products down to order 2^-16 accumulated in FP32. */
int lsk_gauss_sketch(lsk_ctx* ctx, const float* SA, int64_t r, int64_t d,
                     int64_t k, uint64_t seed, int32_t prec, float* GSA);

/* Both stages of CountGauss in one pass over A (Alg. 3, which forms S*A a
 * block of r at a time and adds G_i (S_i A), so that only one block of S*A
 * exists at once): GSA = G * (S * A) with S, G as in lsk_cs_sketch and
 * lsk_gauss_sketch in the LSK_PREC_BF16 mode (same hash, signs and draws);
 * S*A is never written to device memory -- each 32-bucket block is summed
 * on chip, split into bfloat16 hi + lo and multiplied on the tensor cores at
 * once.  A: dense, 32 <= d <= 256, d and ld multiples of 4,
 * values 16-byte aligned (else LSK_ERR_UNSUPPORTED); 1 <= k <= 512,
 * 1 <= r < 2^31.  GSA: device k*d floats row-major, overwritten.  Agrees
 * with lsk_cs_sketch + lsk_gauss_sketch(LSK_PREC_BF16) up to FP32 rounding
 * (the order of the rows within a bucket is not fixed).  k outside [1, 512]
 * or a NULL GSA: LSK_ERR_INVALID_ARG; a device wait that gives up (1 s):
 * LSK_ERR_TIMEOUT from lsk_sync.  Faster than the two separate stages for
 * wide (d > 192), tall (n >= 8 r) problems with r >= 8 * 32 buckets per pair
 * of SMs (4M x 256, r = 65,536, k = 512 on GB300: 0.70 ms against 0.92 ms);
 * slower for narrower or smaller ones. */
int lsk_count_gauss(lsk_ctx* ctx, const lsk_mat* A, int64_t r, int64_t k,
                    uint64_t seed, float* GSA);
/* How lsk_leverage_scores, lsk_leverage_scores_jl, the least-squares driver
 * and the batch's ungrouped problems form their BF16 sketch (k > 0):
 *   0  the two stages (lsk_cs_sketch + lsk_gauss_sketch);
 *   1  the kernel of lsk_count_gauss where the shape favours it (see above),
 *      else the two stages -- the default;
 *   2  the kernel of lsk_count_gauss wherever it applies.
 * The batch's grouped problems always take the two stages (their Gaussian
 * stage is one grouped launch over all of them).  Process-wide; values
 * outside [0, 2] are clamped; returns the previous setting. */
int lsk_set_fused_sketch(int mode);

/* Gram matrix C <- alpha * A^T A + beta * C (csrrk, Sec. 5; Alg. 5 and
 * Alg. 7 for CSR A; the same operation for dense A).  C: device d*d floats
 * row-major, read when beta != 0 and overwritten.  Dense A with d <= 256
 * (d, ld multiples of 4, 16-byte aligned values) runs on the tensor cores as
 * lsk_gram_prec(LSK_PREC_BF16) (about 1e-5 relative Frobenius error: 7e-6 at
 * 4M x 256 with column scales 1e-3 .. 1e3); CSR A and other dense A run in
 * FP32 on the CUDA cores, partial sums folded into FP64 before the final
 * FP32 store (lsk_gram_prec(LSK_PREC_FP32) always takes this path). */
int lsk_gram(lsk_ctx* ctx, const lsk_mat* A, double alpha, double beta,
             float* C);
/* lsk_gram with a precision: LSK_PREC_FP32 on the CUDA cores in FP32 (as
 * lsk_gram for CSR A); LSK_PREC_BF16 (and LSK_PREC_TF32) forms the products of dense
 * A with d <= 256 on the tensor
 * cores from a bfloat16 split of A (a = hi + lo; hi^T hi + hi^T lo + lo^T hi,
 * about 2^-16 relative per product), accumulating at most 1024 rows in FP32
 * before the slices are added (compensated FP32, alpha and beta in FP64).
 * CSR A or d > 256 take the FP32 path.  Workspace: ceil(n / 1024) d*d
 * floats for the BF16 path. */
int lsk_gram_prec(lsk_ctx* ctx, const lsk_mat* A, double alpha, double beta,
                  int32_t prec, float* C);

/* Squared row norms x <- alpha * diag(A B B^T A^T) + beta * x (csrsqn /
 * rmsqn, Sec. 5; Alg. 8 for CSR A).  B: device d*c floats row-major.
 * x: device n floats, read when beta != 0.  A*B is never stored.
 * `upper_triangular` != 0 promises B[i][j] == 0 for i > j (c == d), which
 * lets the dense kernels skip the zero blocks.  prec (dense A):
 * LSK_PREC_FP32 = CUDA-core FP32; LSK_PREC_BF16 = tensor cores with A and B
 * split into bf16 hi + lo, A B ~ AhBh + AhBl + AlBh, FP32 accumulation, for
 * d, c <= 256 (other shapes run the FP32 kernel); LSK_PREC_TF32 = one TF32
 * product on the tensor cores, A streamed by the copy engine (TMA), which
 * rounds each entry to the nearest TF32 on the way (relative error <= 2^-11
 * per entry of A and B; about 3e-4 on the leverage scores of 4M x 256 with
 * column scales 1e-3 .. 1e3; more where a row's score is far below
 * ||A_i|| ||B||, e.g. 1.6e-3 on rows scaled x100 among 4096 x 32 -- the
 * BF16 form keeps ~1e-5 there), for 32 <= d <= 256, c <= 256, n >= 256, ld a
 * multiple of 4 and 16-byte aligned values (other dense shapes run the
 * BF16 form where it applies, else FP32).  CSR A always runs Alg. 8 in
 * FP32. */
int lsk_rownorms_prod(lsk_ctx* ctx, const lsk_mat* A, const float* B,
                      int64_t c, double alpha, double beta,
                      int32_t upper_triangular, int32_t prec, float* x);

/* R of the sketch (Alg. 12 step 2 / Alg. 15 step 3 with a QR in place of
 * the SVD): B = GSA (k x d floats, device, row-major, k >= d) -> R (d x d,
 * upper triangular, R_jj > 0) and R^-1, both FP64 row-major on the device:
 * the Cholesky factor of B^T B (identical to the sign-normalised
 * Householder R in exact arithmetic), to FP64 accuracy.  B^T B is formed
 * with FP64-accurate products; for d <= 256 it is equilibrated by powers of
 * two, factored and inverted in FP32, and the factor and its inverse are
 * corrected by one Newton step with FP64-accurate triangular products (the
 * FP32 error squared, far below what FP64 rounding leaves); for d > 256 the
 * Cholesky factorisation runs in FP64.  Rank deficiency (a pivot <= 0, an
 * FP32 factor that needs a correction larger than 1/4, or min R_jj <=
 * 16 eps64 d max R_jj) sets the deferred LSK_ERR_RANK_DEFICIENT.  Either
 * output may be NULL. */
int lsk_sketch_qr(lsk_ctx* ctx, const float* B, int64_t k, int64_t d,
                  double* R, double* Rinv);

/* Leverage-score estimates (Alg. 15 without the right Gaussian Pi):
 * sketch A to k x d with r CountSketch rows and k Gaussian rows (k == 0:
 * the r x d CountSketch alone, as m = 0 in csrcgs), R from the sketch as in
 * lsk_sketch_qr, then ell_i = ||A_i R^-1||^2 (Alg. 8).  ell: device n
 * floats.  R_out: NULL or device d*d doubles receiving R.  Requires the
 * sketch to have at least d rows.  prec: the Gaussian stage as
 * lsk_gauss_sketch (LSK_PREC_TF32: as LSK_PREC_BF16) and the row norms as
 * lsk_rownorms_prod with B = R^-1. */
int lsk_leverage_scores(lsk_ctx* ctx, const lsk_mat* A, int64_t r, int64_t k,
                        uint64_t seed, int32_t prec, float* ell,
                        double* R_out);

/* ---- row-partitioned (sharded) leverage scores ----------------------------
 * The sketch is linear in A and Def. 3 hashes each row of A by its index:
 * for A split by rows into blocks A_g (row offsets row0_g),
 *     G S A = sum_g G S_g A_g,
 * where S_g holds the columns row0_g .. of S.  So each holder of a block
 * forms its partial sketch with lsk_sketch_rows, the partials are summed
 * (one all-reduce of k*d floats -- the only exchange; Def. 4's reason for a
 * small sketch), every holder forms R from the sum, and scores its own rows
 * with lsk_leverage_scores_from_sketch. */

/* The partial sketch of a block of rows: S_g A (k == 0: r x d) or G S_g A
 * (k > 0: k x d), device floats row-major, into out (accumulate == 0: out is
 * overwritten) or added to it (accumulate != 0: out already holds the sketch
 * of other blocks -- one device holding several blocks, e.g. while later
 * blocks are still being copied in).  Row i of A is row row0 + i of the whole
 * matrix (its CountSketch column).  Same r, k, seed and prec as
 * lsk_leverage_scores; the BF16 mode uses the fused kernel as
 * lsk_set_fused_sketch selects.  row0 >= 0, row0 + n < 2^63. */
int lsk_sketch_rows(lsk_ctx* ctx, const lsk_mat* A, int64_t r, int64_t k,
                    uint64_t seed, int32_t prec, int64_t row0, int32_t accumulate,
                    float* out);

/* R (as lsk_sketch_qr) of a given sketch (rows x d floats, device, e.g. the
 * sum of the partial sketches of all blocks), then ell_i = ||A_i R^-1||^2
 * for the rows of A (Alg. 8; prec as lsk_rownorms_prod).  ell: device n
 * floats.  R_out: NULL or device d*d doubles.  rows >= d, d <= 1024. */
int lsk_leverage_scores_from_sketch(lsk_ctx* ctx, const lsk_mat* A,
                                    const float* sketch, int64_t rows,
                                    int32_t prec, float* ell, double* R_out);

/* Leverage-score estimates of Alg. 15 with its right JL projection: R from
 * the sketch exactly as in lsk_leverage_scores (a QR in place of the SVD of
 * Alg. 15 step 3: both give the same A R^-1 up to a d x d rotation, which
 * the Gaussian Pi does not see), then ell_i = ||A_i R^-1 Pi||^2 (Alg. 8 with
 * B = R^-1 Pi).  Pi is d x m with entries z / sqrt(m), z the standard normal
 * entries of the Gaussian stage's construction drawn on counter stream 2:
 * Pi[i][c] = entry (row c, column i) of that construction with the same
 * seed.  R^-1 Pi is formed in FP64 and stored in FP32.  m in [1, 4096]
 * (else LSK_ERR_INVALID_ARG); with prec = LSK_PREC_BF16 and d, m <= 256 the
 * row norms run on the tensor cores.  ell: device n floats; R_out: NULL or
 * device d*d doubles.  Each estimate is ||A_i R^-1||^2 times a chi^2_m / m
 * variable: unbiased, relative spread sqrt(2/m). */
int lsk_leverage_scores_jl(lsk_ctx* ctx, const lsk_mat* A, int64_t r, int64_t k,
                           int64_t m, uint64_t seed, int32_t prec, float* ell,
                           double* R_out);

/* Exact leverage scores (Alg. 13): B = A^T A in FP64 (FP32 partial sums
 * over row blocks, folded in FP64), R from B (FP64 accurate; Cholesky in
 * place of the SVD of step 2 at full rank), theta_i = ||A_i R^-1||^2
 * (Alg. 8).  theta: device n floats; R_out: NULL or device d*d doubles.
 * Rank deficiency is the deferred LSK_ERR_RANK_DEFICIENT; d <= 1024. */
int lsk_leverage_scores_exact(lsk_ctx* ctx, const lsk_mat* A, int32_t prec,
                              float* theta, double* R_out);

/* Least squares through the Gram matrix (Alg. 10): B = A^T A in FP64, R
 * from B, x = R^-1 R^-T A^T b (the pseudoinverse of step 2 at full rank),
 * then `refine` (0..10) steps x += R^-1 R^-T A^T (b - A x), all in FP64.
 * b: device n doubles; x: device d doubles (written).  The error of the
 * Gram route grows with cond(A)^2; the refinement steps bring it back to
 * cond(A) eps while cond(A)^2 times the Gram's rounding stays below 1. */
int lsk_least_squares_gram(lsk_ctx* ctx, const lsk_mat* A, const double* b,
                           int32_t refine, double* x);

/* Leverage scores with Alg. 15's "truncate if needed" read as a rank-revealing
 * truncation: the numerical rank of the sketch B = G S A is the number of
 * diagonally pivoted Cholesky steps of B^T B (the column-pivoted QR rule, as
 * in lsk_column_select) whose pivot exceeds max(16 eps d, rcond^2) times the
 * largest diagonal entry (rcond ~ a ratio of singular values); the scores
 * are then those of Alg. 15 on the columns K those steps pick (they span the
 * dominant column space): theta_i = ||A[i, K] R^-1||^2 with R from the QR of
 * B[:, K].  rank: NULL or host int64 (written).  Synchronises the context
 * stream to read the rank.  rcond in [0, 1); a numerically zero sketch is
 * LSK_ERR_RANK_DEFICIENT; d <= 1024. */
int lsk_leverage_scores_truncated(lsk_ctx* ctx, const lsk_mat* A, int64_t r,
                                  int64_t k, uint64_t seed, int32_t prec,
                                  double rcond, float* theta, int64_t* rank);

/* Column subset selection (Alg. 9): B = G S A (k > 0; S A when k == 0)
 * with the draws of lsk_leverage_scores, then the first c pivots of a
 * column-pivoted QR of B, taken as the diagonally pivoted Cholesky of
 * B^T B (FP64, exact products): the same pivot rule (largest remaining
 * column norm, lowest index on ties) in exact arithmetic, on a d x d matrix.
 * cols: device c int32 column indices of A, in pivot order (written).
 * c in [1, d], d <= 1024.  A numerically exhausted rank before c pivots
 * sets the deferred LSK_ERR_RANK_DEFICIENT and fills the rest of cols with
 * the remaining columns in order. */
int lsk_column_select(lsk_ctx* ctx, const lsk_mat* A, int64_t r, int64_t k,
                      uint64_t seed, int32_t prec, int64_t c, int32_t* cols);

/* Leverage scores on the columns K selected by lsk_column_select:
 * exact != 0: Alg. 14 -- the exact scores (Alg. 13) of A[:, K]: the Gram
 *   A^T A in FP64, its K x K block, R from it (FP64 accurate; Cholesky in
 *   place of the SVD at full rank), theta_i = ||A[i, K] R^-1||^2;
 * exact == 0: Alg. 16 -- Alg. 15 on A[:, K] with the Alg. 9 sketch
 *   restricted to K (column selection commutes with the left sketch), R
 *   from its QR, theta_i = ||A[i, K] R^-1||^2.
 * The row norms run on A itself with B = E_K R^-1 (d x c, zero outside the
 * rows K): A[:, K] is never copied.  theta: device n floats; cols: NULL or
 * device c int32 (the selection).  Rank deficiency is deferred as above. */
int lsk_leverage_scores_hrn(lsk_ctx* ctx, const lsk_mat* A, int64_t r, int64_t k,
                            uint64_t seed, int32_t prec, int64_t c, int32_t exact,
                            float* theta, int32_t* cols);

/* Gaussian sketch of a CSR matrix (Alg. 4, csrjlt): C = G A, G m x n with
 * entries z / sqrt(m) drawn like the Gaussian stage's G (Philox-4x32-10,
 * 24-bit Box-Muller) on counter stream 3, G[j][i] = entry (row j, column i)
 * of that construction (column index = row index of A); bfloat16-rounded in
 * the BF16 mode.  A: CSR only (LSK_ERR_UNSUPPORTED otherwise; a dense A is a
 * plain GEMM).  C: device m x d floats, row-major (written).  FP32 partial
 * sums over row ranges of A, summed in FP64 in a fixed order.  Malformed
 * CSR sets the deferred LSK_ERR_BAD_CSR.  m in [1, 2^20], d <= 1280. */
int lsk_csrjlt(lsk_ctx* ctx, const lsk_mat* A, int64_t m, uint64_t seed,
               int32_t prec, float* C);

/* Sketch-and-solve least squares (Alg. 11): (A~ b~) = G S (A b) with the
 * sketch sizes and draws of lsk_leverage_scores (k == 0: S (A b)), then
 * x = argmin ||A~ x - b~|| through R of A~ (a QR in place of the SVD of
 * Alg. 11 step 2; same minimiser at full rank): the seminormal equations
 * x = R^-1 R^-T A~^T b~ plus one corrected step, in FP64.  b~ uses the same
 * hash and the same G entries as A~ (bfloat16-rounded in the BF16 mode),
 * accumulated in FP64.  b: device n doubles; x: device d doubles (written).
 * The solution is approximate: ||A x - b|| is within the sketch's distortion
 * of the least-squares residual.  Rank deficiency of A~ is the deferred
 * LSK_ERR_RANK_DEFICIENT (as lsk_sketch_qr); d <= 1024. */
int lsk_sketch_solve(lsk_ctx* ctx, const lsk_mat* A, const double* b, int64_t r,
                     int64_t k, uint64_t seed, int32_t prec, double* x);

/* ---- batches of independent problems ------------------------------------ */
/* One problem of a batch: A (dense or CSR, device), its sketch sizes and
 * seed, and its output ell (device, A.n floats). */
typedef struct lsk_batch_item {
    lsk_mat A;
    int64_t r;
    int64_t k;
    uint64_t seed;
    float* ell;
} lsk_batch_item;

#define LSK_BATCH_STREAMS_MASK 0xFF    /* low byte: force this many streams    */
#define LSK_BATCH_GRAPH        0x100   /* capture the batch into a CUDA graph  */
                                       /* (cached; replayed when the same      */
                                       /* items come again)                    */
#define LSK_BATCH_AUTOTUNE     0x200   /* tune the schedule on this batch      */
                                       /* (see lsk_batch_schedule; kept per    */
                                       /* signature, and in the file named by  */
                                       /* LSK_AUTOTUNE_CACHE if set)           */
#define LSK_BATCH_PER_PROBLEM  0x400   /* no grouped stages: every problem's   */
                                       /* whole pipeline on the worker streams */

/* Leverage scores (as lsk_leverage_scores) of `count` independent problems.
 * With prec = LSK_PREC_BF16, problems with k > 0 and d <= 256 run in three
 * phases: their CountSketches on internal worker streams; then the Gaussian
 * stage and the R^-1 of every sketch as grouped launches (one grid per stage
 * over all problems, so the small latency-bound stages of many problems
 * share the GPU); then their row norms on the worker streams.  Other
 * problems run their whole pipeline on the worker streams.  The streams
 * fork from and join back into the context stream (asynchronous; deferred
 * errors as usual).  The grouped phases keep every grouped problem's sketch
 * resident at once (sum of r d 4 bytes plus small buffers).  A batch runs
 * LSK_PREC_TF32 as LSK_PREC_BF16 (its row norms use operands prepared for
 * all problems at once in the BF16x3 layout).
 * Batching is not in the paper: it applies the same per-problem method to
 * many problems at once.  The batch's internal workspaces are owned by the
 * context.  The items array is read during the call only. */
int lsk_batch_leverage_scores(lsk_ctx* ctx, int32_t count, const lsk_batch_item* items,
                              int32_t prec, int32_t flags);
/* Stream count chosen for this batch signature (0 if none yet). */
int lsk_batch_streams(lsk_ctx* ctx, int32_t count, const lsk_batch_item* items, int32_t prec);
/* The schedule of this batch signature, out[4] = {worker streams, most waves
 * of grouped problems, chunks of 32 sketch columns per block of the grouped
 * Gaussian stage, least 128-row tiles per CTA of the dense row norms}.
 * LSK_BATCH_AUTOTUNE picks it by coordinate descent over waves {2, 4, 8, 16},
 * streams {2, 4, 8, 16}, slice {64, 128, 256} and tiles {8, 16, 32}, each
 * candidate timed on the batch itself.  Returns 1 when a tuned schedule is
 * known for the signature (0 and the defaults {8, 4, 128, 16} otherwise). */
int lsk_batch_schedule(lsk_ctx* ctx, int32_t count, const lsk_batch_item* items, int32_t prec, int32_t* out);

/* ---- sketch-and-precondition least squares (Alg. 12) ------------------- */
typedef struct lsk_lsq_opts {
    int64_t r;              /* CountSketch rows (e.g. d*d)                  */
    int64_t k;              /* Gaussian rows (e.g. 2d; 0 = CountSketch only) */
    uint64_t seed;
    int32_t prec;           /* precision of the sketch (LSK_PREC_*)          */
    int32_t max_iter;       /* inner iterations per refinement step           */
    int32_t max_refine;     /* FP64 refinement steps                         */
    double tol;             /* target eta = ||A^T(b-Ax)|| / ||A^T b||         */
    double inner_tol;       /* relative residual of each inner solve          */
} lsk_lsq_opts;

typedef struct lsk_lsq_info {
    int32_t iters;          /* inner iterations in total                      */
    int32_t refinements;    /* FP64 refinement steps taken                   */
    double eta;             /* final normal-equation residual (FP64)         */
    int32_t status;         /* LSK_OK or LSK_ERR_NOT_CONVERGED               */
} lsk_lsq_info;

/* Fill `opts` with defaults for a d-column problem (r = max(d*d, 4d),
 * k = 2d, BF16 sketch, tol 1e-10). */
void lsk_lsq_default_opts(lsk_lsq_opts* opts, int64_t d);

/* Alg. 12: R from the sketch of A, N = R^-1, then FP64 iterative
 * refinement r_t = b - A x_t, g_t = N^T A^T r_t (both FP64), an inner
 * conjugate-gradient solve of N^T A^T A N z = g_t with FP32 products over A
 * (the preconditioned normal equations, CGLS; the Krylov iterates of LSQR
 * on min ||A N y - r_t||), x_{t+1} = x_t + N z, until
 * eta = ||A^T r|| / ||A^T b|| <= opts->tol.  b: device n doubles; x: device
 * d doubles (output).  info may be NULL.  Synchronises the stream (it reads
 * scalars back); LSK_ERR_NOT_CONVERGED when max_refine steps do not reach
 * tol. */
int lsk_sketch_precondition_lsq(lsk_ctx* ctx, const lsk_mat* A,
                                const double* b, double* x,
                                const lsk_lsq_opts* opts, lsk_lsq_info* info);

/* ---- debug / test entry points ----------------------------------------- */
/* The CountSketch hash of rows 0..n-1: bucket[i] = h(i), sign[i] = sigma_i
 * (Def. 3, spec in the header comment).  Device outputs. */
int lsk_debug_hash(lsk_ctx* ctx, int64_t n, int64_t r, uint64_t seed,
                   int32_t* bucket, int8_t* sign);
/* The Gaussian matrix G (k x r floats, device, row-major) as used by
 * lsk_gauss_sketch with the same precision mode. */
int lsk_debug_gauss(lsk_ctx* ctx, int64_t k, int64_t r, uint64_t seed,
                    int32_t prec, float* G);
/* Failure-detection check (no paper counterpart): one block runs the
 * bounded mbarrier wait that every tensor-core pipeline of this library uses,
 * on a barrier nothing arrives on, with a limit of limit_us microseconds
 * (1 .. 1,000,000).  The wait gives up, sets the context's TIMEOUT flag and
 * the kernel returns; the next lsk_sync reports LSK_ERR_TIMEOUT and the
 * context stays usable.  Asynchronous on the context stream. */
int lsk_debug_wait_timeout(lsk_ctx* ctx, int64_t limit_us);

/* ---- fixed-capacity CountSketch (no device allocation) ------------------ */
/* The paper has no counterpart to this call: it is an interface for callers
 * that cannot let a library allocate device memory -- applications whose
 * pool allocator owns all of HBM, or latency-critical loops where
 * cudaMalloc / cudaFree may synchronise the device.
 *
 * Same result as lsk_cs_sketch (S*A, same hash, same layouts), but it takes
 * no context and allocates nothing: its scratch is one 12 MiB array in device
 * global memory (held until the process exits).  The caller passes A and the
 * output SA (device pointers) and the cudaStream_t to launch on (NULL =
 * legacy default).
 *  - Limits: n <= LSK_NOALLOC_MAX_ROWS, 1 <= r <= LSK_NOALLOC_MAX_BUCKETS;
 *    larger sizes return LSK_ERR_UNSUPPORTED before anything is launched.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress, with that device current).  The CUDA runtime
 *    loads device code lazily, so that first call is when the array and the
 *    CountSketch kernels' code are placed on the device: make it during
 *    set-up, before any stream capture.  Later calls allocate nothing.
 *  - Every call shares the array and it keeps the last call's contents (the
 *    bucket counts are cleared at the start of each call), so calls whose
 *    GPU work overlaps -- on two streams or from two threads -- race and
 *    must be serialised by the caller.
 *  - Asynchronous on `stream`.  Out-of-range CSR entries are skipped and not
 *    reported (there is no context to hold an error flag).
 * Returns LSK_OK, LSK_ERR_INVALID_ARG, LSK_ERR_UNSUPPORTED or LSK_ERR_CUDA. */
#define LSK_NOALLOC_MAX_ROWS    (1 << 20)
#define LSK_NOALLOC_MAX_BUCKETS (1 << 18)
int lsk_cs_sketch_noalloc(const lsk_mat* A, int64_t r, uint64_t seed,
                          float* SA, void* stream);

/* ---- tracing ------------------------------------------------------------ */
/* Per-kernel CUDA-event timing on the context's stream (off by default).
 * While on, every kernel launch of a call is bracketed by two events; the
 * totals are resolved (synchronising on the events) by the query calls. */
int lsk_profile_enable(lsk_ctx* ctx, int on);
/* Drop the accumulated totals. */
int lsk_profile_reset(lsk_ctx* ctx);
/* Number of distinct kernel names with recorded launches. */
int lsk_profile_count(lsk_ctx* ctx);
/* Entry idx: kernel name (NUL-terminated, truncated to name_len), number of
 * launches and their summed duration in milliseconds. */
int lsk_profile_get(lsk_ctx* ctx, int idx, char* name, size_t name_len,
                    long long* launches, double* total_ms);

#ifdef __cplusplus
}
#endif
#endif /* LSK_H */
