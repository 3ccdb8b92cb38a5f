// api.cu -- the extern "C" entry points declared in include/lsk.h.
//
// Host-side argument validation, the context's workspace, and the order in
// which the kernels of each call are launched.  No compute happens here.
#include "lsk_internal.cuh"
#include "count_gauss.cuh"

#include <atomic>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

namespace {

// how the BF16 sketch of the leverage-score and least-squares calls is formed
// (process-wide): 0 the two stages, 1 the fused CountSketch + Gaussian kernel
// where the shape favours it, 2 the fused kernel wherever it applies
std::atomic<int> g_fused_sketch{1};

int fail(lsk_ctx* ctx, int code, const char* fmt, ...) {
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

int cuda_fail(lsk_ctx* ctx, cudaError_t e, const char* where) {
    return fail(ctx, LSK_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

// Grow the workspace to `bytes` (stream-ordered: safe for work still queued).
int ws_ensure(lsk_ctx* ctx, size_t bytes) {
    if (bytes <= ctx->ws_bytes) return LSK_OK;
    size_t want = bytes + bytes / 8;
    if (ctx->ws) {
        cudaError_t e = cudaFreeAsync(ctx->ws, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFreeAsync(workspace)");
        ctx->ws = nullptr;
        ctx->ws_bytes = 0;
    }
    void* p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, want, ctx->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, LSK_ERR_OOM, "workspace allocation of %zu bytes failed: %s", want,
                    cudaGetErrorString(e));
    }
    ctx->ws = p;
    ctx->ws_bytes = want;
    return LSK_OK;
}

int check_mat(lsk_ctx* ctx, const lsk_mat* A) {
    if (!A) return fail(ctx, LSK_ERR_INVALID_ARG, "A is NULL");
    if (A->dtype != LSK_F32) return fail(ctx, LSK_ERR_UNSUPPORTED, "only LSK_F32 values are supported");
    if (A->n < 0 || A->d < 1) return fail(ctx, LSK_ERR_INVALID_ARG, "bad shape n=%lld d=%lld",
                                          (long long)A->n, (long long)A->d);
    if (A->n >= (int64_t)1 << 31) return fail(ctx, LSK_ERR_UNSUPPORTED, "n must be < 2^31");
    if (A->kind == LSK_DENSE) {
        if (A->ld < A->d) return fail(ctx, LSK_ERR_INVALID_ARG, "ld < d");
        if (A->n > 0 && !A->values) return fail(ctx, LSK_ERR_INVALID_ARG, "A->values is NULL");
    } else if (A->kind == LSK_CSR) {
        if (!A->rowptr) return fail(ctx, LSK_ERR_INVALID_ARG, "A->rowptr is NULL");
        if (A->nnz < 0) return fail(ctx, LSK_ERR_INVALID_ARG, "nnz < 0");
        if (A->nnz > 0 && (!A->colidx || !A->values))
            return fail(ctx, LSK_ERR_INVALID_ARG, "A->colidx / A->values is NULL");
        if (A->d > INT32_MAX) return fail(ctx, LSK_ERR_UNSUPPORTED, "d too large for int32 column indices");
    } else {
        return fail(ctx, LSK_ERR_INVALID_ARG, "unknown matrix kind %d", (int)A->kind);
    }
    return LSK_OK;
}

int finish(lsk_ctx* ctx, const char* where) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, where);
    return LSK_OK;
}

int flag_to_status(lsk_ctx* ctx, int f) {
    if (f & LSK_FLAG_BAD_CSR) return fail(ctx, LSK_ERR_BAD_CSR, "CSR row pointer or column index out of range");
    if (f & LSK_FLAG_RANK_DEFICIENT)
        return fail(ctx, LSK_ERR_RANK_DEFICIENT, "sketch is numerically rank deficient");
    if (f & LSK_FLAG_TIMEOUT) return fail(ctx, LSK_ERR_TIMEOUT, "a bounded device wait timed out");
    return LSK_OK;
}

}  // namespace

extern "C" {

int lsk_create(lsk_ctx** out, int device, void* stream) {
    if (!out) return LSK_ERR_INVALID_ARG;
    *out = nullptr;
    lsk_ctx* ctx = (lsk_ctx*)calloc(1, sizeof(lsk_ctx));
    if (!ctx) return LSK_ERR_OOM;
    ctx->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->flag, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(ctx->flag, 0, sizeof(int));
    if (e != cudaSuccess) {
        cudaGetLastError();
        free(ctx);
        return LSK_ERR_CUDA;
    }
    ctx->stream = (cudaStream_t)stream;
    *out = ctx;
    return LSK_OK;
}

int lsk_destroy(lsk_ctx* ctx) {
    if (!ctx) return LSK_OK;
    cudaStreamSynchronize(ctx->stream);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->flag) cudaFree(ctx->flag);
    if (ctx->prof) lsk_prof_delete(ctx->prof);
    lsk_batch_free(ctx);
    free(ctx);
    return LSK_OK;
}

int lsk_set_stream(lsk_ctx* ctx, void* stream) {
    if (!ctx) return LSK_ERR_INVALID_ARG;
    ctx->stream = (cudaStream_t)stream;
    return LSK_OK;
}

int lsk_sync(lsk_ctx* ctx) {
    if (!ctx) return LSK_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamSynchronize");
    int f = 0;
    e = cudaMemcpy(&f, ctx->flag, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "reading the device flag");
    if (f) {
        cudaMemset(ctx->flag, 0, sizeof(int));
        return flag_to_status(ctx, f);
    }
    return LSK_OK;
}

const char* lsk_error_string(const lsk_ctx* ctx) { return ctx ? ctx->err : "null context"; }

size_t lsk_workspace_bytes(const lsk_ctx* ctx) { return ctx ? ctx->ws_bytes : 0; }

int lsk_reserve(lsk_ctx* ctx, size_t bytes) {
    if (!ctx) return LSK_ERR_INVALID_ARG;
    return ws_ensure(ctx, bytes);
}

int lsk_cs_sketch(lsk_ctx* ctx, const lsk_mat* A, int64_t r, uint64_t seed, float* SA) {
    if (!ctx) return LSK_ERR_INVALID_ARG;
    ProfGuard pg(ctx);
    int rc = check_mat(ctx, A);
    if (rc) return rc;
    if (r < 1 || r >= ((int64_t)1 << 31)) return fail(ctx, LSK_ERR_INVALID_ARG, "r must be in [1, 2^31)");
    if (!SA) return fail(ctx, LSK_ERR_INVALID_ARG, "SA is NULL");
    if (A->kind == LSK_CSR && A->d > 51200) return fail(ctx, LSK_ERR_UNSUPPORTED, "CSR sketch needs d <= 51200");
    rc = ws_ensure(ctx, cs_workspace_bytes(A->n, r));
    if (rc) return rc;
    cudaError_t e = cs_launch(A, r, seed, SA, ctx->ws, ctx->flag, ctx->sm_count, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lsk_cs_sketch");
    return finish(ctx, "lsk_cs_sketch");
}

int lsk_gauss_sketch(lsk_ctx* ctx, const float* SA, int64_t r, int64_t d, int64_t k, uint64_t seed,
                     int32_t prec, float* GSA) {
    if (!ctx) return LSK_ERR_INVALID_ARG;
    ProfGuard pg(ctx);
    if (!SA || !GSA) return fail(ctx, LSK_ERR_INVALID_ARG, "SA / GSA is NULL");
    if (r < 1 || d < 1 || k < 1) return fail(ctx, LSK_ERR_INVALID_ARG, "r, d, k must be >= 1");
    if (k >= ((int64_t)1 << 32)) return fail(ctx, LSK_ERR_INVALID_ARG, "k too large");
    if (prec != LSK_PREC_FP32 && prec != LSK_PREC_TF32 && prec != LSK_PREC_BF16)
        return fail(ctx, LSK_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
    prec = sketch_prec(prec);
    int rc = ws_ensure(ctx, gauss_workspace_bytes(r, d, k, prec, ctx->sm_count));
    if (rc) return rc;
    cudaError_t e = gauss_launch(SA, r, d, k, seed, prec, GSA, ctx->ws, ctx->sm_count, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lsk_gauss_sketch");
    return finish(ctx, "lsk_gauss_sketch");
}

int lsk_count_gauss(lsk_ctx* ctx, const lsk_mat* A, int64_t r, int64_t k, uint64_t seed, float* GSA) {
    if (!ctx) return LSK_ERR_INVALID_ARG;
    ProfGuard pg(ctx);
    int rc = check_mat(ctx, A);
    if (rc) return rc;
    if (r < 1 || r >= ((int64_t)1 << 31)) return fail(ctx, LSK_ERR_INVALID_ARG, "r must be in [1, 2^31)");
    if (k < 1 || k > 512) return fail(ctx, LSK_ERR_INVALID_ARG, "k must be in [1, 512]");
    if (!GSA) return fail(ctx, LSK_ERR_INVALID_ARG, "GSA is NULL");
    if (!count_gauss_supported(A, r, k))
        return fail(ctx, LSK_ERR_UNSUPPORTED,
                    "the fused sketch needs dense A, 32 <= d <= 256, d and ld multiples of 4, 16-byte alignment");
    rc = ws_ensure(ctx, count_gauss_workspace_bytes(A, r, k, ctx->sm_count));
    if (rc) return rc;
    cudaError_t e = count_gauss_launch(A, r, k, seed, GSA, ctx->ws, ctx->flag, ctx->sm_count, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lsk_count_gauss");
    return finish(ctx, "lsk_count_gauss");
}

int lsk_set_fused_sketch(int mode) { return g_fused_sketch.exchange(mode < 0 ? 0 : mode > 2 ? 2 : mode); }

}  // extern "C"
namespace {
// A^T A on the CUDA cores in FP32 (partials folded in FP64); CSR: Alg. 7
int gram_fp32(lsk_ctx* ctx, const lsk_mat* A, double alpha, double beta, float* C) {
    ProfGuard pg(ctx);
    int rc = check_mat(ctx, A);
    if (rc) return rc;
    if (!C) return fail(ctx, LSK_ERR_INVALID_ARG, "C is NULL");
    rc = ws_ensure(ctx, gram_workspace_bytes(A, ctx->sm_count));
    if (rc) return rc;
    cudaError_t e = gram_launch(A, alpha, beta, C, ctx->ws, ctx->flag, ctx->sm_count, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lsk_gram");
    return finish(ctx, "lsk_gram");
}
}  // namespace
extern "C" {

int lsk_gram(lsk_ctx* ctx, const lsk_mat* A, double alpha, double beta, float* C) {
    if (!ctx) return LSK_ERR_INVALID_ARG;
    // dense, d <= 256: the tensor cores (BF16x3, ~1e-5 relative); else FP32
    if (A && A->kind == LSK_DENSE && A->dtype == LSK_F32 && gram_tc_supported(A))
        return lsk_gram_prec(ctx, A, alpha, beta, LSK_PREC_BF16, C);
    return gram_fp32(ctx, A, alpha, beta, C);
}

int lsk_gram_prec(lsk_ctx* ctx, const lsk_mat* A, double alpha, double beta, int32_t prec, float* C) {
    if (!ctx) return LSK_ERR_INVALID_ARG;
    if (prec != LSK_PREC_FP32 && prec != LSK_PREC_TF32 && prec != LSK_PREC_BF16)
        return fail(ctx, LSK_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
    prec = sketch_prec(prec);   // TF32: the BF16x3 tensor-core Gram
    if (prec != LSK_PREC_BF16) return gram_fp32(ctx, A, alpha, beta, C);
    ProfGuard pg(ctx);
    int rc = check_mat(ctx, A);
    if (rc) return rc;
    if (!C) return fail(ctx, LSK_ERR_INVALID_ARG, "C is NULL");
    if (!gram_tc_supported(A)) return gram_fp32(ctx, A, alpha, beta, C);   // CSR or d > 256: the FP32 path
    rc = ws_ensure(ctx, gram_tc_workspace_bytes(A, ctx->sm_count));
    if (rc) return rc;
    cudaError_t e = gram_tc_launch(A, alpha, beta, C, ctx->ws, ctx->flag, ctx->sm_count, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lsk_gram_prec");
    return finish(ctx, "lsk_gram_prec");
}

int lsk_rownorms_prod(lsk_ctx* ctx, const lsk_mat* A, const float* B, int64_t c, double alpha,
                      double beta, int32_t upper_triangular, int32_t prec, float* x) {
    if (!ctx) return LSK_ERR_INVALID_ARG;
    ProfGuard pg(ctx);
    int rc = check_mat(ctx, A);
    if (rc) return rc;
    if (!B || !x) return fail(ctx, LSK_ERR_INVALID_ARG, "B / x is NULL");
    if (c < 1) return fail(ctx, LSK_ERR_INVALID_ARG, "c must be >= 1");
    if (upper_triangular && c != A->d) return fail(ctx, LSK_ERR_INVALID_ARG, "upper_triangular needs c == d");
    if (prec != LSK_PREC_FP32 && prec != LSK_PREC_TF32 && prec != LSK_PREC_BF16)
        return fail(ctx, LSK_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
    rc = ws_ensure(ctx, rownorms_workspace_bytes(A, c, upper_triangular, prec));
    if (rc) return rc;
    cudaError_t e = rownorms_launch(A, B, c, alpha, beta, upper_triangular, prec, x, ctx->ws, ctx->flag,
                                    ctx->sm_count, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lsk_rownorms_prod");
    return finish(ctx, "lsk_rownorms_prod");
}

int lsk_sketch_qr(lsk_ctx* ctx, const float* B, int64_t k, int64_t d, double* R, double* Rinv) {
    if (!ctx) return LSK_ERR_INVALID_ARG;
    ProfGuard pg(ctx);
    if (!B) return fail(ctx, LSK_ERR_INVALID_ARG, "B is NULL");
    if (d < 1 || k < d) return fail(ctx, LSK_ERR_INVALID_ARG, "need k >= d >= 1");
    if (d > 1024) return fail(ctx, LSK_ERR_UNSUPPORTED, "sketch QR supports d <= 1024");
    int rc = ws_ensure(ctx, qr_workspace_bytes(k, d));
    if (rc) return rc;
    cudaError_t e = qr_launch(B, k, d, R, Rinv, nullptr, ctx->ws, ctx->flag, ctx->sm_count, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lsk_sketch_qr");
    return finish(ctx, "lsk_sketch_qr");
}

// Workspace layout shared by leverage_scores and the LSQ driver:
//   [SA r*d f32][GSA k*d f32][Rinv64 d*d][Rinv32 d*d][R64 d*d][stage scratch]
namespace {
struct SketchBufs {
    float* SA;
    float* GSA;
    double* Rinv64;
    float* Rinv32;
    double* R64;
    void* scratch;
};

size_t stage_scratch(const lsk_mat* A, int64_t r, int64_t k, int32_t prec, int sm) {
    size_t s = cs_workspace_bytes(A->n, r);
    if (k > 0) {
        const size_t g = gauss_workspace_bytes(r, A->d, k, prec, sm);
        if (g > s) s = g;
    }
    if (k > 0 && prec == LSK_PREC_BF16) {
        const size_t f = count_gauss_workspace_bytes(A, r, k, sm);
        if (f > s) s = f;
    }
    const size_t q = qr_workspace_bytes(k > 0 ? k : r, A->d);
    if (q > s) s = q;
    const size_t rn = rownorms_workspace_bytes(A, A->d, 1, prec);
    if (rn > s) s = rn;
    return s;
}

size_t sketch_bytes(const lsk_mat* A, int64_t r, int64_t k, int32_t prec, int sm, size_t extra) {
    const int64_t d = A->d;
    return ws_round((size_t)r * d * 4) + ws_round((size_t)(k > 0 ? k : 1) * d * 4) +
           ws_round((size_t)d * d * 8) * 2 + ws_round((size_t)d * d * 4) +
           (stage_scratch(A, r, k, prec, sm) > extra ? stage_scratch(A, r, k, prec, sm) : extra) + 4096;
}

SketchBufs carve(void* ws, const lsk_mat* A, int64_t r, int64_t k) {
    const int64_t d = A->d;
    WsCarver wc{(char*)ws, 0};
    SketchBufs b;
    b.SA = wc.take<float>((size_t)r * d);
    b.GSA = wc.take<float>((size_t)(k > 0 ? k : 1) * d);
    b.Rinv64 = wc.take<double>((size_t)d * d);
    b.R64 = wc.take<double>((size_t)d * d);
    b.Rinv32 = wc.take<float>((size_t)d * d);
    b.scratch = wc.take<char>(1);
    return b;
}

// S A (k = 0) into b.SA, or G S A into b.GSA; in the BF16 mode G S A comes
// from the fused kernel where the fused-sketch mode selects it (S A is then
// not formed).  A's rows are columns row0.. of S.  *sk / *rows: the sketch.
cudaError_t sketch_on(const lsk_mat* A, int64_t r, int64_t k, uint64_t seed, int32_t prec, const SketchBufs& b,
                      int* flag, int sm, cudaStream_t st, uint64_t row0, const float** sk, int64_t* rows) {
    const int fused = g_fused_sketch.load();
    if (k > 0 && prec == LSK_PREC_BF16 &&
        ((fused == 1 && count_gauss_preferred(A, r, k, sm)) || (fused == 2 && count_gauss_supported(A, r, k)))) {
        *sk = b.GSA;
        *rows = k;
        return count_gauss_launch(A, r, k, seed, b.GSA, b.scratch, flag, sm, st, row0);
    }
    cudaError_t e = cs_launch(A, r, seed, b.SA, b.scratch, flag, sm, st, row0);
    if (e != cudaSuccess) return e;
    *sk = b.SA;
    *rows = r;
    if (k > 0) {
        e = gauss_launch(b.SA, r, A->d, k, seed, prec, b.GSA, b.scratch, sm, st);
        *sk = b.GSA;
        *rows = k;
    }
    return e;
}

// SA -> (GSA) -> R, R^-1 on the device, all asynchronous.
cudaError_t sketch_and_factor_on(const lsk_mat* A, int64_t r, int64_t k, uint64_t seed, int32_t prec,
                                 const SketchBufs& b, double* R_out, int* flag, int sm, cudaStream_t st) {
    const float* sk = nullptr;
    int64_t rows = 0;
    cudaError_t e = sketch_on(A, r, k, seed, prec, b, flag, sm, st, 0, &sk, &rows);
    if (e != cudaSuccess) return e;
    return qr_launch(sk, rows, A->d, R_out, b.Rinv64, b.Rinv32, b.scratch, flag, sm, st);
}

cudaError_t sketch_and_factor(lsk_ctx* ctx, const lsk_mat* A, int64_t r, int64_t k, uint64_t seed,
                              int32_t prec, const SketchBufs& b, double* R_out) {
    return sketch_and_factor_on(A, r, k, seed, prec, b, R_out, ctx->flag, ctx->sm_count, ctx->stream);
}

int check_sketch_args(lsk_ctx* ctx, const lsk_mat* A, int64_t r, int64_t k, int32_t prec) {
    if (r < 1 || r >= ((int64_t)1 << 31)) return fail(ctx, LSK_ERR_INVALID_ARG, "r must be in [1, 2^31)");
    if (k < 0) return fail(ctx, LSK_ERR_INVALID_ARG, "k must be >= 0");
    const int64_t rows = k > 0 ? k : r;
    if (rows < A->d) return fail(ctx, LSK_ERR_INVALID_ARG, "the sketch needs at least d rows");
    if (A->d > 1024) return fail(ctx, LSK_ERR_UNSUPPORTED, "d <= 1024 is supported");
    if (prec != LSK_PREC_FP32 && prec != LSK_PREC_TF32 && prec != LSK_PREC_BF16)
        return fail(ctx, LSK_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
    return LSK_OK;
}
}  // namespace
}  // extern "C"

// The whole leverage-score pipeline of one problem on (ws, st); used by
// lsk_leverage_scores and by the batch driver.
size_t leverage_workspace_bytes(const lsk_mat* A, int64_t r, int64_t k, int32_t prec, int sm) {
    return sketch_bytes(A, r, k, prec, sm, 0);
}
cudaError_t leverage_pipeline(const lsk_mat* A, int64_t r, int64_t k, uint64_t seed, int32_t prec, float* ell,
                              double* R_out, void* ws, int* flag, int sm, cudaStream_t st) {
    const SketchBufs b = carve(ws, A, r, k);
    cudaError_t e = sketch_and_factor_on(A, r, k, seed, prec, b, R_out, flag, sm, st);
    if (e != cudaSuccess) return e;
    return rownorms_launch(A, b.Rinv32, A->d, 1.0, 0.0, 1, prec, ell, b.scratch, flag, sm, st);
}
int check_leverage_args(lsk_ctx* ctx, const lsk_mat* A, int64_t r, int64_t k, int32_t prec) {
    int rc = check_mat(ctx, A);
    if (rc) return rc;
    return check_sketch_args(ctx, A, r, k, prec);
}

extern "C" {

int lsk_leverage_scores(lsk_ctx* ctx, const lsk_mat* A, int64_t r, int64_t k, uint64_t seed, int32_t prec,
                        float* ell, double* R_out) {
    if (!ctx) return LSK_ERR_INVALID_ARG;
    ProfGuard pg(ctx);
    int rc = check_mat(ctx, A);
    if (rc) return rc;
    rc = check_sketch_args(ctx, A, r, k, prec);
    if (rc) return rc;
    if (!ell && A->n > 0) return fail(ctx, LSK_ERR_INVALID_ARG, "ell is NULL");
    const int32_t rn_prec = prec;   // the row norms keep TF32
    prec = sketch_prec(prec);
    rc = ws_ensure(ctx, sketch_bytes(A, r, k, prec, ctx->sm_count, 0));
    if (rc) return rc;
    const SketchBufs b = carve(ctx->ws, A, r, k);
    cudaError_t e = sketch_and_factor(ctx, A, r, k, seed, prec, b, R_out);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lsk_leverage_scores (sketch)");
    e = rownorms_launch(A, b.Rinv32, A->d, 1.0, 0.0, 1, rn_prec, ell, b.scratch, ctx->flag, ctx->sm_count,
                        ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lsk_leverage_scores (row norms)");
    return finish(ctx, "lsk_leverage_scores");
}

int lsk_sketch_rows(lsk_ctx* ctx, const lsk_mat* A, int64_t r, int64_t k, uint64_t seed, int32_t prec, int64_t row0,
                    int32_t accumulate, float* out) {
    if (!ctx) return LSK_ERR_INVALID_ARG;
    ProfGuard pg(ctx);
    int rc = check_mat(ctx, A);
    if (rc) return rc;
    if (r < 1 || r >= ((int64_t)1 << 31)) return fail(ctx, LSK_ERR_INVALID_ARG, "r must be in [1, 2^31)");
    if (k < 0 || k >= ((int64_t)1 << 32)) return fail(ctx, LSK_ERR_INVALID_ARG, "k must be in [0, 2^32)");
    if (prec != LSK_PREC_FP32 && prec != LSK_PREC_TF32 && prec != LSK_PREC_BF16)
        return fail(ctx, LSK_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
    if (row0 < 0 || A->n > INT64_MAX - row0) return fail(ctx, LSK_ERR_INVALID_ARG, "row0 must be >= 0 and row0 + n < 2^63");
    if (!out) return fail(ctx, LSK_ERR_INVALID_ARG, "out is NULL");
    if (A->kind == LSK_CSR && A->d > 51200) return fail(ctx, LSK_ERR_UNSUPPORTED, "CSR sketch needs d <= 51200");
    prec = sketch_prec(prec);
    cudaError_t e;
    if (k == 0) {   // S A straight into out (the gather adds into it when accumulating)
        rc = ws_ensure(ctx, cs_workspace_bytes(A->n, r));
        if (rc) return rc;
        e = cs_launch(A, r, seed, out, ctx->ws, ctx->flag, ctx->sm_count, ctx->stream, (uint64_t)row0, accumulate != 0);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "lsk_sketch_rows");
        return finish(ctx, "lsk_sketch_rows");
    }
    rc = ws_ensure(ctx, sketch_bytes(A, r, k, prec, ctx->sm_count, 0));
    if (rc) return rc;
    const SketchBufs b = carve(ctx->ws, A, r, k);
    const float* sk = nullptr;
    int64_t rows = 0;
    e = sketch_on(A, r, k, seed, prec, b, ctx->flag, ctx->sm_count, ctx->stream, (uint64_t)row0, &sk, &rows);
    if (e == cudaSuccess)
        e = accumulate ? add_into_launch(out, sk, rows * A->d, ctx->stream)
                       : cudaMemcpyAsync(out, sk, (size_t)rows * A->d * 4, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lsk_sketch_rows");
    return finish(ctx, "lsk_sketch_rows");
}

int lsk_leverage_scores_from_sketch(lsk_ctx* ctx, const lsk_mat* A, const float* sketch, int64_t rows, int32_t prec,
                                    float* ell, double* R_out) {
    if (!ctx) return LSK_ERR_INVALID_ARG;
    ProfGuard pg(ctx);
    int rc = check_mat(ctx, A);
    if (rc) return rc;
    if (!sketch) return fail(ctx, LSK_ERR_INVALID_ARG, "sketch is NULL");
    if (rows < A->d) return fail(ctx, LSK_ERR_INVALID_ARG, "the sketch needs at least d rows");
    if (A->d > 1024) return fail(ctx, LSK_ERR_UNSUPPORTED, "d <= 1024 is supported");
    if (prec != LSK_PREC_FP32 && prec != LSK_PREC_TF32 && prec != LSK_PREC_BF16)
        return fail(ctx, LSK_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
    if (!ell && A->n > 0) return fail(ctx, LSK_ERR_INVALID_ARG, "ell is NULL");
    const int32_t rn_prec = prec;   // the row norms keep TF32
    prec = sketch_prec(prec);
    const int64_t d = A->d;
    const size_t q = qr_workspace_bytes(rows, d), rn = rownorms_workspace_bytes(A, d, 1, rn_prec);
    rc = ws_ensure(ctx, ws_round((size_t)d * d * 8) + ws_round((size_t)d * d * 4) + (q > rn ? q : rn) + 1024);
    if (rc) return rc;
    WsCarver wc{(char*)ctx->ws, 0};
    double* Rinv64 = wc.take<double>((size_t)d * d);
    float* Rinv32 = wc.take<float>((size_t)d * d);
    void* scratch = wc.take<char>(1);
    cudaError_t e = qr_launch(sketch, rows, d, R_out, Rinv64, Rinv32, scratch, ctx->flag, ctx->sm_count, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lsk_leverage_scores_from_sketch (R)");
    e = rownorms_launch(A, Rinv32, d, 1.0, 0.0, 1, rn_prec, ell, scratch, ctx->flag, ctx->sm_count, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lsk_leverage_scores_from_sketch (row norms)");
    return finish(ctx, "lsk_leverage_scores_from_sketch");
}

int lsk_leverage_scores_jl(lsk_ctx* ctx, const lsk_mat* A, int64_t r, int64_t k, int64_t m, uint64_t seed,
                           int32_t prec, float* ell, double* R_out) {
    if (!ctx) return LSK_ERR_INVALID_ARG;
    ProfGuard pg(ctx);
    int rc = check_mat(ctx, A);
    if (rc) return rc;
    rc = check_sketch_args(ctx, A, r, k, prec);
    if (rc) return rc;
    if (m < 1 || m > 4096) return fail(ctx, LSK_ERR_INVALID_ARG, "m must be in [1, 4096]");
    if (!ell && A->n > 0) return fail(ctx, LSK_ERR_INVALID_ARG, "ell is NULL");
    const int32_t rn_prec = prec;   // the row norms keep TF32
    prec = sketch_prec(prec);
    // stage scratch after the factorisation: [X = R^-1 Pi, d*m f32][Pi | row-norm workspace]
    const size_t xb = ws_round((size_t)A->d * m * 4);
    const size_t jw = jl_workspace_bytes(A->d, m);
    const size_t rw = rownorms_workspace_bytes(A, m, 0, rn_prec);
    rc = ws_ensure(ctx, sketch_bytes(A, r, k, prec, ctx->sm_count, xb + (jw > rw ? jw : rw)));
    if (rc) return rc;
    const SketchBufs b = carve(ctx->ws, A, r, k);
    cudaError_t e = sketch_and_factor(ctx, A, r, k, seed, prec, b, R_out);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lsk_leverage_scores_jl (sketch)");
    float* X = (float*)b.scratch;
    void* rest = (char*)b.scratch + xb;
    e = jl_launch(b.Rinv64, A->d, m, seed, X, rest, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lsk_leverage_scores_jl (R^-1 Pi)");
    e = rownorms_launch(A, X, m, 1.0, 0.0, 0, rn_prec, ell, rest, ctx->flag, ctx->sm_count, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lsk_leverage_scores_jl (row norms)");
    return finish(ctx, "lsk_leverage_scores_jl");
}

int lsk_csrjlt(lsk_ctx* ctx, const lsk_mat* A, int64_t m, uint64_t seed, int32_t prec, float* C) {
    if (!ctx) return LSK_ERR_INVALID_ARG;
    ProfGuard pg(ctx);
    int rc = check_mat(ctx, A);
    if (rc) return rc;
    if (A->kind != LSK_CSR) return fail(ctx, LSK_ERR_UNSUPPORTED, "lsk_csrjlt takes a CSR matrix");
    if (!C) return fail(ctx, LSK_ERR_INVALID_ARG, "C is NULL");
    prec = sketch_prec(prec);
    if (prec != LSK_PREC_FP32 && prec != LSK_PREC_BF16)
        return fail(ctx, LSK_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
    if (m < 1 || !jlt_supported(A->d, m)) return fail(ctx, LSK_ERR_UNSUPPORTED, "m in [1, 2^20], d <= 1280");
    rc = ws_ensure(ctx, jlt_workspace_bytes(A->n, A->d, m, ctx->sm_count));
    if (rc) return rc;
    cudaError_t e = jlt_launch(A, m, seed, prec, C, ctx->ws, ctx->flag, ctx->sm_count, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lsk_csrjlt");
    return finish(ctx, "lsk_csrjlt");
}

int lsk_sketch_solve(lsk_ctx* ctx, const lsk_mat* A, const double* b, int64_t r, int64_t k, uint64_t seed,
                     int32_t prec, double* x) {
    if (!ctx) return LSK_ERR_INVALID_ARG;
    ProfGuard pg(ctx);
    int rc = check_mat(ctx, A);
    if (rc) return rc;
    rc = check_sketch_args(ctx, A, r, k, prec);
    if (rc) return rc;
    if (!x || (!b && A->n > 0)) return fail(ctx, LSK_ERR_INVALID_ARG, "b / x is NULL");
    prec = sketch_prec(prec);
    rc = ws_ensure(ctx, sketch_bytes(A, r, k, prec, ctx->sm_count, solve_workspace_bytes(r, k, A->d)));
    if (rc) return rc;
    const SketchBufs bufs = carve(ctx->ws, A, r, k);
    cudaError_t e = sketch_and_factor(ctx, A, r, k, seed, prec, bufs, nullptr);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lsk_sketch_solve (sketch)");
    e = solve_launch(A, b, r, k, seed, prec, k > 0 ? bufs.GSA : bufs.SA, bufs.Rinv64, x, bufs.scratch,
                     ctx->sm_count, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lsk_sketch_solve (solve)");
    return finish(ctx, "lsk_sketch_solve");
}

// ---- column subset selection (Alg. 9) and Alg. 14 / 16 -------------------
namespace {

// S A (k = 0) or G S A into the sketch buffers, without factoring it
cudaError_t sketch_only(lsk_ctx* ctx, const lsk_mat* A, int64_t r, int64_t k, uint64_t seed, int32_t prec,
                        const SketchBufs& b, const float** sk, int64_t* rows) {
    cudaError_t e = cs_launch(A, r, seed, b.SA, b.scratch, ctx->flag, ctx->sm_count, ctx->stream);
    if (e != cudaSuccess) return e;
    *sk = b.SA;
    *rows = r;
    if (k > 0) {
        e = gauss_launch(b.SA, r, A->d, k, seed, prec, b.GSA, b.scratch, ctx->sm_count, ctx->stream);
        *sk = b.GSA;
        *rows = k;
    }
    return e;
}

// scratch after the sketch: [C = B^T B][its partials][pivoted factor][columns K]
struct CssBufs {
    double* C;
    void* gpart;
    void* L;
    int32_t* cols;
    void* rest;
};
size_t css_bytes(int64_t rows, int64_t d, int64_t c) {
    return ws_round((size_t)d * d * 8) + ws_round(sketch_gram64_workspace_bytes(rows, d)) +
           ws_round(pivchol_workspace_bytes(d, c)) + ws_round((size_t)c * 4) + 1024;
}
CssBufs css_carve(void* scratch, int64_t rows, int64_t d, int64_t c) {
    WsCarver wc{(char*)scratch, 0};
    CssBufs b;
    b.C = wc.take<double>((size_t)d * d);
    b.gpart = wc.take<char>(sketch_gram64_workspace_bytes(rows, d));
    b.L = wc.take<char>(pivchol_workspace_bytes(d, c));
    b.cols = wc.take<int32_t>((size_t)c);
    b.rest = wc.take<char>(0);
    return b;
}

int css_checks(lsk_ctx* ctx, const lsk_mat* A, int64_t r, int64_t k, int32_t prec, int64_t c) {
    int rc = check_mat(ctx, A);
    if (rc) return rc;
    rc = check_sketch_args(ctx, A, r, k, prec);
    if (rc) return rc;
    if (c < 1 || c > A->d) return fail(ctx, LSK_ERR_INVALID_ARG, "c must be in [1, d]");
    if (A->d > 1024) return fail(ctx, LSK_ERR_UNSUPPORTED, "column selection supports d <= 1024");
    return LSK_OK;
}

// Alg. 9 into scratch: returns the sketch (for Alg. 16) and the CSS buffers
cudaError_t css_run(lsk_ctx* ctx, const lsk_mat* A, int64_t r, int64_t k, uint64_t seed, int32_t prec, int64_t c,
                    const SketchBufs& b, const float** sk, int64_t* rows, CssBufs* cb) {
    cudaError_t e = sketch_only(ctx, A, r, k, seed, prec, b, sk, rows);
    if (e != cudaSuccess) return e;
    *cb = css_carve(b.scratch, *rows, A->d, c);
    e = sketch_gram64_launch(*sk, *rows, A->d, cb->C, cb->gpart, ctx->sm_count, ctx->stream);
    if (e != cudaSuccess) return e;
    return pivchol_launch(cb->C, A->d, c, 0.0, 1, cb->cols, nullptr, cb->L, ctx->flag, ctx->stream);
}

}  // namespace

int lsk_leverage_scores_truncated(lsk_ctx* ctx, const lsk_mat* A, int64_t r, int64_t k, uint64_t seed,
                                  int32_t prec, double rcond, float* theta, int64_t* rank) {
    if (!ctx) return LSK_ERR_INVALID_ARG;
    ProfGuard pg(ctx);
    const int64_t d = A ? A->d : 0;
    int rc = css_checks(ctx, A, r, k, prec, d);
    if (rc) return rc;
    if (!theta && A->n > 0) return fail(ctx, LSK_ERR_INVALID_ARG, "theta is NULL");
    if (!(rcond >= 0.0 && rcond < 1.0)) return fail(ctx, LSK_ERR_INVALID_ARG, "rcond must be in [0, 1)");
    const int32_t rn_prec = prec;   // the row norms keep TF32
    prec = sketch_prec(prec);
    const int64_t rows = k > 0 ? k : r;
    const size_t tail = ws_round((size_t)rows * d * 4) + ws_round(qr_workspace_bytes(rows, d)) +
                        ws_round((size_t)d * d * 4) + ws_round(rownorms_workspace_bytes(A, d, 0, rn_prec)) +
                        ws_round(4) + 4096;
    rc = ws_ensure(ctx, sketch_bytes(A, r, k, prec, ctx->sm_count, css_bytes(rows, d, d) + tail));
    if (rc) return rc;
    const SketchBufs b = carve(ctx->ws, A, r, k);
    const float* sk;
    int64_t sr;
    cudaError_t e = sketch_only(ctx, A, r, k, seed, prec, b, &sk, &sr);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lsk_leverage_scores_truncated (sketch)");
    const CssBufs cb = css_carve(b.scratch, rows, d, d);
    WsCarver wc{(char*)cb.rest, 0};
    int* dev_rank = wc.take<int>(1);
    e = sketch_gram64_launch(sk, rows, d, cb.C, cb.gpart, ctx->sm_count, ctx->stream);
    if (e == cudaSuccess)
        e = pivchol_launch(cb.C, d, d, rcond, 0, cb.cols, dev_rank, cb.L, ctx->flag, ctx->stream);
    int h_rank = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_rank, dev_rank, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lsk_leverage_scores_truncated (rank)");
    if (rank) *rank = h_rank;
    if (h_rank < 1) return fail(ctx, LSK_ERR_RANK_DEFICIENT, "the sketch is numerically zero");
    const int64_t c = h_rank;
    // Alg. 15 on the c columns that carry the numerical rank
    float* Bk = wc.take<float>((size_t)rows * c);
    void* qw = wc.take<char>(qr_workspace_bytes(rows, c));
    float* Bf = wc.take<float>((size_t)d * c);
    void* rw = wc.take<char>(rownorms_workspace_bytes(A, c, 0, rn_prec));
    e = gather_cols_launch(sk, rows, d, cb.cols, c, Bk, ctx->stream);
    if (e == cudaSuccess)
        e = qr_launch(Bk, rows, c, nullptr, b.Rinv64, b.Rinv32, qw, ctx->flag, ctx->sm_count, ctx->stream);
    if (e == cudaSuccess) e = embed_rows_launch(b.Rinv32, c, cb.cols, d, Bf, ctx->stream);
    if (e == cudaSuccess)
        e = rownorms_launch(A, Bf, c, 1.0, 0.0, 0, rn_prec, theta, rw, ctx->flag, ctx->sm_count, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lsk_leverage_scores_truncated (row norms)");
    return finish(ctx, "lsk_leverage_scores_truncated");
}

int lsk_column_select(lsk_ctx* ctx, const lsk_mat* A, int64_t r, int64_t k, uint64_t seed, int32_t prec,
                      int64_t c, int32_t* cols) {
    if (!ctx) return LSK_ERR_INVALID_ARG;
    ProfGuard pg(ctx);
    int rc = css_checks(ctx, A, r, k, prec, c);
    if (rc) return rc;
    if (!cols) return fail(ctx, LSK_ERR_INVALID_ARG, "cols is NULL");
    prec = sketch_prec(prec);
    const int64_t rows = k > 0 ? k : r;
    rc = ws_ensure(ctx, sketch_bytes(A, r, k, prec, ctx->sm_count, css_bytes(rows, A->d, c)));
    if (rc) return rc;
    const SketchBufs b = carve(ctx->ws, A, r, k);
    const float* sk;
    int64_t sr;
    CssBufs cb;
    cudaError_t e = css_run(ctx, A, r, k, seed, prec, c, b, &sk, &sr, &cb);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cols, cb.cols, (size_t)c * 4, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lsk_column_select");
    return finish(ctx, "lsk_column_select");
}

int lsk_leverage_scores_hrn(lsk_ctx* ctx, const lsk_mat* A, int64_t r, int64_t k, uint64_t seed, int32_t prec,
                            int64_t c, int32_t exact, float* theta, int32_t* cols) {
    if (!ctx) return LSK_ERR_INVALID_ARG;
    ProfGuard pg(ctx);
    int rc = css_checks(ctx, A, r, k, prec, c);
    if (rc) return rc;
    if (!theta && A->n > 0) return fail(ctx, LSK_ERR_INVALID_ARG, "theta is NULL");
    const int32_t rn_prec = prec;   // the row norms keep TF32
    prec = sketch_prec(prec);
    const int64_t d = A->d, rows = k > 0 ? k : r;
    // after the selection: [Gram of A or B[:, K]][its workspace][C_KK][factor ws][E_K R^-1][row-norm ws]
    const size_t gws = exact ? ws_round(gram_workspace_bytes(A, ctx->sm_count)) + ws_round((size_t)d * d * 8)
                             : ws_round((size_t)rows * c * 4) + ws_round(qr_workspace_bytes(rows, c));
    const size_t tail = gws + ws_round((size_t)c * c * 8) + ws_round(qr_from_gram_workspace_bytes(c)) +
                        ws_round((size_t)d * c * 4) + ws_round(rownorms_workspace_bytes(A, c, 0, rn_prec)) + 4096;
    rc = ws_ensure(ctx, sketch_bytes(A, r, k, prec, ctx->sm_count, css_bytes(rows, d, c) + tail));
    if (rc) return rc;
    const SketchBufs b = carve(ctx->ws, A, r, k);
    const float* sk;
    int64_t sr;
    CssBufs cb;
    cudaError_t e = css_run(ctx, A, r, k, seed, prec, c, b, &sk, &sr, &cb);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lsk_leverage_scores_hrn (selection)");
    WsCarver wc{(char*)cb.rest, 0};
    if (exact) {
        // Alg. 14: Alg. 13 on A[:, K] -- the Gram of A in FP64, its K x K block,
        // R from it (FP64 accurate) and ||A_i E_K R^-1||^2
        void* gw = wc.take<char>(gram_workspace_bytes(A, ctx->sm_count));
        double* G = wc.take<double>((size_t)d * d);
        double* Csub = wc.take<double>((size_t)c * c);
        void* qw = wc.take<char>(qr_from_gram_workspace_bytes(c));
        e = gram64_launch(A, G, gw, ctx->flag, ctx->sm_count, ctx->stream);
        if (e == cudaSuccess) e = gather_sub_gram_launch(G, d, cb.cols, c, Csub, ctx->stream);
        if (e == cudaSuccess) e = qr_from_gram_launch(Csub, c, nullptr, b.Rinv64, b.Rinv32, qw, ctx->flag, ctx->stream);
    } else {
        // Alg. 16: Alg. 15 on A[:, K] with the sketch restricted to K
        float* Bk = wc.take<float>((size_t)rows * c);
        void* qw = wc.take<char>(qr_workspace_bytes(rows, c));
        e = gather_cols_launch(sk, rows, d, cb.cols, c, Bk, ctx->stream);
        if (e == cudaSuccess)
            e = qr_launch(Bk, rows, c, nullptr, b.Rinv64, b.Rinv32, qw, ctx->flag, ctx->sm_count, ctx->stream);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lsk_leverage_scores_hrn (factor)");
    float* Bf = wc.take<float>((size_t)d * c);
    void* rw = wc.take<char>(rownorms_workspace_bytes(A, c, 0, rn_prec));
    e = embed_rows_launch(b.Rinv32, c, cb.cols, d, Bf, ctx->stream);
    if (e == cudaSuccess)
        e = rownorms_launch(A, Bf, c, 1.0, 0.0, 0, rn_prec, theta, rw, ctx->flag, ctx->sm_count, ctx->stream);
    if (e == cudaSuccess && cols)
        e = cudaMemcpyAsync(cols, cb.cols, (size_t)c * 4, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lsk_leverage_scores_hrn (row norms)");
    return finish(ctx, "lsk_leverage_scores_hrn");
}

// ---- Alg. 13 and Alg. 10: through the FP64 Gram of A ----------------------
namespace {
// G = A^T A (FP64) and R^-1 from it into Rinv64 / Rinv32 (d x d); scratch carved after
cudaError_t gram_factor(lsk_ctx* ctx, const lsk_mat* A, double* G, void* gws, void* qws, double* R_out,
                        double* Rinv64, float* Rinv32) {
    cudaError_t e = gram64_launch(A, G, gws, ctx->flag, ctx->sm_count, ctx->stream);
    if (e != cudaSuccess) return e;
    return qr_from_gram_launch(G, A->d, R_out, Rinv64, Rinv32, qws, ctx->flag, ctx->stream);
}
size_t gram_factor_bytes(const lsk_mat* A, int sm) {
    return ws_round((size_t)A->d * A->d * 8) * 3 + ws_round((size_t)A->d * A->d * 4) +
           ws_round(gram_workspace_bytes(A, sm)) + ws_round(qr_from_gram_workspace_bytes(A->d)) + 2048;
}
}  // namespace

int lsk_leverage_scores_exact(lsk_ctx* ctx, const lsk_mat* A, int32_t prec, float* theta, double* R_out) {
    if (!ctx) return LSK_ERR_INVALID_ARG;
    ProfGuard pg(ctx);
    int rc = check_mat(ctx, A);
    if (rc) return rc;
    if (A->d > 1024) return fail(ctx, LSK_ERR_UNSUPPORTED, "d <= 1024");
    if (!theta && A->n > 0) return fail(ctx, LSK_ERR_INVALID_ARG, "theta is NULL");
    const int32_t rn_prec = prec;   // the row norms keep TF32
    prec = sketch_prec(prec);
    if (prec != LSK_PREC_FP32 && prec != LSK_PREC_BF16)
        return fail(ctx, LSK_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
    const int64_t d = A->d;
    rc = ws_ensure(ctx, gram_factor_bytes(A, ctx->sm_count) + ws_round(rownorms_workspace_bytes(A, d, 1, rn_prec)));
    if (rc) return rc;
    WsCarver wc{(char*)ctx->ws, 0};
    double* G = wc.take<double>((size_t)d * d);
    double* Rinv64 = wc.take<double>((size_t)d * d);
    float* Rinv32 = wc.take<float>((size_t)d * d);
    void* gws = wc.take<char>(gram_workspace_bytes(A, ctx->sm_count));
    void* qws = wc.take<char>(qr_from_gram_workspace_bytes(d));
    void* rws = wc.take<char>(rownorms_workspace_bytes(A, d, 1, rn_prec));
    cudaError_t e = gram_factor(ctx, A, G, gws, qws, R_out, Rinv64, Rinv32);
    if (e == cudaSuccess)
        e = rownorms_launch(A, Rinv32, d, 1.0, 0.0, 1, rn_prec, theta, rws, ctx->flag, ctx->sm_count, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lsk_leverage_scores_exact");
    return finish(ctx, "lsk_leverage_scores_exact");
}

int lsk_least_squares_gram(lsk_ctx* ctx, const lsk_mat* A, const double* b, int32_t refine, double* x) {
    if (!ctx) return LSK_ERR_INVALID_ARG;
    ProfGuard pg(ctx);
    int rc = check_mat(ctx, A);
    if (rc) return rc;
    if (A->d > 1024) return fail(ctx, LSK_ERR_UNSUPPORTED, "d <= 1024");
    if (!x || (!b && A->n > 0)) return fail(ctx, LSK_ERR_INVALID_ARG, "b / x is NULL");
    if (refine < 0 || refine > 10) return fail(ctx, LSK_ERR_INVALID_ARG, "refine must be in [0, 10]");
    const int64_t d = A->d;
    rc = ws_ensure(ctx, gram_factor_bytes(A, ctx->sm_count) + ws_round(atr64_workspace_bytes(A)) +
                            ws_round((size_t)d * 8));
    if (rc) return rc;
    WsCarver wc{(char*)ctx->ws, 0};
    double* G = wc.take<double>((size_t)d * d);
    double* Rinv64 = wc.take<double>((size_t)d * d);
    float* Rinv32 = wc.take<float>((size_t)d * d);
    void* gws = wc.take<char>(gram_workspace_bytes(A, ctx->sm_count));
    void* qws = wc.take<char>(qr_from_gram_workspace_bytes(d));
    void* aws = wc.take<char>(atr64_workspace_bytes(A));
    double* atr = wc.take<double>((size_t)d);
    cudaError_t e = gram_factor(ctx, A, G, gws, qws, nullptr, Rinv64, Rinv32);
    // x = R^-1 R^-T A^T b, then refinement steps on the residual
    for (int t = 0; t <= refine && e == cudaSuccess; ++t) {
        e = atr64_launch(A, b, t ? x : nullptr, atr, aws, ctx->flag, ctx->sm_count, ctx->stream);
        if (e == cudaSuccess) e = seminormal_launch(atr, Rinv64, d, t ? 1 : 0, x, ctx->stream);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lsk_least_squares_gram");
    return finish(ctx, "lsk_least_squares_gram");
}

void lsk_lsq_default_opts(lsk_lsq_opts* o, int64_t d) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->r = d * d > 4 * d ? d * d : 4 * d;
    o->k = 2 * d;
    o->seed = 0;
    o->prec = LSK_PREC_BF16;
    o->max_iter = 100;
    o->max_refine = 8;
    o->tol = 1e-10;
    o->inner_tol = 1e-6;
}

int lsk_sketch_precondition_lsq(lsk_ctx* ctx, const lsk_mat* A, const double* b, double* x,
                                const lsk_lsq_opts* opts, lsk_lsq_info* info) {
    if (!ctx) return LSK_ERR_INVALID_ARG;
    ProfGuard pg(ctx);
    int rc = check_mat(ctx, A);
    if (rc) return rc;
    if (!opts) return fail(ctx, LSK_ERR_INVALID_ARG, "opts is NULL");
    if (!x || (!b && A->n > 0)) return fail(ctx, LSK_ERR_INVALID_ARG, "b / x is NULL");
    int32_t prec = sketch_prec(opts->prec);
    rc = check_sketch_args(ctx, A, opts->r, opts->k, prec);
    if (rc) return rc;
    if (opts->max_iter < 1 || opts->max_refine < 0 || !(opts->tol > 0.0))
        return fail(ctx, LSK_ERR_INVALID_ARG, "bad LSQ options");
    rc = ws_ensure(ctx, sketch_bytes(A, opts->r, opts->k, prec, ctx->sm_count, lsq_workspace_bytes(A)));
    if (rc) return rc;
    const SketchBufs bufs = carve(ctx->ws, A, opts->r, opts->k);
    cudaError_t e = sketch_and_factor(ctx, A, opts->r, opts->k, opts->seed, prec, bufs, nullptr);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lsk_sketch_precondition_lsq (sketch)");
    // the factor must be valid before iterating: read the flag now
    e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lsk_sketch_precondition_lsq (sync)");
    int f = 0;
    cudaMemcpy(&f, ctx->flag, sizeof(int), cudaMemcpyDeviceToHost);
    if (f) {
        cudaMemset(ctx->flag, 0, sizeof(int));
        return flag_to_status(ctx, f);
    }
    lsk_lsq_info tmp;
    rc = lsq_run(ctx, A, b, x, opts, bufs.Rinv64, bufs.Rinv32, bufs.scratch, info ? info : &tmp);
    if (rc == LSK_ERR_CUDA) return fail(ctx, rc, "lsk_sketch_precondition_lsq: CUDA error %s",
                                        cudaGetErrorString(cudaGetLastError()));
    if (rc == LSK_ERR_NOT_CONVERGED) return fail(ctx, rc, "least squares did not reach tol");
    cudaMemcpy(&f, ctx->flag, sizeof(int), cudaMemcpyDeviceToHost);
    if (f) {
        cudaMemset(ctx->flag, 0, sizeof(int));
        return flag_to_status(ctx, f);
    }
    return rc;
}

int lsk_debug_hash(lsk_ctx* ctx, int64_t n, int64_t r, uint64_t seed, int32_t* bucket, int8_t* sign) {
    if (!ctx) return LSK_ERR_INVALID_ARG;
    if (n < 0 || r < 1 || r >= ((int64_t)1 << 32)) return fail(ctx, LSK_ERR_INVALID_ARG, "bad n / r");
    if (n > 0 && (!bucket || !sign)) return fail(ctx, LSK_ERR_INVALID_ARG, "NULL output");
    cudaError_t e = cs_hash_launch(n, r, seed, bucket, sign, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lsk_debug_hash");
    return finish(ctx, "lsk_debug_hash");
}

int lsk_debug_wait_timeout(lsk_ctx* ctx, int64_t limit_us) {
    if (!ctx) return LSK_ERR_INVALID_ARG;
    if (limit_us < 1 || limit_us > 1000000) return fail(ctx, LSK_ERR_INVALID_ARG, "limit_us must be in [1, 1e6]");
    cudaError_t e = debug_wait_timeout_launch(limit_us, ctx->flag, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lsk_debug_wait_timeout");
    return finish(ctx, "lsk_debug_wait_timeout");
}

int lsk_debug_gauss(lsk_ctx* ctx, int64_t k, int64_t r, uint64_t seed, int32_t prec, float* G) {
    if (!ctx) return LSK_ERR_INVALID_ARG;
    if (k < 1 || r < 1 || !G) return fail(ctx, LSK_ERR_INVALID_ARG, "bad k / r / G");
    cudaError_t e = gauss_debug_launch(k, r, seed, sketch_prec(prec) == LSK_PREC_BF16 ? LSK_PREC_BF16 : LSK_PREC_FP32, G,
                                       ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lsk_debug_gauss");
    return finish(ctx, "lsk_debug_gauss");
}

}  // extern "C"

int fused_sketch_on() { return g_fused_sketch.load(); }
