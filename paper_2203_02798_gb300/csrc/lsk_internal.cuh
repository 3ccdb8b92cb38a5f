// lsk_internal.cuh -- shared declarations of the CUDA library behind lsk.h.
//
// Device helpers (counter-based random draws, warp reductions) and the
// internal launchers each .cu file provides to the C-ABI layer (api.cu).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stddef.h>
#include <string.h>

#include <vector>

#include "../../include/lsk.h"
#include "prof.cuh"

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
// Device-side error flag bits (OR-ed by kernels, read by lsk_sync).
enum : int {
    LSK_FLAG_BAD_CSR = 1,
    LSK_FLAG_RANK_DEFICIENT = 2,
    LSK_FLAG_TIMEOUT = 4,
};

struct lsk_ctx {
    int device;
    int sm_count;
    cudaStream_t stream;
    void* ws;             // workspace (device), stream-ordered allocation
    size_t ws_bytes;
    int* flag;            // device int, OR of LSK_FLAG_*
    LskProf* prof;        // per-kernel event timings (NULL until enabled)
    int prof_on;
    struct LskBatch* batch;   // batch driver state (streams, workspaces, graph)
    char err[512];
};
void lsk_batch_free(lsk_ctx* ctx);

LskProf* lsk_prof_new();
void lsk_prof_delete(LskProf* p);

// Points lsk_prof_current at the context's profiler while a call runs.
struct ProfGuard {
    ProfGuard(lsk_ctx* ctx) { lsk_prof_current = (ctx && ctx->prof_on) ? ctx->prof : nullptr; }
    ~ProfGuard() { lsk_prof_current = nullptr; }
};

// Bump allocator over the context workspace (256-byte aligned pieces).
struct WsCarver {
    char* base;
    size_t off;
    template <class T>
    T* take(size_t count) {
        off = (off + 255) & ~size_t(255);
        T* p = reinterpret_cast<T*>(base + off);
        off += count * sizeof(T);
        return p;
    }
};
inline size_t ws_round(size_t b) { return (b + 255) & ~size_t(255); }

// Allow `fn` the largest dynamic shared memory it can use on the current
// device (the opt-in maximum less its static shared memory), once per function
// and device.  The attribute is process-wide: setting it to each launch's own
// size would race between host threads launching different sizes (a launch
// could see another thread's smaller limit and fail with invalid argument).
cudaError_t allow_dynamic_smem(const void* fn);
template <class F>
inline cudaError_t allow_dynamic_smem(F* fn) { return allow_dynamic_smem(reinterpret_cast<const void*>(fn)); }

// ---------------------------------------------------------------------------
// grouped launches: one grid runs the blocks of many independent problems.
// Problem p owns blocks [off[p], off[p + 1]); off has count + 1 ascending
// entries.  Per-problem parameters and offsets are packed on the host into one
// table (HostTable), copied to the device once per batch plan, and read by the
// grouped kernels through offsets into that device copy.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int group_of(const int* __restrict__ off, int count, int b) {
    int lo = 0, hi = count;   // off[lo] <= b < off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(off + mid) <= b) lo = mid;
        else hi = mid;
    }
    return lo;
}

struct HostTable {
    std::vector<unsigned char> bytes;
    template <class T>
    size_t put(const T* p, size_t n) {
        const size_t o = (bytes.size() + 15) & ~size_t(15);
        bytes.resize(o + sizeof(T) * n);
        if (n) memcpy(bytes.data() + o, p, sizeof(T) * n);
        return o;
    }
};

// Offsets of `count` problems with blocks[p] blocks each; returns the total.
inline int group_offsets(const std::vector<int>& blocks, std::vector<int>& off) {
    off.assign(blocks.size() + 1, 0);
    for (size_t p = 0; p < blocks.size(); ++p) off[p + 1] = off[p] + blocks[p];
    return off.back();
}

// ---------------------------------------------------------------------------
// Philox-4x32-10 (Salmon et al., SC'11).  Round: multiply words 0 and 2 by
// the two Philox multipliers, recombine high/low halves with words 1, 3 and
// the key; the key advances by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int rnd = 0; rnd < 10; ++rnd) {
        if (rnd) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// CountSketch column i (Def. 3): bucket h(i) in [0, r) by multiply-shift of
// the first word, sign from the top bit of the second word.
__device__ __forceinline__ void cs_hash(uint64_t i, uint32_t r, uint32_t k0, uint32_t k1,
                                        uint32_t& bucket, uint32_t& negative) {
    const uint4 w = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)(i >> 32), 0u, 0u), k0, k1);
    bucket = __umulhi(w.x, r);
    negative = w.y >> 31;
}

// Box-Muller pair from two 32-bit words: 24-bit uniforms u1 = (a+1) 2^-24,
// u2 = b 2^-24 (both exact in float32), z0 = rho cos(2 pi u2), z1 = rho sin.
__device__ __forceinline__ float2 box_muller24(uint32_t wa, uint32_t wb) {
    const float u1 = (float)((wa >> 8) + 1u) * 5.9604644775390625e-08f;   // 2^-24, exact
    const float rho = sqrtf(-2.0f * logf(u1));
    float s, co;
    sincospif((float)(wb >> 8) * 1.1920928955078125e-07f, &s, &co);      // 2 u2 = b 2^-23, exact
    return make_float2(rho * co, rho * s);
}

// Four Gaussian entries G[4q + t, c], t = 0..3, unscaled (pairs (w0, w1) and
// (w2, w3); even rows take the cosine branch).  stream: the third counter
// word (1 for the Gaussian stage G, 2 for the right projection Pi of Alg. 15).
__device__ __forceinline__ float4 gauss4(uint64_t c, uint32_t q, uint32_t k0, uint32_t k1, uint32_t stream = 1u) {
    const uint4 w = philox4x32_10(make_uint4((uint32_t)c, (uint32_t)(c >> 32), stream, q), k0, k1);
    const float2 z01 = box_muller24(w.x, w.y);
    const float2 z23 = box_muller24(w.z, w.w);
    return make_float4(z01.x, z01.y, z23.x, z23.y);
}

__device__ __forceinline__ float bf16_round(float x) {
    return __bfloat162float(__float2bfloat16_rn(x));
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void set_flag(int* flag, int bit) {
    if (flag) atomicOr(flag, bit);
}

// ---------------------------------------------------------------------------
// internal launchers (all asynchronous on `st`)
// ---------------------------------------------------------------------------
// countsketch.cu
size_t cs_workspace_bytes(int64_t n, int64_t r);          // with the two-level sort's scratch
size_t cs_workspace_bytes_atomic(int64_t n, int64_t r);   // count / scan / place with L2 atomics only
// row0: global index of A's first row (A is a block of rows of a larger matrix);
// accumulate: SA += S A (SA holds a previous block's sketch) instead of SA = S A
// cidx / ccount (both or neither): compact SA to the non-empty buckets in
// bucket order -- row j of SA is bucket cidx[j], *ccount rows in all (the rows
// past it are left as they were); not with accumulate
cudaError_t cs_launch(const lsk_mat* A, int64_t r, uint64_t seed, float* SA, void* ws,
                      int* flag, int sm_count, cudaStream_t st, uint64_t row0 = 0, bool accumulate = false,
                      uint32_t* cidx = nullptr, uint32_t* ccount = nullptr, bool rx = true);
cudaError_t cs_hash_launch(int64_t n, int64_t r, uint64_t seed, int32_t* bucket, int8_t* sign,
                           cudaStream_t st);
// The gather step alone (S A from a prepared permutation: off[b] .. off[b+1]
// of perm are bucket b's rows, local row index | sign << 31; cpos: compact to
// the non-empty buckets' ranks).
cudaError_t cs_gather_launch(const lsk_mat* A, int64_t r, const uint32_t* off, const uint32_t* perm,
                             const uint32_t* cpos, float* SA, int* flag, int sm_count, cudaStream_t st,
                             bool accumulate = false);
// Grouped preparation of many problems' CountSketch permutations (count, one
// scan, place, compaction) in a handful of launches; problem j then gathers
// with off = g.off + jobs[j].cnt_base, perm = g.perm, cpos = g.cpos +
// jobs[j].cnt_base when it compacts.
struct CsJob {
    int64_t n, r;
    uint64_t seed;
    uint32_t* cidx;       // cs_launch's compaction outputs (or null)
    uint32_t* ccount;
    int64_t cnt_base;     // set by cs_group_build
};
struct CsGroup {
    size_t params_off = 0, rowoff_off = 0;
    int count = 0;
    int64_t rows = 0, counters = 0;
    bool any_compact = false;
    uint32_t *cnt = nullptr, *off = nullptr, *cursor = nullptr, *cpos = nullptr, *perm = nullptr, *tmp = nullptr;
};
size_t cs_group_ws_bytes(int64_t rows, int64_t counters);
void cs_group_build(std::vector<CsJob>& jobs, void* ws, HostTable& t, CsGroup& g);
cudaError_t cs_group_launch(const CsGroup& g, const unsigned char* table, int sm_count, cudaStream_t st);

// gauss_tc.cu: grouped Gaussian stage (BF16) over many sketches
struct GaussJob {
    const float* SA;
    int64_t r, d, k;
    uint64_t seed;
    float* GSA;
    float* part;             // gauss_group_part_bytes(r, d, k, slice_chunks) bytes
    int slice_chunks;        // chunks of 32 columns of r per block (0: the default, 128)
    // compacted sketch (cs_launch's cidx / ccount): SA's row j is bucket idx[j]
    // of *rcount rows; r is then an upper bound (the slices are planned on it)
    const uint32_t* idx = nullptr;
    const uint32_t* rcount = nullptr;
};
struct GaussGroup {
    size_t params_off, off_off, roff_off;
    int count, blocks, rblocks;
    size_t smem;
};
// terms = 1: the BF16 mode; 3: the FP32 mode on the tensor cores
bool gauss_tc_supported(int64_t r, int64_t d, int64_t k, int terms = 1);
size_t gauss_group_part_bytes(int64_t r, int64_t d, int64_t k, int slice_chunks = 0);
void gauss_group_build(const std::vector<GaussJob>& jobs, HostTable& t, GaussGroup& g);
cudaError_t gauss_group_launch(const GaussGroup& g, const unsigned char* table, cudaStream_t st);

// gauss.cu
size_t gauss_workspace_bytes(int64_t r, int64_t d, int64_t k, int32_t prec, int sm_count);
cudaError_t gauss_launch(const float* SA, int64_t r, int64_t d, int64_t k, uint64_t seed,
                         int32_t prec, float* GSA, void* ws, int sm_count, cudaStream_t st);
cudaError_t add_into_launch(float* dst, const float* src, int64_t len, cudaStream_t st);
cudaError_t gauss_debug_launch(int64_t k, int64_t r, uint64_t seed, int32_t prec, float* G,
                               cudaStream_t st);

// gram.cu
size_t gram_workspace_bytes(const lsk_mat* A, int sm_count);
// A^T A with FP64 output (the same partials, summed and stored in FP64)
cudaError_t gram64_launch(const lsk_mat* A, double* C, void* ws, int* flag, int sm_count, cudaStream_t st);
cudaError_t gram_launch(const lsk_mat* A, double alpha, double beta, float* C, void* ws,
                        int* flag, int sm_count, cudaStream_t st);

// gram_tc.cu (dense, d <= 256, BF16x3 on tcgen05)
bool gram_tc_supported(const lsk_mat* A);
size_t gram_tc_workspace_bytes(const lsk_mat* A, int sm_count);
cudaError_t gram_tc_launch(const lsk_mat* A, double alpha, double beta, float* C, void* ws, int* flag,
                           int sm_count, cudaStream_t st);

// LSK_PREC_TF32 is the BF16 mode with the row-norm GEMM A B in TF32: every
// stage other than the row norms takes the BF16 arithmetic
inline int32_t sketch_prec(int32_t prec) { return prec == LSK_PREC_TF32 ? LSK_PREC_BF16 : prec; }

// rownorms.cu
size_t rownorms_workspace_bytes(const lsk_mat* A, int64_t c, int upper_tri, int32_t prec);
// min_tiles: the dense tensor-core form launches CTAs for at least that many
// 128-row tiles each (a small problem leaves SMs to concurrent work)
// prepared (nullable): B's operand built beforehand by a grouped launch -- the
// tensor-core image (rownorms_image_group_launch) for dense BF16, B B^T
// (bbt_group_launch) for CSR -- so this launch skips building it
cudaError_t rownorms_launch(const lsk_mat* A, const float* B, int64_t c, double alpha,
                            double beta, int upper_tri, int32_t prec, float* x, void* ws, int* flag,
                            int sm_count, cudaStream_t st, int min_tiles = 16, const void* prepared = nullptr);
struct BbtJob {
    const float* B;
    int64_t d, c;
    float* M;            // d x d
};
struct BbtGroup {
    size_t params_off = 0, off_off = 0;
    int count = 0, blocks = 0;
};
void bbt_group_build(const std::vector<BbtJob>& jobs, HostTable& t, BbtGroup& g);
cudaError_t bbt_group_launch(const BbtGroup& g, const unsigned char* table, cudaStream_t st);
// rownorms_tc.cu; tf32: the TMA-fed CTA-pair kernel with one TF32 product
// (A rounded to the nearest TF32 in shared memory) instead of BF16x3 (the
// same workspace; img_ready is for the BF16x3 form only)
bool rownorms_tc_supported(const lsk_mat* A, int64_t c, int upper_tri, bool tf32 = false);
size_t rownorms_tc_workspace_bytes(const lsk_mat* A, int64_t c, int upper_tri);
cudaError_t rownorms_tc_launch(const lsk_mat* A, const float* B, int64_t c, float alpha, float beta,
                               int upper_tri, float* x, void* ws, int* flag, int sm_count, cudaStream_t st,
                               int min_tiles = 16, const uint8_t* img_ready = nullptr, bool tf32 = false);
// the tensor-core images of many problems' B (rownorms_tc_workspace_bytes each)
struct RnImageJob {
    lsk_mat A;
    const float* B;
    int64_t c;
    int upper_tri;
    uint8_t* img;
};
struct RnImageGroup {
    size_t params_off = 0, off_off = 0;
    int count = 0, blocks = 0;
};
void rownorms_image_group_build(const std::vector<RnImageJob>& jobs, HostTable& t, RnImageGroup& g);
cudaError_t rownorms_image_group_launch(const RnImageGroup& g, const unsigned char* table, cudaStream_t st);

// qr.cu
size_t qr_workspace_bytes(int64_t k, int64_t d);
// the two halves of qr_launch: C = B^T B in FP64 (pair-FP32 products), then
// R, R^-1 from an FP64 Gram C (d <= 1024; C is overwritten when d > 256)
size_t sketch_gram64_workspace_bytes(int64_t k, int64_t d);
// Cp (nullable): the same Gram as FP32 pairs (hi + lo)
cudaError_t sketch_gram64_launch(const float* B, int64_t k, int64_t d, double* C, void* ws, int sm_count,
                                 cudaStream_t st, float2* Cp = nullptr);
size_t qr_from_gram_workspace_bytes(int64_t d);
cudaError_t qr_from_gram_launch(double* C, int64_t d, double* R, double* Rinv, float* Rinv32, void* ws, int* flag,
                                cudaStream_t st, const float2* Cp = nullptr);
cudaError_t qr_launch(const float* B, int64_t k, int64_t d, double* R, double* Rinv,
                      float* Rinv32, void* ws, int* flag, int sm_count, cudaStream_t st);

// Grouped R^-1 of many sketches (d <= 256, the mixed-precision path): every
// stage of qr_launch, each one grid over all problems.  R is not formed.
struct QrJob {
    const float* B;          // sketch, k x d row-major
    int64_t k, rows_per;
    int d, nchunks, ntiles;
    double* part;            // Gram partials
    double* C;               // FP64 Gram
    float2* Cp;              // the Gram as FP32 pairs (hi + lo)
    float2 *X, *W, *M, *Y;   // pair matrices of the correction step
    float* Lpk;              // packed FP32 Cholesky factor
    int* e;                  // equilibration exponents
    double* Rinv;            // nullable
    float* Rinv32;
    int* flag;
};
enum QrShape { QS_GRAM, QS_GRAMRED, QS_ONE, QS_TRINV, QS_TRI, QS_N };
struct QrGroup {
    size_t jobs_off, off_off[QS_N];
    int count, blocks[QS_N], dmax;
};
bool qr_group_supported(int64_t k, int64_t d);
void qr_group_job(QrJob& j, const float* B, int64_t k, int64_t d, void* ws, double* Rinv, float* Rinv32, int* flag);
void qr_group_build(const std::vector<QrJob>& jobs, HostTable& t, QrGroup& g);
cudaError_t qr_group_launch(const QrGroup& g, const unsigned char* table, cudaStream_t st);
// qr_mixed.cu (pieces of the grouped path)
void qr_mixed_carve(QrJob& j, void* ws);
int qr_mixed_blocks(int d, int shape);
cudaError_t qr_mixed_group_launch(const QrGroup& g, const unsigned char* table, cudaStream_t st);

// lsq.cu
size_t lsq_workspace_bytes(const lsk_mat* A);
int lsq_run(lsk_ctx* ctx, const lsk_mat* A, const double* b, double* x, const lsk_lsq_opts* o,
            const double* Rinv64, const float* Rinv32, void* ws, lsk_lsq_info* info);

// jl.cu: X = R^-1 Pi for Alg. 15 (Pi: d x m Gaussian / sqrt(m), stream 2)
size_t jl_workspace_bytes(int64_t d, int64_t m);
cudaError_t jl_launch(const double* Rinv64, int64_t d, int64_t m, uint64_t seed, float* X32, void* ws,
                      cudaStream_t st);

// css.cu: column subset selection (Alg. 9) pieces
size_t pivchol_workspace_bytes(int64_t d, int64_t c);
cudaError_t pivchol_launch(const double* C, int64_t d, int64_t c, double rcond, int flag_rank, int32_t* cols,
                           int* rank_out, void* ws, int* flag, cudaStream_t st);
cudaError_t gather_sub_gram_launch(const double* C, int64_t d, const int32_t* cols, int64_t c, double* Csub,
                                   cudaStream_t st);
cudaError_t gather_cols_launch(const float* B, int64_t rows, int64_t d, const int32_t* cols, int64_t c, float* Bk,
                               cudaStream_t st);
cudaError_t embed_rows_launch(const float* X, int64_t c, const int32_t* cols, int64_t d, float* Bf, cudaStream_t st);

// jlt.cu: Gaussian sketch of a CSR matrix (Alg. 4), C = G A, stream 3
bool jlt_supported(int64_t d, int64_t m);
size_t jlt_workspace_bytes(int64_t n, int64_t d, int64_t m, int sm_count);
cudaError_t jlt_launch(const lsk_mat* A, int64_t m, uint64_t seed, int32_t prec, float* C, void* ws, int* flag,
                       int sm_count, cudaStream_t st);

// lsq.cu: atr = A^T (b - A x) in FP64 (x == nullptr: x = 0)
size_t atr64_workspace_bytes(const lsk_mat* A);
cudaError_t atr64_launch(const lsk_mat* A, const double* b, const double* x, double* atr, void* ws, int* flag,
                         int sm_count, cudaStream_t st);
// solve.cu: x (+)= R^-1 R^-T c (one block, d <= 1024)
cudaError_t seminormal_launch(const double* c, const double* Rinv64, int64_t d, int add, double* x, cudaStream_t st);

// solve.cu: sketch-and-solve (Alg. 11) given the sketch A~ of A and R^-1
size_t solve_workspace_bytes(int64_t r, int64_t k, int64_t d);
cudaError_t solve_launch(const lsk_mat* A, const double* b, int64_t r, int64_t k, uint64_t seed, int32_t prec,
                         const float* At, const double* Rinv64, double* x, void* ws, int sm_count, cudaStream_t st);

// debug_wait.cu
cudaError_t debug_wait_timeout_launch(int64_t limit_us, int* flag, cudaStream_t st);

// api.cu (used by the batch driver)
size_t leverage_workspace_bytes(const lsk_mat* A, int64_t r, int64_t k, int32_t prec, int sm);
cudaError_t leverage_pipeline(const lsk_mat* A, int64_t r, int64_t k, uint64_t seed, int32_t prec, float* ell,
                              double* R_out, void* ws, int* flag, int sm, cudaStream_t st);
int check_leverage_args(lsk_ctx* ctx, const lsk_mat* A, int64_t r, int64_t k, int32_t prec);
// the process-wide fused-sketch switch (lsk_set_fused_sketch)
int fused_sketch_on();
