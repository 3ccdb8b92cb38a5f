// lsq.cu -- sketch-and-precondition least squares (Alg. 12).
//
// Alg. 12 leaves the "parallel preconditioned iterative method" open; the
// reading used here is a preconditioned Krylov solve with N = R^-1 from the
// sketch, wrapped in FP64 iterative refinement:
//     r_t = b - A x_t   (FP64, A's FP32 values taken exactly)
//     g_t = N^T A^T r_t (FP64, from the same pass)
//     eta_t = ||A^T r_t|| / ||A^T b||          stop when eta_t <= tol
//     z = CG(N^T A^T A N, g_t) to inner_tol;  x_{t+1} = x_t + N z   (FP64)
// The inner solve is conjugate gradients on the preconditioned normal
// equations (CGLS, Hestenes & Stiefel 1952), mathematically the same Krylov
// iterates as LSQR on min ||A N y - r_t||, but with the right-hand side g_t
// formed in FP64: its FP32 products are then relative to the correction
// being sought, not to r_t, so a refinement step gains ~inner_tol even when
// the residual is large (LSQR's FP32 vectors carry r_t and stall at about
// eps32 sqrt(n) there).  Each CG iteration makes ONE pass over A: the block
// that forms u_i = A_i p immediately adds u_i A_i^T into its partial of A^T u
// while the row is still in registers.  The FP64 residual pass likewise forms
// r_i and accumulates r_i A_i^T in the same read.  Scalars live on the
// device; the host reads them back every few iterations for the stop test.
#include "lsk_internal.cuh"

#include <math.h>

#include <algorithm>
#include <string.h>

namespace {

struct LsqrState {
    double alpha, beta, rhobar, phibar, anorm2, atb_norm, eta, bnorm;
    double arnorm, rnorm;
    int done, it;
    double rho, rho0;   // CG on the normal equations: ||s||^2 now and at the start
};

constexpr int kPassThreads = 256;

// ---- FP64 residual + A^T r, dense: warp per row ---------------------------
__global__ void __launch_bounds__(kPassThreads) resid64_dense_kernel(
    const float* __restrict__ A, int64_t lda, int64_t n, int64_t d, const double* __restrict__ b,
    const double* __restrict__ x, float* __restrict__ u32, double* __restrict__ qpart,
    double* __restrict__ sspart) {
    extern __shared__ double sh[];   // x (d) then per-warp q (8 * d)
    double* xs = sh;
    double* qs = sh + d;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t j = threadIdx.x; j < d; j += blockDim.x) xs[j] = x[j];
    for (int64_t j = threadIdx.x; j < 8 * d; j += blockDim.x) qs[j] = 0.0;
    __syncthreads();
    double* qw = qs + w * d;
    double ss = 0.0;
    const int64_t wid = (int64_t)blockIdx.x * 8 + w, nw = (int64_t)gridDim.x * 8;
    for (int64_t i = wid; i < n; i += nw) {
        const float* row = A + i * lda;
        double dot = 0.0;
        for (int64_t j = lane; j < d; j += 32) dot = fma((double)row[j], xs[j], dot);
        dot = warp_sum(dot);
        const double ri = b[i] - dot;
        if (lane == 0) u32[i] = (float)ri;
        ss = fma(ri, ri, ss);
        for (int64_t j = lane; j < d; j += 32) qw[j] = fma((double)row[j], ri, qw[j]);
    }
    __syncthreads();
    for (int64_t j = threadIdx.x; j < d; j += blockDim.x) {
        double s = 0.0;
        for (int t = 0; t < 8; ++t) s += qs[t * d + j];
        qpart[(int64_t)blockIdx.x * d + j] = s;
    }
    // each warp's ss is replicated across lanes (ri is uniform): lane 0 adds
    __shared__ double ssw[8];
    if (lane == 0) ssw[w] = ss;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int t = 0; t < 8; ++t) s += ssw[t];
        sspart[blockIdx.x] = s;
    }
}

// ---- FP64 residual + A^T r, CSR: thread per row ----------------------------
__global__ void __launch_bounds__(kPassThreads) resid64_csr_kernel(
    const float* __restrict__ V, const int32_t* __restrict__ J, const int64_t* __restrict__ I,
    int64_t n, int64_t nnz, int64_t d, const double* __restrict__ b, const double* __restrict__ x,
    float* __restrict__ u32, double* __restrict__ qpart, double* __restrict__ sspart, int* flag) {
    extern __shared__ double sh[];
    double* xs = sh;
    double* qs = sh + d;
    for (int64_t j = threadIdx.x; j < d; j += blockDim.x) {
        xs[j] = x[j];
        qs[j] = 0.0;
    }
    __syncthreads();
    double ss = 0.0;
    bool bad = false;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int64_t k0 = I[i], k1 = I[i + 1];
        double dot = 0.0;
        const bool ok = !(k0 < 0 || k1 < k0 || k1 > nnz);
        if (!ok) bad = true;
        if (ok)
            for (int64_t p = k0; p < k1; ++p) {
                const int32_t j = J[p];
                if (j >= 0 && j < d) dot = fma((double)V[p], xs[j], dot);
                else bad = true;
            }
        const double ri = b[i] - dot;
        u32[i] = (float)ri;
        ss = fma(ri, ri, ss);
        if (ok)
            for (int64_t p = k0; p < k1; ++p) {
                const int32_t j = J[p];
                if (j >= 0 && j < d) atomicAdd(&qs[j], (double)V[p] * ri);
            }
    }
    if (bad) set_flag(flag, LSK_FLAG_BAD_CSR);
    ss = warp_sum(ss);
    __shared__ double ssw[kPassThreads / 32];
    if ((threadIdx.x & 31) == 0) ssw[threadIdx.x >> 5] = ss;
    __syncthreads();
    for (int64_t j = threadIdx.x; j < d; j += blockDim.x) qpart[(int64_t)blockIdx.x * d + j] = qs[j];
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int t = 0; t < kPassThreads / 32; ++t) s += ssw[t];
        sspart[blockIdx.x] = s;
    }
}

// out[j] = sum_z part[z][j] in z order groups: with blockDim >= 4d the
// partials are split four ways (z mod 4) and the four sums added in order.
__device__ __forceinline__ void reduce_partials(const float* __restrict__ part, int nblocks, int64_t d,
                                                float* __restrict__ out) {
    __shared__ float red4[4][256];
    if (d <= 256 && blockDim.x >= 4 * d) {
        const int j = threadIdx.x % d, g = threadIdx.x / d;
        if (g < 4) {
            float s = 0.f;
            for (int z = g; z < nblocks; z += 4) s += part[(int64_t)z * d + j];
            red4[g][j] = s;
        }
        __syncthreads();
        if (threadIdx.x < d) out[threadIdx.x] = (red4[0][threadIdx.x] + red4[1][threadIdx.x]) +
                                                (red4[2][threadIdx.x] + red4[3][threadIdx.x]);
    } else {
        for (int64_t j = threadIdx.x; j < d; j += blockDim.x) {
            float s = 0.f;
            for (int z = 0; z < nblocks; ++z) s += part[(int64_t)z * d + j];
            out[j] = s;
        }
    }
}

// u <- A p - (alpha/beta) u; partial sums of u^2 and of A^T u.  Dense,
// d <= 256: a warp takes RB rows at a time (all RB rows' loads in flight
// before any arithmetic), lane l owns columns l, l + 32, ... (CPL of them),
// so p and the warp's share of A^T u stay in registers.
template <int CPL, int RB>
__global__ void __launch_bounds__(kPassThreads, 2) lsqr_pass_dense_rows_kernel(
    const float* __restrict__ A, int64_t lda, int64_t n, int64_t d, const float* __restrict__ p,
    const LsqrState* __restrict__ st, float* __restrict__ u, float* __restrict__ qpart,
    double* __restrict__ sspart) {
    __shared__ float qs[kPassThreads / 32][CPL * 32];
    __shared__ double ssw[kPassThreads / 32];
    if (st->done) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float pr[CPL], q[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
        const int j = lane + 32 * c;
        pr[c] = j < d ? p[j] : 0.f;
        q[c] = 0.f;
    }
    const float ab = (st->beta > 0.0) ? (float)(st->alpha / st->beta) : 0.f;
    double ss = 0.0;
    const int64_t nw = (int64_t)gridDim.x * (kPassThreads / 32);
    for (int64_t i0 = ((int64_t)blockIdx.x * (kPassThreads / 32) + w) * RB; i0 < n; i0 += nw * RB) {
        float a[RB][CPL];
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            const int64_t row = i0 + r;
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
                const int j = lane + 32 * c;
                a[r][c] = (row < n && j < d) ? __ldg(A + row * lda + j) : 0.f;
            }
        }
        const float uold = (lane < RB && i0 + lane < n) ? u[i0 + lane] : 0.f;
        float dot[RB];
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            float t = 0.f;
#pragma unroll
            for (int c = 0; c < CPL; ++c) t = fmaf(a[r][c], pr[c], t);
            dot[r] = t;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1)
#pragma unroll
            for (int r = 0; r < RB; ++r) dot[r] += __shfl_xor_sync(0xffffffffu, dot[r], o);
        float unew = 0.f;
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            const float ui = (i0 + r < n) ? dot[r] - ab * __shfl_sync(0xffffffffu, uold, r) : 0.f;
            if (lane == r) unew = ui;
#pragma unroll
            for (int c = 0; c < CPL; ++c) q[c] = fmaf(a[r][c], ui, q[c]);
        }
        if (lane < RB && i0 + lane < n) {
            u[i0 + lane] = unew;
            ss = fma((double)unew, (double)unew, ss);
        }
    }
#pragma unroll
    for (int c = 0; c < CPL; ++c) qs[w][lane + 32 * c] = q[c];
    ss = warp_sum(ss);
    if (lane == 0) ssw[w] = ss;
    __syncthreads();
    for (int64_t j = threadIdx.x; j < d; j += blockDim.x) {
        float t = 0.f;
#pragma unroll
        for (int z = 0; z < kPassThreads / 32; ++z) t += qs[z][j];
        qpart[(int64_t)blockIdx.x * d + j] = t;
    }
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int z = 0; z < kPassThreads / 32; ++z) t += ssw[z];
        sspart[blockIdx.x] = t;
    }
}

// u <- A p - (alpha/beta) u; partial sums of u^2 and of A^T u.  Dense, any d:
// warp per row.
__global__ void __launch_bounds__(kPassThreads) lsqr_pass_dense_kernel(
    const float* __restrict__ A, int64_t lda, int64_t n, int64_t d, const float* __restrict__ p,
    const LsqrState* __restrict__ st, float* __restrict__ u, float* __restrict__ qpart,
    double* __restrict__ sspart) {
    extern __shared__ float shf[];   // p (d) then per-warp q (8 * d)
    if (st->done) return;
    float* ps = shf;
    float* qs = shf + d;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t j = threadIdx.x; j < d; j += blockDim.x) ps[j] = p[j];
    for (int64_t j = threadIdx.x; j < 8 * d; j += blockDim.x) qs[j] = 0.f;
    __syncthreads();
    const float ab = (st->beta > 0.0) ? (float)(st->alpha / st->beta) : 0.f;
    float* qw = qs + w * d;
    double ss = 0.0;
    const int64_t wid = (int64_t)blockIdx.x * 8 + w, nw = (int64_t)gridDim.x * 8;
    for (int64_t i = wid; i < n; i += nw) {
        const float* row = A + i * lda;
        float dot = 0.f;
        for (int64_t j = lane; j < d; j += 32) dot = fmaf(row[j], ps[j], dot);
        dot = warp_sum(dot);
        const float ui = dot - ab * u[i];
        __syncwarp();
        if (lane == 0) u[i] = ui;
        ss = fma((double)ui, (double)ui, ss);
        for (int64_t j = lane; j < d; j += 32) qw[j] = fmaf(row[j], ui, qw[j]);
    }
    __syncthreads();
    for (int64_t j = threadIdx.x; j < d; j += blockDim.x) {
        float s = 0.f;
        for (int t = 0; t < 8; ++t) s += qs[t * d + j];
        qpart[(int64_t)blockIdx.x * d + j] = s;
    }
    __shared__ double ssw[8];
    if (lane == 0) ssw[w] = ss;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int t = 0; t < 8; ++t) s += ssw[t];
        sspart[blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(kPassThreads) lsqr_pass_csr_kernel(
    const float* __restrict__ V, const int32_t* __restrict__ J, const int64_t* __restrict__ I,
    int64_t n, int64_t nnz, int64_t d, const float* __restrict__ p, const LsqrState* __restrict__ st,
    float* __restrict__ u, float* __restrict__ qpart, double* __restrict__ sspart) {
    extern __shared__ float shf[];
    if (st->done) return;
    float* ps = shf;
    float* qs = shf + d;
    for (int64_t j = threadIdx.x; j < d; j += blockDim.x) {
        ps[j] = p[j];
        qs[j] = 0.f;
    }
    __syncthreads();
    const float ab = (st->beta > 0.0) ? (float)(st->alpha / st->beta) : 0.f;
    double ss = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int64_t k0 = I[i], k1 = I[i + 1];
        const bool ok = !(k0 < 0 || k1 < k0 || k1 > nnz);
        float dot = 0.f;
        if (ok)
            for (int64_t q = k0; q < k1; ++q) {
                const int32_t j = J[q];
                if (j >= 0 && j < d) dot = fmaf(V[q], ps[j], dot);
            }
        const float ui = dot - ab * u[i];
        u[i] = ui;
        ss = fma((double)ui, (double)ui, ss);
        if (ok)
            for (int64_t q = k0; q < k1; ++q) {
                const int32_t j = J[q];
                if (j >= 0 && j < d) atomicAdd(&qs[j], V[q] * ui);
            }
    }
    ss = warp_sum(ss);
    __shared__ double ssw[kPassThreads / 32];
    if ((threadIdx.x & 31) == 0) ssw[threadIdx.x >> 5] = ss;
    __syncthreads();
    for (int64_t j = threadIdx.x; j < d; j += blockDim.x) qpart[(int64_t)blockIdx.x * d + j] = qs[j];
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int t = 0; t < kPassThreads / 32; ++t) s += ssw[t];
        sspart[blockIdx.x] = s;
    }
}

// ---- inner solve: CG on the preconditioned normal equations ----------------
// N^T A^T A N z = g with g = N^T A^T r formed in FP64 by the residual pass.
// The pass kernels run with alpha = 0 (u = A p): u = A N p_cg, A^T u and
// ||u||^2 in FP32 / FP64; the d-vectors (z, s, p_cg) stay in FP64.  Unlike
// LSQR on min ||A N y - r||, whose FP32 n-vectors carry r itself (mostly
// orthogonal to range(A) when the residual is large), every FP32 quantity
// here is relative to the correction being sought, so each refinement step
// gains ~inner_tol whatever the size of the residual.

// p = N v for an FP64 d-vector staged in shared memory (N upper triangular):
// one warp per row of N, so consecutive lanes read consecutive entries
__device__ __forceinline__ void apply_n(const double* __restrict__ N64, int64_t d, const double* vs, float* p) {
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int64_t i = threadIdx.x >> 5; i < d; i += nw) {
        double t = 0.0;
        for (int64_t j = i + lane; j < d; j += 32) t = fma(N64[i * d + j], vs[j], t);
        t = warp_sum(t);
        if (lane == 0) p[i] = (float)t;
    }
}

// Start of an inner solve after the residual pass: A^T r, eta,
// g = N^T A^T r, s = p_cg = g, z = 0, p = N p_cg.  One block.
__global__ void cg_start_kernel(const double* __restrict__ qpart, int nblocks, int64_t d,
                                const double* __restrict__ N64, int first, LsqrState* st,
                                double* __restrict__ s, double* __restrict__ pc, double* __restrict__ z,
                                double* __restrict__ atr, float* __restrict__ p) {
    __shared__ double red[32];
    __shared__ double pcs[1024];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t j = threadIdx.x; j < d; j += blockDim.x) {
        double t = 0.0;
        for (int q = 0; q < nblocks; ++q) t += qpart[(int64_t)q * d + j];
        atr[j] = t;
    }
    __syncthreads();
    double a2 = 0.0, g2 = 0.0;
    for (int64_t j = threadIdx.x; j < d; j += blockDim.x) {
        a2 = fma(atr[j], atr[j], a2);
        double t = 0.0;
        for (int64_t i = 0; i <= j; ++i) t = fma(N64[i * d + j], atr[i], t);   // (N^T A^T r)_j
        s[j] = t;
        pc[j] = t;
        pcs[j] = t;
        z[j] = 0.0;
        g2 = fma(t, t, g2);
    }
    a2 = warp_sum(a2);
    g2 = warp_sum(g2);
    if (lane == 0) {
        red[wid] = a2;
        red[16 + wid] = g2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double A2 = 0.0, G2 = 0.0;
        for (int t = 0; t < nw; ++t) {
            A2 += red[t];
            G2 += red[16 + t];
        }
        const double atrn = sqrt(A2);
        if (first) st->atb_norm = atrn;
        st->eta = (st->atb_norm > 0.0) ? atrn / st->atb_norm : 0.0;
        st->alpha = 0.0;           // the pass forms u = A p
        st->beta = 1.0;
        st->rho = G2;
        st->rho0 = G2;
        st->it = 0;
        st->done = (G2 == 0.0) ? 1 : 0;
    }
    __syncthreads();
    apply_n(N64, d, pcs, p);
}

// One CG step after the pass: gamma = ||A N p_cg||^2, w = N^T (A^T u),
// z += a p_cg, s -= a w, p_cg = s + b p_cg, p = N p_cg.  One block.
__global__ void cg_step_kernel(const float* __restrict__ qpart, const double* __restrict__ sspart, int nblocks,
                               int64_t d, const double* __restrict__ N64, LsqrState* st, double* __restrict__ s,
                               double* __restrict__ pc, double* __restrict__ z, float* __restrict__ qtmp,
                               double inner_tol, float* __restrict__ p) {
    __shared__ double red[32];
    __shared__ double sc[2];
    __shared__ double pcs[1024];
    if (st->done) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double g2 = 0.0;
    for (int q = threadIdx.x; q < nblocks; q += blockDim.x) g2 += sspart[q];
    g2 = warp_sum(g2);
    if (lane == 0) red[wid] = g2;
    reduce_partials(qpart, nblocks, d, qtmp);   // A^T u
    __syncthreads();
    if (threadIdx.x == 0) {
        double G = 0.0;
        for (int t = 0; t < nw; ++t) G += red[t];
        sc[0] = (G > 0.0) ? st->rho / G : 0.0;   // step length
    }
    __syncthreads();
    const double a = sc[0];
    double r2 = 0.0;
    for (int64_t j = threadIdx.x; j < d; j += blockDim.x) {
        double w = 0.0;
        for (int64_t i = 0; i <= j; ++i) w = fma(N64[i * d + j], (double)qtmp[i], w);   // (N^T A^T u)_j
        z[j] = fma(a, pc[j], z[j]);
        const double sj = fma(-a, w, s[j]);
        s[j] = sj;
        r2 = fma(sj, sj, r2);
    }
    r2 = warp_sum(r2);
    __syncthreads();
    if (lane == 0) red[wid] = r2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double R2 = 0.0;
        for (int t = 0; t < nw; ++t) R2 += red[t];
        sc[1] = (st->rho > 0.0) ? R2 / st->rho : 0.0;
        st->rho = R2;
        st->it += 1;
        if (a == 0.0 || R2 <= inner_tol * inner_tol * st->rho0) st->done = 1;
    }
    __syncthreads();
    if (st->done) return;
    const double bta = sc[1];
    for (int64_t j = threadIdx.x; j < d; j += blockDim.x) {
        const double v = fma(bta, pc[j], s[j]);
        pc[j] = v;
        pcs[j] = v;
    }
    __syncthreads();
    apply_n(N64, d, pcs, p);
}

// x <- x + N y (FP64).  One block.
__global__ void update_x_kernel(const double* __restrict__ N64, int64_t d, const double* __restrict__ y,
                                double* __restrict__ x) {
    __shared__ double ys[1024];
    for (int64_t j = threadIdx.x; j < d; j += blockDim.x) ys[j] = y[j];
    __syncthreads();
    for (int64_t i = threadIdx.x; i < d; i += blockDim.x) {
        double s = 0.0;
        for (int64_t j = i; j < d; ++j) s = fma(N64[i * d + j], ys[j], s);
        x[i] += s;
    }
}

constexpr int kMaxPassBlocks = 2432;   // >= 8 x the SM count of any sm_103 part

// Blocks of a pass over A: enough to keep every SM streaming, few enough
// that each block covers several row groups (fewer partials to reduce).
int pass_grid(const lsk_mat* A, int sm_count) {
    const int64_t n = A->n;
    const bool rows_kernel = A->kind == LSK_DENSE && A->d <= 256;
    const int64_t per_block = rows_kernel ? (kPassThreads / 32) * (A->d <= 64 ? 16 : 8) * 2 : kPassThreads * 2;
    int64_t g = (n + per_block - 1) / per_block;
    const int64_t cap = std::min<int64_t>(rows_kernel ? 4 * sm_count : 8 * sm_count, kMaxPassBlocks);
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

template <int CPL, int RB>
void launch_rows_pass(const lsk_mat* A, int nb, const float* p, const LsqrState* S, float* u, float* qpart,
                      double* sspart, cudaStream_t st) {
    LSK_PROF("lsq_pass", st) lsqr_pass_dense_rows_kernel<CPL, RB><<<nb, kPassThreads, 0, st>>>(
        (const float*)A->values, A->ld, A->n, A->d, p, S, u, qpart, sspart);
}

void lsqr_pass(const lsk_mat* A, int nb, size_t sh32, const float* p, const LsqrState* S, float* u,
               float* qpart, double* sspart, cudaStream_t st) {
    const int64_t n = A->n, d = A->d;
    if (A->kind == LSK_DENSE && d <= 256) {
        switch ((d + 31) / 32) {
            case 1: launch_rows_pass<1, 16>(A, nb, p, S, u, qpart, sspart, st); break;
            case 2: launch_rows_pass<2, 16>(A, nb, p, S, u, qpart, sspart, st); break;
            case 3: launch_rows_pass<3, 8>(A, nb, p, S, u, qpart, sspart, st); break;
            case 4: launch_rows_pass<4, 8>(A, nb, p, S, u, qpart, sspart, st); break;
            case 5: launch_rows_pass<5, 8>(A, nb, p, S, u, qpart, sspart, st); break;
            case 6: launch_rows_pass<6, 8>(A, nb, p, S, u, qpart, sspart, st); break;
            case 7: launch_rows_pass<7, 8>(A, nb, p, S, u, qpart, sspart, st); break;
            default: launch_rows_pass<8, 8>(A, nb, p, S, u, qpart, sspart, st); break;
        }
    } else if (A->kind == LSK_DENSE) {
        LSK_PROF("lsq_pass", st) lsqr_pass_dense_kernel<<<nb, kPassThreads, sh32, st>>>(
            (const float*)A->values, A->ld, n, d, p, S, u, qpart, sspart);
    } else {
        LSK_PROF("lsq_pass", st) lsqr_pass_csr_kernel<<<nb, kPassThreads, sh32, st>>>(
            (const float*)A->values, A->colidx, A->rowptr, n, A->nnz, d, p, S, u, qpart, sspart);
    }
}

}  // namespace

// atr = A^T (b - A x) in FP64 (the residual pass of the refinement loop,
// reduced in block order); x == nullptr means x = 0.
namespace {
__global__ void sum_qpart_kernel(const double* __restrict__ qpart, int nblocks, int64_t d, double* __restrict__ atr) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < d; j += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int z = 0; z < nblocks; ++z) s += qpart[(int64_t)z * d + j];
        atr[j] = s;
    }
}
}  // namespace

size_t atr64_workspace_bytes(const lsk_mat* A) {
    const int nb = kMaxPassBlocks;
    return ws_round((size_t)(A->n > 0 ? A->n : 1) * 4) + ws_round((size_t)nb * A->d * 8) + ws_round((size_t)nb * 8) +
           ws_round((size_t)A->d * 8) + 1024;
}

cudaError_t atr64_launch(const lsk_mat* A, const double* b, const double* x, double* atr, void* ws, int* flag,
                         int sm_count, cudaStream_t st) {
    const int64_t n = A->n, d = A->d;
    const int nb = pass_grid(A, sm_count);
    WsCarver wc{(char*)ws, 0};
    float* u = wc.take<float>(n > 0 ? n : 1);
    double* qpart = wc.take<double>((size_t)nb * d);
    double* sspart = wc.take<double>(nb);
    double* zero = wc.take<double>(d);
    cudaError_t e = cudaSuccess;
    if (!x) {
        if ((e = cudaMemsetAsync(zero, 0, (size_t)d * 8, st)) != cudaSuccess) return e;
        x = zero;
    }
    const bool dense = A->kind == LSK_DENSE;
    const size_t sh64 = dense ? (size_t)9 * d * 8 : (size_t)2 * d * 8;
    if (sh64 > 48 * 1024) {
        if ((e = allow_dynamic_smem(resid64_dense_kernel)) != cudaSuccess) return e;
        if ((e = allow_dynamic_smem(resid64_csr_kernel)) != cudaSuccess) return e;
    }
    if (dense)
        LSK_PROF("lsq_resid64", st) resid64_dense_kernel<<<nb, kPassThreads, sh64, st>>>((const float*)A->values, A->ld, n, d, b, x,
                                                                                          u, qpart, sspart);
    else
        LSK_PROF("lsq_resid64", st) resid64_csr_kernel<<<nb, kPassThreads, sh64, st>>>((const float*)A->values, A->colidx, A->rowptr,
                                                                                        n, A->nnz, d, b, x, u, qpart, sspart, flag);
    LSK_PROF("lsq_small", st) sum_qpart_kernel<<<(unsigned)((d + 255) / 256), 256, 0, st>>>(qpart, nb, d, atr);
    return cudaGetLastError();
}

size_t lsq_workspace_bytes(const lsk_mat* A) {
    const int64_t n = A->n, d = A->d;
    const int nb = kMaxPassBlocks;
    return ws_round(sizeof(LsqrState)) + ws_round((size_t)n * 4) + 6 * ws_round((size_t)d * 8) +
           ws_round((size_t)nb * d * 8) + ws_round((size_t)nb * 8) + 3 * ws_round((size_t)d * 4) +
           ws_round((size_t)2 * d * 4) + 4096;
}

int lsq_run(lsk_ctx* ctx, const lsk_mat* A, const double* b, double* x, const lsk_lsq_opts* o,
            const double* Rinv64, const float* /* FP32 factor: not used, the inner solve runs on Rinv64 */,
            void* ws, lsk_lsq_info* info) {
    cudaStream_t st = ctx->stream;
    const int64_t n = A->n, d = A->d;
    const int nb = pass_grid(A, ctx->sm_count);
    WsCarver wc{(char*)ws, 0};
    LsqrState* S = wc.take<LsqrState>(1);
    float* u = wc.take<float>(n > 0 ? n : 1);
    double* y = wc.take<double>(d);
    double* atr = wc.take<double>(d);
    double* qpart64 = wc.take<double>((size_t)nb * d);
    double* sspart = wc.take<double>(nb);
    float* p = wc.take<float>(d);
    float* qtmp = wc.take<float>(2 * d);
    double* cg_s = wc.take<double>(d);
    double* cg_p = wc.take<double>(d);
    float* qpart32 = reinterpret_cast<float*>(qpart64);   // reused by the FP32 pass

    LsqrState h{};
    cudaError_t e = cudaMemsetAsync(x, 0, (size_t)d * 8, st);
    if (e != cudaSuccess) return LSK_ERR_CUDA;
    const bool dense = A->kind == LSK_DENSE;
    const size_t sh64 = dense ? (size_t)9 * d * 8 : (size_t)2 * d * 8;
    const size_t sh32 = dense ? (size_t)9 * d * 4 : (size_t)2 * d * 4;
    if (sh64 > 48 * 1024) {
        if (allow_dynamic_smem(resid64_dense_kernel) != cudaSuccess ||
            allow_dynamic_smem(resid64_csr_kernel) != cudaSuccess)
            return LSK_ERR_CUDA;
    }
    if (sh32 > 48 * 1024) {
        if (allow_dynamic_smem(lsqr_pass_dense_kernel) != cudaSuccess ||
            allow_dynamic_smem(lsqr_pass_csr_kernel) != cudaSuccess)
            return LSK_ERR_CUDA;
    }
    int total_it = 0, refinements = 0, status = LSK_ERR_NOT_CONVERGED;
    double eta = INFINITY;
    for (int t = 0; t <= o->max_refine; ++t) {
        if (dense)
            LSK_PROF("lsq_resid64", st) resid64_dense_kernel<<<nb, kPassThreads, sh64, st>>>((const float*)A->values, A->ld, n, d, b, x, u,
                                                                 qpart64, sspart);
        else
            LSK_PROF("lsq_resid64", st) resid64_csr_kernel<<<nb, kPassThreads, sh64, st>>>((const float*)A->values, A->colidx, A->rowptr, n,
                                                               A->nnz, d, b, x, u, qpart64, sspart, ctx->flag);
        LSK_PROF("lsq_small", st) cg_start_kernel<<<1, 256, 0, st>>>(qpart64, nb, d, Rinv64, t == 0 ? 1 : 0, S, cg_s, cg_p, y, atr, p);
        e = cudaMemcpyAsync(&h, S, sizeof(h), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return LSK_ERR_CUDA;
        eta = h.eta;
        refinements = t;
        if (!(eta > o->tol)) {
            status = LSK_OK;
            break;
        }
        if (t == o->max_refine) break;
        // the inner solve need only reduce its residual by the factor left to
        // reach tol (with a margin of 10), and never by less than inner_tol
        double stop_rel = 0.1 * o->tol / eta;
        if (stop_rel < o->inner_tol) stop_rel = o->inner_tol;
        if (stop_rel > 0.5) stop_rel = 0.5;
        int it = 0;
        while (!h.done && it < o->max_iter) {
            lsqr_pass(A, nb, sh32, p, S, u, qpart32, sspart, st);
            LSK_PROF("lsq_small", st) cg_step_kernel<<<1, 1024, 0, st>>>(qpart32, sspart, nb, d, Rinv64, S, cg_s, cg_p, y, qtmp,
                                               stop_rel, p);
            ++it;
            if ((it & 3) == 0 || it >= o->max_iter) {   // stopping test every 4 iterations
                e = cudaMemcpyAsync(&h, S, sizeof(h), cudaMemcpyDeviceToHost, st);
                if (e == cudaSuccess) e = cudaStreamSynchronize(st);
                if (e != cudaSuccess) return LSK_ERR_CUDA;
            }
        }
        e = cudaMemcpyAsync(&h, S, sizeof(h), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return LSK_ERR_CUDA;
        total_it += h.it;
        LSK_PROF("lsq_small", st) update_x_kernel<<<1, 256, 0, st>>>(Rinv64, d, y, x);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return LSK_ERR_CUDA;
    if (info) {
        info->iters = total_it;
        info->refinements = refinements;
        info->eta = eta;
        info->status = status;
    }
    return status;
}
