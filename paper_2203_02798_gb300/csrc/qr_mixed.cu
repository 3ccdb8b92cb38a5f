// qr_mixed.cu -- R of the sketch with FP32 factorisation and one FP64 correction.
//
// FP64 on this part is slow and, worse, has long dependent-operation
// latency, so the serial chain of a Cholesky factorisation is run in FP32
// and FP64 is used only in parallel matrix products:
//   1. C = B^T B in FP64 (qr.cu), equilibrated by powers of two:
//      Ct = D^-1 C D^-1, D_j = 2^round(log2 sqrt(C_jj))            (exact)
//   2. Ct ~ Rt^T Rt by FP32 Cholesky (one CTA, packed lower triangle in
//      shared memory), X = Rt^-1 by FP32 back substitution
//   3. one correction step with FP64-accurate products of triangular matrices
//      (FP32-pair arithmetic on the FP32 units, FP64 inputs and outputs):
//        M = X^T Ct X = I + E,  U = strict_upper(E) + diag(E)/2
//        Y = X (I - U)                         (= (R D^-1)^-1 to O(|E|^2))
//        Z = Rt + Rt (I - Y Rt)                (Newton step for Y^-1)
//   4. R = Z D, R^-1 = D^-1 Y
// In exact arithmetic R is the Cholesky factor of C, i.e. the sign-normalised
// Householder R of B.  Rank deficiency is reported when an FP32 pivot is not
// positive, when the FP32 factor needs a correction larger than 1/4 (the
// equilibrated sketch is numerically singular at FP32 precision), or when
// the equilibrated diag(R) spans more than 2^20.
#include "lsk_internal.cuh"

#include <algorithm>

namespace {

constexpr int TT = 16;   // tile edge of the FP64 triangular products (one output per thread)

// e_j = floor(log2 sqrt(C_jj)) and the exact scale 2^-e_j.
__device__ __forceinline__ void equil_exponents_body(const double* __restrict__ C, int d, int* __restrict__ e,
                                       double* __restrict__ sc, int* flag, const int blk, const int nblk) {
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        const double c = C[(int64_t)j * d + j];
        int ex = 0;
        if (c > 0.0 && isfinite(c)) {
            int b2;
            frexp(c, &b2);                  // c = m 2^b2, m in [0.5, 1)
            ex = (b2 - 1) >> 1;
        } else {
            set_flag(flag, LSK_FLAG_RANK_DEFICIENT);
        }
        e[j] = ex;
        sc[j] = ldexp(1.0, -ex);
    }
}

// Ct64 = C 2^{-e_i-e_j} (two exact multiplications), Ct32 = float(Ct64).
__device__ __forceinline__ void equil_scale_body(const double* __restrict__ C, int d, const double* __restrict__ sc,
                                   double* __restrict__ Ct64, float* __restrict__ Ct32, const int blk, const int nblk) {
    for (int t = blk * blockDim.x + threadIdx.x; t < d * d; t += nblk * blockDim.x) {
        const double v = C[t] * sc[t / d] * sc[t % d];
        Ct64[t] = v;
        Ct32[t] = (float)v;
    }
}

// FP32 Cholesky of Ct (d <= 256) in one CTA, blocked by 32: the lower
// triangle lives in shared memory as 32 x 33 (padded) tiles T(I, J), I >= J.
// Per block column K: warp 0 factors T(K, K) with its rows in registers,
// one thread per row solves the panel T(I, K) L_KK^-T, and the rank-32
// trailing update T(I, J) -= L_IK L_JK^T runs one tile per warp with each
// lane's column of L_JK in registers.  Dimensions beyond d are padded with
// the identity.  Writes Rt = L^T (FP64 values, d x d, zeros below) and the
// packed rows of L (row l at offset l(l+1)/2) for the inverse.
constexpr int CB = 32;
constexpr int CP = CB + 1;

// Unblocked Cholesky of one 32 x 32 tile by one warp, row `lane` in a[]:
// compile-time recursion over (j, k) keeps every index static, so a[] stays
// in registers (a nested #pragma unroll of this size is not fully unrolled).
template <int J, int K>
struct DiagUpdate {
    static __device__ __forceinline__ void run(float (&a)[CB], float lij, int lane) {
        const float lkj = __shfl_sync(0xffffffffu, lij, K);   // L[K][J] from lane K
        if (K <= lane) a[K] -= lij * lkj;
        DiagUpdate<J, K + 1>::run(a, lij, lane);
    }
};
template <int J>
struct DiagUpdate<J, CB> {
    static __device__ __forceinline__ void run(float (&)[CB], float, int) {}
};
template <int J>
struct DiagStep {
    static __device__ __forceinline__ void run(float (&a)[CB], int lane, int* flag) {
        float piv = __shfl_sync(0xffffffffu, a[J], J);
        if (!(piv > 0.f) || !isfinite(piv)) {
            if (lane == 0) set_flag(flag, LSK_FLAG_RANK_DEFICIENT);
            piv = 1.f;
        }
        const float il = rsqrtf(piv), l = piv * il;   // FP32 factor: the FP64 correction absorbs its rounding
        if (lane == J) a[J] = l;
        if (lane > J) a[J] *= il;
        DiagUpdate<J, J + 1>::run(a, a[J], lane);
        DiagStep<J + 1>::run(a, lane, flag);
    }
};
template <>
struct DiagStep<CB> {
    static __device__ __forceinline__ void run(float (&)[CB], int, int*) {}
};
__device__ __forceinline__ float* ctile(float* S, int I, int J) { return S + (I * (I + 1) / 2 + J) * (CB * CP); }

__device__ __forceinline__ void chol32_body(const float* __restrict__ Ct32, int d, double* __restrict__ Rt,
                                                      float* __restrict__ Lpk, int* flag, const int blk, const int nblk) {
    extern __shared__ float S[];
    __shared__ float rdiag[CB];
    const int nt = (d + CB - 1) / CB;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    {   // all tiles at once: flat index over (tile, element), tile -> (I, J) from a
        // small table, eight independent loads in flight per thread
        __shared__ unsigned char tI[36], tJ[36];   // nt <= 8
        const int ntl = nt * (nt + 1) / 2;
        if (threadIdx.x < ntl) {
            int I = 0, t = threadIdx.x;
            while (t > I) t -= ++I;
            tI[threadIdx.x] = (unsigned char)I;
            tJ[threadIdx.x] = (unsigned char)t;
        }
        __syncthreads();
#pragma unroll 8
        for (int t = threadIdx.x; t < ntl * CB * CB; t += blockDim.x) {
            const int tl = t >> 10, e = t & 1023;
            const int r = e >> 5, c = e & 31, i = tI[tl] * CB + r, j = tJ[tl] * CB + c;
            S[tl * (CB * CP) + r * CP + c] = (i < d && j < d) ? __ldg(Ct32 + i * d + j) : (i == j ? 1.f : 0.f);
        }
    }
    __syncthreads();
    for (int K = 0; K < nt; ++K) {
        float* D = ctile(S, K, K);
        if (w == 0) {   // (1) diagonal tile: row `lane` in registers (fully unrolled)
            float a[CB];
#pragma unroll
            for (int k = 0; k < CB; ++k) a[k] = D[lane * CP + k];
            DiagStep<0>::run(a, lane, flag);
#pragma unroll
            for (int k = 0; k < CB; ++k) D[lane * CP + k] = a[k];
            __syncwarp();
            rdiag[lane] = 1.f / D[lane * CP + lane];
            __syncwarp();
        }
        __syncthreads();
        // (2) panel: thread per row of T(I, K), I > K
        {
            const int rows = (nt - K - 1) * CB;
            for (int t = threadIdx.x; t < rows; t += blockDim.x) {
                const int I = K + 1 + t / CB, r = t % CB;
                float* T = ctile(S, I, K);
                float x[CB];
#pragma unroll
                for (int j = 0; j < CB; ++j) {
                    float v = T[r * CP + j];
#pragma unroll
                    for (int l = 0; l < j; ++l) v -= x[l] * D[j * CP + l];
                    x[j] = v * rdiag[j];
                }
#pragma unroll
                for (int j = 0; j < CB; ++j) T[r * CP + j] = x[j];
            }
        }
        __syncthreads();
        // (3) trailing update, one tile (I, J), K < J <= I, per warp
        {
            const int T0 = nt - K - 1;
            const int ntile = T0 * (T0 + 1) / 2;
            for (int t = w; t < ntile; t += nw) {
                int I = 0, tt = t;
                while (tt > I) {   // lower pairs (J <= I) over the trailing blocks
                    tt -= I + 1;
                    ++I;
                }
                const int J = tt;
                I += K + 1;
                const int Jg = J + K + 1;
                const float* LI = ctile(S, I, K);
                const float* LJ = ctile(S, Jg, K);
                float* T = ctile(S, I, Jg);
                float lj[CB];
#pragma unroll
                for (int k = 0; k < CB; ++k) lj[k] = LJ[lane * CP + k];   // column `lane` of L_JK^T
                for (int a = 0; a < CB; a += 4) {   // four independent chains
                    float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;
#pragma unroll
                    for (int k = 0; k < CB; ++k) {
                        acc0 = fmaf(LI[a * CP + k], lj[k], acc0);
                        acc1 = fmaf(LI[(a + 1) * CP + k], lj[k], acc1);
                        acc2 = fmaf(LI[(a + 2) * CP + k], lj[k], acc2);
                        acc3 = fmaf(LI[(a + 3) * CP + k], lj[k], acc3);
                    }
                    T[a * CP + lane] -= acc0;
                    T[(a + 1) * CP + lane] -= acc1;
                    T[(a + 2) * CP + lane] -= acc2;
                    T[(a + 3) * CP + lane] -= acc3;
                }
            }
        }
        __syncthreads();
    }
    // Rt[i][j] = L[j][i] for j >= i (only when the caller forms R), then the
    // packed rows of L (row l at l(l+1)/2): warp per row, lanes along it
    if (Rt) {
        for (int i = w; i < d; i += nw)
            for (int j = lane; j < d; j += 32)
                Rt[(int64_t)i * d + j] = (j >= i) ? (double)ctile(S, j >> 5, i >> 5)[(j & 31) * CP + (i & 31)] : 0.0;
    }
    for (int l = w; l < d; l += nw) {
        float* dst = Lpk + l * (l + 1) / 2;
        for (int i = lane; i <= l; i += 32) dst[i] = ctile(S, l >> 5, i >> 5)[(l & 31) * CP + (i & 31)];
    }
}

// Back substitution steps l = min(j, 32 SL + 31) .. 32 SL of column j: the
// rows of block SL hold the pivot; rows i < l of blocks <= SL are updated.
template <int SL>
__device__ __forceinline__ void trinv_block(float (&xr)[8], const float* P, const float* rdiag, int j, int lane) {
    if (j < 32 * SL) return;
    const int top = j < 32 * SL + 31 ? j : 32 * SL + 31;
    for (int l = top; l >= 32 * SL; --l) {
        const int owner = l & 31;
        const float xl = __shfl_sync(0xffffffffu, xr[SL], owner) * rdiag[l];
        if (lane == owner) xr[SL] = xl;
        const float* col = P + l * (l + 1) / 2;   // Rt[i][l] = L[l][i]
#pragma unroll
        for (int s = 0; s <= SL; ++s) {
            const int i = lane + 32 * s;
            if (i < l) xr[s] = fmaf(-col[i], xl, xr[s]);
        }
    }
}

// X = Rt^-1 (upper) in FP32, one warp per column; stored as FP64 values.
// The packed factor (row l of L = column l of Rt at offset l(l+1)/2) is
// staged in shared memory (once per block of 4 or 16 columns) so the
// back-substitution chain sees shared-memory latency.
__device__ __forceinline__ void store_x(double* X, int64_t at, float v) { X[at] = (double)v; }
__device__ __forceinline__ void store_x(float2* X, int64_t at, float v) { X[at] = make_float2(v, 0.f); }
template <class T>
__device__ __forceinline__ void trinv32_body(const float* __restrict__ Lpk, int d, T* __restrict__ X, const int blk, const int nblk) {
    extern __shared__ float P[];
    __shared__ float rdiag[256];
    {   // stage the packed factor with 16-byte loads, several in flight per thread
        const int np = d * (d + 1) / 2, n4 = np >> 2;
        const float4* src4 = reinterpret_cast<const float4*>(Lpk);
        float4* P4 = reinterpret_cast<float4*>(P);
#pragma unroll 4
        for (int t = threadIdx.x; t < n4; t += blockDim.x) P4[t] = __ldg(src4 + t);
        for (int t = 4 * n4 + threadIdx.x; t < np; t += blockDim.x) P[t] = __ldg(Lpk + t);
    }
    __syncthreads();
    for (int l = threadIdx.x; l < d; l += blockDim.x) rdiag[l] = 1.f / P[l * (l + 1) / 2 + l];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int j = (int)(((int64_t)blk * blockDim.x + threadIdx.x) >> 5);
    if (j >= d) return;
    float xr[8];
#pragma unroll
    for (int s = 0; s < 8; ++s) xr[s] = (lane + 32 * s == j) ? 1.f : 0.f;
    // row blocks from the top one down; within block SL the pivot entry is
    // xr[SL], a static index (no per-step selection among the 8 registers)
    trinv_block<7>(xr, P, rdiag, j, lane);
    trinv_block<6>(xr, P, rdiag, j, lane);
    trinv_block<5>(xr, P, rdiag, j, lane);
    trinv_block<4>(xr, P, rdiag, j, lane);
    trinv_block<3>(xr, P, rdiag, j, lane);
    trinv_block<2>(xr, P, rdiag, j, lane);
    trinv_block<1>(xr, P, rdiag, j, lane);
    trinv_block<0>(xr, P, rdiag, j, lane);
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        const int i = lane + 32 * s;
        if (i < d) store_x(X, (int64_t)i * d + j, (i <= j) ? xr[s] : 0.f);
    }
}
// X = Rt^-1 as FP32 pairs (the single-sketch chain keeps its matrices in pair form)
__global__ void __launch_bounds__(512) trinv32_pair_kernel(const float* __restrict__ Lpk, int d, float2* __restrict__ X) {
    trinv32_body(Lpk, d, X, blockIdx.x, gridDim.x);
}

// Out = alpha * op(A) * B + beta * Cin + diag_add * I on the upper triangle
// (tiles I <= J).  op(A) = A or A^T.  The reduction index is limited to
// where both factors can be non-zero: a_upper (op(A) upper: k >= i),
// a_lower (op(A) lower: k <= i), b_upper (B upper: k <= j).  Entries below
// the diagonal of Out are written as zero.
//
// Arithmetic: the FP64 inputs are split into FP32 pairs (x = hi + lo, ~48
// bits), each product is formed as hi*hi exactly (one FMA gives its rounding
// error) plus the cross terms, and the sum is kept as an FP32 pair (TwoSum),
// renormalised every 16 terms: about 2^-46 relative per product and d 2^-47
// of max |term| in the sum -- far inside what the correction step needs --
// on the FP32 units (FP64 runs at 1/64 of that rate on this part).  alpha,
// beta and the final combination are FP64.
struct TriGemm {
    const double* A;
    const double* B;
    const double* Cin;
    double* Out;
    int d, transA, a_upper, a_lower, b_upper;
    double alpha, beta, diag_add;
};

__device__ __forceinline__ float2 split_pair(double x) {
    const float h = (float)x;
    return make_float2(h, (float)(x - (double)h));
}
// (s, c) += a * b with a, b FP32 pairs
__device__ __forceinline__ void pair_mac(float2 a, float2 b, float& s, float& c) {
    const float p = __fmul_rn(a.x, b.x);
    const float e = fmaf(a.x, b.x, -p);                       // a.x b.x = p + e exactly
    const float cross = fmaf(a.x, b.y, __fmul_rn(a.y, b.x));
    const float t = __fadd_rn(s, p);
    const float z = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
    c = __fadd_rn(c, __fadd_rn(err, __fadd_rn(e, cross)));
    s = t;
}
__device__ __forceinline__ void pair_renorm(float& s, float& c) {
    const float t = __fadd_rn(s, c);
    const float z = __fsub_rn(t, s);
    c = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(c, z));
    s = t;
}

__device__ __forceinline__ void tri_gemm64_body(const TriGemm g, const int blk, const int nblk) {
    const int nt = (g.d + TT - 1) / TT;
    int t = blk, I = 0;
    while (t >= nt - I) {   // upper tile pairs (I <= J)
        t -= nt - I;
        ++I;
    }
    const int J = I + t;
    __shared__ float2 As[TT][TT + 1], Bs[TT][TT + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // output (ty, tx)
    const int i0 = I * TT, j0 = J * TT;
    int klo = 0, khi = g.d;
    if (g.a_upper) klo = i0;
    if (g.a_lower) khi = min(khi, i0 + TT);
    if (g.b_upper) khi = min(khi, j0 + TT);
    float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f;   // two chains for latency
    for (int k0 = klo - (klo % TT); k0 < khi; k0 += TT) {
        {
            const int r = threadIdx.x / TT, c = threadIdx.x % TT;
            const int ia = i0 + r, ka = k0 + c;
            double a = 0.0;
            if (ia < g.d && ka < g.d) a = g.transA ? g.A[(int64_t)ka * g.d + ia] : g.A[(int64_t)ia * g.d + ka];
            As[r][c] = split_pair(a);
            const int kb = k0 + r, jb = j0 + c;
            Bs[r][c] = split_pair((kb < g.d && jb < g.d) ? g.B[(int64_t)kb * g.d + jb] : 0.0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TT; kk += 2) {
            pair_mac(As[ty][kk], Bs[kk][tx], s0, c0);
            pair_mac(As[ty][kk + 1], Bs[kk + 1][tx], s1, c1);
        }
        pair_renorm(s0, c0);
        pair_renorm(s1, c1);
        __syncthreads();
    }
    const int i = i0 + ty, j = j0 + tx;
    if (i >= g.d || j >= g.d) return;
    double r = 0.0;
    if (j >= i) {
        r = g.alpha * (((double)s0 + (double)s1) + ((double)c0 + (double)c1));
        if (g.beta != 0.0) r += g.beta * g.Cin[(int64_t)i * g.d + j];
        if (i == j) r += g.diag_add;
    }
    g.Out[(int64_t)i * g.d + j] = r;
}

// U = strict_upper(M - I) + diag(M - I) / 2, in place.  |M - I| > 1/4
// anywhere means the FP32 factor was too far off for one correction: the
// equilibrated sketch is numerically rank deficient at FP32 precision.
__device__ __forceinline__ void correction_body(double* __restrict__ M, int d, int* flag, const int blk, const int nblk) {
    bool big = false;
    for (int t = blk * blockDim.x + threadIdx.x; t < d * d; t += nblk * blockDim.x) {
        const int i = t / d, j = t % d;
        if (i <= j) {
            const double e = M[t] - (i == j ? 1.0 : 0.0);
            if (!(fabs(e) <= 0.25)) big = true;
            M[t] = (i == j) ? 0.5 * e : e;
        } else {
            M[t] = 0.0;
        }
    }
    if (big) set_flag(flag, LSK_FLAG_RANK_DEFICIENT);
}

// R = Z D, R^-1 = D^-1 Y (exact power-of-two scalings); FP32 copy of R^-1.
__device__ __forceinline__ void unscale_body(const double* __restrict__ Z, const double* __restrict__ Y, const int* __restrict__ e,
                               int d, double* __restrict__ R, double* __restrict__ Rinv, float* __restrict__ Rinv32, const int blk, const int nblk) {
    for (int t = blk * blockDim.x + threadIdx.x; t < d * d; t += nblk * blockDim.x) {
        const int i = t / d, j = t % d;
        const bool up = j >= i;
        const double r = (up && Z) ? ldexp(Z[t], e[j]) : 0.0;
        const double ri = up ? ldexp(Y[t], -e[i]) : 0.0;
        if (R) R[t] = r;
        if (Rinv) Rinv[t] = ri;
        if (Rinv32) Rinv32[t] = (float)ri;
    }
}

// min_j Rt_jj <= 2^-20 max_j Rt_jj on the equilibrated factor, with
// Rt_jj = 1 / Y_jj: beyond that conditioning a factor of the Gram cannot
// resolve the sketch in FP64.
__device__ __forceinline__ void rank_check_r_body(const double* __restrict__ Y, int d, int* flag, const int blk, const int nblk) {
    double mn = INFINITY, mx = 0.0;
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        const double v = 1.0 / Y[(int64_t)j * d + j];
        mn = fmin(mn, v);
        mx = fmax(mx, v);
    }
    for (int o = 16; o; o >>= 1) {
        mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    __shared__ double smn[32], smx[32];
    if ((threadIdx.x & 31) == 0) {
        smn[threadIdx.x >> 5] = mn;
        smx[threadIdx.x >> 5] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            mn = fmin(mn, smn[w]);
            mx = fmax(mx, smx[w]);
        }
        if (!(mn > 9.5367431640625e-07 * mx) || !isfinite(mx)) set_flag(flag, LSK_FLAG_RANK_DEFICIENT);
    }
}

// ---- grouped: one grid per stage over many sketches (QrJob table) --------
__device__ __forceinline__ const QrJob& job_of(const QrJob* jobs, const int* off, int count, int& blk, int& nblk) {
    const int g = group_of(off, count, blockIdx.x);
    const int b0 = __ldg(off + g);
    blk = (int)blockIdx.x - b0;
    nblk = __ldg(off + g + 1) - b0;
    return jobs[g];
}

__global__ void equil_exponents_grouped_kernel(const QrJob* __restrict__ jobs, const int* __restrict__ off, int count) {
    int blk, nblk;
    const QrJob& j = job_of(jobs, off, count, blk, nblk);
    equil_exponents_body(j.C, j.d, j.e, j.sc, j.flag, blk, nblk);
}
__global__ void equil_scale_grouped_kernel(const QrJob* __restrict__ jobs, const int* __restrict__ off, int count) {
    int blk, nblk;
    const QrJob& j = job_of(jobs, off, count, blk, nblk);
    equil_scale_body(j.C, j.d, j.sc, j.Ct, j.Ct32, blk, nblk);
}
__global__ void __launch_bounds__(512) chol32_grouped_kernel(const QrJob* __restrict__ jobs, const int* __restrict__ off,
                                                             int count) {
    int blk, nblk;
    const QrJob& j = job_of(jobs, off, count, blk, nblk);
    chol32_body(j.Ct32, j.d, nullptr, j.Lpk, j.flag, blk, nblk);   // R is not formed in a group
}
__global__ void __launch_bounds__(512) trinv32_grouped_kernel(const QrJob* __restrict__ jobs, const int* __restrict__ off,
                                                              int count) {
    int blk, nblk;
    const QrJob& j = job_of(jobs, off, count, blk, nblk);
    trinv32_body(j.Lpk, j.d, j.X, blk, nblk);
}
// which: 0 W = Ct X, 1 M = X^T W, 2 Y = X - X U (the products of qr_mixed_launch without the Newton step)
__global__ void __launch_bounds__(256) tri_gemm64_grouped_kernel(const QrJob* __restrict__ jobs,
                                                                 const int* __restrict__ off, int count, int which) {
    int blk, nblk;
    const QrJob& j = job_of(jobs, off, count, blk, nblk);
    TriGemm g;
    if (which == 0) g = TriGemm{j.Ct, j.X, nullptr, j.W, j.d, 0, 0, 0, 1, 1.0, 0.0, 0.0};
    else if (which == 1) g = TriGemm{j.X, j.W, nullptr, j.M, j.d, 1, 0, 1, 1, 1.0, 0.0, 0.0};
    else g = TriGemm{j.X, j.M, j.X, j.Y, j.d, 0, 1, 0, 1, -1.0, 1.0, 0.0};
    tri_gemm64_body(g, blk, nblk);
}
__global__ void correction_grouped_kernel(const QrJob* __restrict__ jobs, const int* __restrict__ off, int count) {
    int blk, nblk;
    const QrJob& j = job_of(jobs, off, count, blk, nblk);
    correction_body(j.M, j.d, j.flag, blk, nblk);
}
__global__ void unscale_grouped_kernel(const QrJob* __restrict__ jobs, const int* __restrict__ off, int count) {
    int blk, nblk;
    const QrJob& j = job_of(jobs, off, count, blk, nblk);
    unscale_body(nullptr, j.Y, j.e, j.d, nullptr, j.Rinv, j.Rinv32, blk, nblk);
}
__global__ void rank_check_r_grouped_kernel(const QrJob* __restrict__ jobs, const int* __restrict__ off, int count) {
    int blk, nblk;
    const QrJob& j = job_of(jobs, off, count, blk, nblk);
    rank_check_r_body(j.Y, j.d, j.flag, blk, nblk);
}

// ---- single-sketch path: fewer launches, no FP64 arithmetic -----------------
// FP64 runs at 1/64 of the FP32 rate on this part, so the chain of one
// sketch keeps its matrices as FP32 pairs (x = hi + lo, |lo| <= ulp(hi) / 2,
// ~48 bits) from the Gram on, and touches FP64 only to write R and R^-1.
//
// Pair arithmetic (FP32 throughout): TwoSum for exact sums, one FMA for the
// rounding error of a product.
__device__ __forceinline__ void two_sum_acc(float& S, float& E, float s, float c) {
    const float t = __fadd_rn(S, s);
    const float z = __fsub_rn(t, S);
    E = __fadd_rn(E, __fadd_rn(__fadd_rn(__fsub_rn(S, __fsub_rn(t, z)), __fsub_rn(s, z)), c));
    S = t;
}
__device__ __forceinline__ float2 pair_norm(float S, float E) {
    const float h = __fadd_rn(S, E);
    return make_float2(h, __fsub_rn(E, __fsub_rn(h, S)));
}

// chol_eq: the pair Gram Cp -> exponents e_j = floor(log2 sqrt(C_jj)) (the
// scaling 2^-e is exact), the equilibrated FP32 tiles, the FP32 Cholesky
// factorisation, the rank check on its diagonal, and the packed factor (and
// Rt as pairs when R is wanted).  One CTA of 512 threads; tile rows padded to
// 36 floats so that a row of a tile is eight aligned 16-byte vectors (the
// trailing update reads L_IK rows as float4 broadcasts).
constexpr int QP = 36;
__device__ __forceinline__ float* qtile(float* S, int I, int J) { return S + (I * (I + 1) / 2 + J) * (CB * QP); }

size_t chol_eq_smem(int d) {
    const int nt = (d + CB - 1) / CB;
    return (size_t)nt * (nt + 1) / 2 * CB * QP * 4;
}

// warp-wide FP32 Cholesky of the diagonal tile D (row `lane` in registers)
__device__ __forceinline__ void chol_diag_tile(float* D, float* rdiag, int lane, int* flag) {
    float a[CB];
#pragma unroll
    for (int k = 0; k < CB; ++k) a[k] = D[lane * QP + k];
    DiagStep<0>::run(a, lane, flag);
#pragma unroll
    for (int k = 0; k < CB; ++k) D[lane * QP + k] = a[k];
    __syncwarp();
    rdiag[lane] = 1.f / D[lane * QP + lane];
    __syncwarp();
}

// T(I, J) -= L_IK L_JK^T for one 32 x 32 tile by one warp: lane = column of
// the tile, rows of L_IK read as float4 broadcasts
__device__ __forceinline__ void chol_tile_update(float* S, int I, int J, int K, int lane) {
    const float* LI = qtile(S, I, K);
    const float* LJ = qtile(S, J, K);
    float* T = qtile(S, I, J);
    float lj[CB];
#pragma unroll
    for (int k = 0; k < CB; ++k) lj[k] = LJ[lane * QP + k];
#pragma unroll 1
    for (int a = 0; a < CB; ++a) {
        const float4* row = reinterpret_cast<const float4*>(LI + a * QP);
        float acc0 = 0.f, acc1 = 0.f;
#pragma unroll
        for (int q = 0; q < CB / 4; q += 2) {
            const float4 u = row[q], v = row[q + 1];
            acc0 = fmaf(u.x, lj[4 * q], acc0);
            acc1 = fmaf(u.y, lj[4 * q + 1], acc1);
            acc0 = fmaf(u.z, lj[4 * q + 2], acc0);
            acc1 = fmaf(u.w, lj[4 * q + 3], acc1);
            acc0 = fmaf(v.x, lj[4 * q + 4], acc0);
            acc1 = fmaf(v.y, lj[4 * q + 5], acc1);
            acc0 = fmaf(v.z, lj[4 * q + 6], acc0);
            acc1 = fmaf(v.w, lj[4 * q + 7], acc1);
        }
        T[a * QP + lane] -= acc0 + acc1;
    }
}

__global__ void __launch_bounds__(512) chol_eq_kernel(const float2* __restrict__ Cp, int d, int* __restrict__ e_out,
                                                      float2* __restrict__ Rt, float* __restrict__ Lpk, int* flag) {
    extern __shared__ __align__(16) float S[];
    __shared__ float rdiag[CB];
    __shared__ float scf[256];
    __shared__ unsigned char tI[36], tJ[36];
    __shared__ float dmin[32], dmax[32];
    const int nt = (d + CB - 1) / CB;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // (0) equilibration exponents from the diagonal; scf_j = 2^-e_j (a float:
    //     e_j is in [-75, 64] for a finite positive FP32 C_jj)
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        const float c = Cp[(int64_t)j * d + j].x;
        int ex = 0;
        if (c > 0.f && isfinite(c)) {
            int b2;
            frexpf(c, &b2);                 // c = m 2^b2, m in [0.5, 1)
            ex = (b2 - 1) >> 1;
        } else {
            set_flag(flag, LSK_FLAG_RANK_DEFICIENT);
        }
        e_out[j] = ex;
        scf[j] = ldexpf(1.f, -ex);
    }
    const int ntl = nt * (nt + 1) / 2;
    if (threadIdx.x < ntl) {
        int I = 0, t = threadIdx.x;
        while (t > I) t -= ++I;
        tI[threadIdx.x] = (unsigned char)I;
        tJ[threadIdx.x] = (unsigned char)t;
    }
    __syncthreads();
    // (1) the lower tiles of Ct = D^-1 C D^-1 in FP32 (beyond d: the identity):
    //     the FP32 rounding of C times two exact powers of two, in rounds of
    //     24 loads per thread, all issued before any is used
    {
        constexpr int kR = 24;
        const int total = ntl * CB * CB;
        for (int t0 = 0; t0 < total; t0 += kR * 512) {
            float v[kR];
#pragma unroll
            for (int q = 0; q < kR; ++q) {
                const int t = t0 + q * 512 + (int)threadIdx.x;
                const int tl = t >> 10, el = t & 1023;
                const int i = tI[tl < 36 ? tl : 0] * CB + (el >> 5), j = tJ[tl < 36 ? tl : 0] * CB + (el & 31);
                v[q] = (t < total && i < d && j < d) ? __ldg(&Cp[(int64_t)i * d + j].x) : 0.f;
            }
#pragma unroll
            for (int q = 0; q < kR; ++q) {
                const int t = t0 + q * 512 + (int)threadIdx.x;
                if (t < total) {
                    const int tl = t >> 10, el = t & 1023;
                    const int r = el >> 5, c = el & 31, i = tI[tl] * CB + r, j = tJ[tl] * CB + c;
                    S[tl * (CB * QP) + r * QP + c] = (i < d && j < d) ? v[q] * scf[i] * scf[j] : (i == j ? 1.f : 0.f);
                }
            }
        }
    }
    __syncthreads();
    // K = -1 factors the first diagonal tile only; every later pass: the panel
    // of K, then the trailing update with the next diagonal tile looked ahead
    // (one call site of the unrolled diagonal factorisation keeps the code small)
    for (int K = -1; K < nt; ++K) {
        const float* D = qtile(S, K < 0 ? 0 : K, K < 0 ? 0 : K);
        // (2) panel: thread per row of T(I, K), I > K (forward substitution with L_KK)
        if (K >= 0) {
            const int rows = (nt - K - 1) * CB;
            for (int t = threadIdx.x; t < rows; t += blockDim.x) {
                const int I = K + 1 + t / CB, r = t % CB;
                float* T = qtile(S, I, K);
                float x[CB];
#pragma unroll
                for (int j = 0; j < CB; ++j) {
                    float v = T[r * QP + j];
#pragma unroll
                    for (int l = 0; l < j; ++l) v -= x[l] * D[j * QP + l];
                    x[j] = v * rdiag[j];
                }
#pragma unroll
                for (int j = 0; j < CB; ++j) T[r * QP + j] = x[j];
            }
        }
        __syncthreads();
        // (3) trailing update with look-ahead: warp 0 updates the next diagonal
        //     tile (K+1, K+1) and factors it at once, while the other warps
        //     update the rest of the trailing tiles (I, J), K < J <= I
        {
            const int T0 = nt - K - 1;
            const int ntile = K < 0 ? 0 : T0 * (T0 + 1) / 2;
            if (w == 0) {
                if (T0 > 0) {
                    if (K >= 0) chol_tile_update(S, K + 1, K + 1, K, lane);
                    __syncwarp();
                    chol_diag_tile(qtile(S, K + 1, K + 1), rdiag, lane, flag);
                }
            } else {
                for (int t = w; t < ntile; t += nw - 1) {   // t = 0 is the diagonal tile
                    int I = 0, tt = t;
                    while (tt > I) {
                        tt -= I + 1;
                        ++I;
                    }
                    chol_tile_update(S, I + K + 1, tt + K + 1, K, lane);
                }
            }
        }
        __syncthreads();
    }
    // (5) rank check on the equilibrated FP32 factor: min_j L_jj <= 2^-20 max_j
    //     L_jj (one correction step resolves no more than that)
    {
        float mn = INFINITY, mx = 0.f;
        for (int j = threadIdx.x; j < d; j += blockDim.x) {
            const float v = qtile(S, j >> 5, j >> 5)[(j & 31) * QP + (j & 31)];
            mn = fminf(mn, v);
            mx = fmaxf(mx, v);
        }
        for (int o = 16; o; o >>= 1) {
            mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
        if (lane == 0) {
            dmin[w] = mn;
            dmax[w] = mx;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int q = 1; q < nw; ++q) {
                mn = fminf(mn, dmin[q]);
                mx = fmaxf(mx, dmax[q]);
            }
            if (!(mn > 9.5367431640625e-07f * mx) || !isfinite(mx)) set_flag(flag, LSK_FLAG_RANK_DEFICIENT);
        }
    }
    // (6) Rt[i][j] = L[j][i] for j >= i (only when R is wanted), packed rows of L
    if (Rt) {
        for (int i = w; i < d; i += nw)
            for (int j = lane; j < d; j += 32)
                Rt[(int64_t)i * d + j] =
                    make_float2((j >= i) ? qtile(S, j >> 5, i >> 5)[(j & 31) * QP + (i & 31)] : 0.f, 0.f);
    }
    for (int l = w; l < d; l += nw) {
        float* dst = Lpk + l * (l + 1) / 2;
        for (int i = lane; i <= l; i += 32) dst[i] = qtile(S, l >> 5, i >> 5)[(l & 31) * QP + (i & 31)];
    }
}

// Out = alpha op(A) B + beta Cin + diag_add I on the upper triangle (the
// TriGemm operation on pair matrices), with the whole reduction range of a
// 16 x 16 output tile staged in shared memory at once and split between two
// threads per output; A optionally scaled exactly (A_ik 2^(-e_i - e_k)); an
// epilogue finishes a step of the correction:
//   kPlain:   Out as above;
//   kCorrect: Out = U = strict_upper(E) + diag(E) / 2, E = result - I, and
//             the rank flag when |E| > 1/4 (the correction of the FP32 factor);
//   kInverse: Out = Y = result, R64 / R32 = 2^-e_i Y (R^-1 in FP64 and FP32);
//   kFactor:  R64 = 2^e_j result (R; Out unused).
// R64 and R32 are written whole: an off-diagonal tile also writes the zeros
// of its mirror below the diagonal (no lower tile is launched).
enum TriEpi { kPlain = 0, kCorrect = 1, kInverse = 2, kFactor = 3 };
struct TriGemmP {
    const float2* A;
    const float2* B;
    const float2* Cin;
    float2* Out;
    const int* ea;      // nullable: A_ik scaled by 2^(-ea_i - ea_k)
    int d, transA, a_upper, a_lower, b_upper, epi;
    float alpha;        // +1 or -1
    int beta, diag_add; // 0 or 1
    const int* e;
    double* R64;
    float* R32;
    int* flag;
};
constexpr int kTgThreads = 512;
size_t tri_gemm_pair_smem(int d) {
    const int kmax = ((d + TT - 1) / TT) * TT;
    return (size_t)TT * (kmax + 1) * 8 + (size_t)kmax * (TT + 1) * 8 + (size_t)TT * TT * 4 * 4;
}

__global__ void __launch_bounds__(kTgThreads) tri_gemm_pair_kernel(const TriGemmP g) {
    extern __shared__ __align__(16) float2 smp[];
    const int nt = (g.d + TT - 1) / TT;
    const int kmax = nt * TT;
    int t = blockIdx.x, I = 0;
    while (t >= nt - I) {
        t -= nt - I;
        ++I;
    }
    const int J = I + t;
    const int i0 = I * TT, j0 = J * TT;
    int klo = 0, khi = g.d;
    if (g.a_upper) klo = i0;
    if (g.a_lower) khi = min(khi, i0 + TT);
    if (g.b_upper) khi = min(khi, j0 + TT);
    klo -= klo % TT;
    // whole 16-wide chunks (entries past d are zero; past khi within the last
    // chunk the stored zeros of the triangular factors contribute nothing)
    const int klen = khi > klo ? ((khi - klo + TT - 1) / TT) * TT : 0;
    float2* As = smp;                                // [TT][kmax + 1]
    float2* Bs = smp + TT * (kmax + 1);              // [kmax][TT + 1]
    float* red = reinterpret_cast<float*>(Bs + kmax * (TT + 1));   // [TT * TT][4]
    // stage A[i0.., klo..) (a row of 16 per pass, lanes along k) and B[klo.., j0..)
    const int lg = klen > 0 ? klen : 1;
#pragma unroll 4
    for (int q = threadIdx.x; q < TT * klen; q += kTgThreads) {
        const int r = q / lg, c = q - r * lg;
        const int ia = i0 + r, ka = klo + c;
        float2 a = make_float2(0.f, 0.f);
        if (ia < g.d && ka < g.d) {
            a = g.transA ? g.A[(int64_t)ka * g.d + ia] : g.A[(int64_t)ia * g.d + ka];
            if (g.ea) {
                const int sh = -g.ea[ia] - g.ea[ka];
                a = make_float2(ldexpf(a.x, sh), ldexpf(a.y, sh));
            }
        }
        As[r * (kmax + 1) + c] = a;
        const int kr = q >> 4, jc = q & 15;
        const int kb = klo + kr, jb = j0 + jc;
        Bs[kr * (TT + 1) + jc] = (kb < g.d && jb < g.d) ? g.B[(int64_t)kb * g.d + jb] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const int h = threadIdx.x >> 8, o = threadIdx.x & 255, ty = o >> 4, tx = o & 15;
    const int half = ((klen / 2 + TT - 1) / TT) * TT;
    const int kb0 = h ? half : 0, kb1 = h ? klen : min(half, klen);
    float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f;
    for (int k0 = kb0; k0 < kb1; k0 += TT) {
#pragma unroll
        for (int kk = 0; kk < TT; kk += 2) {
            pair_mac(As[ty * (kmax + 1) + k0 + kk], Bs[(k0 + kk) * (TT + 1) + tx], s0, c0);
            pair_mac(As[ty * (kmax + 1) + k0 + kk + 1], Bs[(k0 + kk + 1) * (TT + 1) + tx], s1, c1);
        }
        pair_renorm(s0, c0);
        pair_renorm(s1, c1);
    }
    if (h) {
        red[o * 4 + 0] = s0;
        red[o * 4 + 1] = c0;
        red[o * 4 + 2] = s1;
        red[o * 4 + 3] = c1;
    }
    __syncthreads();
    if (h) return;
    const int i = i0 + ty, j = j0 + tx;
    if (i >= g.d || j >= g.d) return;
    const bool up = j >= i;
    float2 r = make_float2(0.f, 0.f);
    if (up) {
        float S = s0, E = c0;
        two_sum_acc(S, E, s1, c1);
        two_sum_acc(S, E, red[o * 4 + 0], red[o * 4 + 1]);
        two_sum_acc(S, E, red[o * 4 + 2], red[o * 4 + 3]);
        S *= g.alpha;
        E *= g.alpha;
        if (g.beta) {
            const float2 ci = g.Cin[(int64_t)i * g.d + j];
            two_sum_acc(S, E, ci.x, ci.y);
        }
        if (i == j && g.diag_add) two_sum_acc(S, E, 1.f, 0.f);
        r = pair_norm(S, E);
    }
    const int64_t at = (int64_t)i * g.d + j;
    const int64_t mirror = (I < J) ? (int64_t)j * g.d + i : -1;
    if (g.epi == kCorrect) {
        if (up) {
            float S = r.x, E = r.y;
            if (i == j) two_sum_acc(S, E, -1.f, 0.f);
            r = pair_norm(S, E);
            if (!(fabsf(r.x) <= 0.25f)) set_flag(g.flag, LSK_FLAG_RANK_DEFICIENT);
            if (i == j) r = make_float2(0.5f * r.x, 0.5f * r.y);
        }
        g.Out[at] = r;
    } else if (g.epi == kInverse) {
        g.Out[at] = r;
        if (g.R64) g.R64[at] = up ? ldexp((double)r.x + (double)r.y, -g.e[i]) : 0.0;
        if (g.R32) g.R32[at] = up ? ldexpf(r.x, -g.e[i]) : 0.f;
        if (mirror >= 0) {
            if (g.R64) g.R64[mirror] = 0.0;
            if (g.R32) g.R32[mirror] = 0.f;
        }
    } else if (g.epi == kFactor) {
        g.R64[at] = up ? ldexp((double)r.x + (double)r.y, g.e[j]) : 0.0;
        if (mirror >= 0) g.R64[mirror] = 0.0;
    } else {
        g.Out[at] = r;
    }
}

// C (FP64, d x d) -> FP32 pairs, for callers that start from an FP64 Gram
__global__ void to_pair_kernel(const double* __restrict__ C, int64_t len, float2* __restrict__ Cp) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < len; t += (int64_t)gridDim.x * blockDim.x) {
        const double x = C[t];
        const float h = (float)x;
        Cp[t] = make_float2(h, (float)(x - (double)h));
    }
}

size_t chol32_smem(int d) {
    const int nt = (d + CB - 1) / CB;
    return (size_t)nt * (nt + 1) / 2 * CB * CP * 4;
}


}  // namespace

size_t qr_mixed_workspace_bytes(int64_t d) {
    return 6 * ws_round((size_t)d * d * 8) + ws_round((size_t)d * d * 4) + ws_round((size_t)d * (d + 1) / 2 * 4) +
           ws_round((size_t)d * 4) + ws_round((size_t)d * 8) + 4096;
}

void qr_mixed_carve(QrJob& j, void* ws) {
    const size_t d = (size_t)j.d;
    WsCarver wc{(char*)ws, 0};   // the same layout as qr_mixed_launch
    j.Ct = wc.take<double>(d * d);
    j.Ct32 = wc.take<float>(d * d);
    j.Lpk = wc.take<float>(d * (d + 1) / 2);
    j.Rt = wc.take<double>(d * d);
    j.X = wc.take<double>(d * d);
    j.W = wc.take<double>(d * d);
    j.M = wc.take<double>(d * d);
    j.Y = wc.take<double>(d * d);
    j.e = wc.take<int>(d);
    j.sc = wc.take<double>(d);
}

int qr_mixed_blocks(int d, int shape) {
    switch (shape) {
        case QS_ONE: return 1;
        case QS_EW: return std::min((d * d + 255) / 256, 64);
        case QS_TRINV: return (d * 32 + 511) / 512;
        case QS_TRI: {
            const int nt = (d + TT - 1) / TT;
            return nt * (nt + 1) / 2;
        }
        default: return 0;
    }
}

cudaError_t qr_mixed_group_launch(const QrGroup& g, const unsigned char* table, cudaStream_t st) {
    const QrJob* jobs = reinterpret_cast<const QrJob*>(table + g.jobs_off);
    const int* one = reinterpret_cast<const int*>(table + g.off_off[QS_ONE]);
    const int* ew = reinterpret_cast<const int*>(table + g.off_off[QS_EW]);
    const int* tinv = reinterpret_cast<const int*>(table + g.off_off[QS_TRINV]);
    const int* tri = reinterpret_cast<const int*>(table + g.off_off[QS_TRI]);
    const int n = g.count;
    LSK_PROF("qr_equil", st) equil_exponents_grouped_kernel<<<g.blocks[QS_ONE], 256, 0, st>>>(jobs, one, n);
    LSK_PROF("qr_equil", st) equil_scale_grouped_kernel<<<g.blocks[QS_EW], 256, 0, st>>>(jobs, ew, n);
    const size_t tiles = chol32_smem(g.dmax);
    cudaError_t err = allow_dynamic_smem(chol32_grouped_kernel);
    if (err != cudaSuccess) return err;
    LSK_PROF("qr_chol32", st) chol32_grouped_kernel<<<g.blocks[QS_ONE], 512, tiles, st>>>(jobs, one, n);
    const size_t pk = (size_t)g.dmax * (g.dmax + 1) / 2 * 4;
    err = allow_dynamic_smem(trinv32_grouped_kernel);
    if (err != cudaSuccess) return err;
    LSK_PROF("qr_trinv32", st) trinv32_grouped_kernel<<<g.blocks[QS_TRINV], 512, pk, st>>>(jobs, tinv, n);
    LSK_PROF("qr_refine64", st) tri_gemm64_grouped_kernel<<<g.blocks[QS_TRI], 256, 0, st>>>(jobs, tri, n, 0);
    LSK_PROF("qr_refine64", st) tri_gemm64_grouped_kernel<<<g.blocks[QS_TRI], 256, 0, st>>>(jobs, tri, n, 1);
    LSK_PROF("qr_refine64", st) correction_grouped_kernel<<<g.blocks[QS_EW], 256, 0, st>>>(jobs, ew, n);
    LSK_PROF("qr_refine64", st) tri_gemm64_grouped_kernel<<<g.blocks[QS_TRI], 256, 0, st>>>(jobs, tri, n, 2);
    LSK_PROF("qr_finish", st) unscale_grouped_kernel<<<g.blocks[QS_EW], 256, 0, st>>>(jobs, ew, n);
    LSK_PROF("qr_finish", st) rank_check_r_grouped_kernel<<<g.blocks[QS_ONE], 256, 0, st>>>(jobs, one, n);
    return cudaGetLastError();
}

// C: FP64 Gram of the sketch (d x d, full); Cp: the same as FP32 pairs, or
// NULL (then formed here).  Outputs as qr_launch; R is only formed (one
// Newton step) when requested.  Launches: chol_eq (equilibration, FP32
// factor, rank check), trinv32, then W = Ct X, M = X^T W (epilogue: U),
// Y = X - X U (epilogue: R^-1) and, for R, P = I - Y Rt, Z = Rt + Rt P
// (epilogue: R).  Every matrix between them is a pair matrix.
cudaError_t qr_mixed_launch(const double* C, const float2* Cp, int64_t d64, double* R, double* Rinv, float* Rinv32,
                            void* ws, int* flag, cudaStream_t st) {
    const int d = (int)d64;
    const size_t dd = (size_t)d * d;
    WsCarver wc{(char*)ws, 0};
    float2* Cq = wc.take<float2>(dd);
    float* Lpk = wc.take<float>((size_t)d * (d + 1) / 2);
    float2* Rt = wc.take<float2>(dd);
    float2* X = wc.take<float2>(dd);
    float2* W = wc.take<float2>(dd);
    float2* M = wc.take<float2>(dd);
    float2* Y = wc.take<float2>(dd);
    int* e = wc.take<int>(d);
    cudaError_t err;
    if (!Cp) {
        const int64_t g = (int64_t)((dd + 255) / 256) < 1024 ? (int64_t)((dd + 255) / 256) : 1024;
        LSK_PROF("qr_equil", st) to_pair_kernel<<<(unsigned)g, 256, 0, st>>>(C, (int64_t)dd, Cq);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        Cp = Cq;
    }
    if ((err = allow_dynamic_smem(chol_eq_kernel)) != cudaSuccess) return err;
    LSK_PROF("qr_chol32", st) chol_eq_kernel<<<1, 512, chol_eq_smem(d), st>>>(Cp, d, e, R ? Rt : nullptr, Lpk, flag);
    const size_t pk = (size_t)d * (d + 1) / 2 * 4;
    if ((err = allow_dynamic_smem(trinv32_pair_kernel)) != cudaSuccess) return err;
    LSK_PROF("qr_trinv32", st) trinv32_pair_kernel<<<(d * 32 + 127) / 128, 128, pk, st>>>(Lpk, d, X);
    if ((err = allow_dynamic_smem(tri_gemm_pair_kernel)) != cudaSuccess) return err;
    const int nt = (d + TT - 1) / TT;
    const unsigned tiles = (unsigned)(nt * (nt + 1) / 2);
    const size_t tsm = tri_gemm_pair_smem(d);
    auto run = [&](const TriGemmP& g) {
        LSK_PROF("qr_refine64", st) tri_gemm_pair_kernel<<<tiles, kTgThreads, tsm, st>>>(g);
        return cudaGetLastError();
    };
    // W = Ct X on the upper triangle (only k <= j is needed by M); Ct = D^-1 C D^-1 on the fly
    if ((err = run(TriGemmP{Cp, X, nullptr, W, e, d, 0, 0, 0, 1, kPlain, 1.f, 0, 0, nullptr, nullptr, nullptr, flag})) !=
        cudaSuccess)
        return err;
    // M = X^T W, epilogue U
    if ((err = run(TriGemmP{X, W, nullptr, M, nullptr, d, 1, 0, 1, 1, kCorrect, 1.f, 0, 0, nullptr, nullptr, nullptr,
                            flag})) != cudaSuccess)
        return err;
    // Y = X - X U, epilogue R^-1 = D^-1 Y
    if ((err = run(TriGemmP{X, M, X, Y, nullptr, d, 0, 1, 0, 1, kInverse, -1.f, 1, 0, e, Rinv, Rinv32, flag})) !=
        cudaSuccess)
        return err;
    if (R) {
        // P = I - Y Rt ; Z = Rt + Rt P (Newton step for Y^-1), epilogue R = Z D
        if ((err = run(TriGemmP{Y, Rt, nullptr, W, nullptr, d, 0, 1, 0, 1, kPlain, -1.f, 0, 1, nullptr, nullptr,
                                nullptr, flag})) != cudaSuccess)
            return err;
        if ((err = run(TriGemmP{Rt, W, Rt, M, nullptr, d, 0, 1, 0, 1, kFactor, 1.f, 1, 0, e, R, nullptr, flag})) !=
            cudaSuccess)
            return err;
    }
    return cudaGetLastError();
}
