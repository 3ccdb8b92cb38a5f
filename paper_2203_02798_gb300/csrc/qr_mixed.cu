// qr_mixed.cu -- R of the sketch (d <= 256) with an FP32 factorisation and
// one correction step in FP32-pair arithmetic.
//
// FP64 on this part runs at 1/64 of the FP32 rate and has long dependent-
// operation latency, so no step below computes in FP64; the matrices are
// FP32 pairs (x = hi + lo, ~48 bits) and FP64 appears only where R and R^-1
// are written:
//   1. Cp = B^T B as pairs (qr.cu), equilibrated by powers of two:
//      Ct = D^-1 C D^-1, D_j = 2^floor(log2 sqrt(C_jj))           (exact)
//   2. Ct ~ Rt^T Rt by FP32 Cholesky (one CTA, the lower triangle in shared
//      memory), X = Rt^-1 by FP32 back substitution
//   3. one correction step with pair-accurate products of triangular matrices:
//        M = X^T Ct X = I + E,  U = strict_upper(E) + diag(E)/2
//        Y = X (I - U)                         (= (R D^-1)^-1 to O(|E|^2))
//        Z = Rt + Rt (I - Y Rt)                (Newton step for Y^-1, when R is wanted)
//   4. R = Z D, R^-1 = D^-1 Y
// One sketch runs the chain as five to seven launches; a batch runs the same
// kernels grouped (one grid per step over all sketches, R not formed).
// In exact arithmetic R is the Cholesky factor of C, i.e. the sign-normalised
// Householder R of B.  Rank deficiency is reported when an FP32 pivot is not
// positive, when the equilibrated FP32 factor's diagonal spans more than 2^20,
// or when the FP32 factor needs a correction larger than 1/4 (the
// equilibrated sketch is numerically singular at FP32 precision).
#include "lsk_internal.cuh"

#include <algorithm>

namespace {

constexpr int TT = 16;   // tile edge of the triangular pair products (16 x 16 outputs a block)

// FP32 Cholesky pieces: 32 x 32 tiles (CB) of the lower triangle.
constexpr int CB = 32;

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

// Pair arithmetic for the triangular products (FP32 throughout, x = hi + lo
// ~48 bits): each product is formed as hi*hi exactly (one FMA gives its
// rounding error) plus the cross terms, and the sum is kept as an FP32 pair
// (TwoSum), renormalised every 16 terms.
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

__device__ __forceinline__ void chol_eq_body(const float2* __restrict__ Cp, int d, int* __restrict__ e_out,
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

__global__ void __launch_bounds__(512) chol_eq_kernel(const float2* __restrict__ Cp, int d, int* __restrict__ e_out,
                                                      float2* __restrict__ Rt, float* __restrict__ Lpk, int* flag) {
    chol_eq_body(Cp, d, e_out, Rt, Lpk, flag);
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

__device__ __forceinline__ void tri_gemm_pair_body(const TriGemmP& g, const int tile) {
    extern __shared__ __align__(16) float2 smp[];
    const int nt = (g.d + TT - 1) / TT;
    const int kmax = nt * TT;
    int t = tile, I = 0;
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

__global__ void __launch_bounds__(kTgThreads) tri_gemm_pair_kernel(const TriGemmP g) { tri_gemm_pair_body(g, blockIdx.x); }

// ---- grouped: one grid per stage over many sketches (QrJob table), the
// same pair chain as one sketch's (R is not formed in a group) -------------
__device__ __forceinline__ const QrJob& job_of(const QrJob* jobs, const int* off, int count, int& blk, int& nblk) {
    const int g = group_of(off, count, blockIdx.x);
    const int b0 = __ldg(off + g);
    blk = (int)blockIdx.x - b0;
    nblk = __ldg(off + g + 1) - b0;
    return jobs[g];
}
__global__ void __launch_bounds__(512) chol_eq_grouped_kernel(const QrJob* __restrict__ jobs, const int* __restrict__ off,
                                                              int count) {
    int blk, nblk;
    const QrJob& j = job_of(jobs, off, count, blk, nblk);
    chol_eq_body(j.Cp, j.d, j.e, nullptr, j.Lpk, j.flag);
}
__global__ void __launch_bounds__(512) trinv32_pair_grouped_kernel(const QrJob* __restrict__ jobs,
                                                                   const int* __restrict__ off, int count) {
    int blk, nblk;
    const QrJob& j = job_of(jobs, off, count, blk, nblk);
    trinv32_body(j.Lpk, j.d, j.X, blk, nblk);
}
// which: 0 W = Ct X, 1 M = X^T W (epilogue U), 2 Y = X - X U (epilogue R^-1)
__global__ void __launch_bounds__(kTgThreads) tri_gemm_pair_grouped_kernel(const QrJob* __restrict__ jobs,
                                                                           const int* __restrict__ off, int count,
                                                                           int which) {
    int blk, nblk;
    const QrJob& j = job_of(jobs, off, count, blk, nblk);
    TriGemmP g;
    if (which == 0)
        g = TriGemmP{j.Cp, j.X, nullptr, j.W, j.e, j.d, 0, 0, 0, 1, kPlain, 1.f, 0, 0, nullptr, nullptr, nullptr, j.flag};
    else if (which == 1)
        g = TriGemmP{j.X, j.W, nullptr, j.M, nullptr, j.d, 1, 0, 1, 1, kCorrect, 1.f, 0, 0, nullptr, nullptr, nullptr,
                     j.flag};
    else
        g = TriGemmP{j.X, j.M, j.X, j.Y, nullptr, j.d, 0, 1, 0, 1, kInverse, -1.f, 1, 0, j.e, j.Rinv, j.Rinv32, j.flag};
    tri_gemm_pair_body(g, blk);
}

// C (FP64, d x d) -> FP32 pairs, for callers that start from an FP64 Gram
__global__ void to_pair_kernel(const double* __restrict__ C, int64_t len, float2* __restrict__ Cp) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < len; t += (int64_t)gridDim.x * blockDim.x) {
        const double x = C[t];
        const float h = (float)x;
        Cp[t] = make_float2(h, (float)(x - (double)h));
    }
}



}  // namespace

size_t qr_mixed_workspace_bytes(int64_t d) {
    return 6 * ws_round((size_t)d * d * 8) + ws_round((size_t)d * d * 4) + ws_round((size_t)d * (d + 1) / 2 * 4) +
           ws_round((size_t)d * 4) + ws_round((size_t)d * 8) + 4096;
}

void qr_mixed_carve(QrJob& j, void* ws) {
    const size_t d = (size_t)j.d;
    WsCarver wc{(char*)ws, 0};   // within qr_mixed_workspace_bytes(d)
    j.Cp = wc.take<float2>(d * d);
    j.Lpk = wc.take<float>(d * (d + 1) / 2);
    j.X = wc.take<float2>(d * d);
    j.W = wc.take<float2>(d * d);
    j.M = wc.take<float2>(d * d);
    j.Y = wc.take<float2>(d * d);
    j.e = wc.take<int>(d);
}

int qr_mixed_blocks(int d, int shape) {
    switch (shape) {
        case QS_ONE: return 1;
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
    const int* tinv = reinterpret_cast<const int*>(table + g.off_off[QS_TRINV]);
    const int* tri = reinterpret_cast<const int*>(table + g.off_off[QS_TRI]);
    const int n = g.count;
    cudaError_t err;
    if ((err = allow_dynamic_smem(chol_eq_grouped_kernel)) != cudaSuccess) return err;
    LSK_PROF("qr_chol32", st) chol_eq_grouped_kernel<<<g.blocks[QS_ONE], 512, chol_eq_smem(g.dmax), st>>>(jobs, one, n);
    const size_t pk = (size_t)g.dmax * (g.dmax + 1) / 2 * 4;
    if ((err = allow_dynamic_smem(trinv32_pair_grouped_kernel)) != cudaSuccess) return err;
    LSK_PROF("qr_trinv32", st) trinv32_pair_grouped_kernel<<<g.blocks[QS_TRINV], 512, pk, st>>>(jobs, tinv, n);
    if ((err = allow_dynamic_smem(tri_gemm_pair_grouped_kernel)) != cudaSuccess) return err;
    const size_t tsm = tri_gemm_pair_smem(g.dmax);
    for (int which = 0; which < 3; ++which) {
        LSK_PROF("qr_refine64", st) tri_gemm_pair_grouped_kernel<<<g.blocks[QS_TRI], kTgThreads, tsm, st>>>(jobs, tri,
                                                                                                          n, which);
    }
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
