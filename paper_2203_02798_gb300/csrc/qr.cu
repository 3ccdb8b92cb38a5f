// qr.cu -- R of the sketch and R^-1 in FP64 (Alg. 12 step 2, Alg. 15 step 3).
//
// The paper factors the small sketch B (k x d) with an SVD; the reading used
// here takes the QR factor R with a positive diagonal, computed as the
// Cholesky factor of B^T B:
//   1. C = B^T B with exact products of the FP32 values summed in FP32
//      pairs (near-FP64 accuracy at FP32 rates), split over row chunks of B
//      and tiles of C, chunk partials added in FP64 in a fixed order;
//   2. C = L L^T by right-looking blocked Cholesky, 16x16 blocks, two
//      launches per block column (panel, trailing update), so the FP64 work
//      is spread over the whole GPU (FP64 is scarce on this part);
//   3. R = L^T; rank check min R_jj <= 16 eps d max R_jj (flag);
//   4. R^-1 column by column (one warp per column, back substitution).
// In exact arithmetic this R equals the sign-normalised Householder R of B.
// For d <= 256 steps 2-4 are replaced by the mixed-precision factorisation of
// qr_mixed.cu (FP32 Cholesky + one FP64 correction made of parallel
// triangular products), which avoids FP64 dependency chains; the all-FP64
// blocked path below serves larger d.
#include "lsk_internal.cuh"

#include <algorithm>

size_t qr_mixed_workspace_bytes(int64_t d);
cudaError_t qr_mixed_launch(const double* C, const float2* Cp, int64_t d, double* R, double* Rinv, float* Rinv32,
                            void* ws, int* flag, cudaStream_t st);

namespace {

constexpr int QT = 32;   // tile edge of the sketch Gram
constexpr int NB = 16;   // Cholesky block

__device__ __forceinline__ void utile_of(int t, int nt, int& ta, int& tb) {
    ta = 0;
    while (t >= nt - ta) {
        t -= nt - ta;
        ++ta;
    }
    tb = ta + t;
}

// s + c += x y in FP32 pairs: the product is split exactly (x y = p + e,
// one FMA) and the sum s + p by TwoSum, whose rounding error goes to c.
// The _rn intrinsics keep the compiler from fusing any of these steps.
__device__ __forceinline__ void df_mac(float x, float y, float& s, float& c) {
    const float p = __fmul_rn(x, y);
    const float e = fmaf(x, y, -p);
    const float t = __fadd_rn(s, p);
    const float z = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
    c = __fadd_rn(c, __fadd_rn(err, e));
    s = t;
}

// (s, c) <- TwoSum(s, c): keeps |c| at most half an ulp of s.
__device__ __forceinline__ void df_renorm(float& s, float& c) {
    const float t = __fadd_rn(s, c);
    const float z = __fsub_rn(t, s);
    c = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(c, z));
    s = t;
}

// Block (tile, chunk): upper tile `tile` of C over row chunk `chunk` of B.
// Each product of two FP32 values is formed exactly and summed in FP32
// pairs, renormalised every 32 rows: the error is of order k 2^-48 relative
// to sum |x y| (FP64 summation: k 2^-53), and the FP64 units, scarce on
// this part, are not used.  The chunk partials are written as FP64 (s + c).
__device__ __forceinline__ void sketch_gram64_body(const float* __restrict__ B, int64_t k, int64_t d, int64_t rows_per,
                                                   double* __restrict__ part, const int tile, const int chunk) {
    __shared__ float Xa[QT][QT + 1];
    __shared__ float Xb[QT][QT + 1];
    const int nt = (int)((d + QT - 1) / QT);
    int ta, tb;
    utile_of(tile, nt, ta, tb);
    const int64_t a0 = (int64_t)ta * QT, b0 = (int64_t)tb * QT;
    const int tid = threadIdx.x;
    const int ty = tid >> 4, tx = tid & 15;   // outputs (2ty+u, 2tx+v)
    const int64_t r0 = (int64_t)chunk * rows_per;
    const int64_t r1 = min(k, r0 + rows_per);
    float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, cmp[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
    for (int64_t i0 = r0; i0 < r1; i0 += QT) {
#pragma unroll
        for (int t = 0; t < (QT * QT) / 256; ++t) {
            const int idx = tid + 256 * t;
            const int rr = idx / QT, cc = idx % QT;
            const int64_t i = i0 + rr;
            Xa[rr][cc] = (i < r1 && a0 + cc < d) ? B[i * d + a0 + cc] : 0.f;
            Xb[rr][cc] = (i < r1 && b0 + cc < d) ? B[i * d + b0 + cc] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int rr = 0; rr < QT; ++rr) {
            const float x0 = Xa[rr][2 * ty], x1 = Xa[rr][2 * ty + 1];
            const float y0 = Xb[rr][2 * tx], y1 = Xb[rr][2 * tx + 1];
            df_mac(x0, y0, acc[0][0], cmp[0][0]);
            df_mac(x0, y1, acc[0][1], cmp[0][1]);
            df_mac(x1, y0, acc[1][0], cmp[1][0]);
            df_mac(x1, y1, acc[1][1], cmp[1][1]);
        }
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int v = 0; v < 2; ++v) df_renorm(acc[u][v], cmp[u][v]);
        __syncthreads();
    }
    const int ntiles = nt * (nt + 1) / 2;
    double* P = part + ((int64_t)chunk * ntiles + tile) * QT * QT;
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) P[(2 * ty + u) * QT + 2 * tx + v] = (double)acc[u][v] + (double)cmp[u][v];
}

__device__ __forceinline__ void sketch_gram64_reduce_body(const double* __restrict__ part, int64_t nchunks, int64_t d,
                                                          double* __restrict__ C, const int blk, const int nblk,
                                                          float2* __restrict__ Cp = nullptr) {
    const int nt = (int)((d + QT - 1) / QT);
    const int ntiles = nt * (nt + 1) / 2;
    const int64_t len = d * d;
    const int64_t stride = (int64_t)nblk * blockDim.x;
    for (int64_t e = (int64_t)blk * blockDim.x + threadIdx.x; e < len; e += stride) {
        int64_t a = e / d, b = e % d;
        if (a > b) {
            const int64_t t = a;
            a = b;
            b = t;
        }
        const int ta = (int)(a / QT), tb = (int)(b / QT);
        const int tile = ta * nt - ta * (ta - 1) / 2 + (tb - ta);
        const int64_t w = (a % QT) * QT + (b % QT);
        double s = 0.0;
        for (int64_t z = 0; z < nchunks; ++z) s += part[(z * ntiles + tile) * QT * QT + w];
        C[e] = s;
        if (Cp) {   // the same as an FP32 pair (hi + lo, ~48 bits)
            const float h = (float)s;
            Cp[e] = make_float2(h, (float)(s - (double)h));
        }
    }
}

__global__ void __launch_bounds__(256) sketch_gram64_kernel(const float* __restrict__ B, int64_t k, int64_t d,
                                                            int64_t rows_per, double* __restrict__ part) {
    sketch_gram64_body(B, k, d, rows_per, part, blockIdx.x, blockIdx.y);
}
__global__ void sketch_gram64_reduce_kernel(const double* __restrict__ part, int64_t nchunks, int64_t d,
                                            double* __restrict__ C, float2* __restrict__ Cp) {
    sketch_gram64_reduce_body(part, nchunks, d, C, blockIdx.x, gridDim.x, Cp);
}
// grouped over QrJob tables: local block b of a job = (tile b % ntiles, chunk b / ntiles)
__global__ void __launch_bounds__(256) sketch_gram64_grouped_kernel(const QrJob* __restrict__ jobs,
                                                                    const int* __restrict__ off, int count) {
    const int g = group_of(off, count, blockIdx.x);
    const QrJob& j = jobs[g];
    const int b = (int)blockIdx.x - __ldg(off + g);
    sketch_gram64_body(j.B, j.k, j.d, j.rows_per, j.part, b % j.ntiles, b / j.ntiles);
}
__global__ void sketch_gram64_reduce_grouped_kernel(const QrJob* __restrict__ jobs, const int* __restrict__ off,
                                                    int count) {
    const int g = group_of(off, count, blockIdx.x);
    const QrJob& j = jobs[g];
    const int b0 = __ldg(off + g);
    sketch_gram64_reduce_body(j.part, j.nchunks, j.d, j.C, (int)blockIdx.x - b0, __ldg(off + g + 1) - b0, j.Cp);
}

// Factor the diagonal block K of C (lower part) in shared memory.  Every
// block of the panel launch does this redundantly (it is 16x16).  A pivot
// that is not positive and finite flags rank deficiency and is replaced by 1.
__device__ void factor_diag_block(double* C, int64_t d, int64_t kb, double (*L)[NB + 1], int m,
                                  int* flag) {
    const int tid = threadIdx.x;
    for (int e = tid; e < NB * NB; e += blockDim.x) {
        const int i = e / NB, j = e % NB;
        L[i][j] = (i < m && j < m && j <= i) ? C[(kb + i) * d + kb + j] : 0.0;
    }
    __syncthreads();
    if (tid < 32) {
        const int i = tid;
        for (int j = 0; j < m; ++j) {
            double piv = L[j][j];
            if (!(piv > 0.0) || !isfinite(piv)) {
                if (i == 0) set_flag(flag, LSK_FLAG_RANK_DEFICIENT);
                piv = 1.0;
            }
            const double ljj = sqrt(piv);
            __syncwarp();
            if (i == j) L[j][j] = ljj;
            if (i > j && i < m) L[i][j] /= ljj;
            __syncwarp();
            if (i > j && i < m)
                for (int l = j + 1; l <= i; ++l) L[i][l] -= L[i][j] * L[l][j];
            __syncwarp();
        }
    }
    __syncthreads();
}

// Block 0 stores L_KK in `Ldiag` (not in C: the other blocks of this launch
// are still reading A_KK from C); copy_diag_kernel moves it into C at the end.
__global__ void chol_panel_kernel(double* __restrict__ C, int64_t d, int64_t K,
                                  double* __restrict__ Ldiag, int* flag) {
    __shared__ double L[NB][NB + 1];
    const int64_t kb = K * NB;
    const int m = (int)min((int64_t)NB, d - kb);
    factor_diag_block(C, d, kb, L, m, flag);
    if (blockIdx.x == 0) {
        double* D = Ldiag + K * NB * NB;
        for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
            const int i = e / NB, j = e % NB;
            D[e] = (j <= i && i < m) ? L[i][j] : 0.0;
        }
        return;
    }
    // row block I = K + blockIdx.x: L_IK = A_IK L_KK^-T (forward substitution per row)
    const int64_t ib = kb + (int64_t)blockIdx.x * NB;
    if (ib >= d) return;
    const int mi = (int)min((int64_t)NB, d - ib);
    const int t = threadIdx.x;
    if (t < mi) {
        double x[NB];
        double* row = C + (ib + t) * d + kb;
        for (int j = 0; j < m; ++j) {
            double s = row[j];
            for (int l = 0; l < j; ++l) s -= x[l] * L[j][l];
            x[j] = s / L[j][j];
        }
        for (int j = 0; j < m; ++j) row[j] = x[j];
    }
}

// Trailing update of the lower triangle: A_IJ -= L_IK L_JK^T for I >= J > K.
__global__ void chol_update_kernel(double* __restrict__ C, int64_t d, int64_t K) {
    const int64_t nbk = (d + NB - 1) / NB;
    const int T = (int)(nbk - K - 1);
    int t = blockIdx.x, I = 0;
    // lower-triangular tile pairs (J <= I) over the trailing T blocks
    while (t > I) {
        t -= I + 1;
        ++I;
    }
    const int J = t;
    const int64_t ib = (K + 1 + I) * NB, jb = (K + 1 + J) * NB, kb = K * NB;
    __shared__ double Li[NB][NB + 1], Lj[NB][NB + 1];
    const int mk = (int)min((int64_t)NB, d - kb);
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        const int a = e / NB, b = e % NB;
        Li[a][b] = (ib + a < d && b < mk) ? C[(ib + a) * d + kb + b] : 0.0;
        Lj[a][b] = (jb + a < d && b < mk) ? C[(jb + a) * d + kb + b] : 0.0;
    }
    __syncthreads();
    (void)T;
    const int a = threadIdx.x / NB, b = threadIdx.x % NB;
    if (ib + a < d && jb + b < d && (I != J || b <= a)) {
        double s = 0.0;
#pragma unroll
        for (int l = 0; l < NB; ++l) s = fma(Li[a][l], Lj[b][l], s);
        C[(ib + a) * d + jb + b] -= s;
    }
}

__global__ void copy_diag_kernel(double* __restrict__ C, int64_t d,
                                 const double* __restrict__ Ldiag) {
    const int64_t kb = (int64_t)blockIdx.x * NB;
    const double* D = Ldiag + (int64_t)blockIdx.x * NB * NB;
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        const int i = e / NB, j = e % NB;
        if (kb + i < d && kb + j < d) C[(kb + i) * d + kb + j] = D[e];
    }
}

__global__ void rank_check_kernel(const double* __restrict__ Lm, int64_t d, int* flag) {
    double mn = INFINITY, mx = 0.0;
    for (int64_t j = threadIdx.x; j < d; j += blockDim.x) {
        const double v = fabs(Lm[j * d + j]);
        mn = fmin(mn, v);
        mx = fmax(mx, v);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    __shared__ double smn[32], smx[32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        smn[w] = mn;
        smx[w] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
            mn = fmin(mn, smn[i]);
            mx = fmax(mx, smx[i]);
        }
        mn = fmin(mn, smn[0]);
        mx = fmax(mx, smx[0]);
        const double eps = 2.220446049250313e-16;
        if (!(mn > 16.0 * eps * (double)d * mx) || !isfinite(mx)) set_flag(flag, LSK_FLAG_RANK_DEFICIENT);
    }
}

// X = R^-1 with R = L^T: warp per column j, lane owns rows i = lane + 32 s.
template <int S>
__global__ void trinv_kernel(const double* __restrict__ Lm, int64_t d, double* __restrict__ X64,
                             float* __restrict__ X32, double* __restrict__ Rout) {
    const int lane = threadIdx.x & 31;
    const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (j >= d) return;
    double xr[S];
#pragma unroll
    for (int s = 0; s < S; ++s) xr[s] = ((int64_t)(lane + 32 * s) == j) ? 1.0 : 0.0;
    for (int64_t l = j; l >= 0; --l) {
        const int owner = (int)(l & 31), slot = (int)(l >> 5);
        double v = 0.0;
#pragma unroll
        for (int s = 0; s < S; ++s)
            if (s == slot) v = xr[s];
        v = __shfl_sync(0xffffffffu, v, owner);
        const double xl = v / Lm[l * d + l];
#pragma unroll
        for (int s = 0; s < S; ++s)
            if (s == slot && lane == owner) xr[s] = xl;
        const double* Lrow = Lm + l * d;   // R[i][l] = L[l][i]
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int64_t i = lane + 32 * s;
            if (i < l) xr[s] = fma(-Lrow[i], xl, xr[s]);
        }
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int64_t i = lane + 32 * s;
        if (i < d) {
            const double v = (i <= j) ? xr[s] : 0.0;
            if (X64) X64[i * d + j] = v;
            if (X32) X32[i * d + j] = (float)v;
            if (Rout) Rout[i * d + j] = (i <= j) ? Lm[j * d + i] : 0.0;
        }
    }
}

struct QrPlan {
    int ntiles;
    int64_t nchunks, rows_per;
};
QrPlan qr_plan(int64_t k, int64_t d) {
    QrPlan p;
    const int nt = (int)((d + QT - 1) / QT);
    p.ntiles = nt * (nt + 1) / 2;
    int64_t want = (600 + p.ntiles - 1) / p.ntiles;
    int64_t rows = (k + want - 1) / want;
    rows = ((rows + QT - 1) / QT) * QT;
    if (rows < QT) rows = QT;
    p.rows_per = rows;
    p.nchunks = (k + rows - 1) / rows;
    if (p.nchunks < 1) p.nchunks = 1;
    return p;
}

}  // namespace

size_t sketch_gram64_workspace_bytes(int64_t k, int64_t d) {
    const QrPlan p = qr_plan(k, d);
    return ws_round((size_t)p.nchunks * p.ntiles * QT * QT * 8);
}

cudaError_t sketch_gram64_launch(const float* B, int64_t k, int64_t d, double* C, void* ws, int sm_count,
                                 cudaStream_t st, float2* Cp) {
    const QrPlan p = qr_plan(k, d);
    double* part = (double*)ws;
    LSK_PROF("qr_gram64", st) sketch_gram64_kernel<<<dim3((unsigned)p.ntiles, (unsigned)p.nchunks), 256, 0, st>>>(B, k, d, p.rows_per,
                                                                                      part);
    int64_t g = (d * d + 255) / 256;
    if (g > 8 * (int64_t)sm_count) g = 8 * (int64_t)sm_count;
    LSK_PROF("qr_gram64", st) sketch_gram64_reduce_kernel<<<(unsigned)g, 256, 0, st>>>(part, p.nchunks, d, C, Cp);
    return cudaGetLastError();
}

size_t qr_from_gram_workspace_bytes(int64_t d) {
    const int64_t nbk = (d + NB - 1) / NB;
    size_t rest = ws_round((size_t)nbk * NB * NB * 8);
    if (d <= 256 && qr_mixed_workspace_bytes(d) > rest) rest = qr_mixed_workspace_bytes(d);
    return rest;
}

cudaError_t qr_from_gram_launch(double* C, int64_t d, double* R, double* Rinv, float* Rinv32, void* ws, int* flag,
                                cudaStream_t st, const float2* Cp) {
    if (d > 1024) return cudaErrorInvalidValue;
    if (d <= 256) return qr_mixed_launch(C, Cp, d, R, Rinv, Rinv32, ws, flag, st);
    const int64_t nbk = (d + NB - 1) / NB;
    double* Ldiag = (double*)ws;
    for (int64_t K = 0; K < nbk; ++K) {
        const unsigned panel_blocks = (unsigned)(nbk - K);   // diag + blocks below
        LSK_PROF("qr_cholesky", st) chol_panel_kernel<<<panel_blocks, 64, 0, st>>>(C, d, K, Ldiag, flag);
        const int64_t T = nbk - K - 1;
        if (T > 0) LSK_PROF("qr_cholesky", st) chol_update_kernel<<<(unsigned)(T * (T + 1) / 2), NB * NB, 0, st>>>(C, d, K);
    }
    LSK_PROF("qr_cholesky", st) copy_diag_kernel<<<(unsigned)nbk, NB * NB, 0, st>>>(C, d, Ldiag);
    LSK_PROF("qr_rank", st) rank_check_kernel<<<1, 256, 0, st>>>(C, d, flag);
    const unsigned tg = (unsigned)((d * 32 + 127) / 128);
    LSK_PROF("qr_trinv", st) trinv_kernel<32><<<tg, 128, 0, st>>>(C, d, Rinv, Rinv32, R);
    return cudaGetLastError();
}

size_t qr_workspace_bytes(int64_t k, int64_t d) {
    return ws_round((size_t)d * d * 8) * 2 + sketch_gram64_workspace_bytes(k, d) + qr_from_gram_workspace_bytes(d);
}

cudaError_t qr_launch(const float* B, int64_t k, int64_t d, double* R, double* Rinv, float* Rinv32,
                      void* ws, int* flag, int sm_count, cudaStream_t st) {
    if (d > 1024) return cudaErrorInvalidValue;
    WsCarver wc{(char*)ws, 0};
    double* C = wc.take<double>((size_t)d * d);
    float2* Cp = wc.take<float2>((size_t)d * d);
    void* part = wc.take<char>(sketch_gram64_workspace_bytes(k, d));
    void* rest = wc.take<char>(qr_from_gram_workspace_bytes(d));
    cudaError_t e = sketch_gram64_launch(B, k, d, C, part, sm_count, st, d <= 256 ? Cp : nullptr);
    if (e != cudaSuccess) return e;
    return qr_from_gram_launch(C, d, R, Rinv, Rinv32, rest, flag, st, d <= 256 ? Cp : nullptr);
}

bool qr_group_supported(int64_t k, int64_t d) { return d >= 1 && d <= 256 && k >= d; }

// The same workspace layout as qr_launch (C, Gram partials, then the
// mixed-precision factorisation's buffers).
void qr_group_job(QrJob& j, const float* B, int64_t k, int64_t d, void* ws, double* Rinv, float* Rinv32, int* flag) {
    const QrPlan p = qr_plan(k, d);
    WsCarver wc{(char*)ws, 0};
    j.B = B;
    j.k = k;
    j.d = (int)d;
    j.rows_per = p.rows_per;
    j.nchunks = (int)p.nchunks;
    j.ntiles = p.ntiles;
    j.C = wc.take<double>((size_t)d * d);
    j.part = wc.take<double>((size_t)p.nchunks * p.ntiles * QT * QT);
    const int64_t nbk = (d + NB - 1) / NB;
    void* rest = wc.take<double>((size_t)nbk * NB * NB);
    qr_mixed_carve(j, rest);
    j.Rinv = Rinv;
    j.Rinv32 = Rinv32;
    j.flag = flag;
}

void qr_group_build(const std::vector<QrJob>& jobs, HostTable& t, QrGroup& g) {
    g.count = (int)jobs.size();
    g.dmax = 1;
    std::vector<int> blocks(jobs.size()), off;
    for (int s = 0; s < QS_N; ++s) {
        for (size_t i = 0; i < jobs.size(); ++i) {
            const QrJob& j = jobs[i];
            if (j.d > g.dmax) g.dmax = j.d;
            if (s == QS_GRAM) blocks[i] = j.ntiles * j.nchunks;
            else if (s == QS_GRAMRED) blocks[i] = std::min((j.d * j.d + 255) / 256, 64);
            else blocks[i] = qr_mixed_blocks(j.d, s);
        }
        g.blocks[s] = group_offsets(blocks, off);
        g.off_off[s] = t.put(off.data(), off.size());
    }
    g.jobs_off = t.put(jobs.data(), jobs.size());
}

cudaError_t qr_group_launch(const QrGroup& g, const unsigned char* table, cudaStream_t st) {
    if (g.count == 0) return cudaSuccess;
    const QrJob* jobs = reinterpret_cast<const QrJob*>(table + g.jobs_off);
    LSK_PROF("qr_gram64", st) sketch_gram64_grouped_kernel<<<g.blocks[QS_GRAM], 256, 0, st>>>(
        jobs, reinterpret_cast<const int*>(table + g.off_off[QS_GRAM]), g.count);
    LSK_PROF("qr_gram64", st) sketch_gram64_reduce_grouped_kernel<<<g.blocks[QS_GRAMRED], 256, 0, st>>>(
        jobs, reinterpret_cast<const int*>(table + g.off_off[QS_GRAMRED]), g.count);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return qr_mixed_group_launch(g, table, st);
}
