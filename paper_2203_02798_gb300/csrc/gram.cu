// gram.cu -- C <- alpha A^T A + beta C (csrrk semantics; Alg. 5 and Alg. 7).
//
// Both forms follow Alg. 7's structure -- row blocks of A produce private
// partial Gram matrices which are then summed -- with GPU-sized grains:
//
//  dense: a block owns one 64x64 tile of the upper triangle of C and one
//         chunk of rows; FP32 products are accumulated in registers and
//         folded into FP64 every kFold rows (bounding FP32 chain length), the
//         FP64 partials of the chunks are added in a fixed order.
//  CSR:   a block owns a slice of rows of C held in shared memory (the
//         "private d x d" of Alg. 7, sliced so it fits) and a range of rows
//         of A; each thread runs Alg. 5 on its rows (the upper-triangle
//         outer products of the row's nonzeros, shared-memory atomics), the
//         FP32 slices of all blocks are then summed in FP64 in a fixed order
//         and mirrored.
#include "lsk_internal.cuh"

namespace {

constexpr int GT = 64;       // tile edge of C
constexpr int GK = 16;       // rows of A per step
constexpr int kFold = 64;    // steps (of GK rows) between FP32 -> FP64 folds

__device__ __forceinline__ void tile_of(int t, int nt, int& ta, int& tb) {
    // enumerate the upper-triangular tile pairs (ta <= tb) row by row
    ta = 0;
    while (t >= nt - ta) {
        t -= nt - ta;
        ++ta;
    }
    tb = ta + t;
}

__global__ void __launch_bounds__(256) gram_dense_kernel(const float* __restrict__ A, int64_t lda,
                                                         int64_t n, int64_t d, int64_t rows_per,
                                                         double* __restrict__ part) {
    __shared__ __align__(16) float As[GK][GT];
    __shared__ __align__(16) float Bs[GK][GT];
    const int nt = (int)((d + GT - 1) / GT);
    int ta, tb;
    tile_of(blockIdx.x, nt, ta, tb);
    const int64_t a0 = (int64_t)ta * GT, b0 = (int64_t)tb * GT;
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const int64_t i_begin = (int64_t)blockIdx.y * rows_per;
    const int64_t i_end = min(n, i_begin + rows_per);
    float acc[4][4];
    double acc64[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            acc[a][b] = 0.f;
            acc64[a][b] = 0.0;
        }
    int steps = 0;
    for (int64_t i0 = i_begin; i0 < i_end; i0 += GK) {
#pragma unroll
        for (int t = 0; t < (GK * GT) / 256; ++t) {
            const int idx = tid + 256 * t;
            const int kr = idx / GT, cc = idx % GT;
            const int64_t i = i0 + kr;
            const bool rok = i < i_end;
            As[kr][cc] = (rok && a0 + cc < d) ? __ldg(A + i * lda + a0 + cc) : 0.f;
            Bs[kr][cc] = (rok && b0 + cc < d) ? __ldg(A + i * lda + b0 + cc) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            const float4 x = *reinterpret_cast<const float4*>(&As[kk][4 * ty]);
            const float4 y = *reinterpret_cast<const float4*>(&Bs[kk][4 * tx]);
            const float xa[4] = {x.x, x.y, x.z, x.w}, yb[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(xa[a], yb[b], acc[a][b]);
        }
        __syncthreads();
        if (++steps == kFold) {
            steps = 0;
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    acc64[a][b] += (double)acc[a][b];
                    acc[a][b] = 0.f;
                }
        }
    }
    const int ntiles = nt * (nt + 1) / 2;
    double* P = part + ((int64_t)blockIdx.y * ntiles + blockIdx.x) * GT * GT;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) P[(4 * ty + a) * GT + 4 * tx + b] = acc64[a][b] + (double)acc[a][b];
}

// C[a][b] = C[b][a] = alpha sum_z part[z][tile(a, b)][w] + beta C (a <= b):
// a block takes 32 consecutive entries; thread (g, x) adds the chunks z = g,
// g + 8, ... of entry x, then the 8 group sums are added in order
// (deterministic).
template <typename OutT>
__global__ void __launch_bounds__(256) gram_dense_reduce_kernel(const double* __restrict__ part, int64_t nchunks,
                                                                 int64_t d, double alpha, double beta,
                                                                 OutT* __restrict__ C) {
    __shared__ double acc[8][33];
    const int nt = (int)((d + GT - 1) / GT);
    const int ntiles = nt * (nt + 1) / 2;
    const int x = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int64_t e = (int64_t)blockIdx.x * 32 + x;
    const int64_t a = e / d, b = e % d;
    const bool upper = e < d * d && a <= b;
    double s = 0.0;
    if (upper) {
        const int ta = (int)(a / GT), tb = (int)(b / GT);
        const int tile = ta * nt - ta * (ta - 1) / 2 + (tb - ta);
        const double* src = part + (int64_t)tile * GT * GT + (a % GT) * GT + (b % GT);
        const int64_t zs = (int64_t)ntiles * GT * GT;   // one chunk
        int64_t z = g;
        for (; z + 24 < nchunks; z += 32) {   // four loads in flight
            const double x0 = src[z * zs], x1 = src[(z + 8) * zs], x2 = src[(z + 16) * zs], x3 = src[(z + 24) * zs];
            s += x0;
            s += x1;
            s += x2;
            s += x3;
        }
        for (; z < nchunks; z += 8) s += src[z * zs];
    }
    acc[g][x] = s;
    __syncthreads();
    if (g == 0 && upper) {
        double t = 0.0;
        for (int k = 0; k < 8; ++k) t += acc[k][x];
        const double ab = alpha * t;
        C[a * d + b] = (OutT)(beta != 0.0 ? ab + beta * (double)C[a * d + b] : ab);
        if (a != b) C[b * d + a] = (OutT)(beta != 0.0 ? ab + beta * (double)C[b * d + a] : ab);
    }
}

// ---- CSR ------------------------------------------------------------------
// Alg. 5 on the rows of one block: for each pair of nonzeros p <= q of a row
// (positions in the row), v_p v_q is added to the upper-triangle entry
// (min(j_p, j_q), max(j_p, j_q)) of the block's shared-memory slice -- twice
// when p < q share a column, once on the diagonal -- so each off-diagonal
// product is formed once.  1024 threads a block (one block per SM: the slice
// is up to 192 KB), one row a thread.
__global__ void __launch_bounds__(1024) gram_csr_kernel(const float* __restrict__ V, const int32_t* __restrict__ J,
                                                       const int64_t* __restrict__ I, int64_t n, int64_t nnz,
                                                       int64_t d, int64_t slice_rows, int64_t rows_per,
                                                       float* __restrict__ part, int* flag) {
    extern __shared__ float S[];
    const int64_t j0 = (int64_t)blockIdx.y * slice_rows;
    const int64_t j1 = min(d, j0 + slice_rows);
    const int64_t sl = j1 - j0;
    for (int64_t e = threadIdx.x; e < sl * d; e += blockDim.x) S[e] = 0.f;
    __syncthreads();
    const int64_t i_begin = (int64_t)blockIdx.x * rows_per;
    const int64_t i_end = min(n, i_begin + rows_per);
    bool bad = false;
    for (int64_t i = i_begin + threadIdx.x; i < i_end; i += blockDim.x) {
        const int64_t k0 = I[i], k1 = I[i + 1];
        if (k0 < 0 || k1 < k0 || k1 > nnz) {
            bad = true;
            continue;
        }
        for (int64_t pp = k0; pp < k1; ++pp) {
            const int32_t jp = __ldg(J + pp);
            if (jp < 0 || jp >= d) {
                bad = true;
                continue;
            }
            const float vp = __ldg(V + pp);
            for (int64_t qq = pp; qq < k1; ++qq) {
                const int32_t jq = __ldg(J + qq);
                if (jq < 0 || jq >= d) continue;
                const int32_t a = jp < jq ? jp : jq, b = jp < jq ? jq : jp;
                if (a < j0 || a >= j1) continue;
                const float w = vp * __ldg(V + qq);
                atomicAdd(&S[(a - j0) * d + b], (qq != pp && jp == jq) ? 2.f * w : w);
            }
        }
    }
    if (bad) set_flag(flag, LSK_FLAG_BAD_CSR);
    __syncthreads();
    float* P = part + (int64_t)blockIdx.x * d * d + j0 * d;
    for (int64_t e = threadIdx.x; e < sl * d; e += blockDim.x) P[e] = S[e];
}

// C[a][b] = C[b][a] = alpha sum_z part[z][a][b] + beta C (a <= b): a block
// takes 32 consecutive entries; thread (g, x) adds the partials z = g, g + 8,
// ... of entry x in FP64, then the 8 group sums are added in order
// (deterministic).
template <typename OutT>
__global__ void __launch_bounds__(256) gram_csr_reduce_kernel(const float* __restrict__ part, int64_t nblocks,
                                                               int64_t d, double alpha, double beta,
                                                               OutT* __restrict__ C) {
    __shared__ double acc[8][33];
    const int x = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int64_t len = d * d;
    const int64_t e = (int64_t)blockIdx.x * 32 + x;
    const int64_t a = e / d, b = e % d;
    const bool upper = e < len && a <= b;
    double s = 0.0;
    if (upper) {
        int64_t z = g;
        for (; z + 24 < nblocks; z += 32) {   // four loads in flight
            const float x0 = part[z * len + e], x1 = part[(z + 8) * len + e];
            const float x2 = part[(z + 16) * len + e], x3 = part[(z + 24) * len + e];
            s += (double)x0;
            s += (double)x1;
            s += (double)x2;
            s += (double)x3;
        }
        for (; z < nblocks; z += 8) s += (double)part[z * len + e];
    }
    acc[g][x] = s;
    __syncthreads();
    if (g == 0 && upper) {
        double t = 0.0;
        for (int k = 0; k < 8; ++k) t += acc[k][x];
        const double ab = alpha * t;
        C[a * d + b] = (OutT)(beta != 0.0 ? ab + beta * (double)C[a * d + b] : ab);
        if (a != b) C[b * d + a] = (OutT)(beta != 0.0 ? ab + beta * (double)C[b * d + a] : ab);
    }
}

struct DensePlan {
    int ntiles;
    int64_t nchunks, rows_per;
};
DensePlan dense_plan(int64_t n, int64_t d, int sm_count) {
    DensePlan p;
    const int nt = (int)((d + GT - 1) / GT);
    p.ntiles = nt * (nt + 1) / 2;
    int64_t want = (4 * (int64_t)sm_count + p.ntiles - 1) / p.ntiles;
    int64_t rows = (n + want - 1) / want;
    rows = ((rows + GK - 1) / GK) * GK;
    if (rows < GK) rows = GK;
    p.rows_per = rows;
    p.nchunks = (n + rows - 1) / rows;
    if (p.nchunks < 1) p.nchunks = 1;
    return p;
}

struct CsrPlan {
    int64_t slice_rows, nslices, nblocks, rows_per;
    size_t smem;
};
CsrPlan csr_plan(int64_t n, int64_t d, int sm_count) {
    CsrPlan p;
    const int64_t max_floats = 48 * 1024;  // 192 KB of shared memory
    p.slice_rows = max_floats / d;
    if (p.slice_rows > d) p.slice_rows = d;
    if (p.slice_rows < 1) p.slice_rows = 1;
    p.nslices = (d + p.slice_rows - 1) / p.slice_rows;
    // one 1024-thread block per SM
    int64_t nb = ((int64_t)sm_count + p.nslices - 1) / p.nslices;
    if (nb < 1) nb = 1;
    p.rows_per = (n + nb - 1) / nb;
    if (p.rows_per < 1) p.rows_per = 1;
    p.nblocks = (n + p.rows_per - 1) / p.rows_per;
    if (p.nblocks < 1) p.nblocks = 1;
    p.smem = (size_t)p.slice_rows * d * 4;
    return p;
}

}  // namespace

size_t gram_workspace_bytes(const lsk_mat* A, int sm_count) {
    if (A->kind == LSK_DENSE) {
        const DensePlan p = dense_plan(A->n, A->d, sm_count);
        return ws_round((size_t)p.nchunks * p.ntiles * GT * GT * 8);
    }
    const CsrPlan p = csr_plan(A->n, A->d, sm_count);
    return ws_round((size_t)p.nblocks * A->d * A->d * 4);
}

template <typename OutT>
cudaError_t gram_launch_t(const lsk_mat* A, double alpha, double beta, OutT* C, void* ws, int* flag,
                          int sm_count, cudaStream_t st) {
    const int64_t n = A->n, d = A->d;
    const int64_t len = d * d;
    if (A->kind == LSK_DENSE) {
        const DensePlan p = dense_plan(n, d, sm_count);
        double* part = (double*)ws;
        dim3 grid((unsigned)p.ntiles, (unsigned)p.nchunks);
        LSK_PROF("gram_dense", st) gram_dense_kernel<<<grid, 256, 0, st>>>((const float*)A->values, A->ld, n, d, p.rows_per, part);
        LSK_PROF("gram_reduce", st) gram_dense_reduce_kernel<OutT>
            <<<(unsigned)((len + 31) / 32), 256, 0, st>>>(part, p.nchunks, d, alpha, beta, C);
    } else {
        const CsrPlan p = csr_plan(n, d, sm_count);
        if (p.smem > 48 * 1024) {
            cudaError_t e = allow_dynamic_smem(gram_csr_kernel);
            if (e != cudaSuccess) return e;
        }
        float* part = (float*)ws;
        dim3 grid((unsigned)p.nblocks, (unsigned)p.nslices);
        LSK_PROF("gram_csr", st) gram_csr_kernel<<<grid, 1024, p.smem, st>>>((const float*)A->values, A->colidx,
                                                                            A->rowptr, n, A->nnz, d, p.slice_rows,
                                                                            p.rows_per, part, flag);
        LSK_PROF("gram_reduce", st) gram_csr_reduce_kernel<OutT>
            <<<(unsigned)((len + 31) / 32), 256, 0, st>>>(part, p.nblocks, d, alpha, beta, C);
    }
    return cudaGetLastError();
}

cudaError_t gram_launch(const lsk_mat* A, double alpha, double beta, float* C, void* ws, int* flag,
                        int sm_count, cudaStream_t st) {
    return gram_launch_t<float>(A, alpha, beta, C, ws, flag, sm_count, st);
}

cudaError_t gram64_launch(const lsk_mat* A, double* C, void* ws, int* flag, int sm_count, cudaStream_t st) {
    return gram_launch_t<double>(A, 1.0, 0.0, C, ws, flag, sm_count, st);
}
