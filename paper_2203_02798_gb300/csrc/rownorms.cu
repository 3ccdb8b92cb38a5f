// rownorms.cu -- x <- alpha * diag(A B B^T A^T) + beta * x (csrsqn / rmsqn).
//
// dense (rmsqn): a block owns 128 rows of A and sweeps the columns of B in
//   tiles of 64; each product tile A_blk * B_tile stays in registers, is
//   squared and summed into per-row partials, so A*B never exists outside
//   registers (the memory-efficient form of Alg. 8 for dense A).  When B is
//   upper triangular (B = R^-1) the k-loop of column tile [c0, c0+64) stops
//   at c0+64, skipping the zero blocks.  This is the CUDA-core (SIMT) path
//   (LSK_PREC_FP32); the tensor-core path lives in rownorms_tc.cu.
// CSR (csrsqn, Alg. 8): Btilde = B B^T is formed once (FP32, 16 x 16 output
//   tiles); then one thread per row evaluates
//   sum_{p,q in row} v_p v_q Btilde[J_p, J_q] using the symmetry of Btilde.
#include "lsk_internal.cuh"

namespace {

constexpr int RM = 128;   // rows of A per block
constexpr int RN = 64;    // columns of B per tile
constexpr int RK = 16;    // reduction step
constexpr int RMP = RM + 4;

// thread (ty, tx) = (tid / 16, tid % 16): rows 8*ty..8*ty+7, cols 4*tx..4*tx+3
__global__ void __launch_bounds__(256) rownorm_dense_kernel(
    const float* __restrict__ A, int64_t lda, int64_t n, int64_t d, const float* __restrict__ B,
    int64_t c, int upper_tri, float alpha, float beta, float* __restrict__ x) {
    __shared__ __align__(16) float As[RK][RMP];
    __shared__ __align__(16) float Bs[RK][RN];
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const int64_t i0 = (int64_t)blockIdx.x * RM;
    float rowsum[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) rowsum[a] = 0.f;

    for (int64_t c0 = 0; c0 < c; c0 += RN) {
        const int64_t kmax = upper_tri ? min(d, c0 + RN) : d;
        float acc[8][4];
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
        for (int64_t k0 = 0; k0 < kmax; k0 += RK) {
#pragma unroll
            for (int t = 0; t < (RM * RK) / 256; ++t) {
                const int idx = tid + 256 * t;
                const int row = idx / RK, kk = idx % RK;
                const int64_t i = i0 + row, kx = k0 + kk;
                As[kk][row] = (i < n && kx < kmax) ? __ldg(A + i * lda + kx) : 0.f;
            }
#pragma unroll
            for (int t = 0; t < (RK * RN) / 256; ++t) {
                const int idx = tid + 256 * t;
                const int kk = idx / RN, cc = idx % RN;
                const int64_t kx = k0 + kk, cx = c0 + cc;
                Bs[kk][cc] = (kx < kmax && cx < c) ? __ldg(B + kx * c + cx) : 0.f;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < RK; ++kk) {
                const float4 a0 = *reinterpret_cast<const float4*>(&As[kk][8 * ty]);
                const float4 a1 = *reinterpret_cast<const float4*>(&As[kk][8 * ty + 4]);
                const float4 bv = *reinterpret_cast<const float4*>(&Bs[kk][4 * tx]);
                const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float bb[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
                for (int a = 0; a < 8; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(av[a], bb[b], acc[a][b]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) rowsum[a] = fmaf(acc[a][b], acc[a][b], rowsum[a]);
    }
    // the 16 threads of a half-warp share rows: reduce across tx
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        float v = rowsum[a];
#pragma unroll
        for (int o = 8; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        rowsum[a] = v;
    }
    if (tx == 0) {
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const int64_t i = i0 + 8 * ty + a;
            if (i < n) x[i] = (beta != 0.f) ? fmaf(alpha, rowsum[a], beta * x[i]) : alpha * rowsum[a];
        }
    }
}

// Btilde[a][b] = sum_j B[a][j] B[b][j], FP32, 16 x 16 output tiles (one
// output per thread, two accumulation chains).
__device__ __forceinline__ void bbt_body(const float* __restrict__ B, int64_t d, int64_t c, float* __restrict__ M,
                                         int64_t a0, int64_t b0) {
    __shared__ float Ba[16][17], Bb[16][17];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc0 = 0.f, acc1 = 0.f;
    for (int64_t j0 = 0; j0 < c; j0 += 16) {
        const int64_t ja = j0 + tx;
        Ba[ty][tx] = (a0 + ty < d && ja < c) ? __ldg(B + (a0 + ty) * c + ja) : 0.f;
        Bb[ty][tx] = (b0 + ty < d && ja < c) ? __ldg(B + (b0 + ty) * c + ja) : 0.f;
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 16; j += 2) {
            acc0 = fmaf(Ba[ty][j], Bb[tx][j], acc0);
            acc1 = fmaf(Ba[ty][j + 1], Bb[tx][j + 1], acc1);
        }
        __syncthreads();
    }
    if (a0 + ty < d && b0 + tx < d) M[(a0 + ty) * d + b0 + tx] = acc0 + acc1;
}
__global__ void __launch_bounds__(256) bbt_kernel(const float* __restrict__ B, int64_t d, int64_t c,
                                                  float* __restrict__ M) {
    bbt_body(B, d, c, M, (int64_t)blockIdx.y * 16, (int64_t)blockIdx.x * 16);
}
// B B^T of many problems in one launch: problem g's 16 x 16 tiles are blocks
// off[g] .. off[g + 1] - 1, row-major over the tile grid
__global__ void __launch_bounds__(256) bbt_grouped_kernel(const BbtJob* __restrict__ jobs, const int* __restrict__ off,
                                                          int count) {
    const int g = group_of(off, count, blockIdx.x);
    const BbtJob& j = jobs[g];
    const int64_t tiles = (j.d + 15) / 16, t = (int64_t)blockIdx.x - __ldg(off + g);
    bbt_body(j.B, j.d, j.c, j.M, (t / tiles) * 16, (t % tiles) * 16);
}

__global__ void rownorm_csr_kernel(const float* __restrict__ V, const int32_t* __restrict__ J,
                                   const int64_t* __restrict__ I, int64_t n, int64_t nnz, int64_t d,
                                   const float* __restrict__ M, float alpha, float beta,
                                   float* __restrict__ x, int* flag) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int64_t k0 = I[i], k1 = I[i + 1];
        float q = 0.f;
        if (k0 < 0 || k1 < k0 || k1 > nnz) {
            bad = true;
        } else {
            for (int64_t p = k0; p < k1; ++p) {
                const int32_t jp = __ldg(J + p);
                if (jp < 0 || jp >= d) {
                    bad = true;
                    continue;
                }
                const float vp = __ldg(V + p);
                const float* Mrow = M + (int64_t)jp * d;
                float s = vp * __ldg(Mrow + jp);  // diagonal term once
                for (int64_t t = p + 1; t < k1; ++t) {
                    const int32_t jt = __ldg(J + t);
                    if (jt < 0 || jt >= d) continue;
                    s = fmaf(2.0f * __ldg(V + t), __ldg(Mrow + jt), s);
                }
                q = fmaf(vp, s, q);
            }
        }
        x[i] = (beta != 0.f) ? fmaf(alpha, q, beta * x[i]) : alpha * q;
    }
    if (bad) set_flag(flag, LSK_FLAG_BAD_CSR);
}

}  // namespace

size_t rownorms_workspace_bytes(const lsk_mat* A, int64_t c, int upper_tri, int32_t prec) {
    if (A->kind == LSK_DENSE) {
        // the BF16x3 and TF32 images have the same size
        if ((prec == LSK_PREC_BF16 || prec == LSK_PREC_TF32) &&
            (rownorms_tc_supported(A, c, upper_tri) || rownorms_tc_supported(A, c, upper_tri, true)))
            return rownorms_tc_workspace_bytes(A, c, upper_tri);
        return 0;
    }
    return ws_round((size_t)A->d * A->d * 4);
}

cudaError_t rownorms_launch(const lsk_mat* A, const float* B, int64_t c, double alpha, double beta,
                            int upper_tri, int32_t prec, float* x, void* ws, int* flag, int sm_count,
                            cudaStream_t st, int min_tiles, const void* prepared) {
    const int64_t n = A->n, d = A->d;
    if (n == 0) return cudaSuccess;
    // TF32: the one-product TF32 kernel where A suits TMA, else BF16x3 (more
    // accurate), else FP32 on the CUDA cores (an operand prepared by a grouped
    // launch is a BF16x3 image)
    if (A->kind == LSK_DENSE && prec == LSK_PREC_TF32 && !prepared && rownorms_tc_supported(A, c, upper_tri, true))
        return rownorms_tc_launch(A, B, c, (float)alpha, (float)beta, upper_tri, x, ws, flag, sm_count, st,
                                  min_tiles, nullptr, true);
    if (A->kind == LSK_DENSE && (prec == LSK_PREC_BF16 || prec == LSK_PREC_TF32) &&
        rownorms_tc_supported(A, c, upper_tri))
        return rownorms_tc_launch(A, B, c, (float)alpha, (float)beta, upper_tri, x, ws, flag, sm_count, st,
                                  min_tiles, (const uint8_t*)prepared);
    if (A->kind == LSK_DENSE) {
        const unsigned grid = (unsigned)((n + RM - 1) / RM);
        LSK_PROF("rownorm_dense_simt", st) rownorm_dense_kernel<<<grid, 256, 0, st>>>((const float*)A->values, A->ld, n, d, B, c,
                                                   upper_tri ? 1 : 0, (float)alpha, (float)beta, x);
    } else {
        float* M = prepared ? (float*)prepared : (float*)ws;   // prepared: built by bbt_group_launch
        const dim3 bg((unsigned)((d + 15) / 16), (unsigned)((d + 15) / 16));
        if (!prepared) LSK_PROF("rownorm_bbt", st) bbt_kernel<<<bg, 256, 0, st>>>(B, d, c, M);
        int64_t gr = (n + 255) / 256;
        if (gr > 16 * (int64_t)sm_count) gr = 16 * (int64_t)sm_count;
        LSK_PROF("rownorm_csr", st) rownorm_csr_kernel<<<(unsigned)gr, 256, 0, st>>>((const float*)A->values, A->colidx, A->rowptr,
                                                         n, A->nnz, d, M, (float)alpha, (float)beta, x,
                                                         flag);
    }
    return cudaGetLastError();
}

void bbt_group_build(const std::vector<BbtJob>& jobs, HostTable& t, BbtGroup& g) {
    std::vector<int> blocks, off;
    for (const BbtJob& j : jobs) {
        const int tiles = (int)((j.d + 15) / 16);
        blocks.push_back(tiles * tiles);
    }
    g.count = (int)jobs.size();
    g.blocks = group_offsets(blocks, off);
    g.params_off = t.put(jobs.data(), jobs.size());
    g.off_off = t.put(off.data(), off.size());
}

cudaError_t bbt_group_launch(const BbtGroup& g, const unsigned char* table, cudaStream_t st) {
    if (g.count == 0) return cudaSuccess;
    LSK_PROF("rownorm_bbt", st) bbt_grouped_kernel<<<g.blocks, 256, 0, st>>>(
        reinterpret_cast<const BbtJob*>(table + g.params_off), reinterpret_cast<const int*>(table + g.off_off),
        g.count);
    return cudaGetLastError();
}
