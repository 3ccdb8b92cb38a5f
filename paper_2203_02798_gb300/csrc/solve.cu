// solve.cu -- sketch-and-solve least squares (Alg. 11).
//
// (A~ b~) = G S (A b) (k > 0) or S (A b) (k = 0): A~ is the sketch of A that
// the leverage / preconditioning path already forms (CountSketch + Gaussian
// stage), and b~ applies the same S (same hash) and the same G (same draws,
// bf16-rounded in the BF16 mode) to b, accumulated in FP64.  Then x minimises
// ||A~ x - b~||: with R (A~ = Q R, FP64 accurate) x = R^-1 R^-T A~^T b~, the
// seminormal equations, followed by one corrected step
// x += R^-1 R^-T A~^T (b~ - A~ x), which brings the error to that of a QR
// solve (Bjorck, BIT 27 (1987)).  The paper's SVD (Alg. 11 step 2) gives the
// same minimiser when A~ has full rank, which the factorisation checks.
#include "lsk_internal.cuh"

namespace {

constexpr int kColsPerBlock = 512;   // columns of G per partial of G (S b)
constexpr int kRowsPerPart = 2048;   // rows of A~ per partial of A~^T v

unsigned grid_for(int64_t items, int threads, int sm_count) {
    const int64_t g = (items + threads - 1) / threads;
    const int64_t cap = (int64_t)sm_count * 8;
    return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

// S b: row i adds sign_i b_i into bucket h(i) (FP64 atomics)
__global__ void cs_vec_kernel(int64_t n, uint32_t r, uint32_t k0, uint32_t k1, const double* __restrict__ b,
                              double* __restrict__ Sb) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        uint32_t bucket, neg;
        cs_hash((uint64_t)i, r, k0, k1, bucket, neg);
        atomicAdd(Sb + bucket, neg ? -b[i] : b[i]);
    }
}

// part[blk][j] = sum over the block's columns c of G[j, c] (S b)[c]; thread per
// row quad of G, the draws exactly those of the Gaussian stage
__global__ void gauss_vec_kernel(const double* __restrict__ Sb, int64_t r, int k, uint32_t k0, uint32_t k1,
                                 float scale, int bf16, double* __restrict__ part) {
    const int64_t c0 = (int64_t)blockIdx.x * kColsPerBlock;
    const int64_t c1 = c0 + kColsPerBlock < r ? c0 + kColsPerBlock : r;
    const int nq = (k + 3) / 4;
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        for (int64_t c = c0; c < c1; ++c) {
            const double s = Sb[c];
            if (s == 0.0) continue;
            const float4 z = gauss4((uint64_t)c, (uint32_t)q, k0, k1);
            float g[4] = {z.x * scale, z.y * scale, z.z * scale, z.w * scale};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (bf16) g[e] = bf16_round(g[e]);
                acc[e] = fma((double)g[e], s, acc[e]);
            }
        }
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (4 * q + e < k) part[(int64_t)blockIdx.x * k + 4 * q + e] = acc[e];
    }
}

// out[j] = sum over blocks of part[blk][j], in block order
__global__ void sum_parts_kernel(const double* __restrict__ part, int nblk, int len, double* __restrict__ out) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < len; j += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * len + j];
        out[j] = s;
    }
}

// part[blk][j] = sum over the block's rows i of At[i][j] v[i]
__global__ void atv_kernel(const float* __restrict__ At, int64_t rows, int d, const double* __restrict__ v,
                           double* __restrict__ part) {
    const int64_t i0 = (int64_t)blockIdx.x * kRowsPerPart;
    const int64_t i1 = i0 + kRowsPerPart < rows ? i0 + kRowsPerPart : rows;
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        double s = 0.0;
        for (int64_t i = i0; i < i1; ++i) s = fma((double)At[i * d + j], v[i], s);
        part[(int64_t)blockIdx.x * d + j] = s;
    }
}

// res[i] = bt[i] - At[i] x
__global__ void residual_kernel(const float* __restrict__ At, int64_t rows, int d, const double* __restrict__ bt,
                                const double* __restrict__ x, double* __restrict__ res) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += stride) {
        double s = bt[i];
        for (int j = 0; j < d; ++j) s = fma(-(double)At[i * d + j], x[j], s);
        res[i] = s;
    }
}

// x (+)= R^-1 R^-T c: y = R^-T c, then R^-1 y (one block; d <= 1024)
__global__ void __launch_bounds__(1024) seminormal_kernel(const double* __restrict__ c, const double* __restrict__ Rinv,
                                                          int d, int add, double* __restrict__ x) {
    __shared__ double cs[1024], ys[1024];
    for (int j = threadIdx.x; j < d; j += blockDim.x) cs[j] = c[j];
    __syncthreads();
    for (int i = threadIdx.x; i < d; i += blockDim.x) {
        double s = 0.0;
        for (int j = 0; j <= i; ++j) s = fma(Rinv[(int64_t)j * d + i], cs[j], s);
        ys[i] = s;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        double s = 0.0;
        for (int i = j; i < d; ++i) s = fma(Rinv[(int64_t)j * d + i], ys[i], s);
        x[j] = add ? x[j] + s : s;
    }
}

}  // namespace

cudaError_t seminormal_launch(const double* c, const double* Rinv64, int64_t d, int add, double* x, cudaStream_t st) {
    if (d > 1024) return cudaErrorInvalidValue;
    LSK_PROF("solve_small", st) seminormal_kernel<<<1, 1024, 0, st>>>(c, Rinv64, (int)d, add, x);
    return cudaGetLastError();
}

size_t solve_workspace_bytes(int64_t r, int64_t k, int64_t d) {
    const int64_t rows = k > 0 ? k : r;
    const int64_t gblk = (r + kColsPerBlock - 1) / kColsPerBlock;
    const int64_t ablk = (rows + kRowsPerPart - 1) / kRowsPerPart;
    return ws_round((size_t)r * 8) + ws_round((size_t)(k > 0 ? gblk * k : 1) * 8) + ws_round((size_t)rows * 8) * 2 +
           ws_round((size_t)ablk * d * 8) + ws_round((size_t)d * 8) + 4096;
}

cudaError_t solve_launch(const lsk_mat* A, const double* b, int64_t r, int64_t k, uint64_t seed, int32_t prec,
                         const float* At, const double* Rinv64, double* x, void* ws, int sm_count, cudaStream_t st) {
    const int64_t n = A->n, d = A->d, rows = k > 0 ? k : r;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const int64_t gblk = (r + kColsPerBlock - 1) / kColsPerBlock;
    const int64_t ablk = (rows + kRowsPerPart - 1) / kRowsPerPart;
    WsCarver wc{(char*)ws, 0};
    double* Sb = wc.take<double>(r);
    double* gpart = wc.take<double>(k > 0 ? gblk * k : 1);
    double* bt = wc.take<double>(rows);
    double* res = wc.take<double>(rows);
    double* apart = wc.take<double>(ablk * d);
    double* c = wc.take<double>(d);
    cudaError_t e = cudaMemsetAsync(Sb, 0, (size_t)r * 8, st);
    if (e != cudaSuccess) return e;
    if (n > 0)
        LSK_PROF("solve_sketch_b", st) cs_vec_kernel<<<grid_for(n, 256, sm_count), 256, 0, st>>>(n, (uint32_t)r, k0, k1, b, Sb);
    if (k > 0) {
        const float scale = (float)(1.0 / sqrt((double)k));
        LSK_PROF("solve_gauss_b", st) gauss_vec_kernel<<<(unsigned)gblk, 128, 0, st>>>(
            Sb, r, (int)k, k0, k1, scale, prec == LSK_PREC_BF16 ? 1 : 0, gpart);
        LSK_PROF("solve_small", st) sum_parts_kernel<<<(unsigned)((k + 255) / 256), 256, 0, st>>>(gpart, (int)gblk, (int)k, bt);
    } else {
        e = cudaMemcpyAsync(bt, Sb, (size_t)r * 8, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
    }
    // x = R^-1 R^-T A~^T b~, then one corrected step on the residual
    for (int step = 0; step < 2; ++step) {
        const double* v = bt;
        if (step == 1) {
            LSK_PROF("solve_small", st) residual_kernel<<<grid_for(rows, 256, sm_count), 256, 0, st>>>(At, rows, (int)d, bt, x, res);
            v = res;
        }
        LSK_PROF("solve_atv", st) atv_kernel<<<(unsigned)ablk, 256, 0, st>>>(At, rows, (int)d, v, apart);
        LSK_PROF("solve_small", st) sum_parts_kernel<<<(unsigned)((d + 255) / 256), 256, 0, st>>>(apart, (int)ablk, (int)d, c);
        LSK_PROF("solve_small", st) seminormal_kernel<<<1, 1024, 0, st>>>(c, Rinv64, (int)d, step, x);
    }
    return cudaGetLastError();
}
