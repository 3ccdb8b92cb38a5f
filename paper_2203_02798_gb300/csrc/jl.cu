// jl.cu -- the right JL projection of Alg. 15: X = R^-1 Pi.
//
// Pi is d x m with entries z / sqrt(m), z drawn as the Gaussian entries of
// the Gaussian stage (Philox-4x32-10, 24-bit Box-Muller) on counter stream 2:
// Pi[i][c] is the entry (row c, column i) of that construction.  X = R^-1 Pi
// (R^-1 upper triangular, FP64) is formed in FP64 and stored in FP32 for the
// row-norm pass (Alg. 8), so the scores are ||A_i R^-1 Pi||^2.
#include "lsk_internal.cuh"

namespace {

// Pi (d x m, row-major): thread per (i, row quad cq) -> Pi[i][4 cq .. 4 cq + 3]
__global__ void jl_pi_kernel(int d, int m, uint32_t k0, uint32_t k1, float scale, float* __restrict__ Pi) {
    const int nq = (m + 3) / 4;
    const int64_t total = (int64_t)d * nq;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / nq), cq = (int)(t % nq);
        const float4 z = gauss4((uint64_t)i, (uint32_t)cq, k0, k1, 2u);
        const float v[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (4 * cq + e < m) Pi[(int64_t)i * m + 4 * cq + e] = v[e] * scale;
    }
}

// X[j][c] = sum_{i >= j} Rinv[j][i] Pi[i][c] (FP64), stored as FP32
__global__ void jl_x_kernel(const double* __restrict__ Rinv, const float* __restrict__ Pi, int d, int m,
                            float* __restrict__ X) {
    const int64_t total = (int64_t)d * m;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(t / m), c = (int)(t % m);
        double s = 0.0;
        for (int i = j; i < d; ++i) s = fma(Rinv[(int64_t)j * d + i], (double)Pi[(int64_t)i * m + c], s);
        X[t] = (float)s;
    }
}

}  // namespace

size_t jl_workspace_bytes(int64_t d, int64_t m) { return ws_round((size_t)d * m * 4); }

cudaError_t jl_launch(const double* Rinv64, int64_t d, int64_t m, uint64_t seed, float* X32, void* ws,
                      cudaStream_t st) {
    float* Pi = (float*)ws;
    const int64_t nq = (m + 3) / 4;
    const unsigned g1 = (unsigned)((d * nq + 255) / 256 < 4096 ? (d * nq + 255) / 256 : 4096);
    LSK_PROF("jl_pi", st) jl_pi_kernel<<<g1, 256, 0, st>>>((int)d, (int)m, (uint32_t)seed, (uint32_t)(seed >> 32),
                                                          (float)(1.0 / sqrt((double)m)), Pi);
    const unsigned g2 = (unsigned)((d * m + 255) / 256 < 4096 ? (d * m + 255) / 256 : 4096);
    LSK_PROF("jl_x", st) jl_x_kernel<<<g2, 256, 0, st>>>(Rinv64, Pi, (int)d, (int)m, X32);
    return cudaGetLastError();
}
