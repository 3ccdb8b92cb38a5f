// gauss.cu -- the Gaussian stage of CountGauss, GSA = G * SA (Alg. 3).
//
// G (k x r) is never stored: every tile of G is regenerated in registers
// from Philox + Box-Muller (the spec in lsk.h) right before it is used,
// which is the memory-free form of Alg. 3's "set new i.i.d. elements in G"
// batch loop.  The r dimension (the reduction of the product) is split
// across thread blocks; each block writes a k x d partial and a final pass
// adds the partials in a fixed order in FP64, so the result is
// deterministic.
//
// This file holds the CUDA-core (SIMT) path used for LSK_PREC_FP32; the
// BF16 tensor-core path lives in gauss_tc.cu.
#include "lsk_internal.cuh"

namespace {

constexpr int BM = 64;    // rows of G per block
constexpr int BN = 128;   // columns of SA per block
constexpr int BK = 16;    // reduction step

// Thread (ty, tx) = (tid / 16, tid % 16) owns rows 4*ty..4*ty+3 and columns
// {4*tx..4*tx+3} U {64+4*tx..64+4*tx+3} of the block tile.
__global__ void __launch_bounds__(256, 2) gauss_simt_kernel(
    const float* __restrict__ SA, int64_t r, int64_t d, int64_t k, uint32_t k0, uint32_t k1,
    float scale, int bf16, int64_t kc, float* __restrict__ part) {
    __shared__ __align__(16) float Gs[BK][BM];
    __shared__ __align__(16) float Ss[BK][BN];
    const int tid = threadIdx.x;
    const int ty = tid >> 4, tx = tid & 15;
    const int64_t n0 = (int64_t)blockIdx.x * BN;
    const int64_t j0 = (int64_t)blockIdx.y * BM;
    const int64_t c_begin = (int64_t)blockIdx.z * kc;
    const int64_t c_end = min(r, c_begin + kc);

    float acc[4][8];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;

    // generator assignment: thread -> (column cl of the K step, row quad ql)
    const int gl_c = tid >> 4;   // 0..15
    const int gl_q = tid & 15;   // rows 4*gl_q .. 4*gl_q+3 of the tile

    // the SA tile of the next step is loaded into registers while the current
    // one is multiplied (thread: elements tid + 256 t of the BK x BN tile)
    float sa[(BK * BN) / 256];
    const auto load_sa = [&](int64_t c0) {
#pragma unroll
        for (int t = 0; t < (BK * BN) / 256; ++t) {
            const int idx = tid + 256 * t;
            const int kr = idx / BN, cc = idx % BN;
            const int64_t c = c0 + kr, n = n0 + cc;
            sa[t] = (c < c_end && n < d) ? __ldg(SA + c * d + n) : 0.f;
        }
    };
    if (c_begin < c_end) load_sa(c_begin);
    for (int64_t c0 = c_begin; c0 < c_end; c0 += BK) {
        {   // G tile (transposed: Gs[c][j])
            const int64_t c = c0 + gl_c;
            const int64_t jq = j0 + 4 * gl_q;
            float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
            if (c < c_end && jq < k) {
                g = gauss4((uint64_t)c, (uint32_t)(jq >> 2), k0, k1);
                g.x *= scale;
                g.y *= scale;
                g.z *= scale;
                g.w *= scale;
                if (bf16) {
                    g.x = bf16_round(g.x);
                    g.y = bf16_round(g.y);
                    g.z = bf16_round(g.z);
                    g.w = bf16_round(g.w);
                }
                if (jq + 1 >= k) g.y = 0.f;
                if (jq + 2 >= k) g.z = 0.f;
                if (jq + 3 >= k) g.w = 0.f;
            }
            *reinterpret_cast<float4*>(&Gs[gl_c][4 * gl_q]) = g;
        }
#pragma unroll
        for (int t = 0; t < (BK * BN) / 256; ++t) {  // SA tile
            const int idx = tid + 256 * t;
            Ss[idx / BN][idx % BN] = sa[t];
        }
        __syncthreads();
        if (c0 + BK < c_end) load_sa(c0 + BK);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            const float4 gv = *reinterpret_cast<const float4*>(&Gs[kk][4 * ty]);
            const float4 s0 = *reinterpret_cast<const float4*>(&Ss[kk][4 * tx]);
            const float4 s1 = *reinterpret_cast<const float4*>(&Ss[kk][64 + 4 * tx]);
            const float g[4] = {gv.x, gv.y, gv.z, gv.w};
            const float s[8] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(g[a], s[b], acc[a][b]);
        }
        __syncthreads();
    }
    float* P = part + (int64_t)blockIdx.z * k * d;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int64_t j = j0 + 4 * ty + a;
        if (j >= k) continue;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const int64_t n = n0 + (b < 4 ? 4 * tx + b : 64 + 4 * tx + (b - 4));
            if (n < d) P[j * d + n] = acc[a][b];
        }
    }
}

// GSA[e] = sum_z part[z][e] in FP64, in increasing z.
__global__ void reduce_partials_kernel(const float* __restrict__ part, int64_t nz, int64_t len,
                                       float* __restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += stride) {
        double s = 0.0;
        for (int64_t z = 0; z < nz; ++z) s += (double)part[z * len + e];
        out[e] = (float)s;
    }
}

__global__ void gauss_debug_kernel(int64_t k, int64_t r, uint32_t k0, uint32_t k1, float scale,
                                   int bf16, float* __restrict__ G) {
    const int64_t nq = (k + 3) / 4;
    const int64_t total = nq * r;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
        const int64_t q = t / r, c = t % r;
        float4 g = gauss4((uint64_t)c, (uint32_t)q, k0, k1);
        float v[4] = {g.x * scale, g.y * scale, g.z * scale, g.w * scale};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t j = 4 * q + u;
            if (j < k) G[j * r + c] = bf16 ? bf16_round(v[u]) : v[u];
        }
    }
}

struct Plan {
    int64_t tiles_n, tiles_m, nz, kc;
};

Plan make_plan(int64_t r, int64_t d, int64_t k, int sm_count) {
    Plan p;
    p.tiles_n = (d + BN - 1) / BN;
    p.tiles_m = (k + BM - 1) / BM;
    const int64_t tiles = p.tiles_n * p.tiles_m;
    // r-slices so that the grid fills whole waves of 2 blocks per SM (a
    // partial last wave costs a whole block time), at least 128 columns each
    int64_t want = 2 * (int64_t)sm_count / tiles;
    if (want > (r + 127) / 128) want = (r + 127) / 128;
    if (want < 1) want = 1;
    int64_t kc = (r + want - 1) / want;
    kc = ((kc + BK - 1) / BK) * BK;
    if (kc < BK) kc = BK;
    p.kc = kc;
    p.nz = (r + kc - 1) / kc;
    return p;
}

}  // namespace

cudaError_t gauss_tc_launch(const float* SA, int64_t r, int64_t d, int64_t k, uint64_t seed,
                            float* GSA, void* ws, int sm_count, cudaStream_t st, int terms);
size_t gauss_tc_workspace_bytes(int64_t r, int64_t d, int64_t k, int sm_count, int terms);

// The FP32 mode (and TF32, which runs as FP32) on the tensor cores -- G and
// SA as three bf16 terms each -- where the shape fits and the sketch is long
// enough for its slices to fill the GPU; the SIMT tiles otherwise.
bool fp32_on_tensor_cores(int64_t r, int64_t d, int64_t k, int32_t prec) {
    return (prec == LSK_PREC_FP32 || prec == LSK_PREC_TF32) && r >= 8192 && gauss_tc_supported(r, d, k, 3);
}

size_t gauss_workspace_bytes(int64_t r, int64_t d, int64_t k, int32_t prec, int sm_count) {
    if (prec == LSK_PREC_BF16 && gauss_tc_supported(r, d, k))
        return gauss_tc_workspace_bytes(r, d, k, sm_count, 1);
    if (fp32_on_tensor_cores(r, d, k, prec)) return gauss_tc_workspace_bytes(r, d, k, sm_count, 3);
    const Plan p = make_plan(r, d, k, sm_count);
    return ws_round((size_t)p.nz * k * d * 4);
}

cudaError_t gauss_launch(const float* SA, int64_t r, int64_t d, int64_t k, uint64_t seed,
                         int32_t prec, float* GSA, void* ws, int sm_count, cudaStream_t st) {
    if (prec == LSK_PREC_BF16 && gauss_tc_supported(r, d, k))
        return gauss_tc_launch(SA, r, d, k, seed, GSA, ws, sm_count, st, 1);
    if (fp32_on_tensor_cores(r, d, k, prec)) return gauss_tc_launch(SA, r, d, k, seed, GSA, ws, sm_count, st, 3);
    const Plan p = make_plan(r, d, k, sm_count);
    const float scale = (float)(1.0 / sqrt((double)k));
    dim3 grid((unsigned)p.tiles_n, (unsigned)p.tiles_m, (unsigned)p.nz);
    float* part = (float*)ws;
    LSK_PROF("gauss_simt", st) gauss_simt_kernel<<<grid, 256, 0, st>>>(SA, r, d, k, (uint32_t)seed, (uint32_t)(seed >> 32),
                                            scale, prec == LSK_PREC_BF16 ? 1 : 0, p.kc, part);
    const int64_t len = k * d;
    int64_t g = (len + 255) / 256;
    if (g > 8 * (int64_t)sm_count) g = 8 * (int64_t)sm_count;
    LSK_PROF("gauss_reduce", st) reduce_partials_kernel<<<(unsigned)g, 256, 0, st>>>(part, p.nz, len, GSA);
    return cudaGetLastError();
}

cudaError_t gauss_debug_launch(int64_t k, int64_t r, uint64_t seed, int32_t prec, float* G,
                               cudaStream_t st) {
    const float scale = (float)(1.0 / sqrt((double)k));
    const int64_t total = ((k + 3) / 4) * r;
    int64_t g = (total + 255) / 256;
    if (g > 4096) g = 4096;
    gauss_debug_kernel<<<(unsigned)g, 256, 0, st>>>(k, r, (uint32_t)seed, (uint32_t)(seed >> 32),
                                                   scale, prec == LSK_PREC_BF16 ? 1 : 0, G);
    return cudaGetLastError();
}

// dst[i] += src[i] (the sum of the partial sketches of row blocks)
namespace {
__global__ void add_into_kernel(float* __restrict__ dst, const float* __restrict__ src, int64_t len) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] += src[i];
}
}  // namespace
cudaError_t add_into_launch(float* dst, const float* src, int64_t len, cudaStream_t st) {
    if (len <= 0) return cudaSuccess;
    const int64_t g = (len + 255) / 256 < 1024 ? (len + 255) / 256 : 1024;
    LSK_PROF("sketch_add", st) add_into_kernel<<<(unsigned)g, 256, 0, st>>>(dst, src, len);
    return cudaGetLastError();
}
