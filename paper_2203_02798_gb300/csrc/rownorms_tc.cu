// rownorms_tc.cu -- fused tensor-core row norms x_i = alpha ||A_i B||^2 + beta x_i.
//
// The memory-efficient dense form of Alg. 8 (rmsqn) on tcgen05: A*B is
// formed 128 rows at a time in tensor memory and squared / summed there, so
// it never reaches HBM.  Precision: A and B are split into bfloat16 pairs,
// x = hi + lo (about 16 significant bits), and
//     A B ~= A_hi B_hi + A_hi B_lo + A_lo B_hi     (FP32 accumulation),
// the dropped A_lo B_lo term being ~2^-18 relative.
//
// Persistent kernel, one CTA per SM (416 threads):
//   warps 0-3   epilogue: tcgen05.ld the accumulator rows, square, sum, store
//   warp  4     TMEM allocation; lane 0 issues every MMA and commit
//   warps 5-12  converters: stream A from HBM (two K-chunks of loads in
//               flight per thread), split into bf16 hi/lo and write the
//               128-byte-swizzled K-major operand tiles of the current stage
// B (hi and lo) stays resident in shared memory for the whole kernel; when
// B is upper triangular (B = R^-1) only the blocks on or above the diagonal
// are stored and multiplied: K-chunk q (rows 64q..64q+63 of B) only touches
// columns >= 64q.  TMEM holds two 128 x 256 FP32 accumulators so the
// epilogue of one tile overlaps the MMAs of the next.
#include "tc_common.cuh"

namespace {

constexpr int kRows = 128;
constexpr int kStages = 2;
constexpr int kConvWarps = 8;
constexpr int kEpiWarps = 4;
constexpr int kMmaWarp = 4;
constexpr int kConvWarp0 = 5;
constexpr int kThreads = (kEpiWarps + 1 + kConvWarps) * 32;
constexpr uint32_t kHalfStage = kRows * 128;        // one bf16 tile, 64 K-columns
constexpr uint32_t kStageBytes = 2 * kHalfStage;    // hi + lo
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kAccCols = 256;
constexpr size_t kSmemLimit = 232448;

struct RnParams {
    const float* A;
    int64_t lda;
    int64_t n;
    float* x;
    float alpha, beta;
    int d, c, nq, npad, ntiles;
    uint32_t n0[4], nn[4], boff[4];
    uint32_t b_bytes;
    int* flag;
};

// B (d x c, row-major) -> the shared-memory image of its bf16 hi / lo parts:
// per K-chunk q, an (nn[q] x 64) K-major tile whose row r is column n0[q]+r.
__global__ void rownorm_tc_prep_kernel(const float* __restrict__ B, const RnParams p, uint8_t* __restrict__ img) {
    uint32_t total = 0;
    for (int q = 0; q < p.nq; ++q) total += p.nn[q] * 32;
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        int q = 0;
        uint32_t el = e;
        while (el >= p.nn[q] * 32) {
            el -= p.nn[q] * 32;
            ++q;
        }
        const uint32_t r = el >> 5, kl = (el & 31) * 2;
        const int j = (int)(p.n0[q] + r), k = 64 * q + (int)kl;
        const float b0 = (k < p.d && j < p.c) ? B[(int64_t)k * p.c + j] : 0.f;
        const float b1 = (k + 1 < p.d && j < p.c) ? B[(int64_t)(k + 1) * p.c + j] : 0.f;
        uint32_t hi, lo;
        tc::split_bf16x2(b0, b1, hi, lo);
        const uint32_t off = p.boff[q] + tc::sw128_offset(r, kl);
        *reinterpret_cast<uint32_t*>(img + off) = hi;
        *reinterpret_cast<uint32_t*>(img + p.b_bytes + off) = lo;
    }
}

template <bool VEC>
__device__ __forceinline__ void load_chunk(const RnParams& p, int tile, int q, int ct, float4 (&v)[4][2]) {
#pragma unroll
    for (int it = 0; it < 4; ++it) {
        const int idx = ct + 256 * it;
        const int m = idx >> 3, cc = idx & 7;
        const int64_t row = (int64_t)tile * kRows + m;
        const int k = 64 * q + 8 * cc;
        v[it][0] = make_float4(0.f, 0.f, 0.f, 0.f);
        v[it][1] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (row < p.n && k < p.d) {
            const float* src = p.A + row * p.lda + k;
            if constexpr (VEC) {
                asm("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
                    : "=f"(v[it][0].x), "=f"(v[it][0].y), "=f"(v[it][0].z), "=f"(v[it][0].w)
                    : "l"(src));
                asm("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
                    : "=f"(v[it][1].x), "=f"(v[it][1].y), "=f"(v[it][1].z), "=f"(v[it][1].w)
                    : "l"(src + 4));
            } else {
                float t[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) t[e] = (k + e < p.d) ? __ldg(src + e) : 0.f;
                v[it][0] = make_float4(t[0], t[1], t[2], t[3]);
                v[it][1] = make_float4(t[4], t[5], t[6], t[7]);
            }
        }
    }
}

__device__ __forceinline__ void store_chunk(uint8_t* stage, int ct, const float4 (&v)[4][2]) {
#pragma unroll
    for (int it = 0; it < 4; ++it) {
        const int idx = ct + 256 * it;
        const uint32_t m = idx >> 3, cc = idx & 7;
        uint4 hi, lo;
        tc::split_bf16x2(v[it][0].x, v[it][0].y, hi.x, lo.x);
        tc::split_bf16x2(v[it][0].z, v[it][0].w, hi.y, lo.y);
        tc::split_bf16x2(v[it][1].x, v[it][1].y, hi.z, lo.z);
        tc::split_bf16x2(v[it][1].z, v[it][1].w, hi.w, lo.w);
        const uint32_t off = tc::sw128_offset(m, 8 * cc);
        *reinterpret_cast<uint4*>(stage + off) = hi;
        *reinterpret_cast<uint4*>(stage + kHalfStage + off) = lo;
    }
}

// lane 0 waits, the warp follows its verdict
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
    int ok = 0;
    if ((threadIdx.x & 31) == 0) ok = tc::mbar_wait(bar, parity, abort) ? 1 : 0;
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

template <bool VEC>
__global__ void __launch_bounds__(kThreads, 1) rownorm_tc_kernel(const RnParams p, const uint8_t* __restrict__ img) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
    uint8_t* sA = smem;
    uint8_t* sB = smem + kStages * kStageBytes;            // hi image, then lo image
    uint64_t* bars = reinterpret_cast<uint64_t*>(sB + 2 * p.b_bytes);
    uint64_t* full = bars;        // [2] stage filled     (kConvWarps arrivals)
    uint64_t* empty = bars + 2;   // [2] stage consumed   (MMA commit)
    uint64_t* tfull = bars + 4;   // [2] accumulator done (MMA commit)
    uint64_t* tempty = bars + 6;  // [2] accumulator read (kEpiWarps arrivals)
    uint64_t* fin = bars + 8;     // all MMAs complete    (MMA commit)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 9);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < 2; ++s) {
            tc::mbar_init(full + s, kConvWarps);
            tc::mbar_init(empty + s, 1);
            tc::mbar_init(tfull + s, 1);
            tc::mbar_init(tempty + s, kEpiWarps);
        }
        tc::mbar_init(fin, 1);
        *abort = 0;
        tc::fence_mbar_init();
    }
    if (warp == kMmaWarp) {
        tc::tmem_alloc(tmem_slot, kTmemCols);
        tc::tmem_relinquish();
    }
    {   // resident B (hi and lo images), 16-byte copies
        const uint4* src = reinterpret_cast<const uint4*>(img);
        uint4* dst = reinterpret_cast<uint4*>(sB);
        const uint32_t n16 = (2 * p.b_bytes) >> 4;
        for (uint32_t i = threadIdx.x; i < n16; i += kThreads) dst[i] = __ldg(src + i);
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    const int my_tiles = (blockIdx.x < (unsigned)p.ntiles) ? (p.ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

    if (warp < kEpiWarps) {
        // ------------------------------------------------------------ epilogue
        for (int i = 0; i < my_tiles; ++i) {
            const int acc = i & 1;
            if (!warp_wait(tfull + acc, (uint32_t)(i >> 1) & 1u, abort)) break;
            tc::fence_after_sync();
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)acc * kAccCols;
            float sum = 0.f;
            for (int col = 0; col < p.npad; col += 32) {
                float v[32];
                tc::tmem_ld_32x32b_x32(taddr + (uint32_t)col, v);
#pragma unroll
                for (int e = 0; e < 32; ++e) sum = fmaf(v[e], v[e], sum);
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(tempty + acc);
            const int64_t row = ((int64_t)blockIdx.x + (int64_t)i * gridDim.x) * kRows + warp * 32 + lane;
            if (row < p.n) p.x[row] = (p.beta != 0.f) ? fmaf(p.alpha, sum, p.beta * p.x[row]) : p.alpha * sum;
        }
    } else if (warp == kMmaWarp) {
        // ------------------------------------------------------------ MMA issue
        if (lane == 0) {
            const uint32_t sA_u32 = tc::smem_u32(sA), sB_u32 = tc::smem_u32(sB);
            bool ok = true;
            for (int i = 0; i < my_tiles && ok; ++i) {
                const int acc = i & 1;
                if (!tc::mbar_wait(tempty + acc, ((uint32_t)(i >> 1) & 1u) ^ 1u, abort)) break;
                tc::fence_after_sync();
                const uint32_t d_base = tmem + (uint32_t)acc * kAccCols;
                for (int q = 0; q < p.nq; ++q) {
                    const int g = i * p.nq + q;
                    const int s = g & 1;
                    if (!tc::mbar_wait(full + s, (uint32_t)(g >> 1) & 1u, abort)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t a_hi = sA_u32 + (uint32_t)s * kStageBytes, a_lo = a_hi + kHalfStage;
                    const uint32_t b_hi = sB_u32 + p.boff[q], b_lo = b_hi + p.b_bytes;
                    const uint32_t idesc = tc::idesc_bf16_f32(128, p.nn[q]);
                    const uint32_t d_tmem = d_base + p.n0[q];
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const uint32_t ko = 32u * kk;
                        tc::mma_bf16(d_tmem, tc::desc_sw128_kmajor(a_hi + ko), tc::desc_sw128_kmajor(b_hi + ko), idesc,
                                     (q | kk) != 0);
                        tc::mma_bf16(d_tmem, tc::desc_sw128_kmajor(a_hi + ko), tc::desc_sw128_kmajor(b_lo + ko), idesc, 1);
                        tc::mma_bf16(d_tmem, tc::desc_sw128_kmajor(a_lo + ko), tc::desc_sw128_kmajor(b_hi + ko), idesc, 1);
                    }
                    tc::mma_commit(empty + s);
                }
                if (ok) tc::mma_commit(tfull + acc);
            }
            // every MMA issued must be complete before TMEM is released
            tc::mma_commit(fin);
            volatile int never = 0;
            tc::mbar_wait(fin, 0, &never);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ converters
        const int ct = threadIdx.x - kConvWarp0 * 32;   // 0 .. 255
        const int G = my_tiles * p.nq;
        float4 b0[4][2], b1[4][2];
        auto tile_of = [&](int g) { return (int)blockIdx.x + (g / p.nq) * (int)gridDim.x; };
        if (G > 0) load_chunk<VEC>(p, tile_of(0), 0 % p.nq, ct, b0);
        if (G > 1) load_chunk<VEC>(p, tile_of(1), 1 % p.nq, ct, b1);
        for (int g = 0; g < G; g += 2) {
            if (!warp_wait(empty + 0, ((uint32_t)(g >> 1) & 1u) ^ 1u, abort)) break;
            store_chunk(sA, ct, b0);
            tc::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(full + 0);
            if (g + 2 < G) load_chunk<VEC>(p, tile_of(g + 2), (g + 2) % p.nq, ct, b0);
            if (g + 1 >= G) break;
            if (!warp_wait(empty + 1, ((uint32_t)((g + 1) >> 1) & 1u) ^ 1u, abort)) break;
            store_chunk(sA + kStageBytes, ct, b1);
            tc::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(full + 1);
            if (g + 3 < G) load_chunk<VEC>(p, tile_of(g + 3), (g + 3) % p.nq, ct, b1);
        }
    }

    tc::fence_before_sync();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, kTmemCols);
    }
    if (threadIdx.x == 0 && *abort) set_flag(p.flag, LSK_FLAG_TIMEOUT);
}

bool make_plan(const lsk_mat* A, int64_t c, int upper_tri, RnParams& p) {
    const int64_t d = A->d;
    if (A->kind != LSK_DENSE || d < 1 || d > 256 || c < 1 || c > 256) return false;
    if (upper_tri && c != d) return false;
    p.d = (int)d;
    p.c = (int)c;
    p.nq = (int)((d + 63) / 64);
    p.npad = (int)((c + 31) / 32) * 32;
    uint32_t off = 0;
    for (int q = 0; q < 4; ++q) {
        p.n0[q] = 0;
        p.nn[q] = 0;
        p.boff[q] = off;
        if (q < p.nq) {
            p.n0[q] = upper_tri ? (uint32_t)(64 * q) : 0u;
            if ((int)p.n0[q] >= p.npad) return false;
            p.nn[q] = (uint32_t)p.npad - p.n0[q];
            off += p.nn[q] * 128u;
        }
    }
    p.b_bytes = off;
    const size_t smem = (size_t)kStages * kStageBytes + 2 * (size_t)p.b_bytes + 1024 + 128;
    return smem <= kSmemLimit;
}

size_t smem_bytes(const RnParams& p) { return (size_t)kStages * kStageBytes + 2 * (size_t)p.b_bytes + 1024 + 128; }

}  // namespace

bool rownorms_tc_supported(const lsk_mat* A, int64_t c, int upper_tri) {
    RnParams p{};
    return make_plan(A, c, upper_tri, p);
}

size_t rownorms_tc_workspace_bytes(const lsk_mat* A, int64_t c, int upper_tri) {
    RnParams p{};
    if (!make_plan(A, c, upper_tri, p)) return 0;
    return ws_round(2 * (size_t)p.b_bytes);
}

cudaError_t rownorms_tc_launch(const lsk_mat* A, const float* B, int64_t c, float alpha, float beta, int upper_tri,
                               float* x, void* ws, int* flag, int sm_count, cudaStream_t st) {
    RnParams p{};
    if (!make_plan(A, c, upper_tri, p)) return cudaErrorNotSupported;
    p.A = (const float*)A->values;
    p.lda = A->ld;
    p.n = A->n;
    p.x = x;
    p.alpha = alpha;
    p.beta = beta;
    p.flag = flag;
    p.ntiles = (int)((A->n + kRows - 1) / kRows);
    if (p.ntiles == 0) return cudaSuccess;
    uint8_t* img = (uint8_t*)ws;
    LSK_PROF("rownorm_tc_prep", st) rownorm_tc_prep_kernel<<<64, 256, 0, st>>>(B, p, img);
    const size_t smem = smem_bytes(p);
    const bool vec = (p.d % 8 == 0) && (A->ld % 4 == 0) && (((uintptr_t)A->values & 15) == 0);
    const int grid = p.ntiles < sm_count ? p.ntiles : sm_count;
    cudaError_t e;
    if (vec) {
        e = cudaFuncSetAttribute(rownorm_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        LSK_PROF("rownorm_dense_tc", st) rownorm_tc_kernel<true><<<grid, kThreads, smem, st>>>(p, img);
    } else {
        e = cudaFuncSetAttribute(rownorm_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        LSK_PROF("rownorm_dense_tc", st) rownorm_tc_kernel<false><<<grid, kThreads, smem, st>>>(p, img);
    }
    return cudaGetLastError();
}
