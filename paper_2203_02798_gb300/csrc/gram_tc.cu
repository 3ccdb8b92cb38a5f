// gram_tc.cu -- Gram matrix C = alpha A^T A + beta C of a dense A on tcgen05.
//
// The dense form of Alg. 5 / Alg. 7 (rows of A produce partial Gram matrices
// that are then summed), with the partial of a block of rows formed on the
// tensor cores.  Precision: A is split into bfloat16 pairs, a = hi + lo, and
//     A^T A ~= hi^T hi + hi^T lo + lo^T hi        (FP32 accumulation in TMEM)
// (the dropped lo^T lo term is ~2^-17 relative to |a_i||a_j|).
//
// Persistent kernel, one CTA per SM; CTA c takes the slices c, c + grid, ...
// of kSliceRows = 1024 rows each, so no FP32 accumulator sums more than
// 3 x 1024 products (the tensor cores' FP32 accumulation biases long
// all-positive sums, such as the diagonal, at the 1e-5 level by 2048 rows).
// After each slice the epilogue warps add the accumulator into the CTA's
// running FP32 partial in global memory (upper triangle; all CTAs' partials
// together stay in L2), and a second kernel adds the CTAs' partials in order
// with a compensated FP32 sum, then forms alpha * sum + beta * C.
//   warps 0-15  workers: per chunk of 32 rows, load the rows (16-byte loads)
//               into a padded FP32 staging buffer and transpose them into one
//               K-major bf16 hi / lo tile pair (row a of the tile = column a of
//               A, 32 consecutive rows along K) in a 4-stage ring;
//   warp 16     lane 0 issues, for each 128-row M tile t, the products with
//               the tile's rows 128 t .. npad - 1 as the N operand (the same
//               shared-memory tile is both operands; only the upper block
//               triangle is computed);
//   warps 17-24 epilogue: accumulator t is read by the warps whose TMEM lane
//               quarter covers it, added into the running partial, released.
// TMEM holds the two accumulators (N = npad and npad - 128 columns).  Waits
// are bounded; a timeout sets the TIMEOUT flag.
#include "tc_common.cuh"

namespace {

constexpr int kKC = 32;            // rows of A per chunk (the K of the MMAs)
constexpr int kMT = 128;           // rows of an MMA tile (columns of A)
constexpr int kWorkers = 16;
constexpr int kMmaWarp = kWorkers;
constexpr int kEpi0 = kWorkers + 1;
constexpr int kEpiWarps = 8;
constexpr int kThreads = (kWorkers + 1 + kEpiWarps) * 32;
constexpr int kWorkerThreads = kWorkers * 32;
constexpr int kStagePad = 4;
constexpr int kStages = 4;
constexpr int kSliceRows = 1024;   // rows per slice (FP32 accumulation length bound)
constexpr size_t kSmemLimit = 232448;

struct GrParams {
    const float* A;
    int64_t lda, n;
    int d, npad, slices, vec;
    float* part;       // [gridDim][d][d] running partials (upper triangle), zeroed before the launch
    int* flag;
};

__host__ __device__ inline uint32_t half_bytes(int npad) { return (uint32_t)npad * kKC * 2; }   // one bf16 tile
__host__ __device__ inline uint32_t stage_bytes(int npad) { return 2 * half_bytes(npad); }     // hi + lo

__device__ __forceinline__ void named_sync() { asm volatile("bar.sync 1, %0;" ::"r"(kWorkerThreads) : "memory"); }

// Rows i0 .. i0+31 (clipped to r_end) of A into registers: float4 f = wt + 512 j
// -> row f / q4, columns 4 (f % q4).
template <int NPAD>
__device__ __forceinline__ void load_rows(const GrParams& p, int64_t i0, int64_t r_end, int wt, float4 (&a)[4]) {
    constexpr int q4 = NPAD / 4, nf4 = kKC * q4;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        a[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        const int f = wt + kWorkerThreads * j;
        if (f < nf4) {
            const int rr = f / q4, c = 4 * (f % q4);
            const int64_t i = i0 + rr;
            if (i < r_end) {
                const float* src = p.A + i * p.lda + c;
                if (p.vec && c < p.d) {
                    a[j] = __ldg(reinterpret_cast<const float4*>(src));
                } else {
                    a[j].x = c < p.d ? __ldg(src) : 0.f;
                    a[j].y = c + 1 < p.d ? __ldg(src + 1) : 0.f;
                    a[j].z = c + 2 < p.d ? __ldg(src + 2) : 0.f;
                    a[j].w = c + 3 < p.d ? __ldg(src + 3) : 0.f;
                }
            }
        }
    }
}

// NPAD (d rounded up to 32) is a template parameter: every index split below
// is then a division by a constant.
template <int NPAD>
__global__ void __launch_bounds__(kThreads, 1) gram_tc_kernel(const GrParams p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
    const uint32_t sbytes = stage_bytes(NPAD);
    uint8_t* stages = smem;
    float* stagef = reinterpret_cast<float*>(smem + kStages * sbytes);   // kKC x (npad + pad)
    constexpr int ldf = NPAD + kStagePad;
    uint64_t* bars = reinterpret_cast<uint64_t*>(stagef + kKC * ldf);
    uint64_t* full = bars;                 // [kStages] (kWorkers arrivals)
    uint64_t* empty = bars + kStages;      // [kStages] (MMA commit)
    uint64_t* done = bars + 2 * kStages;   // slice accumulated       (MMA commit)
    uint64_t* drained = done + 1;          // accumulator read        (epilogue warp arrivals)
    uint64_t* fin = done + 2;              // every MMA complete      (MMA commit)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
    volatile int* go_on = abort + 1;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int ntiles = (NPAD + kMT - 1) / kMT;   // 1 or 2 M tiles
    const int nepi = 4 * ntiles;                   // epilogue warps in use
    const int my_slices = ((int)blockIdx.x < p.slices) ? (p.slices - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            tc::mbar_init(full + s, kWorkers);
            tc::mbar_init(empty + s, 1);
        }
        tc::mbar_init(done, 1);
        tc::mbar_init(drained, nepi);
        tc::mbar_init(fin, 1);
        *abort = 0;
        tc::fence_mbar_init();
    }
    // accumulator t at column 256 t: N = npad (t = 0), npad - 128 (t = 1)
    constexpr uint32_t tcols = ntiles == 2 ? 512u : NPAD <= 32 ? 32u : NPAD <= 64 ? 64u : 128u;
    if (warp == kMmaWarp) {
        tc::tmem_alloc(tmem_slot, tcols);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp < kWorkers) {
        const int wt = threadIdx.x;
        constexpr int q4 = NPAD / 4;
        constexpr int nf4 = kKC * q4;   // float4 in a chunk (<= 4 per thread)
        int s = 0;
        uint32_t ph = 0;
        for (int z = 0; z < my_slices; ++z) {
            const int64_t r_begin = ((int64_t)blockIdx.x + (int64_t)z * gridDim.x) * kSliceRows;
            const int64_t r_end = min(p.n, r_begin + kSliceRows);
            const int nchunks = (int)((r_end - r_begin + kKC - 1) / kKC);
            bool ok = true;
            // chunk g's rows are loaded while chunk g-1 is staged and transposed
            float4 a[4], nx[4];
            load_rows<NPAD>(p, r_begin, r_end, wt, a);
            for (int g = 0; g < nchunks; ++g) {
                if (g + 1 < nchunks) load_rows<NPAD>(p, r_begin + (int64_t)(g + 1) * kKC, r_end, wt, nx);
                // (2) wait for the stage (one thread decides for all workers)
                if (wt == 0) *go_on = tc::mbar_wait(empty + s, ph ^ 1u, abort) ? 1 : 0;
                named_sync();
                if (!*go_on) {
                    ok = false;
                    break;
                }
                // (3) rows into the FP32 staging buffer
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int f = wt + kWorkerThreads * j;
                    if (f < nf4) {
                        const int rr = f / q4, c = 4 * (f % q4);
                        *reinterpret_cast<float4*>(stagef + rr * ldf + c) = a[j];
                    }
                }
                named_sync();
                // (4) transpose + split: item (column c, row group r8) -> 8 consecutive rows of column c
                uint8_t* th = stages + s * sbytes;
                uint8_t* tl = th + half_bytes(NPAD);
                #pragma unroll
                for (int item = wt; item < NPAD * (kKC / 8); item += kWorkerThreads) {
                    const int c = item % NPAD, r8 = item / NPAD;
                    float v[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) v[e] = stagef[(8 * r8 + e) * ldf + c];
                    uint4 hi, lo;
                    tc::split_bf16x2(v[0], v[1], hi.x, lo.x);
                    tc::split_bf16x2(v[2], v[3], hi.y, lo.y);
                    tc::split_bf16x2(v[4], v[5], hi.z, lo.z);
                    tc::split_bf16x2(v[6], v[7], hi.w, lo.w);
                    const uint32_t off = tc::sw64_offset(c, 8 * r8);
                    *reinterpret_cast<uint4*>(th + off) = hi;
                    *reinterpret_cast<uint4*>(tl + off) = lo;
                }
                tc::fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(full + s);
                if (++s == kStages) {
                    s = 0;
                    ph ^= 1u;
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) a[j] = nx[j];
            }
            if (!ok) break;
        }
    } else if (warp == kMmaWarp) {
        if (lane == 0) {
            const uint32_t base = tc::smem_u32(stages);
            bool okm = true;
            int s = 0;
            uint32_t ph = 0;
            for (int z = 0; z < my_slices && okm; ++z) {
                const int64_t r_begin = ((int64_t)blockIdx.x + (int64_t)z * gridDim.x) * kSliceRows;
                const int64_t r_end = min(p.n, r_begin + kSliceRows);
                const int nchunks = (int)((r_end - r_begin + kKC - 1) / kKC);
                // the previous slice's accumulator has been read out
                if (z > 0 && !tc::mbar_wait(drained, (uint32_t)(z - 1) & 1u, abort)) break;
                tc::fence_after_sync();
                for (int g = 0; g < nchunks; ++g) {
                    if (!tc::mbar_wait(full + s, ph, abort)) {
                        okm = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t hi = base + (uint32_t)s * sbytes, lo = hi + half_bytes(NPAD);
#pragma unroll
                    for (int kk = 0; kk < kKC / 16; ++kk) {
                        const uint32_t ko = 32u * kk;   // 16 bf16 = 32 bytes along the swizzled row
                        for (int t = 0; t < ntiles; ++t) {
                            const uint32_t off = (uint32_t)t * (kMT * kKC * 2) + ko;   // tile rows from 128 t
                            const uint32_t idesc = tc::idesc_bf16_f32(128, (uint32_t)(NPAD - t * kMT));
                            const uint32_t dt = tmem + 256u * t;
                            tc::mma_bf16(dt, tc::desc_sw64_kmajor(hi + off), tc::desc_sw64_kmajor(hi + off), idesc,
                                         (g | kk) != 0);
                            tc::mma_bf16(dt, tc::desc_sw64_kmajor(hi + off), tc::desc_sw64_kmajor(lo + off), idesc, 1);
                            tc::mma_bf16(dt, tc::desc_sw64_kmajor(lo + off), tc::desc_sw64_kmajor(hi + off), idesc, 1);
                        }
                    }
                    tc::mma_commit(empty + s);
                    if (++s == kStages) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
                if (okm) tc::mma_commit(done);
            }
            tc::mma_commit(fin);
            volatile int never = 0;
            tc::mbar_wait(fin, 0, &never);
        }
        __syncwarp();
    } else if (warp - kEpi0 < nepi) {
        // epilogue warp e: accumulator t = e / 4, TMEM lanes of its quarter q = warp % 4
        const int e = warp - kEpi0, t = e >> 2, q = warp & 3;
        const int row = t * kMT + q * 32 + lane;   // column a of A
        const int ncols = NPAD - t * kMT;        // columns b = t*128 .. npad-1
        float* dst = p.part + ((int64_t)blockIdx.x * p.d + row) * p.d + t * kMT;
        for (int z = 0; z < my_slices; ++z) {
            int okw = 0;
            if (lane == 0) okw = tc::mbar_wait(done, (uint32_t)z & 1u, abort) ? 1 : 0;
            if (!__shfl_sync(0xffffffffu, okw, 0)) break;
            tc::fence_after_sync();
            for (int col = 0; col < ncols; col += 32) {
                uint32_t v[32];
                tc::tmem_ld_32x32b_x32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(256 * t + col), v);
                tc::tmem_ld_wait();
                if (row < p.d) {
#pragma unroll
                    for (int k = 0; k < 32; ++k) {
                        const int b = t * kMT + col + k;
                        if (b < p.d && b >= row) dst[col + k] += __uint_as_float(v[k]);
                    }
                }
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(drained);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, tcols);
    }
    if (threadIdx.x == 0 && *abort) set_flag(p.flag, LSK_FLAG_TIMEOUT);
}

// C[a][b] = alpha * sum_c part[c][min][max] + beta * C[a][b]: the CTAs'
// partials in order, compensated FP32 sum (Neumaier), alpha and beta in FP64.
__global__ void gram_tc_reduce_kernel(const float* __restrict__ part, int slices, int d, double alpha, double beta,
                                      float* __restrict__ C) {
    const int64_t len = (int64_t)d * d;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += stride) {
        int a = (int)(e / d), b = (int)(e % d);
        if (a > b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int64_t idx = (int64_t)a * d + b;
        float s = 0.f, c = 0.f;
        for (int z = 0; z < slices; ++z) {
            const float x = part[(int64_t)z * len + idx];
            const float t = s + x;
            c += (fabsf(s) >= fabsf(x)) ? (s - t) + x : (x - t) + s;
            s = t;
        }
        double v = alpha * ((double)s + (double)c);
        if (beta != 0.0) v += beta * (double)C[e];
        C[e] = (float)v;
    }
}

size_t smem_bytes(int npad) {
    return (size_t)kStages * stage_bytes(npad) + (size_t)kKC * (npad + kStagePad) * 4 + 1024 + 128;
}

}  // namespace

bool gram_tc_supported(const lsk_mat* A) {
    return A->kind == LSK_DENSE && A->d >= 1 && A->d <= 256 && smem_bytes((int)((A->d + 31) / 32) * 32) <= kSmemLimit;
}

template <int NPAD>
cudaError_t launch_npad(const GrParams& p, int grid, cudaStream_t st) {
    const size_t smem = smem_bytes(NPAD);
    cudaError_t e = allow_dynamic_smem(gram_tc_kernel<NPAD>);
    if (e != cudaSuccess) return e;
    LSK_PROF("gram_tc", st) gram_tc_kernel<NPAD><<<grid, kThreads, smem, st>>>(p);
    return cudaGetLastError();
}

// one running partial per CTA of the persistent grid
int grid_of(const lsk_mat* A, int sm_count) {
    const int64_t slices = (A->n + kSliceRows - 1) / kSliceRows;
    return (int)(slices < sm_count ? slices : sm_count);
}

size_t gram_tc_workspace_bytes(const lsk_mat* A, int sm_count) {
    const int g = grid_of(A, sm_count);
    return ws_round((size_t)(g > 0 ? g : 1) * A->d * A->d * 4);
}

cudaError_t gram_tc_launch(const lsk_mat* A, double alpha, double beta, float* C, void* ws, int* flag, int sm_count,
                           cudaStream_t st) {
    if (!gram_tc_supported(A)) return cudaErrorNotSupported;
    GrParams p;
    p.A = (const float*)A->values;
    p.lda = A->ld;
    p.n = A->n;
    p.d = (int)A->d;
    p.npad = (int)((A->d + 31) / 32) * 32;
    p.slices = (int)((A->n + kSliceRows - 1) / kSliceRows);
    p.vec = (A->d % 4 == 0) && (A->ld % 4 == 0) && (((uintptr_t)A->values & 15) == 0);
    p.part = (float*)ws;
    p.flag = flag;
    const int grid = grid_of(A, sm_count);
    const int64_t len = A->d * A->d;
    int64_t rg = (len + 255) / 256;
    if (rg > 8 * (int64_t)sm_count) rg = 8 * (int64_t)sm_count;
    cudaError_t e;
    if (grid > 0) {
        e = cudaMemsetAsync(p.part, 0, (size_t)grid * len * 4, st);
        if (e != cudaSuccess) return e;
        switch (p.npad) {
            case 32: e = launch_npad<32>(p, grid, st); break;
            case 64: e = launch_npad<64>(p, grid, st); break;
            case 96: e = launch_npad<96>(p, grid, st); break;
            case 128: e = launch_npad<128>(p, grid, st); break;
            case 160: e = launch_npad<160>(p, grid, st); break;
            case 192: e = launch_npad<192>(p, grid, st); break;
            case 224: e = launch_npad<224>(p, grid, st); break;
            default: e = launch_npad<256>(p, grid, st); break;
        }
        if (e != cudaSuccess) return e;
    }
    LSK_PROF("gram_reduce", st) gram_tc_reduce_kernel<<<(unsigned)rg, 256, 0, st>>>(p.part, grid, p.d, alpha, beta, C);
    return cudaGetLastError();
}
