// rownorms_tc.cu -- fused tensor-core row norms x_i = alpha ||A_i B||^2 + beta x_i.
//
// The memory-efficient dense form of Alg. 8 (rmsqn) on tcgen05: A*B is
// formed 128 rows at a time in tensor memory and squared / summed there, so
// it never reaches HBM.  Precision: A and B are split into bfloat16 pairs,
// x = hi + lo (about 16 significant bits), and
//     A B ~= A_hi B_hi + A_hi B_lo + A_lo B_hi     (FP32 accumulation),
// the dropped A_lo B_lo term being ~2^-18 relative.
//
// Two forms share the pipeline below.  The CTA-pair form (rownorm_tc2_kernel)
// runs M = 256 MMAs across two SMs so each SM holds only half of B and a
// deeper ring; it is used where B is large enough to keep the single-CTA ring
// short of its full depth (d = c = 256 triangular: 5 stages against 9) and
// clusters of two fit.  Single-CTA form:
// Persistent kernel, one CTA per SM (640 threads, 96 registers each):
//   warps 0-3   epilogue: tcgen05.ld the accumulator rows, square, sum, store
//   warp  4     TMEM allocation; lane 0 issues every MMA and commit
//   warps 5-19  converters: each owns every 15th half-chunk (64 rows x 32 K)
//               of the operand stream: it loads its piece from HBM (fully
//               coalesced 16-byte loads), splits it into bf16 hi/lo and
//               writes the 64-byte-swizzled K-major tile into the stage
//               ring.  A warp arrives on the stage barrier only after its own
//               loads have landed (the arrive has release semantics and would
//               otherwise wait for loads still in flight), while the other 14
//               warps keep 7.5 chunks (120 KB) of loads in flight per SM.  The
//               uses of each stage are handed out in order (a per-stage count
//               of stored halves), so no warp waits on a stage barrier more
//               than one phase ahead of it.
// B (hi and lo) stays resident in shared memory for the whole kernel.  K is
// cut into chunks of 32; when B is upper triangular (B = R^-1) K-chunk q
// (rows 32q..32q+31 of B) only touches columns >= 32q, so only those blocks
// are stored and multiplied.  TMEM holds two 128 x 256 FP32 accumulators so
// the epilogue of one tile overlaps the MMAs of the next.
#include "tc_common.cuh"

#include <cuda.h>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>

namespace {

constexpr int kRows = 128;
constexpr int kKC = 32;                              // K per chunk (one 64-byte swizzle row)
constexpr int kMaxQ = 8;                             // d <= 256
constexpr int kConvWarps = 15;      // odd: 20 warps in all, which leaves 96 registers a thread
constexpr int kPieceRows = 64;                       // rows of one converter piece (half a chunk)
constexpr int kPieces = kRows / kPieceRows;          // pieces per chunk (2)
constexpr int kF4 = kPieceRows * kKC / 4 / 32;       // float4 loads per lane per piece (16)
constexpr int kEpiWarps = 4;
constexpr int kMmaWarp = 4;
constexpr int kConvWarp0 = 5;
constexpr int kThreads = (kEpiWarps + 1 + kConvWarps) * 32;
constexpr uint32_t kHalfStage = kRows * kKC * 2;     // one bf16 tile: 8 KB
constexpr uint32_t kStageBytes = 2 * kHalfStage;     // hi + lo
constexpr int kMaxStages = 8;
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kAccCols = 256;
constexpr size_t kSmemLimit = 232448;
constexpr size_t kSmemExtra = 1024 + 256;            // alignment slack + barriers
constexpr int kMaxStages2 = 12;                      // CTA-pair ring
constexpr size_t kSmemExtra2 = 1024 + 1024 + 512;    // alignment slack + pad after B + barriers

struct RnParams {
    const float* A;
    int64_t lda;
    int64_t n;
    float* x;
    float alpha, beta;
    int d, c, nq, npad, ntiles, stages;
    uint32_t n0[kMaxQ], nn[kMaxQ], boff[kMaxQ];
    uint32_t b_bytes;
    int* flag;
    // CTA-pair form: each CTA holds rows [n0 + h nn / 2, n0 + (h + 1) nn / 2)
    // of every K-chunk's B tile (h = its rank in the pair)
    uint32_t hoff[kMaxQ];
    uint32_t hb_bytes;
    int pair, stages2, ntiles2;
    // TF32 form (pair only): each CTA's half of B is one TF32 image of
    // 2 hb_bytes, chunk q at 2 hoff[q] (128-byte rows of 32 FP32 words)
    int tf32;
};

// B (d x c, row-major) -> the shared-memory image of its bf16 hi / lo parts:
// per K-chunk q, an (nn[q] x 32) K-major tile whose row r is column n0[q]+r.
__device__ __forceinline__ void prep_body(const float* __restrict__ B, const RnParams& p, uint8_t* __restrict__ img,
                                          uint32_t blk, uint32_t nblk) {
    if (p.tf32) {
        // B rounded to the nearest TF32 (ties away from zero: half a unit of
        // the 13 dropped bits added to the magnitude, then those bits
        // cleared), in 128-byte-swizzled K-major tiles: element (r, k) of
        // the half tile at 1024 (r / 8) + 128 (r % 8) + 16 ((k / 4) ^ (r % 8))
        // + 4 (k % 4)
        uint32_t total = 0;
        for (int q = 0; q < p.nq; ++q) total += p.nn[q] * kKC;
        for (uint32_t e = blk * blockDim.x + threadIdx.x; e < total; e += nblk * blockDim.x) {
            int q = 0;
            uint32_t el = e;
            while (el >= p.nn[q] * kKC) {
                el -= p.nn[q] * kKC;
                ++q;
            }
            const uint32_t r = el / kKC, kl = el % kKC;
            const int j = (int)(p.n0[q] + r), k = kKC * q + (int)kl;
            const float b = (k < p.d && j < p.c) ? B[(int64_t)k * p.c + j] : 0.f;
            const uint32_t u = (__float_as_uint(b) + 0x1000u) & 0xFFFFE000u;
            const uint32_t hn = p.nn[q] / 2, h = r / hn, rr = r - h * hn;
            const uint32_t off = h * 2 * p.hb_bytes + 2 * p.hoff[q] + (rr >> 3) * 1024u + (rr & 7u) * 128u +
                                 (((kl >> 2) ^ (rr & 7u)) << 4) + (kl & 3u) * 4u;
            *reinterpret_cast<uint32_t*>(img + off) = u;
        }
        return;
    }
    uint32_t total = 0;
    for (int q = 0; q < p.nq; ++q) total += p.nn[q] * (kKC / 2);
    for (uint32_t e = blk * blockDim.x + threadIdx.x; e < total; e += nblk * blockDim.x) {
        int q = 0;
        uint32_t el = e;
        while (el >= p.nn[q] * (kKC / 2)) {
            el -= p.nn[q] * (kKC / 2);
            ++q;
        }
        const uint32_t r = el / (kKC / 2), kl = (el % (kKC / 2)) * 2;
        const int j = (int)(p.n0[q] + r), k = kKC * q + (int)kl;
        const float b0 = (k < p.d && j < p.c) ? B[(int64_t)k * p.c + j] : 0.f;
        const float b1 = (k + 1 < p.d && j < p.c) ? B[(int64_t)(k + 1) * p.c + j] : 0.f;
        uint32_t hi, lo;
        tc::split_bf16x2(b0, b1, hi, lo);
        if (p.pair) {
            // [half 0: hi, lo][half 1: hi, lo], half h = rows h nn / 2 .. of the tile
            const uint32_t hn = p.nn[q] / 2, h = r / hn;
            const uint32_t off = h * 2 * p.hb_bytes + p.hoff[q] + tc::sw64_offset(r - h * hn, kl);
            *reinterpret_cast<uint32_t*>(img + off) = hi;
            *reinterpret_cast<uint32_t*>(img + p.hb_bytes + off) = lo;
        } else {
            const uint32_t off = p.boff[q] + tc::sw64_offset(r, kl);
            *reinterpret_cast<uint32_t*>(img + off) = hi;
            *reinterpret_cast<uint32_t*>(img + p.b_bytes + off) = lo;
        }
    }
}
__global__ void rownorm_tc_prep_kernel(const float* __restrict__ B, const RnParams p, uint8_t* __restrict__ img) {
    prep_body(B, p, img, blockIdx.x, gridDim.x);
}
// the images of many problems' B in one launch (kPrepBlocks blocks a problem)
struct RnPrepJob {
    const float* B;
    RnParams p;
    uint8_t* img;
};
constexpr int kPrepBlocks = 16;
__global__ void rownorm_tc_prep_grouped_kernel(const RnPrepJob* __restrict__ jobs, const int* __restrict__ off,
                                               int count) {
    const int g = group_of(off, count, blockIdx.x);
    const int b0 = __ldg(off + g), b1 = __ldg(off + g + 1);
    prep_body(jobs[g].B, jobs[g].p, jobs[g].img, (uint32_t)((int)blockIdx.x - b0), (uint32_t)(b1 - b0));
}

// Lane l loads float4 number f = l + 32 i of the piece (row f / 8 of the
// piece, columns 4 (f % 8) .. +3): consecutive lanes read consecutive
// 16-byte pieces, four 128-byte row segments per warp instruction.
template <bool VEC, int PR = kPieceRows>
__device__ __forceinline__ void load_piece(const RnParams& p, int64_t rowbase, int q, int half, int lane,
                                           float4 (&v)[PR / 4]) {
    constexpr int F4 = PR / 4;
    const int64_t row0 = rowbase + half * PR + (lane >> 3);
    const int k0 = kKC * q + 4 * (lane & 7);
    if (VEC && row0 - (lane >> 3) + PR <= p.n && kKC * q + kKC <= p.d) {
        // interior piece: no bounds checks, rows 4 apart per step
        const float* src = p.A + row0 * p.lda + k0;
        const int64_t step = 4 * p.lda;
#pragma unroll
        for (int i = 0; i < F4; ++i) {
            asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
                         : "=f"(v[i].x), "=f"(v[i].y), "=f"(v[i].z), "=f"(v[i].w)
                         : "l"(src));
            src += step;
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < F4; ++i) {
        const int f = lane + 32 * i;
        const int m = half * PR + (f >> 3), c4 = f & 7;
        const int64_t row = rowbase + m;
        const int k = kKC * q + 4 * c4;
        v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (row < p.n && k < p.d) {
            const float* src = p.A + row * p.lda + k;
            if constexpr (VEC) {
                // volatile: a prefetch kAhead chunks before its use, issued here
                asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
                             : "=f"(v[i].x), "=f"(v[i].y), "=f"(v[i].z), "=f"(v[i].w)
                             : "l"(src));
            } else {
                v[i].x = __ldg(src);
                v[i].y = (k + 1 < p.d) ? __ldg(src + 1) : 0.f;
                v[i].z = (k + 2 < p.d) ? __ldg(src + 2) : 0.f;
                v[i].w = (k + 3 < p.d) ? __ldg(src + 3) : 0.f;
            }
        }
    }
}

// Element (m, 4 c4) of the piece, m = PR half + 4 i + l8 (l8 = lane / 8,
// c4 = lane % 8), sits at tc::sw64_offset(m, 4 c4).  Because l8 < 4, the row
// atom (m / 8 = (PR / 8) half + i / 2), the row in the atom (4 (i % 2) + l8)
// and the swizzle phase ((m / 2) % 4 = 2 (i % 2) + l8 / 2) split into a
// per-lane part that depends only on the parity of i and a constant 512 (i /
// 2): two base offsets per lane, and every store takes an immediate offset.
template <int PR = kPieceRows>
__device__ __forceinline__ void store_piece(uint8_t* stage, int half, int lane, const float4 (&v)[PR / 4]) {
    const uint32_t l8 = (uint32_t)lane >> 3, c4 = (uint32_t)lane & 7u;
    const uint32_t lane_part = l8 * 64u + (c4 & 1u) * 8u;
    const uint32_t b_even = (uint32_t)half * (PR * 64u) + lane_part + ((((c4 >> 1) ^ (l8 >> 1)) & 3u) << 4);
    const uint32_t b_odd = (uint32_t)half * (PR * 64u) + 256u + lane_part +
                           ((((c4 >> 1) ^ (2u + (l8 >> 1))) & 3u) << 4);
    uint8_t* const s_even = stage + b_even;
    uint8_t* const s_odd = stage + b_odd;
#pragma unroll
    for (int i = 0; i < PR / 4; ++i) {
        uint2 hi, lo;
        tc::split_bf16x2(v[i].x, v[i].y, hi.x, lo.x);
        tc::split_bf16x2(v[i].z, v[i].w, hi.y, lo.y);
        uint8_t* const dst = ((i & 1) ? s_odd : s_even) + (i >> 1) * 512;
        *reinterpret_cast<uint2*>(dst) = hi;
        *reinterpret_cast<uint2*>(dst + kHalfStage) = lo;
    }
}

// lane 0 waits, the warp follows its result
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
    int ok = 0;
    if ((threadIdx.x & 31) == 0) ok = tc::mbar_wait(bar, parity, abort) ? 1 : 0;
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

template <bool VEC>
__global__ void __launch_bounds__(kThreads, 1) rownorm_tc_kernel(const RnParams p, const uint8_t* __restrict__ img) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
    const int S = p.stages;
    uint8_t* sA = smem;                                  // S stages of (hi, lo)
    uint8_t* sB = smem + S * kStageBytes;                // B hi image, then lo image
    uint64_t* bars = reinterpret_cast<uint64_t*>(sB + 2 * p.b_bytes);
    uint64_t* full = bars;                       // [S] stage filled     (kPieces arrivals)
    uint64_t* empty = bars + kMaxStages;         // [S] stage consumed   (MMA commit)
    uint64_t* tfull = bars + 2 * kMaxStages;     // [2] accumulator done (MMA commit)
    uint64_t* tempty = tfull + 2;                // [2] accumulator read (kEpiWarps arrivals)
    uint64_t* fin = tfull + 4;                   // all MMAs complete    (MMA commit)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
    int* stored = const_cast<int*>(abort) + 1;   // [S] halves stored per stage (in use order)

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            tc::mbar_init(full + s, kPieces);
            tc::mbar_init(empty + s, 1);
        }
        for (int a = 0; a < 2; ++a) {
            tc::mbar_init(tfull + a, 1);
            tc::mbar_init(tempty + a, kEpiWarps);
        }
        tc::mbar_init(fin, 1);
        *abort = 0;
        for (int s = 0; s < kMaxStages; ++s) stored[s] = 0;
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
            for (int col = 0; col < p.npad; col += 64) {   // two loads in flight per wait
                uint32_t v0[32], v1[32];
                tc::tmem_ld_32x32b_x32(taddr + (uint32_t)col, v0);
                const bool two = col + 32 < p.npad;
                if (two) tc::tmem_ld_32x32b_x32(taddr + (uint32_t)col + 32u, v1);
                tc::tmem_ld_wait();
#pragma unroll
                for (int e = 0; e < 32; ++e) sum = fmaf(__uint_as_float(v0[e]), __uint_as_float(v0[e]), sum);
                if (two) {
#pragma unroll
                    for (int e = 0; e < 32; ++e) sum = fmaf(__uint_as_float(v1[e]), __uint_as_float(v1[e]), sum);
                }
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
            // One thread issues everything, so its per-chunk instruction chain
            // is on the critical path: stage and phase advance incrementally
            // (no division), and the K-chunk loop is unrolled so the per-chunk
            // constants of p are read with static indices (no local copy).
            const uint32_t sA_u32 = tc::smem_u32(sA), sB_u32 = tc::smem_u32(sB);
            bool ok = true;
            int s = 0;
            uint32_t ph = 0;
            for (int i = 0; i < my_tiles && ok; ++i) {
                const int acc = i & 1;
                if (!tc::mbar_wait(tempty + acc, ((uint32_t)(i >> 1) & 1u) ^ 1u, abort)) break;
                tc::fence_after_sync();
                const uint32_t d_base = tmem + (uint32_t)acc * kAccCols;
#pragma unroll
                for (int q = 0; q < kMaxQ; ++q) {
                    if (q >= p.nq) break;
                    if (!tc::mbar_wait(full + s, ph, abort)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t a_hi = sA_u32 + (uint32_t)s * kStageBytes, a_lo = a_hi + kHalfStage;
                    const uint32_t b_hi = sB_u32 + p.boff[q], b_lo = b_hi + p.b_bytes;
                    const uint32_t idesc = tc::idesc_bf16_f32(128, p.nn[q]);
                    const uint32_t d_tmem = d_base + p.n0[q];
#pragma unroll
                    for (int kk = 0; kk < kKC / 16; ++kk) {
                        const uint32_t ko = 32u * kk;   // 16 bf16 = 32 bytes along the swizzled row
                        tc::mma_bf16(d_tmem, tc::desc_sw64_kmajor(a_hi + ko), tc::desc_sw64_kmajor(b_hi + ko), idesc,
                                     (q | kk) != 0);
                        tc::mma_bf16(d_tmem, tc::desc_sw64_kmajor(a_hi + ko), tc::desc_sw64_kmajor(b_lo + ko), idesc, 1);
                        tc::mma_bf16(d_tmem, tc::desc_sw64_kmajor(a_lo + ko), tc::desc_sw64_kmajor(b_hi + ko), idesc, 1);
                    }
                    tc::mma_commit(empty + s);
                    if (++s == S) {
                        s = 0;
                        ph ^= 1u;
                    }
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
        // piece number pc = kPieces * g + half goes to converter warp pc % kConvWarps
        // (kConvWarps is odd, so a warp's pieces alternate between the halves)
        const int cw = warp - kConvWarp0;
        const int G = my_tiles * p.nq;
        float4 buf[kF4];
        // piece pc: chunk g = pc / 2 = (tile t, K-chunk q), stage s, use u -- advanced without division
        int pc = cw, g = pc / kPieces, t = g / p.nq, q = g % p.nq, s = g % S, u = g / S;
        for (; g < G;) {
            const int half = pc % kPieces;
            load_piece<VEC>(p, ((int64_t)blockIdx.x + (int64_t)t * gridDim.x) * kRows, q, half, lane, buf);
            int ok = 1;
            if (lane == 0) {
                // both halves of this stage's previous use are stored: the stage
                // barriers are now at most one phase behind this use
                ok = tc::counter_wait(reinterpret_cast<volatile int*>(stored + s), kPieces * u, abort) &&
                     tc::mbar_wait(empty + s, ((uint32_t)u & 1u) ^ 1u, abort);
            }
            if (!__shfl_sync(0xffffffffu, ok, 0)) break;
            store_piece(sA + s * kStageBytes, half, lane, buf);
            tc::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
                tc::mbar_arrive(full + s);
                atomicAdd(stored + s, 1);
            }
            pc += kConvWarps;
            const int dg = pc / kPieces - g;
            g += dg;
            for (q += dg; q >= p.nq; q -= p.nq) ++t;
            for (s += dg; s >= S; s -= S) ++u;
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

// CTA-pair form (cluster of 2 SMs, cta_group::2): one M = 256 MMA covers 256
// rows, 128 in each CTA, and each CTA keeps only its half of every K-chunk's B
// tile, so B takes half the shared memory and the ring is nearly twice as
// deep (9 stages at d = 256).  The even CTA's MMA thread issues for both;
// the converters of both CTAs arrive on its stage barriers and its commits
// are multicast to both CTAs' barriers; each CTA's epilogue reads its own
// TMEM rows and reports to the even CTA.
template <bool VEC, int PR>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1)
    rownorm_tc2_kernel(const RnParams p, const uint8_t* __restrict__ img) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
    const int S = p.stages2;
    const uint32_t rank = tc::cluster_ctarank();
    const int cid = (int)tc::cluster_id_x(), ncl = (int)tc::nclusters_x();
    uint8_t* sA = smem;                                  // S stages of (hi, lo), this CTA's 128 rows
    uint8_t* sB = smem + S * kStageBytes;                // this CTA's half of B: hi image, then lo image
    uint64_t* bars = reinterpret_cast<uint64_t*>(sB + 2 * p.hb_bytes + 1024);
    constexpr int NP = kRows / PR;               // pieces per chunk
    uint64_t* full = bars;                       // [S] even CTA: stage filled in both CTAs (2 NP arrivals)
    uint64_t* empty = bars + kMaxStages2;        // [S] stage consumed (multicast commit)
    uint64_t* tfull = bars + 2 * kMaxStages2;    // [2] accumulator done (multicast commit)
    uint64_t* tempty = tfull + 2;                // [2] even CTA: accumulator read in both (2 kEpiWarps arrivals)
    uint64_t* fin = tfull + 4;                   // all MMAs complete (multicast commit)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
    int* stored = const_cast<int*>(abort) + 1;   // [S] halves stored per stage (in use order)

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            tc::mbar_init(full + s, 2 * NP);
            tc::mbar_init(empty + s, 1);
        }
        for (int a = 0; a < 2; ++a) {
            tc::mbar_init(tfull + a, 1);
            tc::mbar_init(tempty + a, 2 * kEpiWarps);
        }
        tc::mbar_init(fin, 1);
        *abort = 0;
        for (int s = 0; s < kMaxStages2; ++s) stored[s] = 0;
        tc::fence_mbar_init();
    }
    if (warp == kMmaWarp) {
        tc::tmem_alloc_pair(tmem_slot, kTmemCols);
        tc::tmem_relinquish_pair();
    }
    {   // this CTA's half of B (hi and lo images), 16-byte copies
        const uint4* src = reinterpret_cast<const uint4*>(img + (size_t)rank * 2 * p.hb_bytes);
        uint4* dst = reinterpret_cast<uint4*>(sB);
        const uint32_t n16 = (2 * p.hb_bytes) >> 4;
        for (uint32_t i = threadIdx.x; i < n16; i += kThreads) dst[i] = __ldg(src + i);
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    tc::cluster_sync();   // barriers of both CTAs initialised, B halves in place
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    const int my_tiles = (cid < p.ntiles2) ? (p.ntiles2 - 1 - cid) / ncl + 1 : 0;

    if (warp < kEpiWarps) {
        // ------------------------------------------------------------ epilogue
        for (int i = 0; i < my_tiles; ++i) {
            const int acc = i & 1;
            if (!warp_wait(tfull + acc, (uint32_t)(i >> 1) & 1u, abort)) break;
            tc::fence_after_sync();
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)acc * kAccCols;
            float sum = 0.f;
            for (int col = 0; col < p.npad; col += 64) {
                uint32_t v0[32], v1[32];
                tc::tmem_ld_32x32b_x32(taddr + (uint32_t)col, v0);
                const bool two = col + 32 < p.npad;
                if (two) tc::tmem_ld_32x32b_x32(taddr + (uint32_t)col + 32u, v1);
                tc::tmem_ld_wait();
#pragma unroll
                for (int e = 0; e < 32; ++e) sum = fmaf(__uint_as_float(v0[e]), __uint_as_float(v0[e]), sum);
                if (two) {
#pragma unroll
                    for (int e = 0; e < 32; ++e) sum = fmaf(__uint_as_float(v1[e]), __uint_as_float(v1[e]), sum);
                }
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) {
                if (rank == 0) tc::mbar_arrive(tempty + acc);
                else tc::mbar_arrive_cluster(tempty + acc, 0);
            }
            const int64_t row = ((int64_t)cid + (int64_t)i * ncl) * (2 * kRows) + rank * kRows + warp * 32 + lane;
            if (row < p.n) p.x[row] = (p.beta != 0.f) ? fmaf(p.alpha, sum, p.beta * p.x[row]) : p.alpha * sum;
        }
    } else if (warp == kMmaWarp) {
        // ------------------------------------------------------------ MMA issue (even CTA)
        if (lane == 0 && rank == 0) {
            const uint32_t sA_u32 = tc::smem_u32(sA), sB_u32 = tc::smem_u32(sB);
            bool ok = true;
            int s = 0;
            uint32_t ph = 0;
            for (int i = 0; i < my_tiles && ok; ++i) {
                const int acc = i & 1;
                if (!tc::mbar_wait_cluster(tempty + acc, ((uint32_t)(i >> 1) & 1u) ^ 1u, abort)) break;
                tc::fence_after_sync();
                const uint32_t d_base = tmem + (uint32_t)acc * kAccCols;
#pragma unroll
                for (int q = 0; q < kMaxQ; ++q) {
                    if (q >= p.nq) break;
                    if (!tc::mbar_wait_cluster(full + s, ph, abort)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t a_hi = sA_u32 + (uint32_t)s * kStageBytes, a_lo = a_hi + kHalfStage;
                    const uint32_t b_hi = sB_u32 + p.hoff[q], b_lo = b_hi + p.hb_bytes;
                    const uint32_t idesc = tc::idesc_bf16_f32(2 * kRows, p.nn[q]);
                    const uint32_t d_tmem = d_base + p.n0[q];
#pragma unroll
                    for (int kk = 0; kk < kKC / 16; ++kk) {
                        const uint32_t ko = 32u * kk;
                        tc::mma_bf16_pair(d_tmem, tc::desc_sw64_kmajor(a_hi + ko), tc::desc_sw64_kmajor(b_hi + ko),
                                          idesc, (q | kk) != 0);
                        tc::mma_bf16_pair(d_tmem, tc::desc_sw64_kmajor(a_hi + ko), tc::desc_sw64_kmajor(b_lo + ko),
                                          idesc, 1);
                        tc::mma_bf16_pair(d_tmem, tc::desc_sw64_kmajor(a_lo + ko), tc::desc_sw64_kmajor(b_hi + ko),
                                          idesc, 1);
                    }
                    tc::mma_commit_pair(empty + s);
                    if (++s == S) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
                if (ok) tc::mma_commit_pair(tfull + acc);
            }
            tc::mma_commit_pair(fin);
        }
        if (lane == 0) {
            // both CTAs: the last multicast commit has landed here, so no
            // arrival is still on its way when the CTA leaves
            volatile int never = 0;
            tc::mbar_wait(fin, 0, &never);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ converters
        // piece number pc = NP * g + part goes to converter warp pc % kConvWarps;
        // the uses of each stage are claimed in piece order (stored[s])
        const int cw = warp - kConvWarp0;
        const int G = my_tiles * p.nq;
        struct Piece {
            int pc, g, t, q, s, u;
        };
        const auto first = [&](int pc) {
            const int g = pc / NP;
            return Piece{pc, g, g / p.nq, g % p.nq, g % S, g / S};
        };
        const auto advance = [&](Piece& x) {
            x.pc += kConvWarps;
            const int dg = x.pc / NP - x.g;
            x.g += dg;
            for (x.q += dg; x.q >= p.nq; x.q -= p.nq) ++x.t;
            for (x.s += dg; x.s >= S; x.s -= S) ++x.u;
        };
        const auto rowbase = [&](const Piece& x) {
            return ((int64_t)cid + (int64_t)x.t * ncl) * (2 * kRows) + rank * kRows;
        };
        // claim the stage for piece x (in order), split and store it, arrive
        const auto put = [&](const Piece& x, const float4 (&v)[PR / 4]) -> bool {
            int ok = 1;
            if (lane == 0) {
                ok = tc::counter_wait(reinterpret_cast<volatile int*>(stored + x.s), NP * x.u, abort) &&
                     tc::mbar_wait(empty + x.s, ((uint32_t)x.u & 1u) ^ 1u, abort);
            }
            if (!__shfl_sync(0xffffffffu, ok, 0)) return false;
            store_piece<PR>(sA + x.s * kStageBytes, x.pc % NP, lane, v);
            tc::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
                if (rank == 0) tc::mbar_arrive(full + x.s);
                else tc::mbar_arrive_cluster(full + x.s, 0);
                atomicAdd(stored + x.s, 1);
            }
            return true;
        };
        // one piece in registers: load it, claim its stage, store it.  (Two
        // 32-row pieces in flight per warp measured slower: twice the claims,
        // fences and arrivals per byte, and the loads were not the limit.)
        float4 buf[PR / 4];
        for (Piece a = first(cw); a.g < G; advance(a)) {
            load_piece<VEC, PR>(p, rowbase(a), a.q, a.pc % NP, lane, buf);
            if (!put(a, buf)) break;
        }
    }

    tc::fence_before_sync();
    __syncthreads();
    tc::cluster_sync();   // no CTA leaves while its peer may still arrive on its barriers
    if (warp == kMmaWarp) {
        tc::fence_after_sync();
        tc::tmem_dealloc_pair(tmem, kTmemCols);
    }
    if (threadIdx.x == 0 && *abort) set_flag(p.flag, LSK_FLAG_TIMEOUT);
}

// CTA-pair form fed by TMA (A row-major FP32 with 16-byte aligned rows).
// One thread per CTA streams the CTA's 128 rows of every K-chunk (128 x 32
// FP32 = 16 KB, 128-byte swizzle) into the stage ring as soon as the MMAs
// have released the stage, so the ring itself is the data in flight (9
// stages = 144 KB per SM at d = c = 256) and no thread holds loads in
// registers.  The converters split a landed chunk into bf16 hi / lo in
// place: a warp owns whole 8-row blocks, and the 1 KB of FP32 of one block is
// exactly the room of its 512-byte hi atom (at +0) and 512-byte lo atom (at
// +512), so the split needs no barrier beyond the warp; the MMAs read the hi
// and lo operands with 8-row atoms 1024 bytes apart.  Converter group i of
// G takes chunks i, i + G, ...; the ring is a multiple of G stages, so each
// stage belongs to one group, which waits on its uses in order (never a
// phase ahead of the barrier).  The MMA issue, the accumulators and
// the epilogue are those of rownorm_tc2_kernel.
constexpr int kTmaWarp = 5;
constexpr int kCvtWarp0 = 6;
template <int GROUPS, int WARPS>
struct TmaShape {
    static constexpr int kGroups = GROUPS;                          // converter groups
    static constexpr int kWarps = WARPS;                            // warps per group
    static constexpr int kBlocks = kRows / 8 / WARPS;               // 8-row blocks per warp
    static constexpr int kThreads = (kCvtWarp0 + GROUPS * WARPS) * 32;
};
constexpr uint32_t kChunkBytes = kRows * kKC * 4;              // one FP32 chunk = one stage
static_assert(kChunkBytes == kStageBytes, "a landed FP32 chunk becomes its own hi / lo stage");


// TF32 = false: the BF16x3 products of the converters' hi / lo split.
// TF32 = true: one kind::tf32 product per K-step straight from the landed
// chunk (A operand) and the TF32 image of B.  The tensor map then has the
// TF32 element type, so the copy engine rounds every FP32 word of A to the
// nearest TF32 on its way into shared memory (the MMA itself would drop the
// 13 low mantissa bits: rounding toward zero, a -3.5e-4 relative bias on
// A's entries on average); the converter warps only pass each landed chunk
// on to the even CTA's MMA thread, group i of G taking chunks i, i + G, ...
template <class T, bool TF32 = false>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(T::kThreads, 1)
    rownorm_tma2_kernel(const RnParams p, const uint8_t* __restrict__ img, const __grid_constant__ CUtensorMap tmA) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
    const int S = p.stages2;
    const uint32_t rank = tc::cluster_ctarank();
    const int cid = (int)tc::cluster_id_x(), ncl = (int)tc::nclusters_x();
    uint8_t* sA = smem;                                  // S stages: FP32 chunk, then its hi / lo blocks
    uint8_t* sB = smem + S * kStageBytes;                // this CTA's half of B: hi image, then lo image
    uint64_t* bars = reinterpret_cast<uint64_t*>(sB + 2 * p.hb_bytes + 1024);
    uint64_t* full = bars;                       // [S] even CTA: chunk split in both CTAs (2 kWarps arrivals)
    uint64_t* empty = bars + kMaxStages2;        // [S] stage consumed (multicast commit)
    uint64_t* landed = bars + 2 * kMaxStages2;   // [S] this CTA's chunk has landed (TMA bytes)
    uint64_t* tfull = bars + 3 * kMaxStages2;    // [2] accumulator done (multicast commit)
    uint64_t* tempty = tfull + 2;                // [2] even CTA: accumulator read in both (2 kEpiWarps arrivals)
    uint64_t* fin = tfull + 4;                   // all MMAs complete (multicast commit)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            tc::mbar_init(full + s, 2 * T::kWarps);
            tc::mbar_init(empty + s, 1);
            tc::mbar_init(landed + s, 1);
        }
        for (int a = 0; a < 2; ++a) {
            tc::mbar_init(tfull + a, 1);
            tc::mbar_init(tempty + a, 2 * kEpiWarps);
        }
        tc::mbar_init(fin, 1);
        *abort = 0;
        tc::fence_mbar_init();
    }
    if (warp == kMmaWarp) {
        tc::tmem_alloc_pair(tmem_slot, kTmemCols);
        tc::tmem_relinquish_pair();
    }
    if (warp == kTmaWarp && lane == 0) tc::prefetch_tmap(&tmA);
    {   // this CTA's half of B (hi and lo images), 16-byte copies
        const uint4* src = reinterpret_cast<const uint4*>(img + (size_t)rank * 2 * p.hb_bytes);
        uint4* dst = reinterpret_cast<uint4*>(sB);
        const uint32_t n16 = (2 * p.hb_bytes) >> 4;
        for (uint32_t i = threadIdx.x; i < n16; i += T::kThreads) dst[i] = __ldg(src + i);
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    tc::cluster_sync();   // barriers of both CTAs initialised, B halves in place
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    const int my_tiles = (cid < p.ntiles2) ? (p.ntiles2 - 1 - cid) / ncl + 1 : 0;
    const int G = my_tiles * p.nq;

    if (warp < kEpiWarps) {
        // ------------------------------------------------------------ epilogue
        for (int i = 0; i < my_tiles; ++i) {
            const int acc = i & 1;
            if (!warp_wait(tfull + acc, (uint32_t)(i >> 1) & 1u, abort)) break;
            tc::fence_after_sync();
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)acc * kAccCols;
            float sum = 0.f;
            for (int col = 0; col < p.npad; col += 64) {
                uint32_t v0[32], v1[32];
                tc::tmem_ld_32x32b_x32(taddr + (uint32_t)col, v0);
                const bool two = col + 32 < p.npad;
                if (two) tc::tmem_ld_32x32b_x32(taddr + (uint32_t)col + 32u, v1);
                tc::tmem_ld_wait();
#pragma unroll
                for (int e = 0; e < 32; ++e) sum = fmaf(__uint_as_float(v0[e]), __uint_as_float(v0[e]), sum);
                if (two) {
#pragma unroll
                    for (int e = 0; e < 32; ++e) sum = fmaf(__uint_as_float(v1[e]), __uint_as_float(v1[e]), sum);
                }
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) {
                if (rank == 0) tc::mbar_arrive(tempty + acc);
                else tc::mbar_arrive_cluster(tempty + acc, 0);
            }
            const int64_t row = ((int64_t)cid + (int64_t)i * ncl) * (2 * kRows) + rank * kRows + warp * 32 + lane;
            if (row < p.n) p.x[row] = (p.beta != 0.f) ? fmaf(p.alpha, sum, p.beta * p.x[row]) : p.alpha * sum;
        }
    } else if (warp == kMmaWarp) {
        // ------------------------------------------------------------ MMA issue (even CTA)
        if (lane == 0 && rank == 0) {
            const uint32_t sA_u32 = tc::smem_u32(sA), sB_u32 = tc::smem_u32(sB);
            bool ok = true;
            int s = 0;
            uint32_t ph = 0;
            for (int i = 0; i < my_tiles && ok; ++i) {
                const int acc = i & 1;
                if (!tc::mbar_wait_cluster(tempty + acc, ((uint32_t)(i >> 1) & 1u) ^ 1u, abort)) break;
                tc::fence_after_sync();
                const uint32_t d_base = tmem + (uint32_t)acc * kAccCols;
#pragma unroll
                for (int q = 0; q < kMaxQ; ++q) {
                    if (q >= p.nq) break;
                    if (!tc::mbar_wait_cluster(full + s, ph, abort)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t d_tmem = d_base + p.n0[q];
                    if constexpr (TF32) {
                        // A: the 128 x 32 FP32 chunk as TMA left it (128-byte
                        // swizzle, 8-row atoms 1024 bytes apart); B: chunk q of
                        // the TF32 image; K = 8 (32 bytes) per MMA
                        const uint32_t a0 = sA_u32 + (uint32_t)s * kStageBytes;
                        const uint32_t b0 = sB_u32 + 2u * p.hoff[q];
                        const uint32_t idesc = tc::idesc_tf32_f32(2 * kRows, p.nn[q]);
#pragma unroll
                        for (int kk = 0; kk < kKC / 8; ++kk)
                            tc::mma_tf32_pair(d_tmem, tc::desc_sw128_kmajor(a0 + 32u * kk),
                                              tc::desc_sw128_kmajor(b0 + 32u * kk), idesc, (q | kk) != 0);
                    } else {
                        const uint32_t a_hi = sA_u32 + (uint32_t)s * kStageBytes, a_lo = a_hi + 512u;
                        const uint32_t b_hi = sB_u32 + p.hoff[q], b_lo = b_hi + p.hb_bytes;
                        const uint32_t idesc = tc::idesc_bf16_f32(2 * kRows, p.nn[q]);
#pragma unroll
                        for (int kk = 0; kk < kKC / 16; ++kk) {
                            const uint32_t ko = 32u * kk;
                            const uint64_t ah = tc::desc_sw64_kmajor_sbo(a_hi + ko, 1024u);
                            const uint64_t al = tc::desc_sw64_kmajor_sbo(a_lo + ko, 1024u);
                            tc::mma_bf16_pair(d_tmem, ah, tc::desc_sw64_kmajor(b_hi + ko), idesc, (q | kk) != 0);
                            tc::mma_bf16_pair(d_tmem, ah, tc::desc_sw64_kmajor(b_lo + ko), idesc, 1);
                            tc::mma_bf16_pair(d_tmem, al, tc::desc_sw64_kmajor(b_hi + ko), idesc, 1);
                        }
                    }
                    tc::mma_commit_pair(empty + s);
                    if (++s == S) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
                if (ok) tc::mma_commit_pair(tfull + acc);
            }
            tc::mma_commit_pair(fin);
        }
        if (lane == 0) {
            volatile int never = 0;
            tc::mbar_wait(fin, 0, &never);
        }
        __syncwarp();
    } else if (warp == kTmaWarp) {
        // ------------------------------------------------------------ TMA producer (both CTAs)
        if (lane == 0) {
            int issued = 0, t = 0, q = 0, s = 0;
            uint32_t u = 0;
            for (int g = 0; g < G; ++g) {
                if (!tc::mbar_wait(empty + s, (u & 1u) ^ 1u, abort)) break;
                tc::mbar_arrive_expect_tx(landed + s, kChunkBytes);
                const int64_t y = ((int64_t)cid + (int64_t)t * ncl) * (2 * kRows) + rank * kRows;
                tc::tma_load_2d(sA + s * kStageBytes, &tmA, kKC * q, (int32_t)y, landed + s);
                ++issued;
                if (++q == p.nq) {
                    q = 0;
                    ++t;
                }
                if (++s == S) {
                    s = 0;
                    ++u;
                }
            }
            // no copy may still be landing when the CTA leaves (only possible
            // after a wait gave up): wait for the last use issued on each stage
            volatile int never = 0;
            for (int st = 0; st < S && st < issued; ++st) {
                const int uses = (issued - 1 - st) / S + 1;
                tc::mbar_wait(landed + st, (uint32_t)(uses - 1) & 1u, &never);
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ converters
        const int cw = warp - kCvtWarp0, grp = cw / T::kWarps, wi = cw % T::kWarps;
        int s = grp % S;
        uint32_t u = (uint32_t)(grp / S);
        for (int g = grp; g < G; g += T::kGroups) {
            if (!warp_wait(landed + s, u & 1u, abort)) break;
            static_assert(T::kBlocks * T::kWarps * 8 == kRows, "the converter warps cover the chunk's rows");
            if constexpr (!TF32) {
                tc::mbar_try_wait(landed + s, u & 1u);   // every lane acquires the landed bytes
                tc::split_blocks_in_place<T::kBlocks>(sA + s * kStageBytes + wi * T::kBlocks * 1024, lane);
                tc::fence_proxy_async_smem();
            }
            __syncwarp();
            if (lane == 0) {
                if (rank == 0) tc::mbar_arrive(full + s);
                else tc::mbar_arrive_cluster(full + s, 0);
            }
            for (s += T::kGroups; s >= S; s -= S) ++u;
        }
    }

    tc::fence_before_sync();
    __syncthreads();
    tc::cluster_sync();   // no CTA leaves while its peer may still arrive on its barriers
    if (warp == kMmaWarp) {
        tc::fence_after_sync();
        tc::tmem_dealloc_pair(tmem, kTmemCols);
    }
    if (threadIdx.x == 0 && *abort) set_flag(p.flag, LSK_FLAG_TIMEOUT);
}

size_t smem_bytes2(const RnParams& p) {
    return (size_t)p.stages2 * kStageBytes + 2 * (size_t)p.hb_bytes + kSmemExtra2;
}

size_t smem_bytes(const RnParams& p) {
    return (size_t)p.stages * kStageBytes + 2 * (size_t)p.b_bytes + kSmemExtra;
}

bool make_plan(const lsk_mat* A, int64_t c, int upper_tri, RnParams& p) {
    const int64_t d = A->d;
    if (A->kind != LSK_DENSE || d < 1 || d > 256 || c < 1 || c > 256) return false;
    if (upper_tri && c != d) return false;
    p.d = (int)d;
    p.c = (int)c;
    p.nq = (int)((d + kKC - 1) / kKC);
    p.npad = (int)((c + 31) / 32) * 32;
    uint32_t off = 0;
    for (int q = 0; q < kMaxQ; ++q) {
        p.n0[q] = 0;
        p.nn[q] = 0;
        p.boff[q] = off;
        if (q < p.nq) {
            p.n0[q] = upper_tri ? (uint32_t)(kKC * q) : 0u;
            if ((int)p.n0[q] >= p.npad) return false;
            p.nn[q] = (uint32_t)p.npad - p.n0[q];
            off += p.nn[q] * (kKC * 2);
        }
    }
    p.b_bytes = off;   // multiple of 2048 (nn multiple of 32, 64-byte rows)
    uint32_t hoff = 0;
    for (int q = 0; q < kMaxQ; ++q) {
        p.hoff[q] = hoff;
        hoff += (p.nn[q] / 2) * (kKC * 2);
    }
    p.hb_bytes = hoff;   // multiple of 1024 (nn / 2 multiple of 16)
    // the deepest rings that fit next to B (at least 2 stages)
    p.stages2 = 0;
    for (int s = kMaxStages2; s >= 2; --s) {
        p.stages2 = s;
        if (smem_bytes2(p) <= kSmemLimit) break;
        p.stages2 = 0;
    }
    p.stages = 0;
    for (int s = kMaxStages; s >= 2; --s) {
        p.stages = s;
        if (smem_bytes(p) <= kSmemLimit) break;
        p.stages = 0;
    }
    return p.stages >= 2 || p.stages2 >= 2;
}

// clusters of two of `fn` (`threads` a CTA) that fit on the device at once
// with this shared memory (0: none; cached per device, kernel and size)
int pair_clusters(const void* fn, int threads, size_t smem) {
    static std::mutex mu;
    static std::map<std::tuple<int, const void*, size_t>, int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_tuple(dev, fn, smem);
    const auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    cudaError_t e = allow_dynamic_smem(fn);
    int n = 0;
    if (e == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(2, 1, 1);
        cfg.blockDim = dim3(threads, 1, 1);
        cfg.dynamicSmemBytes = smem;
        if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) n = 0;
    }
    cudaGetLastError();
    cache[key] = n;
    return n;
}

const void* pair_kernel(bool vec) {
    return vec ? (const void*)rownorm_tc2_kernel<true, kPieceRows> : (const void*)rownorm_tc2_kernel<false, kPieceRows>;
}

// The TMA-fed kernel's converter layouts (groups x warps a group); the
// first is the default, LSK_ROWNORM_TMA_VARIANT=i selects another.
struct TmaVariant {
    const void* fn;
    int threads, groups;
    void (*launch)(int grid, size_t smem, cudaStream_t st, const RnParams& p, const uint8_t* img,
                   const CUtensorMap& tmA);
};
template <int G, int W>
TmaVariant tma_variant_of() {
    using T = TmaShape<G, W>;
    return {(const void*)rownorm_tma2_kernel<T>, T::kThreads, T::kGroups,
            [](int grid, size_t smem, cudaStream_t st, const RnParams& p, const uint8_t* img, const CUtensorMap& tmA) {
                rownorm_tma2_kernel<T><<<grid, T::kThreads, smem, st>>>(p, img, tmA);
            }};
}
const TmaVariant& tma_variant() {
    static const TmaVariant kVariants[] = {tma_variant_of<4, 4>(), tma_variant_of<8, 2>(), tma_variant_of<2, 4>(),
                                           tma_variant_of<3, 4>(), tma_variant_of<4, 2>(), tma_variant_of<3, 2>()};
    const char* v = getenv("LSK_ROWNORM_TMA_VARIANT");
    const int i = v ? atoi(v) : 0;
    return kVariants[(i >= 0 && i < (int)(sizeof(kVariants) / sizeof(kVariants[0]))) ? i : 0];
}

// The TF32 kernel: G one-warp relay groups, the ring G stages deep (the
// deepest of these that fits beside B; one group per stage, so a landed
// chunk never waits behind another chunk's hand-off).
template <int G>
TmaVariant tf32_variant_of() {
    using T = TmaShape<G, 1>;
    return {(const void*)rownorm_tma2_kernel<T, true>, T::kThreads, T::kGroups,
            [](int grid, size_t smem, cudaStream_t st, const RnParams& p, const uint8_t* img, const CUtensorMap& tmA) {
                rownorm_tma2_kernel<T, true><<<grid, T::kThreads, smem, st>>>(p, img, tmA);
            }};
}
const TmaVariant* tf32_variant(int stages2) {
    static const TmaVariant kByDepth[] = {tf32_variant_of<12>(), tf32_variant_of<9>(), tf32_variant_of<6>(),
                                          tf32_variant_of<4>(), tf32_variant_of<2>()};
    for (const TmaVariant& v : kByDepth)
        if (v.groups <= stages2) return &v;
    return nullptr;
}

// The TMA-fed pair form reads A through a tensor map of boxes 32 columns x
// 128 rows: rows must start on 16-byte boundaries, and the row count must
// fit the map's 32-bit coordinates.
bool tma_ok(const lsk_mat* A) {
    return A->d >= kKC && A->n >= 2 * kRows && A->n < ((int64_t)1 << 31) - 4 * kRows && A->ld % 4 == 0 &&
           ((uintptr_t)A->values & 15) == 0 && tc::encode_tiled() != nullptr;
}

bool make_tmap(const RnParams& p, CUtensorMap* m) {
    const tc::EncodeTiledFn fn = tc::encode_tiled();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)p.d, (cuuint64_t)p.n};
    const cuuint64_t strides[1] = {(cuuint64_t)p.lda * 4};
    const cuuint32_t box[2] = {(cuuint32_t)kKC, (cuuint32_t)kRows};
    const cuuint32_t elem[2] = {1, 1};
    // TF32 form: the copy engine rounds FP32 to the nearest TF32
    const CUtensorMapDataType ty = p.tf32 ? CU_TENSOR_MAP_DATA_TYPE_TFLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    return fn(m, ty, 2, const_cast<float*>(p.A), dims, strides, box, elem,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The form a launch takes: the CTA-pair form where B leaves the single-CTA
// ring short of its full depth and clusters of two fit (TMA-fed behind
// LSK_ROWNORM_TMA=1), else the single-CTA form.  The B image's layout follows
// from it, so the grouped image build asks the same question.
struct PairChoice {
    int ncl = 0;        // clusters of two (0: single-CTA form)
    bool tma = false;
    int stages2 = 0;    // the TMA form's ring (a multiple of its converter groups)
};
PairChoice choose_form(const lsk_mat* A, const RnParams& p, bool vec) {
    PairChoice pc;
    // LSK_ROWNORM_SINGLE_CTA=1 selects the single-CTA form (for testing it)
    const char* single = getenv("LSK_ROWNORM_SINGLE_CTA");
    const bool allow_pair = !(single && single[0] == '1');
    // the pair form pays for its cross-SM hand-offs only where B leaves the
    // single-CTA ring short of its full depth
    const bool want_pair = p.stages2 >= 2 && (p.stages < 2 || (allow_pair && p.stages < kMaxStages &&
                                                               p.stages2 > p.stages));
    // LSK_ROWNORM_TMA=1 feeds the pair form by TMA (measured slower at d = c =
    // 256: its in-place ring of 8 stages caps the bytes in flight)
    const char* tma_env = getenv("LSK_ROWNORM_TMA");
    bool use_tma = want_pair && (tma_env && tma_env[0] == '1') && tma_ok(A);
    const TmaVariant& tv = tma_variant();
    // converter group i takes the chunks (and so the stages) i mod groups: with
    // the ring a multiple of the group count, each stage belongs to one group,
    // which then sees every use of it in order (no wait a phase ahead)
    const int stages_tma = (p.stages2 / tv.groups) * tv.groups;
    use_tma = use_tma && stages_tma >= 2;
    RnParams q = p;
    if (use_tma) q.stages2 = stages_tma;
    const void* pfn = use_tma ? tv.fn : pair_kernel(vec);
    pc.ncl = want_pair ? pair_clusters(pfn, use_tma ? tv.threads : kThreads, smem_bytes2(q)) : 0;
    pc.tma = use_tma && pc.ncl > 0;
    pc.stages2 = q.stages2;
    return pc;
}

// The TF32 form: TMA-fed CTA pairs only, the ring a multiple of the
// converter groups; fills p (stages2, pair, tf32) and the clusters that fit.
bool tf32_plan(const lsk_mat* A, RnParams& p, int& ncl, const TmaVariant** tv_out = nullptr) {
    if (!tma_ok(A) || p.stages2 < 2) return false;
    const TmaVariant* tv = tf32_variant(p.stages2);
    if (!tv) return false;
    RnParams q = p;
    q.stages2 = tv->groups;
    q.pair = 1;
    q.tf32 = 1;
    ncl = pair_clusters(tv->fn, tv->threads, smem_bytes2(q));
    if (ncl <= 0) return false;
    p = q;
    if (tv_out) *tv_out = tv;
    return true;
}

}  // namespace

bool rownorms_tc_supported(const lsk_mat* A, int64_t c, int upper_tri, bool tf32) {
    RnParams p{};
    if (!make_plan(A, c, upper_tri, p)) return false;
    if (tf32) {
        int ncl = 0;
        return tf32_plan(A, p, ncl);
    }
    if (p.stages >= 2) return true;
    // only the CTA-pair form fits: it needs clusters of two on this device
    const bool vec = (p.d % 4 == 0) && (A->ld % 4 == 0) && (((uintptr_t)A->values & 15) == 0);
    return pair_clusters(pair_kernel(vec), kThreads, smem_bytes2(p)) > 0;
}

size_t rownorms_tc_workspace_bytes(const lsk_mat* A, int64_t c, int upper_tri) {
    RnParams p{};
    if (!make_plan(A, c, upper_tri, p)) return 0;
    return ws_round(2 * (size_t)p.b_bytes);
}

cudaError_t rownorms_tc_launch(const lsk_mat* A, const float* B, int64_t c, float alpha, float beta, int upper_tri,
                               float* x, void* ws, int* flag, int sm_count, cudaStream_t st, int min_tiles,
                               const uint8_t* img_ready, bool tf32) {
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
    const bool vec = (p.d % 4 == 0) && (A->ld % 4 == 0) && (((uintptr_t)A->values & 15) == 0);
    p.ntiles2 = (int)((A->n + 2 * kRows - 1) / (2 * kRows));
    const int kMinTiles0 = min_tiles > 0 ? min_tiles : 1;
    if (tf32) {
        int ncl = 0;
        const TmaVariant* tv = nullptr;
        if (!tf32_plan(A, p, ncl, &tv)) return cudaErrorNotSupported;
        LSK_PROF("rownorm_tc_prep", st) rownorm_tc_prep_kernel<<<64, 256, 0, st>>>(B, p, img);
        CUtensorMap tmA;
        if (!make_tmap(p, &tmA)) return cudaErrorNotSupported;
        const int want2 = (p.ntiles2 + kMinTiles0 - 1) / kMinTiles0;
        const int grid2 = 2 * (want2 < ncl ? want2 : ncl);
        LSK_PROF("rownorm_dense_tf32", st) tv->launch(grid2, smem_bytes2(p), st, p, img, tmA);
        return cudaGetLastError();
    }
    const PairChoice pc = choose_form(A, p, vec);
    const bool use_tma = pc.tma;
    const TmaVariant& tv = tma_variant();
    const int ncl = pc.ncl;
    if (use_tma) p.stages2 = pc.stages2;
    p.pair = ncl > 0 ? 1 : 0;
    if (!p.pair && p.stages < 2) return cudaErrorNotSupported;
    if (img_ready) img = const_cast<uint8_t*>(img_ready);   // built by rownorms_image_group_launch
    else LSK_PROF("rownorm_tc_prep", st) rownorm_tc_prep_kernel<<<64, 256, 0, st>>>(B, p, img);
    cudaError_t e;
    // CTAs (pairs) for at least min_tiles tiles each: a small problem then
    // leaves SMs to the problems on other streams (its per-CTA set-up -- TMEM,
    // the B image, the ring -- is paid over several tiles); a large one still
    // takes one persistent CTA per SM
    const int kMinTiles = min_tiles > 0 ? min_tiles : 1;
    if (p.pair) {
        const size_t smem2 = smem_bytes2(p);
        const int want2 = (p.ntiles2 + kMinTiles - 1) / kMinTiles;
        const int grid2 = 2 * (want2 < ncl ? want2 : ncl);
        if (use_tma) {
            CUtensorMap tmA;
            if (!make_tmap(p, &tmA)) return cudaErrorNotSupported;
            LSK_PROF("rownorm_dense_tc", st) tv.launch(grid2, smem2, st, p, img, tmA);
        } else if (vec) {
            LSK_PROF("rownorm_dense_tc", st)
                rownorm_tc2_kernel<true, kPieceRows><<<grid2, kThreads, smem2, st>>>(p, img);
        } else {
            LSK_PROF("rownorm_dense_tc", st)
                rownorm_tc2_kernel<false, kPieceRows><<<grid2, kThreads, smem2, st>>>(p, img);
        }
        return cudaGetLastError();
    }
    const size_t smem = smem_bytes(p);
    const int want = (p.ntiles + kMinTiles - 1) / kMinTiles;
    const int grid = want < sm_count ? want : sm_count;
    if (vec) {
        e = allow_dynamic_smem(rownorm_tc_kernel<true>);
        if (e != cudaSuccess) return e;
        LSK_PROF("rownorm_dense_tc", st) rownorm_tc_kernel<true><<<grid, kThreads, smem, st>>>(p, img);
    } else {
        e = allow_dynamic_smem(rownorm_tc_kernel<false>);
        if (e != cudaSuccess) return e;
        LSK_PROF("rownorm_dense_tc", st) rownorm_tc_kernel<false><<<grid, kThreads, smem, st>>>(p, img);
    }
    return cudaGetLastError();
}

void rownorms_image_group_build(const std::vector<RnImageJob>& jobs, HostTable& t, RnImageGroup& g) {
    std::vector<RnPrepJob> js;
    std::vector<int> blocks, off;
    for (const RnImageJob& j : jobs) {
        RnPrepJob r{};
        if (!make_plan(&j.A, j.c, j.upper_tri, r.p)) continue;
        const bool vec = (r.p.d % 4 == 0) && (j.A.ld % 4 == 0) && (((uintptr_t)j.A.values & 15) == 0);
        r.p.pair = choose_form(&j.A, r.p, vec).ncl > 0 ? 1 : 0;
        r.B = j.B;
        r.img = j.img;
        js.push_back(r);
        blocks.push_back(kPrepBlocks);
    }
    g.count = (int)js.size();
    g.blocks = group_offsets(blocks, off);
    g.params_off = t.put(js.data(), js.size());
    g.off_off = t.put(off.data(), off.size());
}

cudaError_t rownorms_image_group_launch(const RnImageGroup& g, const unsigned char* table, cudaStream_t st) {
    if (g.count == 0) return cudaSuccess;
    LSK_PROF("rownorm_tc_prep", st) rownorm_tc_prep_grouped_kernel<<<g.blocks, 256, 0, st>>>(
        reinterpret_cast<const RnPrepJob*>(table + g.params_off), reinterpret_cast<const int*>(table + g.off_off),
        g.count);
    return cudaGetLastError();
}
