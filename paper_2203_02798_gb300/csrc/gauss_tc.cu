// gauss_tc.cu -- Gaussian stage GSA = G * SA on tcgen05 tensor cores.
//
// BF16 mode: G (k x r) is exactly representable in bfloat16 by definition of
// the mode (the bf16 rounding of z / sqrt(k)); SA is split into bf16 hi + lo.
//     GSA = G SA_hi + G SA_lo       (FP32 accumulation in tensor memory)
// FP32 mode (Terms<3>): G and SA each as three bf16 terms, six products.
// A block owns one 256-row band of G (two 128-row MMA tiles) and one slice
// of the r dimension; the k x d partials of the slices are added afterwards
// in a fixed order with a compensated FP32 sum (deterministic).  Per 32-column
// chunk of the slice, each of the 16 worker warps, on its own:
//   - loads rows 2w, 2w+1 of the chunk's 32 rows of SA (16-byte loads);
//   - draws its 64 items of the 256 x 32 G chunk (Philox + Box-Muller, 4 rows
//     per draw, two independent draws per thread) into bf16 words;
//   - claims the ring stage (the MMAs of its previous use are done), writes
//     its G words into the K-major operand tiles and its SA rows, split, into
//     MN-major tiles (SA's rows are the MMA's K, its columns N: no transpose),
//     and arrives;
// lane 0 of warp 16 issues the MMAs (2 K-steps x products x 2 tiles) once all
// 16 warps have arrived.  Drawing G (~90 instructions per entry) is the bound,
// so the workers share no barrier: a warp still drawing does not hold the
// others up, and a warp may run a whole ring ahead.
#include "tc_common.cuh"

namespace {

constexpr int kM = 256;            // rows of G per block (two 128-row MMA tiles sharing each SA chunk)
constexpr int kMT = 128;           // rows per MMA tile
constexpr int kKC = 32;            // r-columns per chunk (64-byte swizzle rows)
constexpr int kWorkers = 16;       // worker warps (also the epilogue, warps 0-7)
constexpr int kMmaWarp = kWorkers;
constexpr int kThreads = (kWorkers + 1) * 32;
constexpr int kWorkerThreads = kWorkers * 32;
constexpr int kMaxN = 256;
// T = 1: the BF16 mode (G exact in bf16, SA as bf16 hi + lo; 2 products a
// K-step).  T = 3: the FP32 mode -- G and SA each split into three bf16 terms
// (x = x1 + x2 + x3 exactly: 3 x 8 significant bits), and the six products
// of order down to 2^-16 accumulated in FP32 (the dropped G2 S3, G3 S2, G3 S3
// are below 2^-23 of |G||SA|): FP32 accuracy on the BF16 tensor pipe.
template <int T>
struct Terms {
    static constexpr int kA = T;                    // G terms
    static constexpr int kB = T == 1 ? 2 : 3;       // SA terms
    static constexpr int kStages = T == 1 ? 4 : 2;
    static constexpr int kProducts = T == 1 ? 2 : 6;
};
constexpr size_t kSmemLimit = 232448;

struct GtParams {
    const float* SA;
    float* part;       // [slices][k][d]
    int64_t r, k;
    int d, npad;
    int64_t kslice;    // r-columns per slice (multiple of kKC)
    int tiles_m, slices;
    uint32_t k0, k1;
    float scale;
    int* flag;
    float* out;        // GSA, k x d (read by the reduction)
    // compacted sketch: SA's row c is bucket idx[c] (its column of G), *rcount
    // rows in all; r bounds *rcount (null: rows are buckets 0 .. r - 1)
    const uint32_t* idx;
    const uint32_t* rcount;
};

__host__ __device__ constexpr uint32_t a_bytes() { return kM * kKC * 2; }               // 16 KB (two tiles) a term
// SA's terms are MN-major (SA's rows are K, its columns N): 128-byte-swizzled
// atoms of 8 rows x 64 columns, 1 KB apart along the columns (nbn of them)
// and nbn KB apart along the rows
__host__ __device__ inline uint32_t b_atoms(int npad) { return (uint32_t)(npad + 63) / 64; }
__host__ __device__ inline uint32_t b_sbo(int npad) { return b_atoms(npad) * 1024u; }
__host__ __device__ inline uint32_t b_bytes(int npad) { return b_sbo(npad) * (kKC / 8); }   // a term
template <int T>
__host__ __device__ inline uint32_t stage_bytes(int npad) {
    return Terms<T>::kA * a_bytes() + Terms<T>::kB * b_bytes(npad);
}
template <int T>
__host__ __device__ inline size_t smem_of(int npad) {
    return (size_t)Terms<T>::kStages * stage_bytes<T>(npad) + 1024 + 128;
}

// x = t1 + t2 + t3 to 24 significant bits (each term the bf16 rounding of the
// remainder): three bf16x2 words for the pair (a, b), a in the low halves.
__device__ __forceinline__ void split3_bf16x2(float a, float b, uint32_t& w1, uint32_t& w2, uint32_t& w3) {
    uint32_t h;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(b), "f"(a));
    const float ra = a - __uint_as_float(h << 16), rb = b - __uint_as_float(h & 0xFFFF0000u);
    uint32_t m;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(m) : "f"(rb), "f"(ra));
    const float sa = ra - __uint_as_float(m << 16), sb = rb - __uint_as_float(m & 0xFFFF0000u);
    uint32_t l;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(l) : "f"(sb), "f"(sa));
    w1 = h;
    w2 = m;
    w3 = l;
}


// One block: row tile and r-slice number `blk` of problem p.
template <int T>
__device__ __forceinline__ void gauss_tc_body(const GtParams& p, const int blk) {
    constexpr int kStages = Terms<T>::kStages, kA = Terms<T>::kA, kB = Terms<T>::kB;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
    const uint32_t sbytes = stage_bytes<T>(p.npad);
    uint8_t* stages = smem;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kStages * sbytes);
    uint64_t* full = bars;              // [kStages] (kWorkers arrivals)
    uint64_t* empty = bars + kStages;   // [kStages] (MMA commit)
    uint64_t* done = bars + 2 * kStages;  // accumulator complete   (MMA commit)
    uint64_t* fin = done + 1;             // every MMA complete     (MMA commit)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mt = blk % p.tiles_m, slice = blk / p.tiles_m;
    const int64_t j0 = (int64_t)mt * kM;
    const int64_t c_begin = (int64_t)slice * p.kslice;
    const int64_t r_rows = p.rcount ? min(p.r, (int64_t)__ldg(p.rcount)) : p.r;   // rows of SA
    const int64_t c_end = min(r_rows, c_begin + p.kslice);
    const int nchunks = c_end > c_begin ? (int)((c_end - c_begin + kKC - 1) / kKC) : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            tc::mbar_init(full + s, kWorkers);
            tc::mbar_init(empty + s, 1);
        }
        tc::mbar_init(done, 1);
        tc::mbar_init(fin, 1);
        *abort = 0;
        tc::fence_mbar_init();
    }
    // two accumulators (one per MMA tile) at columns 0 and npad
    const uint32_t tcols = p.npad <= 16 ? 32u : p.npad <= 32 ? 64u : p.npad <= 64 ? 128u : p.npad <= 128 ? 256u : 512u;
    if (warp == kMmaWarp) {
        tc::tmem_alloc(tmem_slot, tcols);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp < kWorkers) {
        // Each worker warp works alone: per chunk it loads SA rows 2 w, 2 w + 1
        // of the chunk, draws its 64 items of G, claims the stage, writes both
        // and arrives; the warps are held together only by the stage ring.
        const int wt = threadIdx.x;   // 0 .. kWorkerThreads - 1
        constexpr int H = (kMaxN + 127) / 128;          // 128-column halves of a row of SA
        const int nh = (p.npad + 127) / 128;
        const bool vec = (p.d % 4) == 0;
        bool ok = true;
        for (int g = 0; g < nchunks; ++g) {
            const int s = g % kStages;
            const int64_t c0 = c_begin + (int64_t)g * kKC;
            // (1) SA rows c0 + 2 w + e, lane: columns 4 lane + 128 h .. + 3
            float4 sa[2][H];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int64_t c = c0 + 2 * warp + e;
#pragma unroll
                for (int h = 0; h < H; ++h) {
                    sa[e][h] = make_float4(0.f, 0.f, 0.f, 0.f);
                    const int n = 4 * lane + 128 * h;
                    if (h < nh && c < c_end && n < p.d) {
                        const float* src = p.SA + c * p.d + n;
                        if (vec) {
                            sa[e][h] = __ldg(reinterpret_cast<const float4*>(src));
                        } else {
                            sa[e][h].x = __ldg(src);
                            sa[e][h].y = n + 1 < p.d ? __ldg(src + 1) : 0.f;
                            sa[e][h].z = n + 2 < p.d ? __ldg(src + 2) : 0.f;
                            sa[e][h].w = n + 3 < p.d ? __ldg(src + 3) : 0.f;
                        }
                    }
                }
            }
            // (2) G chunk: item = wt + 512 i -> (row quad gq = item / 16, column pair cp = item % 16),
            //     64 x 16 items = the 256 x 32 chunk, two independent draws per worker thread
            static_assert(2 * kWorkerThreads == (kM / 4) * (kKC / 2), "two G items per worker thread");
            uint32_t gw[2][4][kA];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int item = wt + kWorkerThreads * i;
                const int gq = item >> 4, cp = item & 15;
                const int64_t jq = j0 + 4 * gq;
                const int64_t c = c0 + 2 * cp;
                float4 z0 = make_float4(0.f, 0.f, 0.f, 0.f), z1 = z0;
                if (jq < p.k) {
                    // column of G = the row's bucket
                    if (c < c_end)
                        z0 = gauss4((uint64_t)(p.idx ? __ldg(p.idx + c) : c), (uint32_t)(jq >> 2), p.k0, p.k1);
                    if (c + 1 < c_end)
                        z1 = gauss4((uint64_t)(p.idx ? __ldg(p.idx + c + 1) : c + 1), (uint32_t)(jq >> 2), p.k0,
                                    p.k1);
                }
                const float a0[4] = {z0.x, z0.y, z0.z, z0.w}, a1[4] = {z1.x, z1.y, z1.z, z1.w};
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const bool rowok = jq + t < p.k;
                    const float g0 = rowok ? a0[t] * p.scale : 0.f, g1 = rowok ? a1[t] * p.scale : 0.f;
                    if constexpr (kA == 1) {
                        const __nv_bfloat162 h = __floats2bfloat162_rn(g0, g1);
                        gw[i][t][0] = *reinterpret_cast<const uint32_t*>(&h);
                    } else {
                        split3_bf16x2(g0, g1, gw[i][t][0], gw[i][t][1], gw[i][t][2]);
                    }
                }
            }
            // (3) claim the stage (the MMAs of its previous use are done)
            int okw = 1;
            if (lane == 0) okw = tc::mbar_wait(empty + s, ((uint32_t)(g / kStages) & 1u) ^ 1u, abort) ? 1 : 0;
            if (!__shfl_sync(0xffffffffu, okw, 0)) {
                ok = false;
                break;
            }
            uint8_t* st = stages + s * sbytes;
            // (4) G words: row 4 gq + t, columns 2cp, 2cp+1 (rows 128.. are the second tile,
            //     8 KB further on: sw64 offsets continue linearly in the row)
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int item = wt + kWorkerThreads * i;
                const int gq = item >> 4, cp = item & 15;
#pragma unroll
                for (int t = 0; t < 4; ++t)
#pragma unroll
                    for (int a = 0; a < kA; ++a)
                        *reinterpret_cast<uint32_t*>(st + a * a_bytes() + tc::sw64_offset(4 * gq + t, 2 * cp)) =
                            gw[i][t][a];
            }
            // (5) SA rows split into the kB MN-major terms: columns 4 lane .. + 3 of
            //     K-row kr go to atom (col / 64, kr / 8), row kr % 8, 16-byte chunk
            //     ((col % 64) / 8) ^ (kr % 8), bytes 8 (lane % 2) .. + 7
            uint8_t* b0 = st + kA * a_bytes();
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const uint32_t kr = 2u * (uint32_t)warp + (uint32_t)e, rr = kr & 7u;
#pragma unroll
                for (int h = 0; h < H; ++h) {
                    if (h >= nh) break;
                    const uint32_t col = 4u * (uint32_t)lane + 128u * h;
                    if (col >= 64u * b_atoms(p.npad)) continue;   // past the term's atoms (zeros)
                    const uint32_t off = (col >> 6) * 1024u + (kr >> 3) * b_sbo(p.npad) + rr * 128u +
                                         (((((col & 63u) >> 3) ^ rr) & 7u) << 4) + (col & 7u) * 2u;
                    const float4 v = sa[e][h];
                    if constexpr (kB == 2) {
                        uint2 hi, lo;
                        tc::split_bf16x2(v.x, v.y, hi.x, lo.x);
                        tc::split_bf16x2(v.z, v.w, hi.y, lo.y);
                        *reinterpret_cast<uint2*>(b0 + off) = hi;
                        *reinterpret_cast<uint2*>(b0 + b_bytes(p.npad) + off) = lo;
                    } else {
                        uint2 w1, w2, w3;
                        split3_bf16x2(v.x, v.y, w1.x, w2.x, w3.x);
                        split3_bf16x2(v.z, v.w, w1.y, w2.y, w3.y);
                        *reinterpret_cast<uint2*>(b0 + off) = w1;
                        *reinterpret_cast<uint2*>(b0 + b_bytes(p.npad) + off) = w2;
                        *reinterpret_cast<uint2*>(b0 + 2 * b_bytes(p.npad) + off) = w3;
                    }
                }
            }
            tc::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(full + s);
        }
        // epilogue: warps 0-3 read tile 0 (columns 0..npad), warps 4-7 tile 1 (columns npad..2 npad);
        // a warp may only read the TMEM lanes 32 (warp % 4) .. + 31
        if (warp < 8 && nchunks == 0) {
            // a slice past the compacted sketch's rows: its partial is zero
            const int tile = warp >> 2, wq = warp & 3;
            const int64_t j = j0 + tile * kMT + wq * 32 + lane;
            if (j < p.k) {
                float* dst = p.part + ((int64_t)slice * p.k + j) * p.d;
                for (int col = 0; col < p.d; ++col) dst[col] = 0.f;
            }
        } else if (warp < 8) {
            int okw = 0;
            if (lane == 0) okw = (ok && tc::mbar_wait(done, 0, abort)) ? 1 : 0;
            okw = __shfl_sync(0xffffffffu, okw, 0);
            if (okw) {
                tc::fence_after_sync();
                const int tile = warp >> 2, wq = warp & 3;
                const int64_t j = j0 + tile * kMT + wq * 32 + lane;
                float* dst = p.part + ((int64_t)slice * p.k + j) * p.d;
                for (int col = 0; col < p.npad; col += 32) {
                    uint32_t v[32];
                    tc::tmem_ld_32x32b_x32(tmem + ((uint32_t)(wq * 32) << 16) + (uint32_t)(tile * p.npad + col), v);
                    tc::tmem_ld_wait();
                    if (j < p.k) {
#pragma unroll
                        for (int e = 0; e < 32; ++e)
                            if (col + e < p.d) dst[col + e] = __uint_as_float(v[e]);
                    }
                }
            }
        }
    } else if (warp == kMmaWarp) {
        if (lane == 0) {
            const uint32_t base = tc::smem_u32(stages);
            // A (G) K-major, B (SA) MN-major
            const uint32_t idesc = tc::idesc_bf16_f32(128, (uint32_t)p.npad) | (1u << 16);
            bool okm = true;
            for (int g = 0; g < nchunks; ++g) {
                const int s = g % kStages;
                if (!tc::mbar_wait(full + s, (uint32_t)(g / kStages) & 1u, abort)) {
                    okm = false;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t a = base + s * sbytes, b = a + kA * a_bytes();
                // (A term, SA term) of each product: BF16 mode G (SA_hi + SA_lo);
                // FP32 mode the six products of order down to 2^-16
                constexpr int kPA[6] = {0, 0, 1, 0, 1, 2}, kPB[6] = {0, 1, 0, 2, 1, 0};
#pragma unroll
                for (int kk = 0; kk < kKC / 16; ++kk) {
                    const uint32_t ko = 32u * kk;
#pragma unroll
                    for (int t = 0; t < kM / kMT; ++t) {
                        const uint32_t dt = tmem + (uint32_t)(t * p.npad);
#pragma unroll
                        for (int q = 0; q < Terms<T>::kProducts; ++q) {
                            const uint32_t at = a + (uint32_t)kPA[q] * a_bytes() + (uint32_t)t * (kMT * kKC * 2) + ko;
                            const uint32_t bt = b + (uint32_t)kPB[q] * b_bytes(p.npad) + 2u * b_sbo(p.npad) * kk;
                            tc::mma_bf16(dt, tc::desc_sw64_kmajor(at), tc::desc_sw128_mnmajor(bt, 1024u, b_sbo(p.npad)),
                                         idesc, (g | kk | q) != 0);
                        }
                    }
                }
                tc::mma_commit(empty + s);
            }
            if (okm && nchunks > 0) tc::mma_commit(done);
            tc::mma_commit(fin);
            volatile int never = 0;
            tc::mbar_wait(fin, 0, &never);
        }
        __syncwarp();
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, tcols);
    }
    if (threadIdx.x == 0 && *abort) set_flag(p.flag, LSK_FLAG_TIMEOUT);
}

template <int T>
__global__ void __launch_bounds__(kThreads, 1) gauss_tc_kernel(const GtParams p) { gauss_tc_body<T>(p, blockIdx.x); }

// Grouped: the blocks of many problems in one grid.
__global__ void __launch_bounds__(kThreads, 1) gauss_tc_grouped_kernel(const GtParams* __restrict__ ps,
                                                                       const int* __restrict__ off, int count) {
    const int g = group_of(off, count, blockIdx.x);
    gauss_tc_body<1>(ps[g], (int)blockIdx.x - __ldg(off + g));
}

struct Plan {
    int npad, tiles_m, slices;
    int64_t kslice;
    size_t smem;
};

bool make_plan(int64_t r, int64_t d, int64_t k, int sm_count, Plan& P, int terms = 1) {
    if (d < 1 || d > kMaxN || k < 1 || r < 1) return false;
    P.npad = (int)((d + 31) / 32) * 32;
    P.tiles_m = (int)((k + kM - 1) / kM);
    int64_t want = ((int64_t)sm_count + P.tiles_m - 1) / P.tiles_m;   // one wave of blocks
    const int64_t max_slices = (r + 8 * kKC - 1) / (8 * kKC);   // >= 8 chunks per block
    if (want > max_slices) want = max_slices;
    if (want < 1) want = 1;
    int64_t ks = (r + want - 1) / want;
    ks = ((ks + kKC - 1) / kKC) * kKC;
    P.kslice = ks;
    P.slices = (int)((r + ks - 1) / ks);
    P.smem = terms == 3 ? smem_of<3>(P.npad) : smem_of<1>(P.npad);
    return P.smem <= kSmemLimit;
}

__device__ __forceinline__ void reduce_body(const float* __restrict__ part, int slices, int64_t len,
                                            float* __restrict__ out, int blk, int nblk) {
    const int64_t stride = (int64_t)nblk * blockDim.x;
    for (int64_t e = (int64_t)blk * blockDim.x + threadIdx.x; e < len; e += stride) {
        // compensated FP32 sum (Neumaier) in slice order: about two roundings
        // of error in total, without FP64 adds (scarce on this part)
        float s = 0.f, c = 0.f;
        for (int z = 0; z < slices; ++z) {
            const float x = part[(int64_t)z * len + e];
            const float t = s + x;
            c += (fabsf(s) >= fabsf(x)) ? (s - t) + x : (x - t) + s;
            s = t;
        }
        out[e] = s + c;
    }
}
__global__ void gauss_tc_reduce_kernel(const float* __restrict__ part, int slices, int64_t len,
                                       float* __restrict__ out) {
    reduce_body(part, slices, len, out, blockIdx.x, gridDim.x);
}
__global__ void gauss_tc_reduce_grouped_kernel(const GtParams* __restrict__ ps, const int* __restrict__ roff,
                                               int count) {
    const int g = group_of(roff, count, blockIdx.x);
    const int b0 = __ldg(roff + g), b1 = __ldg(roff + g + 1);
    const GtParams& p = ps[g];
    reduce_body(p.part, p.slices, p.k * p.d, p.out, (int)blockIdx.x - b0, b1 - b0);
}

// Grouped plan: the parallelism comes from the many problems, so a block
// takes a longer slice (>= slice_chunks chunks, 128 by default; the batch
// autotuner may pick another) and fewer partials are written.
void plan_grouped(int64_t r, int64_t d, int64_t k, Plan& P, int slice_chunks) {
    P.npad = (int)((d + 31) / 32) * 32;
    P.tiles_m = (int)((k + kM - 1) / kM);
    if (slice_chunks < 1) slice_chunks = 128;
    const int64_t want = (r + (int64_t)slice_chunks * kKC - 1) / ((int64_t)slice_chunks * kKC);
    int64_t ks = (r + want - 1) / want;
    ks = ((ks + kKC - 1) / kKC) * kKC;
    P.kslice = ks;
    P.slices = (int)((r + ks - 1) / ks);
    P.smem = smem_of<1>(P.npad);
}

constexpr int kReduceBlockCap = 64;

}  // namespace

bool gauss_tc_supported(int64_t r, int64_t d, int64_t k, int terms) {
    Plan P;
    return make_plan(r, d, k, 152, P, terms);
}

size_t gauss_tc_workspace_bytes(int64_t r, int64_t d, int64_t k, int sm_count, int terms) {
    Plan P;
    if (!make_plan(r, d, k, sm_count, P, terms)) return 0;
    return ws_round((size_t)P.slices * k * d * 4);
}

cudaError_t gauss_tc_launch(const float* SA, int64_t r, int64_t d, int64_t k, uint64_t seed, float* GSA, void* ws,
                            int sm_count, cudaStream_t st, int terms) {
    Plan P;
    if (!make_plan(r, d, k, sm_count, P, terms)) return cudaErrorNotSupported;
    GtParams p;
    p.SA = SA;
    p.part = (float*)ws;
    p.r = r;
    p.k = k;
    p.d = (int)d;
    p.npad = P.npad;
    p.kslice = P.kslice;
    p.tiles_m = P.tiles_m;
    p.slices = P.slices;
    p.k0 = (uint32_t)seed;
    p.k1 = (uint32_t)(seed >> 32);
    p.scale = (float)(1.0 / sqrt((double)k));
    p.flag = nullptr;
    p.out = GSA;
    p.idx = nullptr;
    p.rcount = nullptr;
    cudaError_t e;
    if (terms == 3) {
        e = allow_dynamic_smem(gauss_tc_kernel<3>);
        if (e != cudaSuccess) return e;
        LSK_PROF("gauss_tc_fp32", st) gauss_tc_kernel<3><<<P.tiles_m * P.slices, kThreads, P.smem, st>>>(p);
    } else {
        e = allow_dynamic_smem(gauss_tc_kernel<1>);
        if (e != cudaSuccess) return e;
        LSK_PROF("gauss_tc", st) gauss_tc_kernel<1><<<P.tiles_m * P.slices, kThreads, P.smem, st>>>(p);
    }
    const int64_t len = k * d;
    int64_t g = (len + 255) / 256;
    if (g > 8 * (int64_t)sm_count) g = 8 * (int64_t)sm_count;
    LSK_PROF("gauss_reduce", st) gauss_tc_reduce_kernel<<<(unsigned)g, 256, 0, st>>>(p.part, P.slices, len, GSA);
    return cudaGetLastError();
}

// The slice-order compensated sum of `slices` partials of len floats each
// (used by the fused CountSketch + Gaussian kernel as well).
cudaError_t gauss_tc_reduce_launch(const float* part, int slices, int64_t len, float* out, int sm_count,
                                   cudaStream_t st) {
    if (len <= 0) return cudaSuccess;
    int64_t g = (len + 255) / 256;
    if (g > 8 * (int64_t)sm_count) g = 8 * (int64_t)sm_count;
    LSK_PROF("gauss_reduce", st) gauss_tc_reduce_kernel<<<(unsigned)g, 256, 0, st>>>(part, slices, len, out);
    return cudaGetLastError();
}

size_t gauss_group_part_bytes(int64_t r, int64_t d, int64_t k, int slice_chunks) {
    Plan P;
    plan_grouped(r, d, k, P, slice_chunks);
    return ws_round((size_t)P.slices * k * d * 4);
}

void gauss_group_build(const std::vector<GaussJob>& jobs, HostTable& t, GaussGroup& g) {
    std::vector<GtParams> ps(jobs.size());
    std::vector<int> blocks(jobs.size()), rblocks(jobs.size()), off, roff;
    g.smem = 0;
    for (size_t i = 0; i < jobs.size(); ++i) {
        const GaussJob& j = jobs[i];
        Plan P;
        plan_grouped(j.r, j.d, j.k, P, j.slice_chunks);
        GtParams& p = ps[i];
        p.SA = j.SA;
        p.part = j.part;
        p.r = j.r;
        p.k = j.k;
        p.d = (int)j.d;
        p.npad = P.npad;
        p.kslice = P.kslice;
        p.tiles_m = P.tiles_m;
        p.slices = P.slices;
        p.k0 = (uint32_t)j.seed;
        p.k1 = (uint32_t)(j.seed >> 32);
        p.scale = (float)(1.0 / sqrt((double)j.k));
        p.flag = nullptr;
        p.out = j.GSA;
        p.idx = j.idx;
        p.rcount = j.rcount;
        blocks[i] = P.tiles_m * P.slices;
        const int64_t rb = (j.k * j.d + 255) / 256;
        rblocks[i] = (int)(rb < kReduceBlockCap ? rb : kReduceBlockCap);
        if (P.smem > g.smem) g.smem = P.smem;
    }
    g.count = (int)jobs.size();
    g.blocks = group_offsets(blocks, off);
    g.rblocks = group_offsets(rblocks, roff);
    g.params_off = t.put(ps.data(), ps.size());
    g.off_off = t.put(off.data(), off.size());
    g.roff_off = t.put(roff.data(), roff.size());
}

cudaError_t gauss_group_launch(const GaussGroup& g, const unsigned char* table, cudaStream_t st) {
    if (g.count == 0) return cudaSuccess;
    const GtParams* ps = reinterpret_cast<const GtParams*>(table + g.params_off);
    const int* off = reinterpret_cast<const int*>(table + g.off_off);
    const int* roff = reinterpret_cast<const int*>(table + g.roff_off);
    cudaError_t e = allow_dynamic_smem(gauss_tc_grouped_kernel);
    if (e != cudaSuccess) return e;
    LSK_PROF("gauss_tc_grouped", st) gauss_tc_grouped_kernel<<<g.blocks, kThreads, g.smem, st>>>(ps, off, g.count);
    LSK_PROF("gauss_reduce_grouped", st) gauss_tc_reduce_grouped_kernel<<<g.rblocks, 256, 0, st>>>(ps, roff, g.count);
    return cudaGetLastError();
}
