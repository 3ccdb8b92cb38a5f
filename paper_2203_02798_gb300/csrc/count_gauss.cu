// count_gauss.cu -- the fused CountSketch + Gaussian stage: GSA = G (S A) in
// one pass over A, with S A never written to HBM.
//
// Alg. 3 forms the sketch in blocks of r: B = S_i A for one block of rows of
// S, then C += G_i B with a fresh Gaussian block G_i, so that only one block
// of S A exists at a time.  Here a block is 32 buckets (one K-chunk of the
// tensor-core product) and it lives in shared memory only.  A cluster of two
// CTAs (a tcgen05 CTA pair) owns one slice of the buckets and the whole
// k x d product of that slice:
//   - producer warp: copies the rows of A bucket by bucket (the order of the
//     CountSketch permutation, steps 1-3 of countsketch.cu) into a ring of
//     row slots with 16-byte asynchronous copies (cp.async, one per lane and
//     row) -- each CTA its half of the columns -- and writes each row's sign
//     beside it;
//   - 4 summing warps: walk the ring in order, add every row (with its sign)
//     to the open bucket's sum (one column per lane), and when a bucket closes
//     write its sum as bf16 hi + lo into the K-major B operand of the chunk;
//   - 8 worker warps: draw this CTA's rows of the chunk's columns of G
//     (the Gaussian stage's Philox + Box-Muller draws, bf16) into the A operand;
//   - the even CTA's MMA thread: M = 256 pair MMAs, G rows [0, 128) of each
//     256-row set from the even CTA and [128, 256) from the odd one, B's first
//     N / 2 = d_pad / 2 rows (S A columns) from the even CTA and the rest from
//     the odd one; each CTA's TMEM holds its 128 rows of every set, so the pair
//     keeps the whole 512 x 256 FP32 accumulator (2 x 512 columns);
//   - the worker warps then copy the accumulator out as the slice's partial,
//     and the partials are summed in slice order (compensated FP32).
// Every wait is bounded (1 s); a timeout sets LSK_FLAG_TIMEOUT and the copies
// in flight are waited for before the CTA leaves.
#include "tc_common.cuh"
#include "count_gauss.cuh"

#include <map>
#include <mutex>
#include <tuple>

namespace {

constexpr int kKC = 32;              // buckets per chunk (one K-major 64-byte swizzle row)
constexpr int kSetRows = 256;        // rows of G per pair MMA (M = 256)
constexpr int kHalfRows = 128;       // ... of which each CTA holds 128
constexpr int kMaxSets = 2;          // k <= 512
constexpr int kWorkers = 8;          // G-drawing warps 0..7 (also the epilogue)
constexpr int kWorkerThreads = kWorkers * 32;
constexpr int kCons0 = kWorkers;     // summing warps 8..11
constexpr int kCons = 4;
constexpr int kProdWarp = kCons0 + kCons;   // 12
constexpr int kMmaWarp = kProdWarp + 1;     // 13
constexpr int kThreads = (kMmaWarp + 1) * 32;
constexpr int kStages = 3;
constexpr int kGroupRows = 8;        // ring rows per barrier
constexpr int kGroups = 24;
constexpr int kRing = kGroups * kGroupRows;   // row slots per CTA
constexpr size_t kSmemLimit = 232448;

static_assert(kCons * 32 >= 128, "the summing warps cover a 128-column half");
static_assert(2 * kMaxSets * kWorkerThreads == kMaxSets * 32 * 16, "two G items per thread and set");

struct CgParams {
    const float* A;
    int64_t lda;
    const uint32_t* off;    // bucket -> first position in perm (r + 1 entries)
    const uint32_t* perm;   // row | sign << 31, grouped by bucket
    float* part;            // [slices][k][d]
    int64_t r, k;
    int d, npad, hw, nsets;
    int64_t kslice;         // buckets per slice (multiple of kKC)
    int slices;
    uint32_t k0, k1;
    float scale;
    uint32_t tcols;
    int* flag;
};

__host__ __device__ constexpr uint32_t a_bytes() { return kMaxSets * kHalfRows * kKC * 2; }   // 16 KB
__host__ __device__ inline uint32_t b_bytes(int hw) { return (uint32_t)hw * kKC * 2; }        // hi or lo
__host__ __device__ inline uint32_t stage_bytes(int hw) { return a_bytes() + 2 * b_bytes(hw); }
inline size_t smem_bytes(int hw) {
    return 1024 + (size_t)kStages * stage_bytes(hw) + (size_t)kRing * hw * 4 + (size_t)kRing * 4 +
           (size_t)(2 * kStages + 2 * kGroups + 2) * 8 + 16;
}

// 16 bytes global -> shared, asynchronous, cached in L2 only (both addresses
// 16-byte aligned)
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_u32(dst)), "l"(src) : "memory");
}
// one arrival on `bar` once every cp.async this thread has issued so far has
// landed (counted in the barrier's expected arrivals)
__device__ __forceinline__ void cp_async_arrive(uint64_t* bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void arrive_even(uint64_t* bar, uint32_t rank) {
    if (rank == 0) tc::mbar_arrive(bar);
    else tc::mbar_arrive_cluster(bar, 0);
}
// x as bf16 hi + lo at element (n, k) of the K-major hi / lo tiles
__device__ __forceinline__ void store_split(uint8_t* bh, uint32_t bbytes, int n, int k, float x) {
    uint32_t h, l;
    tc::split_bf16x2(x, 0.f, h, l);
    const uint32_t o = tc::sw64_offset((uint32_t)n, (uint32_t)k);
    *reinterpret_cast<uint16_t*>(bh + o) = (uint16_t)(h & 0xFFFFu);
    *reinterpret_cast<uint16_t*>(bh + bbytes + o) = (uint16_t)(l & 0xFFFFu);
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1) count_gauss_kernel(const CgParams p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
    const uint32_t rank = tc::cluster_ctarank();
    const int slice = (int)tc::cluster_id_x();
    const uint32_t sbytes = stage_bytes(p.hw), bbytes = b_bytes(p.hw);
    uint8_t* stages = smem;
    float* ring = reinterpret_cast<float*>(smem + kStages * sbytes);   // kRing slots of hw floats
    float* sgn = ring + kRing * p.hw;                                   // kRing signs
    uint64_t* bars = reinterpret_cast<uint64_t*>(sgn + kRing);
    uint64_t* fullS = bars;                  // [kStages] even CTA: chunk operands written in both CTAs
    uint64_t* emptyS = fullS + kStages;      // [kStages] chunk consumed (multicast commit)
    uint64_t* fullR = emptyS + kStages;      // [kGroups] ring group landed (copy bytes)
    uint64_t* emptyR = fullR + kGroups;      // [kGroups] ring group read by the summing warps
    uint64_t* done = emptyR + kGroups;       // accumulator complete (multicast commit)
    uint64_t* fin = done + 1;                // every MMA complete (multicast commit)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t c_begin = (int64_t)slice * p.kslice;
    const int64_t c_end = min(p.r, c_begin + p.kslice);
    const int nchunks = c_begin < c_end ? (int)((c_end - c_begin + kKC - 1) / kKC) : 0;
    const uint32_t T0 = c_begin < c_end ? __ldg(p.off + c_begin) : 0u;
    const uint32_t T = c_begin < c_end ? __ldg(p.off + c_end) - T0 : 0u;   // rows of this slice
    const int col0 = (int)rank * p.hw;                                    // first column of S A here
    const int hv = max(0, min(p.hw, p.d - col0));                         // valid columns here

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            tc::mbar_init(fullS + s, 2 * (kWorkers + kCons));
            tc::mbar_init(emptyS + s, 1);
        }
        for (int g = 0; g < kGroups; ++g) {
            tc::mbar_init(fullR + g, 32 + 1);   // the producer's lanes (copies landed) + its signs
            tc::mbar_init(emptyR + g, kCons);
        }
        tc::mbar_init(done, 1);
        tc::mbar_init(fin, 1);
        *abort = 0;
        tc::fence_mbar_init();
    }
    if (warp == kMmaWarp) {
        tc::tmem_alloc_pair(tmem_slot, p.tcols);
        tc::tmem_relinquish_pair();
    }
    tc::fence_before_sync();
    tc::cluster_sync();   // barriers of both CTAs initialised, TMEM allocated
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp < kWorkers) {
        // ------------------------------------------------------------ G workers
        const int wt = threadIdx.x;
        const int items = p.nsets * 512;   // per set: 32 row quads x 16 column pairs
        bool ok = true;
        for (int g = 0; g < nchunks; ++g) {
            const int s = g % kStages;
            const int64_t c0 = c_begin + (int64_t)g * kKC;
            uint32_t gw[2 * kMaxSets][4];
#pragma unroll
            for (int i = 0; i < 2 * kMaxSets; ++i) {
                const int item = wt + kWorkerThreads * i;
                const int gq = item >> 4, cp = item & 15;
                const int64_t jq = (int64_t)(gq >> 5) * kSetRows + (int64_t)rank * kHalfRows + 4 * (gq & 31);
                const int64_t c = c0 + 2 * cp;
                float4 z0 = make_float4(0.f, 0.f, 0.f, 0.f), z1 = z0;
                if (item < items && jq < p.k) {
                    if (c < c_end) z0 = gauss4((uint64_t)c, (uint32_t)(jq >> 2), p.k0, p.k1);
                    if (c + 1 < c_end) z1 = gauss4((uint64_t)(c + 1), (uint32_t)(jq >> 2), p.k0, p.k1);
                }
                const float a0[4] = {z0.x, z0.y, z0.z, z0.w}, a1[4] = {z1.x, z1.y, z1.z, z1.w};
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const bool rowok = jq + t < p.k;
                    const __nv_bfloat162 h = __floats2bfloat162_rn(rowok ? a0[t] * p.scale : 0.f,
                                                                   rowok ? a1[t] * p.scale : 0.f);
                    gw[i][t] = *reinterpret_cast<const uint32_t*>(&h);
                }
            }
            int w = 1;
            if (lane == 0) w = tc::mbar_wait(emptyS + s, ((uint32_t)(g / kStages) & 1u) ^ 1u, abort) ? 1 : 0;
            if (!__shfl_sync(0xffffffffu, w, 0)) {
                ok = false;
                break;
            }
            uint8_t* st = stages + s * sbytes;
            // local row 4 gq + t: set gq / 32 (the second set's rows follow 8 KB on)
#pragma unroll
            for (int i = 0; i < 2 * kMaxSets; ++i) {
                const int item = wt + kWorkerThreads * i;
                if (item < items) {
                    const int gq = item >> 4, cp = item & 15;
#pragma unroll
                    for (int t = 0; t < 4; ++t)
                        *reinterpret_cast<uint32_t*>(st + tc::sw64_offset(4 * gq + t, 2 * cp)) = gw[i][t];
                }
            }
            tc::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) arrive_even(fullS + s, rank);
        }
        // ------------------------------------------------------------ epilogue
        // warp w reads set w / 4, TMEM lanes 32 (w % 4) .. + 31 (its own lanes)
        const int set = warp >> 2, wq = warp & 3;
        if (set < p.nsets) {
            int okw = 0;
            if (lane == 0) okw = (ok && nchunks > 0 && tc::mbar_wait(done, 0, abort)) ? 1 : 0;
            okw = __shfl_sync(0xffffffffu, okw, 0);
            if (okw) {
                tc::fence_after_sync();
                const int64_t j = (int64_t)set * kSetRows + (int64_t)rank * kHalfRows + wq * 32 + lane;
                float* dst = p.part + ((int64_t)slice * p.k + j) * p.d;
                for (int col = 0; col < p.npad; col += 32) {
                    uint32_t v[32];
                    tc::tmem_ld_32x32b_x32(tmem + ((uint32_t)(wq * 32) << 16) + (uint32_t)(set * p.npad + col), v);
                    tc::tmem_ld_wait();
                    if (j < p.k) {
#pragma unroll
                        for (int e = 0; e < 32; ++e)
                            if (col + e < p.d) dst[col + e] = __uint_as_float(v[e]);
                    }
                }
            }
        }
    } else if (warp < kProdWarp) {
        // ------------------------------------------------------------ summing warps
        const int col = (warp - kCons0) * 32 + lane;   // column of this CTA's half
        const bool colv = col < hv, colb = col < p.hw;
        // lane l: end (row of the slice) of bucket l of chunk g
        auto ends_of = [&](int g) -> uint32_t {
            const int64_t c = c_begin + (int64_t)g * kKC + lane;
            return (g < nchunks && c < c_end) ? __ldg(p.off + c + 1) - T0 : T;
        };
        uint8_t* bh = stages + a_bytes();
        auto claim = [&](int g) -> bool {
            int w = 1;
            if (lane == 0)
                w = tc::mbar_wait(emptyS + g % kStages, ((uint32_t)(g / kStages) & 1u) ^ 1u, abort) ? 1 : 0;
            bh = stages + (g % kStages) * sbytes + a_bytes();
            return __shfl_sync(0xffffffffu, w, 0) != 0;
        };
        uint32_t ends_cur = ends_of(0), ends_nxt = ends_of(1);
        int g = 0, bb = 0;
        int nb = nchunks > 0 ? (int)min((int64_t)kKC, c_end - c_begin) : 0;
        float acc = 0.f;
        uint32_t t = 0;
        bool ok = nchunks > 0 && claim(0);
        uint32_t bend = __shfl_sync(0xffffffffu, ends_cur, 0);
        // close every bucket that ends at row t, and each chunk they complete
        auto advance = [&]() -> bool {
            while (t == bend) {
                if (colb) store_split(bh, bbytes, col, bb, acc);
                acc = 0.f;
                if (++bb == nb) {
                    if (colb)
                        for (int z = nb; z < kKC; ++z) store_split(bh, bbytes, col, z, 0.f);
                    tc::fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) arrive_even(fullS + g % kStages, rank);
                    if (++g == nchunks) {
                        bend = 0xFFFFFFFFu;
                        return true;
                    }
                    bb = 0;
                    nb = (int)min((int64_t)kKC, c_end - (c_begin + (int64_t)g * kKC));
                    ends_cur = ends_nxt;
                    ends_nxt = ends_of(g + 1);
                    if (!claim(g)) return false;
                }
                bend = __shfl_sync(0xffffffffu, ends_cur, bb);
            }
            return true;
        };
        if (ok) ok = advance();
        while (ok && t < T) {
            const uint32_t grp = t / kGroupRows;
            const int gi = (int)(grp % kGroups);
            int w = 1;
            if (lane == 0) w = tc::mbar_wait(fullR + gi, (grp / kGroups) & 1u, abort) ? 1 : 0;
            if (!__shfl_sync(0xffffffffu, w, 0)) {
                ok = false;
                break;
            }
            const uint32_t nr = min((uint32_t)kGroupRows, T - t);
            float v[kGroupRows], sg[kGroupRows];
#pragma unroll
            for (int q = 0; q < kGroupRows; ++q) {
                const uint32_t slot = (t + q) % kRing;
                v[q] = ((uint32_t)q < nr && colv) ? ring[slot * p.hw + col] : 0.f;
                sg[q] = ((uint32_t)q < nr) ? sgn[slot] : 0.f;
            }
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(emptyR + gi);   // the group's slots may be refilled
#pragma unroll
            for (int q = 0; q < kGroupRows; ++q) {
                if ((uint32_t)q < nr && ok) {
                    acc = fmaf(sg[q], v[q], acc);
                    ++t;
                    if (t == bend) ok = advance();
                }
            }
        }
    } else if (warp == kProdWarp) {
        // ------------------------------------------------------------ producer
        // lane l copies columns [4 l, 4 l + 4) of the half row (16-byte copies)
        const bool lanecp = 4 * lane < hv;
        const float* Ah = p.A + col0 + 4 * lane;
        const uint32_t* pp = p.perm + T0;
        uint32_t pf0 = (lane < T) ? __ldg(pp + lane) : 0u;
        uint32_t pf1 = (32u + lane < T) ? __ldg(pp + 32 + lane) : 0u;
        uint32_t pf2 = (64u + lane < T) ? __ldg(pp + 64 + lane) : 0u;
        uint32_t pf3 = (96u + lane < T) ? __ldg(pp + 96 + lane) : 0u;
        uint32_t issued = 0;   // ring groups armed so far
        bool ok = true;
        for (uint32_t t = 0; t < T && ok; t += 32) {
            const uint32_t mine = pf0;   // perm entry of row t + lane
            pf0 = pf1;
            pf1 = pf2;
            pf2 = pf3;
            pf3 = (t + 128u + lane < T) ? __ldg(pp + t + 128 + lane) : 0u;
#pragma unroll
            for (int q8 = 0; q8 < 4; ++q8) {
                const uint32_t tg = t + 8u * q8;
                if (tg >= T) break;
                const uint32_t grp = tg / kGroupRows;
                const int gi = (int)(grp % kGroups);
                const uint32_t nr = min((uint32_t)kGroupRows, T - tg);
                int w = 1;
                if (lane == 0) w = tc::mbar_wait(emptyR + gi, ((grp / kGroups) & 1u) ^ 1u, abort) ? 1 : 0;
                if (!__shfl_sync(0xffffffffu, w, 0)) {
                    ok = false;
                    break;
                }
#pragma unroll
                for (int e = 0; e < kGroupRows; ++e) {
                    const uint32_t pe = __shfl_sync(0xffffffffu, mine, 8 * q8 + e);
                    if ((uint32_t)e < nr) {
                        const uint32_t slot = (tg + e) % kRing;
                        if (lanecp) cp_async16(ring + slot * p.hw + 4 * lane, Ah + (int64_t)(pe & 0x7fffffffu) * p.lda);
                        if (lane == 0) sgn[slot] = (pe >> 31) ? -1.f : 1.f;
                    }
                }
                cp_async_arrive(fullR + gi);
                if (lane == 0) tc::mbar_arrive(fullR + gi);   // the signs (release)
                issued = grp + 1;
            }
        }
        cp_async_wait_all();
        if (lane == 0) {
            // the groups still completing (the last kGroups) complete before the CTA leaves
            volatile int never = 0;
            const uint32_t first = issued > (uint32_t)kGroups ? issued - kGroups : 0u;
            for (uint32_t grp = first; grp < issued; ++grp)
                tc::mbar_wait(fullR + grp % kGroups, (grp / kGroups) & 1u, &never);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ MMA issue (even CTA)
        if (lane == 0 && rank == 0) {
            const uint32_t base = tc::smem_u32(stages);
            const uint32_t idesc = tc::idesc_bf16_f32(kSetRows, (uint32_t)p.npad);
            bool okm = true;
            for (int g = 0; g < nchunks; ++g) {
                const int s = g % kStages;
                if (!tc::mbar_wait_cluster(fullS + s, (uint32_t)(g / kStages) & 1u, abort)) {
                    okm = false;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t a = base + s * sbytes, bh = a + a_bytes(), bl = bh + bbytes;
#pragma unroll
                for (int kk = 0; kk < kKC / 16; ++kk) {
                    const uint32_t ko = 32u * kk;
                    for (int set = 0; set < p.nsets; ++set) {
                        const uint32_t at = a + (uint32_t)set * (kHalfRows * kKC * 2) + ko;
                        const uint32_t dt = tmem + (uint32_t)(set * p.npad);
                        tc::mma_bf16_pair(dt, tc::desc_sw64_kmajor(at), tc::desc_sw64_kmajor(bh + ko), idesc,
                                          (g | kk) != 0);
                        tc::mma_bf16_pair(dt, tc::desc_sw64_kmajor(at), tc::desc_sw64_kmajor(bl + ko), idesc, 1);
                    }
                }
                tc::mma_commit_pair(emptyS + s);
            }
            if (okm && nchunks > 0) tc::mma_commit_pair(done);
            tc::mma_commit_pair(fin);
        }
        if (lane == 0) {
            // both CTAs: the last multicast commit has landed here
            volatile int never = 0;
            tc::mbar_wait(fin, 0, &never);
        }
        __syncwarp();
    }

    tc::fence_before_sync();
    __syncthreads();
    tc::cluster_sync();   // no CTA leaves while its peer may still arrive on its barriers
    if (warp == kMmaWarp) {
        tc::fence_after_sync();
        tc::tmem_dealloc_pair(tmem, p.tcols);
    }
    if (threadIdx.x == 0 && *abort) set_flag(p.flag, LSK_FLAG_TIMEOUT);
}

// clusters of two that fit on the device at once (cached per device and size)
int cg_clusters(size_t smem) {
    static std::mutex mu;
    static std::map<std::tuple<int, size_t>, int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_tuple(dev, smem);
    const auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int n = 0;
    if (allow_dynamic_smem(count_gauss_kernel) == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(2, 1, 1);
        cfg.blockDim = dim3(kThreads, 1, 1);
        cfg.dynamicSmemBytes = smem;
        if (cudaOccupancyMaxActiveClusters(&n, (const void*)count_gauss_kernel, &cfg) != cudaSuccess) n = 0;
    }
    cudaGetLastError();
    cache[key] = n;
    return n;
}

bool shape_ok(const lsk_mat* A, int64_t r, int64_t k) {
    const int64_t d = A->d;
    return A->kind == LSK_DENSE && d >= 32 && d <= 256 && d % 4 == 0 && A->ld % 4 == 0 &&
           ((uintptr_t)A->values & 15) == 0 && k >= 1 && k <= (int64_t)kMaxSets * kSetRows && r >= 1 &&
           r < ((int64_t)1 << 31) && A->n < ((int64_t)1 << 31);
}

// slices of the buckets for `clusters` pairs: one wave, >= 8 chunks a slice
void plan(const lsk_mat* A, int64_t r, int64_t k, int clusters, CgParams& p) {
    const int64_t d = A->d;
    p.d = (int)d;
    p.npad = (int)((d + 31) / 32) * 32;
    p.hw = p.npad / 2;
    p.nsets = (int)((k + kSetRows - 1) / kSetRows);
    uint32_t cols = 32;
    while (cols < (uint32_t)(p.nsets * p.npad)) cols <<= 1;
    p.tcols = cols;
    int64_t want = clusters;
    const int64_t max_slices = (r + 8 * kKC - 1) / (8 * kKC);
    if (want > max_slices) want = max_slices;
    if (want < 1) want = 1;
    int64_t ks = (r + want - 1) / want;
    ks = ((ks + kKC - 1) / kKC) * kKC;
    p.kslice = ks;
    p.slices = (int)((r + ks - 1) / ks);
}

}  // namespace

bool count_gauss_supported(const lsk_mat* A, int64_t r, int64_t k) {
    if (!shape_ok(A, r, k)) return false;
    const int hw = (int)((A->d + 31) / 32) * 16;
    const size_t smem = smem_bytes(hw);
    return smem <= kSmemLimit && cg_clusters(smem) > 0;
}

size_t count_gauss_workspace_bytes(const lsk_mat* A, int64_t r, int64_t k, int sm_count) {
    if (!shape_ok(A, r, k)) return 0;
    CgParams p{};
    plan(A, r, k, sm_count / 2 > 0 ? sm_count / 2 : 1, p);   // most slices any launch uses
    return cs_workspace_bytes(A->n, r) + ws_round((size_t)p.slices * k * A->d * 4);
}

cudaError_t count_gauss_launch(const lsk_mat* A, int64_t r, int64_t k, uint64_t seed, float* GSA, void* ws,
                               int* flag, int sm_count, cudaStream_t st) {
    if (!shape_ok(A, r, k)) return cudaErrorNotSupported;
    CgParams p{};
    const int hw = (int)((A->d + 31) / 32) * 16;
    const size_t smem = smem_bytes(hw);
    const int maxc = cg_clusters(smem);
    if (smem > kSmemLimit || maxc < 1) return cudaErrorNotSupported;
    const int half = sm_count / 2 > 0 ? sm_count / 2 : 1;
    plan(A, r, k, maxc < half ? maxc : half, p);
    const uint32_t* off = nullptr;
    const uint32_t* perm = nullptr;
    cudaError_t e = cs_prep_launch(A->n, r, seed, ws, sm_count, st, &off, &perm);
    if (e != cudaSuccess) return e;
    p.A = (const float*)A->values;
    p.lda = A->ld;
    p.off = off;
    p.perm = perm;
    p.part = reinterpret_cast<float*>((char*)ws + cs_workspace_bytes(A->n, r));
    p.r = r;
    p.k = k;
    p.k0 = (uint32_t)seed;
    p.k1 = (uint32_t)(seed >> 32);
    p.scale = (float)(1.0 / sqrt((double)k));
    p.flag = flag;
    LSK_PROF("count_gauss", st) count_gauss_kernel<<<2 * p.slices, kThreads, smem, st>>>(p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return gauss_tc_reduce_launch(p.part, p.slices, k * A->d, GSA, sm_count, st);
}
