// count_gauss.cu -- the fused CountSketch + Gaussian stage: GSA = G (S A) in
// one pass over A, with S A never written to HBM.
//
// Alg. 3 forms the sketch in blocks of r: B = S_i A for one block of rows of
// S, then C += G_i B with a fresh Gaussian block G_i, so that only one block
// of S A exists at a time.  Here a block is 32 buckets (one K-chunk of the
// tensor-core product) and it lives in shared memory only, as bf16 hi + lo.
// A cluster of two CTAs (a tcgen05 CTA pair) owns one slice of the buckets
// and the whole k x d product of that slice:
//   - 16 gather warps per CTA: CTA `rank` sums buckets [16 rank, 16 rank + 16)
//     of every chunk, one per warp, whole rows at a time.  A bucket's rows are
//     consecutive in the CountSketch permutation (steps 1-3 of countsketch.cu);
//     they stream through a private ring of row slots in shared memory filled
//     with per-lane 16-byte cp.async copies, several rows in flight per warp
//     without holding registers.  When a bucket closes, its first half of
//     columns goes as bf16 hi + lo into the even CTA's B operand of the chunk
//     and its second half into the odd CTA's (distributed shared memory);
//   - 8 worker warps: draw this CTA's rows of the chunk's columns of G (the
//     Gaussian stage's Philox + Box-Muller draws, bf16) into the A operand;
//   - the even CTA's MMA thread: M = 256 pair MMAs, G rows [0, 128) of each
//     256-row set from the even CTA and [128, 256) from the odd one, B's first
//     N / 2 = d_pad / 2 rows (S A columns) from the even CTA and the rest from
//     the odd one; each CTA's TMEM holds its 128 rows of every set, so the pair
//     keeps the whole 512 x 256 FP32 accumulator (2 x 512 columns);
//   - the worker warps then copy the accumulator out as the slice's partial,
//     and the partials are summed in slice order (compensated FP32).
// A ring of kStages chunk operands lets the gather warps and the draws run
// ahead of the MMAs.  Every wait is bounded (1 s); a timeout sets
// LSK_FLAG_TIMEOUT and every warp winds down (a gather warp waits for its own
// copies in flight before it leaves).
//
// Why the rows go through shared memory: the gather is bound by the bytes in
// flight per SM (Little's law: ~45 GB/s per SM at ~2 us loaded latency needs
// ~90 KB).  Loads into registers capped that at 64 KB here (the draws, the
// MMA and TMEM bookkeeping share the register file), 0.84 ms at 4M x 256;
// the cp.async rings hold 80 KB without registers: 0.70 ms.
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
constexpr int kGath0 = kWorkers;     // first gather warp
constexpr int kStages = 3;
constexpr size_t kSmemLimit = 232448;

static_assert(2 * kMaxSets * kWorkerThreads == kMaxSets * 32 * 16, "two G items per thread and set");

// gather warps and rows in flight per gather warp
template <int NG, int kRing, bool kUnroll = true>
struct Shape {
    static constexpr int kMmaWarp = kGath0 + NG;
    static constexpr int kThreads = (kMmaWarp + 1) * 32;
    static_assert(NG == 16, "a CTA sums 16 buckets of a chunk, one per gather warp");
    static_assert(kRing >= 2 && kRing <= 16, "row slots per gather warp");
};

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
// stages, then the gather warps' row rings (16 warps x ring slots x 1 KB), then the barriers
inline size_t smem_bytes(int hw, int ring) {
    return 1024 + (size_t)kStages * stage_bytes(hw) + (size_t)16 * ring * 1024 + (size_t)(2 * kStages + 2) * 8 + 16;
}

__device__ __forceinline__ void arrive_even(uint64_t* bar, uint32_t rank) {
    if (rank == 0) tc::mbar_arrive(bar);
    else tc::mbar_arrive_cluster(bar, 0);
}
// shared::cluster address of the same shared-memory offset in CTA `rank`
__device__ __forceinline__ uint32_t peer_addr(uint32_t local, uint32_t rank) {
    uint32_t a;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"(local), "r"(rank));
    return a;
}
__device__ __forceinline__ void st_cluster_u16(uint32_t addr, uint32_t v) {
    asm volatile("st.shared::cluster.u16 [%0], %1;" ::"r"(addr), "h"((uint16_t)v) : "memory");
}
__device__ __forceinline__ void fence_proxy_async_cluster() {
    asm volatile("fence.proxy.async.shared::cluster;" ::: "memory");
}
// the four sums of a lane (rows n .. n + 3 of a B operand, bucket k of the
// chunk) as bf16 hi + lo into the K-major hi / lo tiles at shared::cluster
// address bh (this CTA's or the peer's)
__device__ __forceinline__ void store_split4(uint32_t bh, uint32_t bbytes, int n, int k, float4 x) {
    uint32_t h01, l01, h23, l23;
    tc::split_bf16x2(x.x, x.y, h01, l01);
    tc::split_bf16x2(x.z, x.w, h23, l23);
    const uint32_t o0 = tc::sw64_offset((uint32_t)n, (uint32_t)k), o1 = tc::sw64_offset((uint32_t)n + 1, (uint32_t)k);
    const uint32_t o2 = tc::sw64_offset((uint32_t)n + 2, (uint32_t)k), o3 = tc::sw64_offset((uint32_t)n + 3, (uint32_t)k);
    st_cluster_u16(bh + o0, h01);
    st_cluster_u16(bh + o1, h01 >> 16);
    st_cluster_u16(bh + o2, h23);
    st_cluster_u16(bh + o3, h23 >> 16);
    st_cluster_u16(bh + bbytes + o0, l01);
    st_cluster_u16(bh + bbytes + o1, l01 >> 16);
    st_cluster_u16(bh + bbytes + o2, l23);
    st_cluster_u16(bh + bbytes + o3, l23 >> 16);
}

template <int NG, int kRing, bool kUnroll>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(Shape<NG, kRing>::kThreads, 1)
    count_gauss_kernel(const CgParams p) {
    constexpr int kMmaWarp = Shape<NG, kRing>::kMmaWarp;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
    const uint32_t rank = tc::cluster_ctarank();
    const int slice = (int)tc::cluster_id_x();
    const uint32_t sbytes = stage_bytes(p.hw), bbytes = b_bytes(p.hw);
    uint8_t* stages = smem;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kStages * sbytes + NG * kRing * 1024);
    uint64_t* fullS = bars;                  // [kStages] even CTA: chunk operands written in both CTAs
    uint64_t* emptyS = fullS + kStages;      // [kStages] chunk consumed (multicast commit)
    uint64_t* done = emptyS + kStages;       // accumulator complete (multicast commit)
    uint64_t* fin = done + 1;                // every MMA complete (multicast commit)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t c_begin = (int64_t)slice * p.kslice;
    const int64_t c_end = min(p.r, c_begin + p.kslice);
    const int nchunks = c_begin < c_end ? (int)((c_end - c_begin + kKC - 1) / kKC) : 0;
    const int col0 = (int)rank * p.hw;                                    // first column of S A here
    const int hv = max(0, min(p.hw, p.d - col0));                         // valid columns here

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            tc::mbar_init(fullS + s, 2 * (kWorkers + NG));
            tc::mbar_init(emptyS + s, 1);
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
            // the ring keeps the workers ahead of the MMAs, so they claim the
            // stage first and draw straight into it (few registers live)
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
                    const int64_t jq = (int64_t)(gq >> 5) * kSetRows + (int64_t)rank * kHalfRows + 4 * (gq & 31);
                    const int64_t c = c0 + 2 * cp;
                    float4 z0 = make_float4(0.f, 0.f, 0.f, 0.f), z1 = z0;
                    if (jq < p.k) {
                        if (c < c_end) z0 = gauss4((uint64_t)c, (uint32_t)(jq >> 2), p.k0, p.k1);
                        if (c + 1 < c_end) z1 = gauss4((uint64_t)(c + 1), (uint32_t)(jq >> 2), p.k0, p.k1);
                    }
                    const float a0[4] = {z0.x, z0.y, z0.z, z0.w}, a1[4] = {z1.x, z1.y, z1.z, z1.w};
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const bool rowok = jq + t < p.k;
                        const __nv_bfloat162 h = __floats2bfloat162_rn(rowok ? a0[t] * p.scale : 0.f,
                                                                       rowok ? a1[t] * p.scale : 0.f);
                        *reinterpret_cast<uint32_t*>(st + tc::sw64_offset(4 * gq + t, 2 * cp)) =
                            *reinterpret_cast<const uint32_t*>(&h);
                    }
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
    } else if (warp < kMmaWarp) {
        // ------------------------------------------------------------ gather warps
        // CTA `rank` sums buckets [16 rank, 16 rank + 16) of every chunk; gather
        // warp gi sums bucket 16 rank + gi of each chunk, whole rows at a time
        // (lane l: columns 4l.. of each half).  A bucket's first half goes to
        // the even CTA's B operand and its second half to the odd CTA's.
        //
        // The rows stream through a private ring of kRing row slots in shared
        // memory: each step the warp issues one row (every lane copies its
        // 2 x 16 bytes with cp.async) and sums the row issued kRing - 1 steps
        // earlier, so kRing - 1 rows are in flight per warp without holding
        // registers.  A lane reads back only the bytes it copied itself, so its
        // own cp.async.wait_group orders the copy before the read.  The copying
        // side walks the warp's buckets (chunk by chunk) ahead of the summing
        // side; every issued row carries its chunk and sign to the summing side
        // (meta), which closes a chunk's bucket when a row of a later chunk
        // arrives (or at the end).
        const int gi = warp - kGath0;
        const int n0 = 4 * lane;
        const bool lv0 = n0 < min(p.hw, p.d);            // columns n0.. of the first half exist
        const bool lv1 = p.hw + n0 < p.d;                // ... of the second half
        const bool lb = n0 < p.hw;                       // rows n0.. of the B operands
        const float* A0 = p.A + n0;
        const float* A1 = p.A + p.hw + n0;
        const uint32_t here = tc::smem_u32(stages);
        const uint32_t tile0 = peer_addr(here, 0);       // the stages of the even CTA (shared::cluster)
        const uint32_t tile1 = peer_addr(here, 1);       // ... of the odd CTA
        const uint32_t ring = here + kStages * sbytes + (uint32_t)(gi * kRing * 1024 + 16 * lane);
        const int kb = 16 * (int)rank + gi;              // this warp's bucket within every chunk
        auto range_of = [&](int g, uint32_t& bs, uint32_t& be) {
            bs = be = 0u;
            if (g < nchunks) {
                const int64_t b = c_begin + (int64_t)g * kKC + kb;
                if (b < c_end) {
                    bs = __ldg(p.off + b);
                    be = __ldg(p.off + b + 1);
                }
            }
        };
        auto window = [&](uint32_t t, uint32_t e) -> uint32_t {
            return (t + lane < e) ? __ldg(p.perm + t + lane) : 0x80000000u;
        };
        // ---- copying side: chunk gp, rows [tp, ep) of its bucket, permutation
        // window [wp, wp + 32) in pwp, the next window (base pnb) in pnp
        int gp = 0;
        uint32_t tp, ep, s1, e1, s2, e2;
        range_of(0, tp, ep);
        range_of(1, s1, e1);
        range_of(2, s2, e2);
        uint32_t wp = tp, pwp = window(tp, ep);
        uint32_t pnb = tp + 32 < ep ? tp + 32 : s1, pne = tp + 32 < ep ? ep : e1;
        uint32_t pnp = window(pnb, pne);
        // window [tp, tp + 32): from pnp when that was loaded for it (the same
        // base and bucket end), and the next one (this bucket's or the next
        // bucket's first) into pnp
        auto open_window = [&]() {
            wp = tp;
            pwp = (pnb == tp && pne == ep) ? pnp : window(tp, ep);
            pnb = tp + 32 < ep ? tp + 32 : s1;
            pne = tp + 32 < ep ? ep : e1;
            pnp = window(pnb, pne);
        };
        // move to the next row to copy: skip finished (and empty) buckets, open windows
        auto normalize = [&]() {
            while (gp < nchunks && tp == ep) {
                ++gp;
                tp = s1;
                ep = e1;
                s1 = s2;
                e1 = e2;
                range_of(gp + 2, s2, e2);
                if (tp < ep) open_window();
            }
            if (gp < nchunks && tp == wp + 32) open_window();
        };
        normalize();
        // ---- summing side: chunk gc, its sums
        int gc = 0;
        float4 acc0 = make_float4(0.f, 0.f, 0.f, 0.f), acc1 = acc0;
        bool ok = true;
        // close chunk gc's bucket: its sums into both CTAs' B operands of the chunk
        auto close = [&]() -> bool {
            const int st = gc % kStages;
            int w = 1;
            if (lane == 0) w = tc::mbar_wait(emptyS + st, ((uint32_t)(gc / kStages) & 1u) ^ 1u, abort) ? 1 : 0;
            if (!__shfl_sync(0xffffffffu, w, 0)) return false;
            const uint32_t so = (uint32_t)st * sbytes + a_bytes();
            if (lb) {
                store_split4(tile0 + so, bbytes, n0, kb, acc0);
                store_split4(tile1 + so, bbytes, n0, kb, acc1);
            }
            fence_proxy_async_cluster();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive_cluster(fullS + st, 0);
            acc0 = make_float4(0.f, 0.f, 0.f, 0.f);
            acc1 = acc0;
            ++gc;
            return true;
        };
        // per slot: chunk << 1 | sign of the row copied there, -1 if none (in
        // registers when the steps of a round are unrolled, else in the
        // thread's local memory: a smaller loop body for the instruction cache)
        int meta[kRing];
#pragma unroll
        for (int i = 0; i < kRing; ++i) meta[i] = -1;
        // rounds of kRing steps; the round that starts with nothing left to copy
        // sums every row still in the ring and is the last
        for (bool last = false; ok && !last;) {
            last = gp >= nchunks;
#pragma unroll(kUnroll ? kRing : 1)
            for (int i = 0; i < kRing; ++i) {
                // (1) sum the row copied kRing - 1 steps ago (slot i + 1)
                const int sl = (i + 1) % kRing;
                asm volatile("cp.async.wait_group %0;" ::"n"(kRing - 2) : "memory");
                const int m = meta[sl];
                if (m >= 0) {
                    while (ok && gc < (m >> 1)) ok = close();
                    const uint32_t a = ring + (uint32_t)sl * 1024u;
                    const float sg = (m & 1) ? -1.0f : 1.0f;
                    if (lv0) {
                        float4 v;
                        asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
                        acc0.x = fmaf(sg, v.x, acc0.x);
                        acc0.y = fmaf(sg, v.y, acc0.y);
                        acc0.z = fmaf(sg, v.z, acc0.z);
                        acc0.w = fmaf(sg, v.w, acc0.w);
                    }
                    if (lv1) {
                        float4 v;
                        asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a + 512u));
                        acc1.x = fmaf(sg, v.x, acc1.x);
                        acc1.y = fmaf(sg, v.y, acc1.y);
                        acc1.z = fmaf(sg, v.z, acc1.z);
                        acc1.w = fmaf(sg, v.w, acc1.w);
                    }
                }
                // (2) copy the next row into slot i (summed in step i - 1, its
                //     values already consumed by the FMAs above)
                meta[i] = -1;
                if (gp < nchunks) {
                    const uint32_t pe = __shfl_sync(0xffffffffu, pwp, (int)(tp - wp));
                    const int64_t ro = (int64_t)(pe & 0x7fffffffu) * p.lda;
                    const uint32_t a = ring + (uint32_t)i * 1024u;
                    if (lv0) asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(a), "l"(A0 + ro) : "memory");
                    if (lv1) asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(a + 512u), "l"(A1 + ro) : "memory");
                    meta[i] = (gp << 1) | (int)(pe >> 31);
                    ++tp;
                    normalize();
                }
                asm volatile("cp.async.commit_group;" ::: "memory");
            }
        }
        while (ok && gc < nchunks) ok = close();         // trailing (empty) buckets
        asm volatile("cp.async.wait_all;" ::: "memory");
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

// the kernel shapes that can be launched (gather warps, row slots per warp)
struct Variant {
    void (*fn)(CgParams);
    int threads;
    int ring;          // row slots per gather warp
};
template <int NG, int R, bool U>
constexpr Variant variant() {
    return Variant{count_gauss_kernel<NG, R, U>, Shape<NG, R>::kThreads, R};
}
// 6 slots (5 rows in flight per warp, 80 KB per SM) measured fastest at
// 4M x 256 (0.70 ms against 0.72 ms for 4 slots and 0.80 ms for 8; the
// 6-slot steps not unrolled, with the slot metadata in local memory: 0.73)
const Variant kVariants[] = {variant<16, 6, true>(), variant<16, 4, true>()};
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);

// LSK_CG_VARIANT=1 selects the 4-slot kernel (a complete kernel; for timing
// comparisons and tests)
int variant_index() {
    static int v = [] {
        const char* s = getenv("LSK_CG_VARIANT");
        const int i = s ? atoi(s) : 0;
        return (i >= 0 && i < kNumVariants) ? i : 0;
    }();
    return v;
}

// clusters of two that fit on the device at once (cached per device, variant and size)
int cg_clusters(int vi, size_t smem) {
    static std::mutex mu;
    static std::map<std::tuple<int, int, size_t>, int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_tuple(dev, vi, smem);
    const auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int n = 0;
    const Variant& v = kVariants[vi];
    if (allow_dynamic_smem(v.fn) == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(2, 1, 1);
        cfg.blockDim = dim3(v.threads, 1, 1);
        cfg.dynamicSmemBytes = smem;
        if (cudaOccupancyMaxActiveClusters(&n, (const void*)v.fn, &cfg) != cudaSuccess) n = 0;
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
    const int vi = variant_index();
    const size_t smem = smem_bytes(hw, kVariants[vi].ring);
    return smem <= kSmemLimit && cg_clusters(vi, smem) > 0;
}

bool count_gauss_preferred(const lsk_mat* A, int64_t r, int64_t k, int sm_count) {
    const int64_t pairs = sm_count / 2 > 0 ? sm_count / 2 : 1;
    return A->kind == LSK_DENSE && A->d > 192 && r >= pairs * 8 * kKC && A->n >= 8 * r &&
           count_gauss_supported(A, r, k);
}

size_t count_gauss_workspace_bytes(const lsk_mat* A, int64_t r, int64_t k, int sm_count) {
    if (!shape_ok(A, r, k)) return 0;
    CgParams p{};
    plan(A, r, k, sm_count / 2 > 0 ? sm_count / 2 : 1, p);   // most slices any launch uses
    return cs_workspace_bytes(A->n, r) + ws_round((size_t)p.slices * k * A->d * 4);
}

cudaError_t count_gauss_launch(const lsk_mat* A, int64_t r, int64_t k, uint64_t seed, float* GSA, void* ws,
                               int* flag, int sm_count, cudaStream_t st, uint64_t row0) {
    if (!shape_ok(A, r, k)) return cudaErrorNotSupported;
    CgParams p{};
    const int hw = (int)((A->d + 31) / 32) * 16;
    const int vi = variant_index();
    const size_t smem = smem_bytes(hw, kVariants[vi].ring);
    const int maxc = cg_clusters(vi, smem);
    if (smem > kSmemLimit || maxc < 1) return cudaErrorNotSupported;
    const int half = sm_count / 2 > 0 ? sm_count / 2 : 1;
    plan(A, r, k, maxc < half ? maxc : half, p);
    const uint32_t* off = nullptr;
    const uint32_t* perm = nullptr;
    cudaError_t e = cs_prep_launch(A->n, r, seed, ws, sm_count, st, &off, &perm, row0, flag);
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
    const Variant& v = kVariants[vi];
    LSK_PROF("count_gauss", st) v.fn<<<2 * p.slices, v.threads, smem, st>>>(p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return gauss_tc_reduce_launch(p.part, p.slices, k * A->d, GSA, sm_count, st);
}
