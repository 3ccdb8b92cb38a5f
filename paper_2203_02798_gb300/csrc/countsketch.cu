// countsketch.cu -- CountSketch S*A for dense and CSR A (Def. 3, Alg. 2).
//
// The paper stores S as a Block (Column) CountSketch and lets each thread
// own whole rows of SA (Alg. 2, the b_r = r case of Sec. 2.3), so that no two
// threads write the same output row.  Here S is never stored: (h(i), sigma_i)
// is recomputed from Philox whenever it is needed, and row ownership is kept
// at the finest grain -- one warp owns one bucket (one row of SA):
//
//   1. count: cnt[h(i)]++ for every row (fire-and-forget atomics)
//   2. scan:  off = exclusive prefix sum of cnt        (bucket -> first slot),
//             and a copy of it as each bucket's fill cursor
//   3. place: perm[cursor[h(i)]++] = i | sigma_bit << 31
//   4. gather (dense): the warp owning bucket b streams the rows listed in
//      perm[off[b] .. off[b+1]) with 16-byte coalesced loads, accumulates them
//      (with their signs) in registers and writes row b of SA exactly once.
//      gather (CSR): same ownership, the row of SA is accumulated in shared
//      memory because CSR columns are scattered.
//
// Every byte of A is read once and every row of SA written once, with no
// global atomics on floating-point data; the only extra traffic is the
// 4 bytes per row of perm.  The per-bucket loads are the Y of Lemma 1:
// expected n/r rows per warp, concentrated as in Lemma 2-3.
#include "lsk_internal.cuh"

namespace {

constexpr int kScanBlock = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanBlock * kScanItems;

// Row i of A is column row0 + i of S: a block of rows of a larger matrix
// (one shard of a row partition) is hashed by its global row index.  Each
// thread takes kPrepRows rows per pass with their atomics independent, so
// several round trips to L2 are in flight per thread.
constexpr int kPrepRows = 4;

__global__ void cs_count_kernel(int64_t n, uint64_t row0, uint32_t r, uint32_t k0, uint32_t k1,
                                uint32_t* __restrict__ cnt) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += stride * kPrepRows) {
#pragma unroll
        for (int q = 0; q < kPrepRows; ++q) {
            const int64_t i = i0 + q * stride;
            if (i < n) {
                uint32_t b, neg;
                cs_hash(row0 + (uint64_t)i, r, k0, k1, b, neg);
                atomicAdd(&cnt[b], 1u);   // result unused: compiled to a reduction (no round trip)
            }
        }
    }
}

// The order of the rows inside a bucket is the order in which their atomics
// reach the cursor (not fixed from run to run); every consumer sums a bucket's
// rows in that order, so S*A is exact for integer-valued data and agrees to
// FP32 rounding otherwise.
__global__ void cs_place_kernel(int64_t n, uint64_t row0, uint32_t r, uint32_t k0, uint32_t k1,
                                uint32_t* __restrict__ cursor, uint32_t* __restrict__ perm) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += stride * kPrepRows) {
        uint32_t slot[kPrepRows], val[kPrepRows];
#pragma unroll
        for (int q = 0; q < kPrepRows; ++q) {
            const int64_t i = i0 + q * stride;
            if (i < n) {
                uint32_t b, neg;
                cs_hash(row0 + (uint64_t)i, r, k0, k1, b, neg);
                slot[q] = atomicAdd(&cursor[b], 1u);
                val[q] = (uint32_t)i | (neg << 31);
            }
        }
#pragma unroll
        for (int q = 0; q < kPrepRows; ++q)
            if (i0 + q * stride < n) perm[slot[q]] = val[q];
    }
}

// Block-local exclusive scan of kScanTile entries; writes the tile total.
__global__ void scan_tiles_kernel(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                  uint32_t* __restrict__ tile_sums, int64_t len) {
    __shared__ uint32_t warp_tot[kScanBlock / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t run = 0;
#pragma unroll
    for (int t = 0; t < kScanItems; ++t) {
        const int64_t i = base + t;
        v[t] = (i < len) ? in[i] : 0u;
        const uint32_t x = v[t];
        v[t] = run;
        run += x;
    }
    // exclusive scan of the per-thread totals across the block
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = (lane < kScanBlock / 32) ? warp_tot[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < kScanBlock / 32) warp_tot[lane] = wi - w;
        if (lane == kScanBlock / 32 - 1) tile_sums[blockIdx.x] = wi;
    }
    __syncthreads();
    const uint32_t excl = warp_tot[wid] + incl - run;
#pragma unroll
    for (int t = 0; t < kScanItems; ++t) {
        const int64_t i = base + t;
        if (i < len) out[i] = v[t] + excl;
    }
}

__global__ void scan_add_kernel(uint32_t* __restrict__ out, const uint32_t* __restrict__ tile_off,
                                int64_t len) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len) out[i] += tile_off[i / kScanTile];
}

// Exclusive scan of `len` uint32 into `out` (may alias nothing); `tmp` must
// hold scan_tmp_words(len) words.
size_t scan_tmp_words(int64_t len) {
    size_t words = 0;
    int64_t l = len;
    while (true) {
        const int64_t tiles = (l + kScanTile - 1) / kScanTile;
        words += 2 * (size_t)tiles + 64;
        if (tiles <= 1) break;
        l = tiles;
    }
    return words;
}

cudaError_t exclusive_scan(const uint32_t* in, uint32_t* out, int64_t len, uint32_t* tmp,
                           cudaStream_t st) {
    if (len <= 0) return cudaSuccess;
    const int64_t tiles = (len + kScanTile - 1) / kScanTile;
    uint32_t* sums = tmp;
    LSK_PROF("cs_scan", st) scan_tiles_kernel<<<(unsigned)tiles, kScanBlock, 0, st>>>(in, out, sums, len);
    if (tiles > 1) {
        uint32_t* sums_off = tmp + tiles + 32;
        cudaError_t e = exclusive_scan(sums, sums_off, tiles, sums_off + tiles + 32, st);
        if (e != cudaSuccess) return e;
        LSK_PROF("cs_scan", st) scan_add_kernel<<<(unsigned)((len + 255) / 256), 256, 0, st>>>(out, sums_off, len);
    }
    return cudaGetLastError();
}

// Single-pass exclusive scan of the counters (decoupled look-back): block b
// takes tile t (the t-th ticket, kScanTile counts), scans it, publishes its
// aggregate, then adds the published values of the tiles before it, nearest
// first and 32 at a time (one warp), until one carries its inclusive prefix,
// and publishes its own.  A
// tile only waits on tiles whose tickets were taken earlier, i.e. by blocks
// already running.  Writes off[i] = cursor[i] = the exclusive prefix and
// off[len] = the total.  state: the ticket, then one word per tile (flag
// << 32 | value; flag 1 = aggregate, 2 = inclusive prefix), zeroed before
// the launch.  A wait that runs out sets the TIMEOUT flag.
constexpr int kLookbackSpins = 1 << 20;
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__global__ void __launch_bounds__(kScanBlock) scan_lookback_kernel(const uint32_t* __restrict__ in,
                                                                   uint32_t* __restrict__ off,
                                                                   uint32_t* __restrict__ cursor, int64_t len,
                                                                   unsigned long long* state, int* flag) {
    __shared__ uint32_t warp_tot[kScanBlock / 32];
    __shared__ uint32_t s_tile, s_prefix;
    if (threadIdx.x == 0) s_tile = atomicAdd(reinterpret_cast<unsigned int*>(state), 1u);
    __syncthreads();
    const int64_t t = s_tile;
    unsigned long long* tiles = state + 1;
    const int64_t base = t * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t run = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        const int64_t i = base + q;
        const uint32_t x = (i < len) ? in[i] : 0u;
        v[q] = run;
        run += x;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const uint32_t w = (lane < kScanBlock / 32) ? warp_tot[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < kScanBlock / 32) warp_tot[lane] = wi - w;
        const uint32_t total = __shfl_sync(0xffffffffu, wi, kScanBlock / 32 - 1);   // the tile's sum
        uint32_t prefix = 0;
        if (t == 0) {
            if (lane == 0) st_release_u64(tiles, (2ull << 32) | total);
        } else {
            if (lane == 0) st_release_u64(tiles + t, (1ull << 32) | total);
            // the warp reads 32 tiles at once, nearest first (lane l: tile p0 - l);
            // before tile 0 counts as an inclusive prefix of 0
            for (int64_t p0 = t - 1;; p0 -= 32) {
                const int64_t p = p0 - lane;
                unsigned long long x = 2ull << 32;
                if (p >= 0) {
                    x = ld_acquire_u64(tiles + p);
                    for (int spin = 0; (x >> 32) == 0 && spin < kLookbackSpins; ++spin) x = ld_acquire_u64(tiles + p);
                    if ((x >> 32) == 0) {
                        set_flag(flag, LSK_FLAG_TIMEOUT);
                        x = 2ull << 32;
                    }
                }
                const unsigned incl_lanes = __ballot_sync(0xffffffffu, (x >> 32) == 2);
                const int stop = incl_lanes ? __ffs(incl_lanes) - 1 : 31;   // the nearest inclusive prefix
                uint32_t val = lane <= stop ? (uint32_t)x : 0u;
#pragma unroll
                for (int o = 16; o; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
                prefix += val;
                if (incl_lanes) break;
            }
            if (lane == 0) st_release_u64(tiles + t, (2ull << 32) | (prefix + total));
        }
        if (lane == 0) {
            s_prefix = prefix;
            if ((t + 1) * kScanTile >= len) off[len] = prefix + total;   // the last tile: the total
        }
    }
    __syncthreads();
    const uint32_t excl = s_prefix + warp_tot[wid] + incl - run;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        const int64_t i = base + q;
        if (i < len) {
            off[i] = v[q] + excl;
            if (cursor) cursor[i] = v[q] + excl;
        }
    }
}

// ---- two-level counting sort of the rows by bucket --------------------------
// The permutation of count / scan / place with the per-row atomics in shared
// memory instead of L2, and every write coalesced: bucket b splits into
// coarse c = b >> shift and fine f = b & (F - 1).  (1) block k hashes its
// chunk of rows, keeps (bucket | sign) per row and counts its rows per
// coarse bucket in shared memory; (2) the counts, laid out coarse bucket by
// coarse bucket and block by block, are scanned in place (the look-back
// scan): each block's offset inside each coarse bucket; (3) each block sorts
// its chunk by coarse bucket in shared memory and writes each coarse bucket's
// run contiguously (row | sign, and f); (4) block c counts coarse bucket c's
// rows per fine bucket, scans the counts (the offsets of its F buckets),
// sorts the rows by fine bucket in shared memory and writes them
// contiguously.  F makes a coarse bucket ~kRxRowsPerCoarse rows on average.
constexpr int kRxThreads = 512;
constexpr int64_t kRxMaxFine = 4096;
constexpr int64_t kRxMaxCoarse = 2048;
constexpr int64_t kRxRowsPerCoarse = 8192;
constexpr int64_t kRxChunk = 16384;        // rows a block sorts in shared memory (step 3)
constexpr int64_t kRxStage = 16384;        // rows of a coarse bucket sorted in shared memory (step 4)
struct RxPlan {
    int64_t F, B, chunk;
    int shift, nct;
};
bool rx_plan(int64_t n, int64_t r, RxPlan& q) {
    if (n <= 0 || n >= ((int64_t)1 << 31) || r < 1) return false;
    int64_t F = 1;
    int sh = 0;
    while (F < kRxMaxFine && n * (F * 2) <= kRxRowsPerCoarse * r) {
        F *= 2;
        ++sh;
    }
    if (n * F > 2 * kRxRowsPerCoarse * r) return false;   // few buckets for many rows: the atomic form
    const int64_t B = (r + F - 1) / F;
    if (B > kRxMaxCoarse) return false;
    int64_t nct = (n + kRxChunk - 1) / kRxChunk;
    if (nct < 256) nct = 256;
    if (B * nct > ((int64_t)1 << 24)) return false;
    q.F = F;
    q.B = B;
    q.shift = sh;
    q.nct = (int)nct;
    q.chunk = (n + nct - 1) / nct;
    return true;
}
size_t rx_scatter_smem(const RxPlan& q) { return (size_t)q.B * 12 + 16 + (size_t)q.chunk * 8; }
size_t rx_fine_smem(const RxPlan& q) { return (size_t)q.F * 4 + (size_t)kRxStage * 4; }

// block-wide exclusive scan of cnt[0 .. len) in shared memory (len <=
// 8 kRxThreads), in place; `tot` receives the total
__device__ __forceinline__ void rx_block_scan(uint32_t* cnt, int len, uint32_t* wsum, uint32_t& tot) {
    const int per = (len + kRxThreads - 1) / kRxThreads;
    const int lo = (int)threadIdx.x * per, hi = min(len, lo + per);
    uint32_t run = 0;
    for (int i = lo; i < hi; ++i) run += cnt[i];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        const uint32_t x = lane < kRxThreads / 32 ? wsum[lane] : 0u;
        uint32_t xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o) xi += y;
        }
        if (lane < kRxThreads / 32) wsum[lane] = xi - x;
        if (lane == 31) wsum[kRxThreads / 32] = xi;
    }
    __syncthreads();
    uint32_t acc = wsum[w] + incl - run;
    for (int i = lo; i < hi; ++i) {
        const uint32_t c = cnt[i];
        cnt[i] = acc;
        acc += c;
    }
    tot = wsum[kRxThreads / 32];
    __syncthreads();
}

__global__ void __launch_bounds__(kRxThreads) rx_count_kernel(int64_t n, uint64_t row0, uint32_t r, uint32_t k0,
                                                              uint32_t k1, RxPlan q, uint32_t* __restrict__ bsign,
                                                              uint32_t* __restrict__ H, unsigned long long* hstate,
                                                              int hstate_words) {
    extern __shared__ uint32_t hs[];
    if (blockIdx.x == 0)   // the scan's state, zeroed for the next launch
        for (int j = threadIdx.x; j < hstate_words; j += blockDim.x) hstate[j] = 0ull;
    for (int64_t c = threadIdx.x; c < q.B; c += blockDim.x) hs[c] = 0u;
    __syncthreads();
    const int64_t i0 = (int64_t)blockIdx.x * q.chunk, i1 = min(n, i0 + q.chunk);
    for (int64_t i = i0 + threadIdx.x; i < i1; i += (int64_t)kPrepRows * kRxThreads) {
        uint32_t b[kPrepRows], neg[kPrepRows];
#pragma unroll
        for (int u = 0; u < kPrepRows; ++u)
            if (i + u * kRxThreads < i1) cs_hash(row0 + (uint64_t)(i + u * kRxThreads), r, k0, k1, b[u], neg[u]);
#pragma unroll
        for (int u = 0; u < kPrepRows; ++u) {
            if (i + u * kRxThreads < i1) {
                bsign[i + u * kRxThreads] = b[u] | (neg[u] << 31);
                atomicAdd(&hs[b[u] >> q.shift], 1u);
            }
        }
    }
    __syncthreads();
    for (int64_t c = threadIdx.x; c < q.B; c += blockDim.x) H[c * q.nct + blockIdx.x] = hs[c];
}

// step 3: shared memory holds the global base and the local offset (then the
// cursor) of every coarse bucket, and the chunk sorted by coarse bucket as
// (row | sign, fine | coarse << 16)
__global__ void __launch_bounds__(kRxThreads) rx_scatter_kernel(int64_t n, RxPlan q,
                                                                const uint32_t* __restrict__ bsign,
                                                                const uint32_t* __restrict__ base,
                                                                uint32_t* __restrict__ T, uint16_t* __restrict__ TF) {
    extern __shared__ uint32_t sm[];
    __shared__ uint32_t wsum[kRxThreads / 32 + 1];
    uint32_t* hb = sm;                 // [B] global start of this block's run in coarse bucket c
    uint32_t* lo = sm + q.B;           // [B] local start of coarse bucket c in the sorted chunk
    uint32_t* cur = sm + 2 * q.B;      // [B] cursor
    uint2* stage = reinterpret_cast<uint2*>(sm + ((3 * q.B + 3) & ~(int64_t)1));
    for (int64_t c = threadIdx.x; c < q.B; c += blockDim.x) {
        const int64_t idx = c * q.nct + blockIdx.x;
        const uint32_t b0 = __ldg(base + idx);
        hb[c] = b0;
        lo[c] = __ldg(base + idx + 1) - b0;   // this block's rows in coarse bucket c
    }
    __syncthreads();
    uint32_t tot;
    rx_block_scan(lo, (int)q.B, wsum, tot);
    for (int64_t c = threadIdx.x; c < q.B; c += blockDim.x) cur[c] = lo[c];
    __syncthreads();
    const int64_t i0 = (int64_t)blockIdx.x * q.chunk, i1 = min(n, i0 + q.chunk);
    const uint32_t fmask = (uint32_t)q.F - 1u;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += kRxThreads) {
        const uint32_t v = __ldg(bsign + i);
        const uint32_t b = v & 0x7fffffffu, c = b >> q.shift;
        const uint32_t p = atomicAdd(&cur[c], 1u);
        stage[p] = make_uint2((uint32_t)i | (v & 0x80000000u), (b & fmask) | (c << 16));
    }
    __syncthreads();
    for (uint32_t p = threadIdx.x; p < tot; p += kRxThreads) {
        const uint2 e = stage[p];
        const uint32_t c = e.y >> 16;
        const uint32_t g = hb[c] + (p - lo[c]);
        T[g] = e.x;
        TF[g] = (uint16_t)(e.y & 0xffffu);
    }
}

// step 4: block c, rows [s, e) of coarse bucket c
__global__ void __launch_bounds__(kRxThreads) rx_fine_kernel(int64_t n, int64_t r, RxPlan q,
                                                             const uint32_t* __restrict__ base,
                                                             const uint32_t* __restrict__ T,
                                                             const uint16_t* __restrict__ TF,
                                                             uint32_t* __restrict__ perm, uint32_t* __restrict__ off) {
    extern __shared__ uint32_t fc[];   // [F] counts, then starts; then the staged rows
    __shared__ uint32_t wsum[kRxThreads / 32 + 1];
    uint32_t* stage = fc + q.F;
    const int64_t c = blockIdx.x;
    const uint32_t s = __ldg(base + c * q.nct);
    const uint32_t e = (c + 1 < q.B) ? __ldg(base + (c + 1) * q.nct) : (uint32_t)n;
    for (int f = threadIdx.x; f < (int)q.F; f += kRxThreads) fc[f] = 0u;
    __syncthreads();
    for (uint32_t i = s + threadIdx.x; i < e; i += kRxThreads) atomicAdd(&fc[__ldg(TF + i)], 1u);
    __syncthreads();
    uint32_t tot;
    rx_block_scan(fc, (int)q.F, wsum, tot);
    for (int f = threadIdx.x; f < (int)q.F; f += kRxThreads) {
        const int64_t b = c * q.F + f;
        if (b < r) off[b] = s + fc[f];
    }
    if (c == q.B - 1 && threadIdx.x == 0) off[r] = (uint32_t)n;
    __syncthreads();
    if (e - s <= (uint32_t)kRxStage) {
        // sorted in shared memory, then written contiguously
        for (uint32_t i = s + threadIdx.x; i < e; i += kRxThreads) {
            const uint32_t p = atomicAdd(&fc[__ldg(TF + i)], 1u);
            stage[p] = __ldg(T + i);
        }
        __syncthreads();
        for (uint32_t p = threadIdx.x; p < e - s; p += kRxThreads) perm[s + p] = stage[p];
    } else {
        for (uint32_t i = s + threadIdx.x; i < e; i += kRxThreads) {
            const uint32_t p = atomicAdd(&fc[__ldg(TF + i)], 1u);
            perm[s + p] = __ldg(T + i);
        }
    }
}

// ---- dense gather ---------------------------------------------------------
// One warp per bucket part.  Lanes own VEC consecutive columns in each of U
// column groups of 32*VEC; the rows are fetched kBatch at a time so that
// each warp keeps kBatch rows of loads in flight.  With few buckets (small r,
// long buckets) each bucket's row list is cut into P contiguous parts, one
// warp each, so that enough warps stream A; their sums are then added into
// SA (zeroed first) atomically.  With P = 1 each warp stores its bucket.
template <int VEC>
struct VecT;
template <>
struct VecT<4> {
    using T = float4;
};
template <>
struct VecT<1> {
    using T = float;
};

__device__ __forceinline__ void vadd(float4& a, const float4& b, float s) {
    a.x = fmaf(s, b.x, a.x);
    a.y = fmaf(s, b.y, a.y);
    a.z = fmaf(s, b.z, a.z);
    a.w = fmaf(s, b.w, a.w);
}
__device__ __forceinline__ void vadd(float& a, const float& b, float s) { a = fmaf(s, b, a); }
__device__ __forceinline__ void vzero(float4& a) { a = make_float4(0.f, 0.f, 0.f, 0.f); }
__device__ __forceinline__ void vzero(float& a) { a = 0.f; }
__device__ __forceinline__ void vatomic_add(float4* p, const float4& v) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}
__device__ __forceinline__ void vatomic_add(float* p, const float& v) { atomicAdd(p, v); }

template <int VEC>
__device__ __forceinline__ typename VecT<VEC>::T ldg_stream(const float* p) {
    if constexpr (VEC == 4) {
        float4 v;
        asm("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
                     : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                     : "l"(p));
        return v;
    } else {
        float v;
        asm("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
        return v;
    }
}

template <int VEC, int U>
__global__ void __launch_bounds__(256) cs_dense_gather_kernel(
    const float* __restrict__ A, int64_t lda, int64_t d, uint32_t r,
    const uint32_t* __restrict__ off, const uint32_t* __restrict__ perm, float* __restrict__ SA, int P,
    int accumulate, const uint32_t* __restrict__ cpos) {
    using V = typename VecT<VEC>::T;
    constexpr int kCols = 32 * VEC * U;  // columns per pass
    constexpr int kBatch = (VEC * U >= 8) ? 8 : 4;   // rows of loads in flight per warp
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t items = (int64_t)r * P;
    for (int64_t vb = warp; vb < items; vb += nwarps) {
        const int64_t b = vb / P;
        const uint32_t part = (uint32_t)(vb % P);
        const uint32_t s0 = off[b], len = off[b + 1] - s0;
        const uint32_t s = s0 + (uint32_t)(((uint64_t)len * part) / P);
        const uint32_t e = s0 + (uint32_t)(((uint64_t)len * (part + 1)) / P);
        if ((P > 1 || accumulate || cpos) && s == e) continue;
        const int64_t orow = cpos ? (int64_t)cpos[b] : b;   // compacted: the bucket's rank among the non-empty
        for (int64_t c0 = 0; c0 < d; c0 += kCols) {
            V acc[U];
#pragma unroll
            for (int u = 0; u < U; ++u) vzero(acc[u]);
            bool colok[U];
#pragma unroll
            for (int u = 0; u < U; ++u) colok[u] = (c0 + (int64_t)(u * 32 + lane) * VEC) < d;
            for (uint32_t t0 = s; t0 < e; t0 += 32) {
                const uint32_t m = min(32u, e - t0);
                const uint32_t mine = (lane < (int)m) ? perm[t0 + lane] : 0u;
                uint32_t j = 0;
                for (; j + kBatch <= m; j += kBatch) {
                    V v[kBatch][U];
                    float sg[kBatch];
#pragma unroll
                    for (int q = 0; q < kBatch; ++q) {
                        const uint32_t p = __shfl_sync(0xffffffffu, mine, j + q);
                        sg[q] = (p >> 31) ? -1.0f : 1.0f;
                        const float* row = A + (int64_t)(p & 0x7fffffffu) * lda + c0;
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            if (colok[u]) v[q][u] = ldg_stream<VEC>(row + (u * 32 + lane) * VEC);
                            else vzero(v[q][u]);
                        }
                    }
#pragma unroll
                    for (int q = 0; q < kBatch; ++q)
#pragma unroll
                        for (int u = 0; u < U; ++u) vadd(acc[u], v[q][u], sg[q]);
                }
                for (; j < m; ++j) {
                    const uint32_t p = __shfl_sync(0xffffffffu, mine, j);
                    const float sg = (p >> 31) ? -1.0f : 1.0f;
                    const float* row = A + (int64_t)(p & 0x7fffffffu) * lda + c0;
#pragma unroll
                    for (int u = 0; u < U; ++u)
                        if (colok[u]) vadd(acc[u], ldg_stream<VEC>(row + (u * 32 + lane) * VEC), sg);
                }
            }
            float* out = SA + orow * d + c0;
            if (P == 1 && !accumulate) {
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (colok[u]) *reinterpret_cast<V*>(out + (u * 32 + lane) * VEC) = acc[u];
            } else {
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (colok[u]) vatomic_add(reinterpret_cast<V*>(out + (u * 32 + lane) * VEC), acc[u]);
            }
        }
    }
}

// ---- CSR gather -----------------------------------------------------------
// One warp per bucket part (P parts per bucket as in the dense gather); the
// part's row of SA lives in shared memory (d floats per warp).  Lane t handles the t-th row of the bucket's list and
// adds its nonzeros with shared-memory atomics (columns of different rows
// may collide).  Out-of-range row pointers or column indices are skipped
// and reported through the BAD_CSR flag.
__global__ void cs_csr_gather_kernel(const float* __restrict__ V, const int32_t* __restrict__ J,
                                     const int64_t* __restrict__ I, int64_t nnz, int64_t d,
                                     uint32_t r, const uint32_t* __restrict__ off,
                                     const uint32_t* __restrict__ perm, float* __restrict__ SA,
                                     int* flag, int P, int accumulate, const uint32_t* __restrict__ cpos) {
    extern __shared__ float srow[];
    const int lane = threadIdx.x & 31;
    float* acc = srow + (int64_t)(threadIdx.x >> 5) * d;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t items = (int64_t)r * P;
    for (int64_t vb = warp; vb < items; vb += nwarps) {
        const int64_t b = vb / P;
        const uint32_t part = (uint32_t)(vb % P);
        const uint32_t s0 = off[b], len = off[b + 1] - s0;
        const uint32_t s = s0 + (uint32_t)(((uint64_t)len * part) / P);
        const uint32_t e = s0 + (uint32_t)(((uint64_t)len * (part + 1)) / P);
        if ((P > 1 || accumulate || cpos) && s == e) continue;
        for (int64_t c = lane; c < d; c += 32) acc[c] = 0.0f;
        __syncwarp();
        bool bad = false;
        for (uint32_t t = s + lane; t < e; t += 32) {
            const uint32_t p = perm[t];
            const float sg = (p >> 31) ? -1.0f : 1.0f;
            const int64_t row = p & 0x7fffffffu;
            const int64_t k0 = I[row], k1 = I[row + 1];
            if (k0 < 0 || k1 < k0 || k1 > nnz) {
                bad = true;
                continue;
            }
            for (int64_t kk = k0; kk < k1; ++kk) {
                const int32_t col = __ldg(J + kk);
                if (col < 0 || col >= d) {
                    bad = true;
                    continue;
                }
                atomicAdd(&acc[col], sg * __ldg(V + kk));
            }
        }
        if (bad) set_flag(flag, LSK_FLAG_BAD_CSR);
        __syncwarp();
        float* out = SA + (cpos ? (int64_t)cpos[b] : b) * d;
        if (P == 1 && !accumulate) {
            for (int64_t c = lane; c < d; c += 32) out[c] = acc[c];
        } else {
            for (int64_t c = lane; c < d; c += 32)
                if (acc[c] != 0.0f) atomicAdd(out + c, acc[c]);
        }
        __syncwarp();
    }
}

__global__ void cs_hash_debug_kernel(int64_t n, uint32_t r, uint32_t k0, uint32_t k1,
                                     int32_t* bucket, int8_t* sign) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        uint32_t b, neg;
        cs_hash((uint64_t)i, r, k0, k1, b, neg);
        bucket[i] = (int32_t)b;
        sign[i] = neg ? (int8_t)-1 : (int8_t)1;
    }
}

// Compaction of the sketch's rows to the non-empty buckets (off[b + 1] >
// off[b]), in bucket order: cpos[b] = the number of non-empty buckets before b,
// cidx[cpos[b]] = b for each non-empty b, *ccount = their number.  One block
// of 1024 threads, rounds of 4096 buckets (4 consecutive a thread) with the
// running total carried across rounds.
__device__ __forceinline__ void compact_body(const uint32_t* __restrict__ off, int64_t r, uint32_t* __restrict__ cpos,
                                             uint32_t* __restrict__ cidx, uint32_t* __restrict__ ccount) {
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t carry_s;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t carry = 0;
    for (int64_t r0 = 0; r0 < r; r0 += 4096) {
        const int64_t b0 = r0 + 4 * (int64_t)threadIdx.x;
        uint32_t f[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) f[q] = (b0 + q < r && off[b0 + q + 1] > off[b0 + q]) ? 1u : 0u;
        const uint32_t run = f[0] + f[1] + f[2] + f[3];
        uint32_t incl = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wsum[w] = incl;
        __syncthreads();
        if (w == 0) {
            uint32_t v = wsum[lane], vi = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, vi, o);
                if (lane >= o) vi += y;
            }
            wsum[lane] = vi - v;   // exclusive warp offsets
            if (lane == 31) carry_s = vi;
        }
        __syncthreads();
        uint32_t pos = carry + wsum[w] + incl - run;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (b0 + q < r) {
                cpos[b0 + q] = pos;
                if (f[q]) cidx[pos] = (uint32_t)(b0 + q);
            }
            pos += f[q];
        }
        carry += carry_s;
        __syncthreads();
    }
    if (threadIdx.x == 0) *ccount = carry;
}
__global__ void __launch_bounds__(1024) cs_compact_kernel(const uint32_t* __restrict__ off, int64_t r,
                                                          uint32_t* __restrict__ cpos, uint32_t* __restrict__ cidx,
                                                          uint32_t* __restrict__ ccount) {
    compact_body(off, r, cpos, cidx, ccount);
}

// ---- grouped preparation: the permutations of many problems, three launches
// The problems' rows are numbered consecutively (problem p owns rows
// rowoff[p] .. rowoff[p + 1] - 1) and their counters too (problem p's r + 1
// counters from cnt_base); one exclusive scan over all the counters then
// gives each bucket its range of the shared permutation, so the problems'
// rows land in consecutive blocks of it and each problem's off[] (its slice
// of the scanned counters) indexes that shared permutation directly.
struct CsGp {
    int64_t n, r, cnt_base;
    uint32_t k0, k1;
    uint32_t* cidx;     // compaction (or null)
    uint32_t* ccount;
};

__device__ __forceinline__ int job_of(const int64_t* __restrict__ rowoff, int count, int64_t g) {
    int lo = 0, hi = count - 1;   // largest p with rowoff[p] <= g
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(rowoff + mid) <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void cs_count_grouped_kernel(const CsGp* __restrict__ ps, const int64_t* __restrict__ rowoff, int count,
                                        int64_t rows, uint32_t* __restrict__ cnt) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < rows; g += stride) {
        const int p = job_of(rowoff, count, g);
        const CsGp& j = ps[p];
        uint32_t b, neg;
        cs_hash((uint64_t)(g - __ldg(rowoff + p)), (uint32_t)j.r, j.k0, j.k1, b, neg);
        atomicAdd(&cnt[j.cnt_base + b], 1u);
    }
}

__global__ void cs_place_grouped_kernel(const CsGp* __restrict__ ps, const int64_t* __restrict__ rowoff, int count,
                                        int64_t rows, uint32_t* __restrict__ cursor, uint32_t* __restrict__ perm) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < rows; g += stride) {
        const int p = job_of(rowoff, count, g);
        const CsGp& j = ps[p];
        const uint32_t i = (uint32_t)(g - __ldg(rowoff + p));
        uint32_t b, neg;
        cs_hash((uint64_t)i, (uint32_t)j.r, j.k0, j.k1, b, neg);
        perm[atomicAdd(&cursor[j.cnt_base + b], 1u)] = i | (neg << 31);
    }
}

// block p: problem p's compaction (if it has one)
__global__ void __launch_bounds__(1024) cs_compact_grouped_kernel(const CsGp* __restrict__ ps,
                                                                  const uint32_t* __restrict__ off,
                                                                  uint32_t* __restrict__ cpos) {
    const CsGp& j = ps[blockIdx.x];
    if (!j.cidx) return;
    compact_body(off + j.cnt_base, j.r, cpos + j.cnt_base, j.cidx, j.ccount);
}

inline unsigned grid_for(int64_t items, int threads, int sm_count, int per_sm = 8) {
    int64_t g = (items + threads - 1) / threads;
    const int64_t cap = (int64_t)sm_count * per_sm;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (unsigned)g;
}

}  // namespace

// the look-back scan's ticket and tile words
size_t scan_state_words(int64_t len) { return (size_t)((len + kScanTile - 1) / kScanTile) + 1; }

// The CountSketch workspace, in this order: the counters and the scan's
// state (zeroed by one memset), the bucket offsets, the cursors, the
// permutation, the multi-level scan's scratch, the compaction positions;
// then, for the two-level sort, the per-row (bucket | sign), the rows
// grouped by coarse bucket with their fine indices, the per-block counts
// (scanned in place) and their scan state.
struct CsWs {
    uint32_t *cnt, *off, *cursor, *perm, *tmp, *cpos;
    unsigned long long* state;
    uint32_t *bsign, *T, *H;
    uint16_t* TF;
    unsigned long long* hstate;
    int hstate_words;
    size_t bytes;
};
CsWs cs_carve(void* ws, int64_t n, int64_t r, const RxPlan* q) {
    WsCarver wc{(char*)ws, 0};
    CsWs w{};
    const size_t nn = n > 0 ? (size_t)n : 1;
    w.cnt = wc.take<uint32_t>(r + 1);
    w.state = wc.take<unsigned long long>(scan_state_words(r));
    w.off = wc.take<uint32_t>(r + 1);
    w.cursor = wc.take<uint32_t>(r + 1);
    w.perm = wc.take<uint32_t>(nn);
    w.tmp = wc.take<uint32_t>(scan_tmp_words(r));
    w.cpos = wc.take<uint32_t>(r + 1);
    if (q) {
        w.bsign = wc.take<uint32_t>(nn);
        w.T = wc.take<uint32_t>(nn);
        w.TF = wc.take<uint16_t>(nn);
        w.H = wc.take<uint32_t>((size_t)q->B * q->nct + 1);
        w.hstate_words = (int)scan_state_words(q->B * q->nct);
        w.hstate = wc.take<unsigned long long>((size_t)w.hstate_words);
    }
    w.bytes = ws_round(wc.off) + 256;
    return w;
}

size_t cs_workspace_bytes(int64_t n, int64_t r) {
    RxPlan q;
    return cs_carve(nullptr, n, r, rx_plan(n, r, q) ? &q : nullptr).bytes;
}
size_t cs_workspace_bytes_atomic(int64_t n, int64_t r) { return cs_carve(nullptr, n, r, nullptr).bytes; }

cudaError_t cs_hash_launch(int64_t n, int64_t r, uint64_t seed, int32_t* bucket, int8_t* sign,
                           cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    cs_hash_debug_kernel<<<grid_for(n, 256, 152, 16), 256, 0, st>>>(
        n, (uint32_t)r, (uint32_t)seed, (uint32_t)(seed >> 32), bucket, sign);
    return cudaGetLastError();
}

// Steps 1-3 (count, scan, place): on return *off_out (r + 1 entries, off[r] = n)
// and *perm_out (n entries, local row indices) point into ws; the launches
// are queued on st.  Row i is hashed as column row0 + i of S.  rx: ws holds
// cs_workspace_bytes (the two-level sort where its plan applies), else
// cs_workspace_bytes_atomic (count / scan / place with L2 atomics).
cudaError_t cs_prep_launch(int64_t n, int64_t r, uint64_t seed, void* ws, int sm_count, cudaStream_t st,
                           const uint32_t** off_out, const uint32_t** perm_out, uint64_t row0, int* flag, bool rx) {
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    RxPlan q;
    const bool two_level = rx && rx_plan(n, r, q);
    const CsWs w = cs_carve(ws, n, r, two_level ? &q : nullptr);
    cudaError_t e;
    if (two_level) {
        if ((e = allow_dynamic_smem(rx_scatter_kernel)) != cudaSuccess) return e;
        if ((e = allow_dynamic_smem(rx_fine_kernel)) != cudaSuccess) return e;
        LSK_PROF("cs_count", st) rx_count_kernel<<<q.nct, kRxThreads, (size_t)q.B * 4, st>>>(
            n, row0, (uint32_t)r, k0, k1, q, w.bsign, w.H, w.hstate, w.hstate_words);
        const int64_t len = q.B * q.nct;
        LSK_PROF("cs_scan", st) scan_lookback_kernel<<<(unsigned)((len + kScanTile - 1) / kScanTile), kScanBlock, 0,
                                                       st>>>(w.H, w.H, nullptr, len, w.hstate, flag);
        LSK_PROF("cs_place", st) rx_scatter_kernel<<<q.nct, kRxThreads, rx_scatter_smem(q), st>>>(n, q, w.bsign, w.H,
                                                                                                  w.T, w.TF);
        LSK_PROF("cs_fine", st) rx_fine_kernel<<<(unsigned)q.B, kRxThreads, rx_fine_smem(q), st>>>(n, r, q, w.H, w.T,
                                                                                                   w.TF, w.perm, w.off);
        *off_out = w.off;
        *perm_out = w.perm;
        return cudaGetLastError();
    }
    // the counters and the scan's state are contiguous: one memset
    e = cudaMemsetAsync(w.cnt, 0, (size_t)((char*)(w.state + scan_state_words(r)) - (char*)w.cnt), st);
    if (e != cudaSuccess) return e;
    if (n > 0) LSK_PROF("cs_count", st) cs_count_kernel<<<grid_for(n, 256, sm_count), 256, 0, st>>>(n, row0, (uint32_t)r, k0, k1, w.cnt);
    const unsigned tiles = (unsigned)((r + kScanTile - 1) / kScanTile);
    LSK_PROF("cs_scan", st) scan_lookback_kernel<<<tiles, kScanBlock, 0, st>>>(w.cnt, w.off, w.cursor, r, w.state, flag);
    if (n > 0) {
        LSK_PROF("cs_place", st) cs_place_kernel<<<grid_for(n, 256, sm_count), 256, 0, st>>>(n, row0, (uint32_t)r, k0, k1, w.cursor, w.perm);
    }
    *off_out = w.off;
    *perm_out = w.perm;
    return cudaGetLastError();
}

cudaError_t cs_launch(const lsk_mat* A, int64_t r, uint64_t seed, float* SA, void* ws, int* flag,
                      int sm_count, cudaStream_t st, uint64_t row0, bool accumulate, uint32_t* cidx,
                      uint32_t* ccount, bool rx) {
    const int64_t n = A->n;
    const uint32_t* off = nullptr;
    const uint32_t* perm = nullptr;
    cudaError_t e = cs_prep_launch(n, r, seed, ws, sm_count, st, &off, &perm, row0, flag, rx);
    if (e != cudaSuccess) return e;
    const bool compact = cidx != nullptr && ccount != nullptr && !accumulate;
    uint32_t* cpos = nullptr;
    if (compact) {
        cpos = cs_carve(ws, n, r, nullptr).cpos;   // the same place in either form
        LSK_PROF("cs_compact", st) cs_compact_kernel<<<1, 1024, 0, st>>>(off, r, cpos, cidx, ccount);
    }
    return cs_gather_launch(A, r, off, perm, cpos, SA, flag, sm_count, st, accumulate);
}

cudaError_t cs_gather_launch(const lsk_mat* A, int64_t r, const uint32_t* off, const uint32_t* perm,
                             const uint32_t* cpos, float* SA, int* flag, int sm_count, cudaStream_t st,
                             bool accumulate) {
    const int64_t n = A->n, d = A->d;
    cudaError_t e = cudaSuccess;
    const bool compact = cpos != nullptr;
    // parts per bucket: enough warps to stream A when there are few buckets,
    // while each part keeps several rows (one part a bucket when compacting)
    int P = 1;
    while (!compact && P < 32 && r * P < 16384 && n >= (int64_t)r * P * 8) P *= 2;
    if (P > 1 && !accumulate && (e = cudaMemsetAsync(SA, 0, (size_t)r * d * 4, st)) != cudaSuccess) return e;
    const int acc = accumulate ? 1 : 0;   // add into SA (the parts add atomically either way)
    const int64_t warps_needed = r * P;
    if (A->kind == LSK_DENSE) {
        const float* Av = (const float*)A->values;
        const bool vec4 = (d % 4 == 0) && (A->ld % 4 == 0) && (((uintptr_t)Av & 15) == 0) &&
                          (((uintptr_t)SA & 15) == 0);
        const unsigned grid = grid_for(warps_needed * 32, 256, sm_count, 8);
        if (vec4) {
            if (d <= 128)
                LSK_PROF("cs_dense_gather", st) cs_dense_gather_kernel<4, 1><<<grid, 256, 0, st>>>(Av, A->ld, d, (uint32_t)r, off, perm, SA, P, acc, cpos);
            else
                LSK_PROF("cs_dense_gather", st) cs_dense_gather_kernel<4, 2><<<grid, 256, 0, st>>>(Av, A->ld, d, (uint32_t)r, off, perm, SA, P, acc, cpos);
        } else {
            if (d <= 32)
                LSK_PROF("cs_dense_gather", st) cs_dense_gather_kernel<1, 1><<<grid, 256, 0, st>>>(Av, A->ld, d, (uint32_t)r, off, perm, SA, P, acc, cpos);
            else
                LSK_PROF("cs_dense_gather", st) cs_dense_gather_kernel<1, 2><<<grid, 256, 0, st>>>(Av, A->ld, d, (uint32_t)r, off, perm, SA, P, acc, cpos);
        }
    } else {
        // shared-memory row per warp: pick warps per block to fit 200 KB
        int warps = 8;
        while (warps > 1 && (size_t)warps * d * 4 > 200 * 1024) warps >>= 1;
        const size_t smem = (size_t)warps * d * 4;
        if (smem > 200 * 1024) return cudaErrorInvalidValue;
        if (smem > 48 * 1024) {
            e = allow_dynamic_smem(cs_csr_gather_kernel);
            if (e != cudaSuccess) return e;
        }
        const int threads = warps * 32;
        int64_t g = (warps_needed + warps - 1) / warps;
        const int64_t cap = (int64_t)sm_count * 32 / warps * 2;
        if (g > cap) g = cap;
        if (g < 1) g = 1;
        LSK_PROF("cs_csr_gather", st) cs_csr_gather_kernel<<<(unsigned)g, threads, smem, st>>>(
            (const float*)A->values, A->colidx, A->rowptr, A->nnz, d, (uint32_t)r, off, perm, SA, flag, P, acc, cpos);
    }
    return cudaGetLastError();
}

size_t cs_group_ws_bytes(int64_t rows, int64_t counters) {
    return ws_round((size_t)counters * 4) * 4 + ws_round((size_t)(rows > 0 ? rows : 1) * 4) +
           ws_round(scan_tmp_words(counters) * 4) + 2048;
}

void cs_group_build(std::vector<CsJob>& jobs, void* ws, HostTable& t, CsGroup& g) {
    std::vector<CsGp> ps(jobs.size());
    std::vector<int64_t> rowoff(jobs.size() + 1, 0);
    int64_t cb = 0;
    g.any_compact = false;
    for (size_t i = 0; i < jobs.size(); ++i) {
        CsJob& j = jobs[i];
        j.cnt_base = cb;
        ps[i] = CsGp{j.n, j.r, cb, (uint32_t)j.seed, (uint32_t)(j.seed >> 32), j.cidx, j.ccount};
        rowoff[i + 1] = rowoff[i] + j.n;
        cb += j.r + 1;
        g.any_compact = g.any_compact || j.cidx != nullptr;
    }
    g.count = (int)jobs.size();
    g.rows = rowoff.back();
    g.counters = cb;
    WsCarver wc{(char*)ws, 0};
    g.cnt = wc.take<uint32_t>((size_t)g.counters);
    g.off = wc.take<uint32_t>((size_t)g.counters);
    g.cursor = wc.take<uint32_t>((size_t)g.counters);
    g.cpos = wc.take<uint32_t>((size_t)g.counters);
    g.perm = wc.take<uint32_t>((size_t)(g.rows > 0 ? g.rows : 1));
    g.tmp = wc.take<uint32_t>(scan_tmp_words(g.counters));
    g.params_off = t.put(ps.data(), ps.size());
    g.rowoff_off = t.put(rowoff.data(), rowoff.size());
}

cudaError_t cs_group_launch(const CsGroup& g, const unsigned char* table, int sm_count, cudaStream_t st) {
    if (g.count == 0) return cudaSuccess;
    const CsGp* ps = reinterpret_cast<const CsGp*>(table + g.params_off);
    const int64_t* rowoff = reinterpret_cast<const int64_t*>(table + g.rowoff_off);
    cudaError_t e = cudaMemsetAsync(g.cnt, 0, (size_t)g.counters * 4, st);
    if (e != cudaSuccess) return e;
    if (g.rows > 0)
        LSK_PROF("cs_count", st) cs_count_grouped_kernel<<<grid_for(g.rows, 256, sm_count), 256, 0, st>>>(
            ps, rowoff, g.count, g.rows, g.cnt);
    e = exclusive_scan(g.cnt, g.off, g.counters, g.tmp, st);
    if (e != cudaSuccess) return e;
    if (g.rows > 0) {
        e = cudaMemcpyAsync(g.cursor, g.off, (size_t)g.counters * 4, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
        LSK_PROF("cs_place", st) cs_place_grouped_kernel<<<grid_for(g.rows, 256, sm_count), 256, 0, st>>>(
            ps, rowoff, g.count, g.rows, g.cursor, g.perm);
    }
    if (g.any_compact)
        LSK_PROF("cs_compact", st) cs_compact_grouped_kernel<<<g.count, 1024, 0, st>>>(ps, g.off, g.cpos);
    return cudaGetLastError();
}
