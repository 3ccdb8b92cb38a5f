// tc_common.cuh -- sm_100-family tensor-core building blocks (inline PTX).
//
// tcgen05 MMA with operands in shared memory (128-byte-swizzled, K-major
// canonical layout), accumulators in tensor memory (TMEM), completion
// tracked with mbarriers.  Every wait is bounded by a wall-clock limit; on
// timeout the caller gets `false`, sets the context's TIMEOUT flag and
// winds down (no trap).
#pragma once
#include "lsk_internal.cuh"

#include <cuda.h>

namespace tc {

constexpr uint64_t kWaitLimitNs = 1000000000ull;   // 1 s per wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---- mbarrier ---------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// try_wait with a suspend-time hint: the thread may sleep (up to `ns`) until
// the phase completes instead of returning at once, so a waiting warp does
// not take issue slots from the working ones.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, uint32_t parity, uint32_t ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}
// Wait for the phase with the given parity to complete.  Gives up (returns
// false) after limit_ns or when *abort becomes non-zero.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort,
                                          uint64_t limit_ns = kWaitLimitNs) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    while (true) {
        if (mbar_try_wait_sleep(bar, parity, 20000u)) return true;
        if (*abort) return false;
        if (globaltimer() - t0 > limit_ns) {
            *abort = 1;
            return false;
        }
    }
}

// ---- CTA pairs (cluster of 2, cta_group::2) --------------------------------
__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_id_x() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t nclusters_x() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}
// every thread of both CTAs (release / acquire at cluster scope)
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// arrive on the barrier at the same shared-memory offset in CTA `rank` of the cluster
__device__ __forceinline__ void mbar_arrive_cluster(uint64_t* bar, uint32_t rank) {
    uint32_t remote;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(smem_u32(bar)), "r"(rank));
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(remote) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_sleep_cluster(uint64_t* bar, uint32_t parity, uint32_t ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}
// mbar_wait for a barrier that threads of the peer CTA arrive on
__device__ __forceinline__ bool mbar_wait_cluster(uint64_t* bar, uint32_t parity, volatile int* abort) {
    const uint64_t t0 = globaltimer();
    while (true) {
        if (mbar_try_wait_sleep_cluster(bar, parity, 20000u)) return true;
        if (*abort) return false;
        if (globaltimer() - t0 > kWaitLimitNs) {
            *abort = 1;
            return false;
        }
    }
}

// Wait until the shared-memory counter *ctr reaches `target` (bounded like
// mbar_wait).  Used to hand out the uses of a pipeline stage in order.
__device__ __forceinline__ bool counter_wait(volatile int* ctr, int target, volatile int* abort) {
    if (*ctr >= target) return true;
    const uint64_t t0 = globaltimer();
    while (*ctr < target) {
        __nanosleep(32);   // yield issue slots to the warps doing work
        if (*abort) return false;
        if (globaltimer() - t0 > kWaitLimitNs) {
            *abort = 1;
            return false;
        }
    }
    return true;
}

// ---- TMA (tensor-map bulk copies) ------------------------------------------
// Arrive on a local barrier and raise its expected transaction bytes: the
// phase completes once the arrivals are in and `bytes` have landed.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// Load the box at coordinates (x, y) of a 2-D tensor map into this CTA's
// shared memory at `dst` (1024-byte aligned for the 128-byte swizzle),
// completing `bytes` on `bar`.  x times the element size must be a multiple
// of 16 bytes; out-of-range elements are filled with zeros.
__device__ __forceinline__ void tma_load_2d(void* dst, const void* tmap, int32_t x, int32_t y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void prefetch_tmap(const void* tmap) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tmap)) : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---- TMEM ---------------------------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// cta_group::2: one warp of each CTA of the pair takes part; both CTAs get
// the same columns
__device__ __forceinline__ void tmem_alloc_pair(uint32_t* dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish_pair() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc_pair(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// ---- descriptors ------------------------------------------------------------
// Shared-memory matrix descriptor, K-major, 128-byte swizzle: rows of 128 B
// (64 bf16 along K), 8-row atoms of 1024 B stacked along M/N (SBO = 1024).
// The atom base must be 1024-byte aligned; a K offset inside the atom is
// applied by advancing the start address (32 B per 16 bf16).
__device__ __forceinline__ uint64_t desc_sw128_kmajor(uint32_t smem_addr) {
    uint64_t d = 0;
    d |= (uint64_t)((smem_addr & 0x3FFFFu) >> 4);        // start address
    d |= (uint64_t)1 << 16;                              // LBO (unused for swizzled K-major)
    d |= (uint64_t)(1024u >> 4) << 32;                   // SBO: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                              // fixed 0b001 (sm_100 descriptor version)
    d |= (uint64_t)2 << 61;                              // 128-byte swizzle
    return d;
}

// Same, 64-byte swizzle: rows of 64 B (32 bf16 along K), 8-row atoms of 512 B
// (SBO = 512); the atom base must be 512-byte aligned.
__device__ __forceinline__ uint64_t desc_sw64_kmajor(uint32_t smem_addr) {
    uint64_t d = 0;
    d |= (uint64_t)((smem_addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(512u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;                              // 64-byte swizzle
    return d;
}

// Same, with the 8-row atoms `sbo` bytes apart (a multiple of 512): two
// operands can then interleave atom by atom (the hi / lo halves of a split
// tile at +0 and +512 of every 1024-byte block).
__device__ __forceinline__ uint64_t desc_sw64_kmajor_sbo(uint32_t smem_addr, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((smem_addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;
    return d;
}

// MN-major operand, 128-byte swizzle: atoms of 8 K-rows x 128 bytes (64 bf16
// along M/N, the row of K-index k at 128 k within the atom), atoms `lbo`
// bytes apart along M/N and `sbo` bytes apart along K (the next 8 rows).
// Atom bases must be 1024-byte aligned.
__device__ __forceinline__ uint64_t desc_sw128_mnmajor(uint32_t smem_addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((smem_addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(uint32_t M, uint32_t N) {
    return (1u << 4)            // D format F32
           | (1u << 7)          // A format BF16
           | (1u << 10)         // B format BF16
           | ((N >> 3) << 17)   // N / 8
           | ((M >> 4) << 24);  // M / 16
}
// Same with both operands MN-major (the transpose bits of A and B).
__host__ __device__ constexpr uint32_t idesc_bf16_f32_mn(uint32_t M, uint32_t N) {
    return idesc_bf16_f32(M, N) | (1u << 15) | (1u << 16);
}
// Instruction descriptor, kind::tf32: D = F32, A = B = TF32 (format code 2,
// 32-bit containers of which the MMA uses sign, exponent and the top 10
// mantissa bits), both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32_f32(uint32_t M, uint32_t N) {
    return (1u << 4)            // D format F32
           | (2u << 7)          // A format TF32
           | (2u << 10)         // B format TF32
           | ((N >> 3) << 17)   // N / 8
           | ((M >> 4) << 24);  // M / 16
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// M = 256 across a CTA pair (issued by the even CTA): A rows 0..127 from
// this CTA's shared memory and 128..255 from the peer's (same offsets), B's
// first N/2 rows (K-major) from this CTA and the other N/2 from the peer;
// each CTA's TMEM receives its own 128 rows x N columns.
__device__ __forceinline__ void mma_bf16_pair(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                              uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// The kind::tf32 form of mma_bf16_pair: K = 8 per instruction (32 bytes of a
// 128-byte operand row).
__device__ __forceinline__ void mma_tf32_pair(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                              uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// Arrive on `bar` in both CTAs of the pair when every pair MMA issued so far
// by this thread has completed.
__device__ __forceinline__ void mma_commit_pair(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            smem_u32(bar)),
        "h"((uint16_t)3)
        : "memory");
}

// Arrive on `bar` when every MMA issued so far by this thread has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// 32 lanes x 32 columns of FP32 from TMEM: thread t of the warp gets row
// (lane base + t), columns [col, col + 32).  Asynchronous: the registers are
// valid after tmem_ld_wait().
__device__ __forceinline__ void tmem_ld_32x32b_x32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
          "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
          "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Byte offset of element (row, k) inside a K-major, 128-byte-swizzled bf16
// tile whose rows hold 64 elements: 16-byte chunk (k / 8) of row r is stored
// at chunk position (k / 8) XOR (r mod 8).
__host__ __device__ __forceinline__ uint32_t sw128_offset(uint32_t row, uint32_t k) {
    return (row >> 3) * 1024u + (row & 7u) * 128u + ((((k >> 3) ^ (row & 7u)) & 7u) << 4) + (k & 7u) * 2u;
}

// Byte offset of element (row, k) inside a K-major, 64-byte-swizzled bf16
// tile whose rows hold 32 elements: 16-byte chunk (k / 8) of row r is stored
// at chunk position (k / 8) XOR ((r / 2) mod 4).
__host__ __device__ __forceinline__ uint32_t sw64_offset(uint32_t row, uint32_t k) {
    return (row >> 3) * 512u + (row & 7u) * 64u + ((((k >> 3) ^ (row >> 1)) & 3u) << 4) + (k & 7u) * 2u;
}

// hi = bf16(x), lo = bf16(x - hi): x = hi + lo to ~16 significant bits.
// Packed as bf16x2 words with a (resp. a - hi_a) in the low half.  Six
// instructions a pair: two round-to-nearest-even conversions (cvt packs its
// first source into the high half), the exact widening of hi by shifting /
// masking the bf16 bit patterns into float position, and two subtractions.
__device__ __forceinline__ void split_bf16x2(float a, float b, uint32_t& hi, uint32_t& lo) {
    uint32_t h, l;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(b), "f"(a));
    const float ha = __uint_as_float(h << 16), hb = __uint_as_float(h & 0xFFFF0000u);
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(l) : "f"(b - hb), "f"(a - ha));
    hi = h;
    lo = l;
}

// ---- in-place bf16 split of a landed FP32 tile -------------------------------
// A 1 KB block of 8 rows x 32 FP32 words, as a 128-byte-swizzled TMA copy
// leaves it, becomes the 512-byte 64-byte-swizzled atom of its bf16 hi parts
// (at +0) and that of its lo parts (at +512): 8 rows x 32 bf16 each.  The
// rows are K for a K-major operand and K for an MN-major one alike (the
// descriptor says which); the bytes are the same.
// Lane l splits row l / 4 of the block, K-elements 8 (l % 4) .. +7: two
// 16-byte reads of the FP32 rows (chunk c of row r at 128 r + 16 (c ^ r) under
// the 128-byte swizzle), one 16-byte write each to the hi and lo atoms (chunk
// kc of row r at 64 r + 16 (kc ^ (r / 2)) under the 64-byte swizzle).  All
// reads of the warp's blocks precede the warp barrier, all writes follow it.
template <int NB>
__device__ __forceinline__ void split_blocks_in_place(uint8_t* first_block, int lane) {
    const uint32_t r = (uint32_t)lane >> 2, kc = (uint32_t)lane & 3u;
    const uint32_t rd0 = 128u * r + 16u * ((2u * kc) ^ r), rd1 = 128u * r + 16u * ((2u * kc + 1u) ^ r);
    const uint32_t wr = 64u * r + 16u * ((kc ^ (r >> 1)) & 3u);
    constexpr int kPass = NB % 4 == 0 ? 4 : NB % 2 == 0 ? 2 : 1;   // blocks held in registers at once
#pragma unroll
    for (int b0 = 0; b0 < NB; b0 += kPass) {
        uint4 hi[kPass], lo[kPass];
#pragma unroll
        for (int b = 0; b < kPass; ++b) {
            const uint8_t* blk = first_block + (b0 + b) * 1024;
            const float4 v0 = *reinterpret_cast<const float4*>(blk + rd0);
            const float4 v1 = *reinterpret_cast<const float4*>(blk + rd1);
            split_bf16x2(v0.x, v0.y, hi[b].x, lo[b].x);
            split_bf16x2(v0.z, v0.w, hi[b].y, lo[b].y);
            split_bf16x2(v1.x, v1.y, hi[b].z, lo[b].z);
            split_bf16x2(v1.z, v1.w, hi[b].w, lo[b].w);
        }
        __syncwarp();
#pragma unroll
        for (int b = 0; b < kPass; ++b) {
            uint8_t* blk = first_block + (b0 + b) * 1024;
            *reinterpret_cast<uint4*>(blk + wr) = hi[b];
            *reinterpret_cast<uint4*>(blk + 512 + wr) = lo[b];
        }
    }
}

// ---- tensor maps ------------------------------------------------------------
// cuTensorMapEncodeTiled from the driver (looked up once; null if absent)
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
inline EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = []() -> EncodeTiledFn {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return reinterpret_cast<EncodeTiledFn>(f);
    }();
    return fn;
}

}  // namespace tc
