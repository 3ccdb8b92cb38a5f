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
// After each slice the epilogue warps read the accumulator out of TMEM, hand
// it back to the MMAs at once, and add it into the CTA's running FP32 partial
// in global memory with fire-and-forget vector reductions (one writer per
// address, in program order, so the sums are deterministic); a second kernel
// adds the CTAs' partials in order with a compensated FP32 sum, then forms
// alpha * sum + beta * C.  Warps:
//   0 .. kWorkers-1
//               workers: each owns every kWorkers-th piece of 8 rows (a
//               quarter of a 32-row chunk) and works alone: 16-byte loads of
//               whole rows, a bf16 hi / lo split, and 8-byte stores into the
//               stage's MN-major tiles (no transpose: a row-major chunk of A
//               is MN-major for both operands of A^T A, the instruction
//               descriptor's transpose bits say so).  The uses of each ring
//               stage are claimed in piece order;
//   kWorkers    lane 0 issues, for each 128-column M tile t, the products
//               with columns 128 t .. npad - 1 as the N operand (the same
//               shared-memory tile is both operands; only the upper block
//               triangle is computed);
//   then 8      epilogue: accumulator t is read by the warps whose TMEM lane
//               quarter covers it.
// TMEM holds the two accumulators (N = npad and npad - 128 columns).  Waits
// are bounded; a timeout sets the TIMEOUT flag.
#include "tc_common.cuh"

namespace {

constexpr int kKC = 32;            // rows of A per chunk (the K of the MMAs)
constexpr int kMT = 128;           // rows of an MMA tile (columns of A)
// warp roles: kWorkers workers, one MMA warp, kEpiWarps epilogue warps
template <int W, int E, int PR = 8>
struct GramShape {
    static constexpr int kPieceRows = PR;   // rows of one worker piece
    static constexpr int kPieces = 32 / PR; // pieces per 32-row chunk
    static constexpr int kWorkers = W;
    static constexpr int kMmaWarp = W;
    static constexpr int kEpi0 = W + 1;
    static constexpr int kEpiWarps = E;   // 4 (both accumulators each) or 8 (one each)
    static constexpr int kThreads = (W + 1 + E) * 32;
};
constexpr int kMaxStages = 8;
constexpr int kSliceRows = 1024;   // rows per slice (FP32 accumulation length bound)
constexpr size_t kSmemLimit = 232448;

struct GrParams {
    const float* A;
    int64_t lda, n;
    int d, npad, slices, vec;   // vec: 16-byte loads
    float* part;       // [gridDim][npad][npad] running partials, zeroed before the launch
    int* flag;
};

// Stage layout, per bf16 tile (hi, then lo): MN-major 128-byte-swizzled atoms
// of 8 rows of A (K) x 64 columns of A (M / N), atom (column block mb, row
// group kg) at mb x 1024 + kg x kSbo(npad).  The column blocks run to a whole
// number of 128-column MMA tiles, so an M = 128 operand never reads past its
// tile (columns past d hold zeros, past npad they feed accumulator rows that
// are never read).
__host__ __device__ constexpr uint32_t mn_blocks(int npad) { return 2u * (uint32_t)((npad + kMT - 1) / kMT); }
__host__ __device__ constexpr uint32_t kSbo(int npad) { return mn_blocks(npad) * 1024u; }   // next 8 rows
__host__ __device__ constexpr uint32_t half_bytes(int npad) { return kSbo(npad) * (kKC / 8); }  // one bf16 tile
__host__ __device__ constexpr uint32_t stage_bytes(int npad) { return 2 * half_bytes(npad); }   // hi + lo
// ring depth that fits next to the barriers
__host__ __device__ constexpr int stages_of(int npad) {
    return (int)((232448 - 2048) / stage_bytes(npad)) < kMaxStages ? (int)((232448 - 2048) / stage_bytes(npad))
                                                                     : kMaxStages;
}

// Rows row0 .. row0 + 7 of A (zeros at and past r_end or d), lane t: float4
// number t + 32 h of each row (columns 4 t + 128 h .. + 3): 512 contiguous
// bytes a row per warp instruction.
template <int NPAD, int PR>
__device__ __forceinline__ void load_piece(const GrParams& p, int64_t row0, int64_t r_end, int lane,
                                           float4 (&v)[PR][(NPAD + kMT - 1) / kMT]) {
    constexpr int H = (NPAD + kMT - 1) / kMT;
#pragma unroll
    for (int r = 0; r < PR; ++r) {
        const int64_t row = row0 + r;
        const float* src = p.A + row * p.lda;
#pragma unroll
        for (int h = 0; h < H; ++h) {
            const int c = 4 * lane + kMT * h;
            v[r][h] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (row < r_end && c < p.d) {
                if (p.vec && c + 3 < p.d) {
                    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
                                 : "=f"(v[r][h].x), "=f"(v[r][h].y), "=f"(v[r][h].z), "=f"(v[r][h].w)
                                 : "l"(src + c));
                } else {
                    v[r][h].x = __ldg(src + c);
                    v[r][h].y = c + 1 < p.d ? __ldg(src + c + 1) : 0.f;
                    v[r][h].z = c + 2 < p.d ? __ldg(src + c + 2) : 0.f;
                    v[r][h].w = c + 3 < p.d ? __ldg(src + c + 3) : 0.f;
                }
            }
        }
    }
}

// Split the piece into bf16 hi / lo and store it as rows PR part .. PR part +
// PR - 1 of the chunk: row k of the chunk is row k % 8 of the atoms of row
// group k / 8; columns 4 t .. 4 t + 3 go to atom (c / 64, k / 8), 16-byte
// chunk ((c % 64) / 8) ^ (k % 8), bytes 8 (t % 2) .. +7.  Sixteen lanes fill
// one 128-byte atom row: two wavefronts a warp instruction.
template <int NPAD, int PR>
__device__ __forceinline__ void store_piece(uint8_t* th, uint8_t* tl, int part, int lane,
                                            const float4 (&v)[PR][(NPAD + kMT - 1) / kMT]) {
    constexpr int H = (NPAD + kMT - 1) / kMT;
    const uint32_t c0 = 4u * (uint32_t)lane;
    const uint32_t k0 = (uint32_t)(PR * part);
    uint8_t* const bh = th + (k0 >> 3) * kSbo(NPAD);
    uint8_t* const bl = tl + (k0 >> 3) * kSbo(NPAD);
#pragma unroll
    for (int r = 0; r < PR; ++r) {
        const uint32_t rr = (k0 & 7u) + (uint32_t)r;   // row in the atom
#pragma unroll
        for (int h = 0; h < H; ++h) {
            const uint32_t c = c0 + kMT * h;
            const uint32_t off = (c >> 6) * 1024u + rr * 128u + (((((c & 63u) >> 3) ^ rr) & 7u) << 4) + (c & 7u) * 2u;
            uint2 hi, lo;
            tc::split_bf16x2(v[r][h].x, v[r][h].y, hi.x, lo.x);
            tc::split_bf16x2(v[r][h].z, v[r][h].w, hi.y, lo.y);
            *reinterpret_cast<uint2*>(bh + off) = hi;
            *reinterpret_cast<uint2*>(bl + off) = lo;
        }
    }
}

// NPAD (d rounded up to 32) is a template parameter: every index split below
// is then a division by a constant.
template <int NPAD, class SH>
__global__ void __launch_bounds__(SH::kThreads, 1) gram_tc_kernel(const GrParams p) {
    constexpr int kWorkers = SH::kWorkers, kMmaWarp = SH::kMmaWarp, kEpi0 = SH::kEpi0, kEpiWarps = SH::kEpiWarps;
    constexpr int kPieceRows = SH::kPieceRows, kPieces = SH::kPieces;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
    constexpr int kStages = stages_of(NPAD);
    const uint32_t sbytes = stage_bytes(NPAD);
    uint8_t* stages = smem;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kStages * sbytes);
    uint64_t* full = bars;                 // [kStages] (kPieces arrivals)
    uint64_t* empty = bars + kStages;      // [kStages] (MMA commit)
    uint64_t* done = bars + 2 * kStages;   // slice accumulated       (MMA commit)
    uint64_t* drained = done + 1;          // accumulator read        (epilogue warp arrivals)
    uint64_t* fin = done + 2;              // every MMA complete      (MMA commit)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
    int* stored = const_cast<int*>(abort) + 1;   // [kStages] pieces stored per stage (in use order)

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int ntiles = (NPAD + kMT - 1) / kMT;   // 1 or 2 M tiles
    const int nepi = 4 * (ntiles < kEpiWarps / 4 ? ntiles : kEpiWarps / 4);   // epilogue warps in use
    const int my_slices = ((int)blockIdx.x < p.slices) ? (p.slices - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            tc::mbar_init(full + s, kPieces);
            tc::mbar_init(empty + s, 1);
            stored[s] = 0;
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
        // the CTA's chunks in order: slice z (rows from (blockIdx.x + z grid)
        // 1024) holds chunks 32 z .. 32 z + 31; only the matrix's last slice
        // is short
        int my_chunks = my_slices * (kSliceRows / kKC);
        if (my_slices > 0 && (int)blockIdx.x + (my_slices - 1) * (int)gridDim.x == p.slices - 1) {
            const int64_t last_rows = p.n - (int64_t)(p.slices - 1) * kSliceRows;
            my_chunks -= kSliceRows / kKC - (int)((last_rows + kKC - 1) / kKC);
        }
        constexpr int H = (NPAD + kMT - 1) / kMT;
        const int npieces = my_chunks * kPieces;
        // piece pc: chunk h = pc / kPieces of the CTA's sequence, rows
        // kPieceRows (pc % kPieces) .. of it
        const auto rows_of = [&](int pc, int64_t& row0, int64_t& r_end) {
            const int h = pc / kPieces;
            const int z = h / (kSliceRows / kKC), cz = h % (kSliceRows / kKC);
            const int64_t r_begin = ((int64_t)blockIdx.x + (int64_t)z * gridDim.x) * kSliceRows;
            r_end = min(p.n, r_begin + kSliceRows);
            row0 = r_begin + (int64_t)cz * kKC + (pc % kPieces) * kPieceRows;
        };
        // claim piece pc's stage (in piece order), store it, arrive
        const auto put = [&](int pc, const float4 (&v)[kPieceRows][H]) -> bool {
            const int h = pc / kPieces, s = h % kStages, u = h / kStages;
            int ok = 1;
            if (lane == 0) {
                ok = tc::counter_wait(reinterpret_cast<volatile int*>(stored + s), kPieces * u, abort) &&
                     tc::mbar_wait(empty + s, ((uint32_t)u & 1u) ^ 1u, abort);
            }
            if (!__shfl_sync(0xffffffffu, ok, 0)) return false;
            uint8_t* th = stages + (size_t)s * sbytes;
            store_piece<NPAD, kPieceRows>(th, th + half_bytes(NPAD), pc % kPieces, lane, v);
            tc::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
                tc::mbar_arrive(full + s);
                atomicAdd(stored + s, 1);
            }
            return true;
        };
        // one piece in registers: load it, claim its stage, store it (two
        // 4-row pieces in flight a warp measured no faster)
        int64_t row0, r_end;
        float4 v[kPieceRows][H];
        for (int pc = warp; pc < npieces; pc += kWorkers) {
            rows_of(pc, row0, r_end);
            load_piece<NPAD, kPieceRows>(p, row0, r_end, lane, v);
            if (!put(pc, v)) break;
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
                        const uint32_t ko = 2u * kSbo(NPAD) * kk;   // 16 rows = two 8-row groups
                        for (int t = 0; t < ntiles; ++t) {
                            const uint32_t off = (uint32_t)t * 2048u + ko;   // columns from 128 t
                            const uint32_t idesc = tc::idesc_bf16_f32_mn(128, (uint32_t)(NPAD - t * kMT));
                            const uint32_t dt = tmem + 256u * t;
                            const uint64_t dh = tc::desc_sw128_mnmajor(hi + off, 1024u, kSbo(NPAD));
                            const uint64_t dl = tc::desc_sw128_mnmajor(lo + off, 1024u, kSbo(NPAD));
                            tc::mma_bf16(dt, dh, dh, idesc, (g | kk) != 0);
                            tc::mma_bf16(dt, dh, dl, idesc, 1);
                            tc::mma_bf16(dt, dl, dh, idesc, 1);
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
        // epilogue warp e: TMEM lane quarter q = warp % 4, accumulators
        // t = e / 4, e / 4 + nepi / 4, ...
        const int e = warp - kEpi0, q = warp & 3;
        for (int z = 0; z < my_slices; ++z) {
            int okw = 0;
            if (lane == 0) okw = tc::mbar_wait(done, (uint32_t)z & 1u, abort) ? 1 : 0;
            if (!__shfl_sync(0xffffffffu, okw, 0)) break;
            tc::fence_after_sync();
            // the accumulator is handed back as soon as it is in registers; the
            // adds into the running partial are fire-and-forget reductions (one
            // writer per address, in program order: deterministic)
            for (int t = e >> 2; t < ntiles; t += nepi >> 2) {
                const int row = t * kMT + q * 32 + lane;   // column a of A
                const int ncols = NPAD - t * kMT;        // columns b = t*128 .. npad-1
                float* dst = p.part + ((int64_t)blockIdx.x * NPAD + row) * NPAD + t * kMT;
                // 64 columns per TMEM round trip (ncols is a multiple of 32)
                for (int col = 0; col < ncols; col += 64) {
                    uint32_t va[32], vb[32];
                    const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(256 * t + col);
                    const bool two = col + 32 < ncols;
                    tc::tmem_ld_32x32b_x32(ta, va);
                    if (two) tc::tmem_ld_32x32b_x32(ta + 32u, vb);
                    tc::tmem_ld_wait();
                    if (t + (nepi >> 2) >= ntiles && col + 64 >= ncols) {
                        tc::fence_before_sync();
                        __syncwarp();
                        if (lane == 0) tc::mbar_arrive(drained);
                    }
                    if (row < p.d) {
#pragma unroll
                        for (int k = 0; k < 64; k += 4) {
                            const uint32_t* w = k < 32 ? va + k : vb + (k - 32);
                            if (k < 32 || two)
                                asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst + col + k),
                                             "f"(__uint_as_float(w[0])), "f"(__uint_as_float(w[1])),
                                             "f"(__uint_as_float(w[2])), "f"(__uint_as_float(w[3]))
                                             : "memory");
                        }
                    }
                }
            }
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
__global__ void gram_tc_reduce_kernel(const float* __restrict__ part, int slices, int d, int npad, double alpha,
                                      double beta, float* __restrict__ C) {
    const int64_t len = (int64_t)d * d, plen = (int64_t)npad * npad;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += stride) {
        int a = (int)(e / d), b = (int)(e % d);
        if (a > b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int64_t idx = (int64_t)a * npad + b;
        float s = 0.f, c = 0.f;
        for (int z = 0; z < slices; ++z) {
            const float x = part[(int64_t)z * plen + idx];
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
    return (size_t)stages_of(npad) * stage_bytes(npad) + 1024 + 256;
}

}  // namespace

bool gram_tc_supported(const lsk_mat* A) {
    return A->kind == LSK_DENSE && A->d >= 1 && A->d <= 256 && smem_bytes((int)((A->d + 31) / 32) * 32) <= kSmemLimit;
}

template <int NPAD, class SH>
cudaError_t launch_shape(const GrParams& p, int grid, cudaStream_t st) {
    const size_t smem = smem_bytes(NPAD);
    cudaError_t e = allow_dynamic_smem(gram_tc_kernel<NPAD, SH>);
    if (e != cudaSuccess) return e;
    LSK_PROF("gram_tc", st) gram_tc_kernel<NPAD, SH><<<grid, SH::kThreads, smem, st>>>(p);
    return cudaGetLastError();
}
// 15 workers and 4 epilogue warps (each reading both accumulators): 640
// threads, 96 registers a thread (11 workers with 8 epilogue warps measured
// 1.3% slower at 4M x 256)
template <int NPAD>
cudaError_t launch_npad(const GrParams& p, int grid, cudaStream_t st) {
    return launch_shape<NPAD, GramShape<15, 4>>(p, grid, st);
}

// one running partial per CTA of the persistent grid
int grid_of(const lsk_mat* A, int sm_count) {
    const int64_t slices = (A->n + kSliceRows - 1) / kSliceRows;
    return (int)(slices < sm_count ? slices : sm_count);
}

size_t gram_tc_workspace_bytes(const lsk_mat* A, int sm_count) {
    const int g = grid_of(A, sm_count);
    const size_t npad = (size_t)((A->d + 31) / 32) * 32;
    return ws_round((size_t)(g > 0 ? g : 1) * npad * npad * 4);
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
    p.vec = (A->ld % 4 == 0) && (((uintptr_t)A->values & 15) == 0);
    p.part = (float*)ws;
    p.flag = flag;
    const int grid = grid_of(A, sm_count);
    const int64_t len = A->d * A->d;
    int64_t rg = (len + 255) / 256;
    if (rg > 8 * (int64_t)sm_count) rg = 8 * (int64_t)sm_count;
    cudaError_t e;
    if (grid > 0) {
        e = cudaMemsetAsync(p.part, 0, (size_t)grid * p.npad * p.npad * 4, st);
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
    LSK_PROF("gram_reduce", st) gram_tc_reduce_kernel<<<(unsigned)rg, 256, 0, st>>>(p.part, grid, p.d, p.npad, alpha, beta, C);
    return cudaGetLastError();
}
