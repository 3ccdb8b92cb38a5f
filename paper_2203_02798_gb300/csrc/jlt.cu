// jlt.cu -- Gaussian sketch of a CSR matrix, C = G A (Alg. 4, csrjlt).
//
// G is m x n with entries z / sqrt(m) drawn like the Gaussian stage's G
// (Philox-4x32-10 + Box-Muller, bfloat16-rounded in the BF16 mode) on
// counter stream 3, with column index = row index of A.  As in Alg. 4 each
// block owns a range of rows of G (JB of them, one per thread) so no two
// threads write the same entry of C: it walks a range of rows of A, 128 rows
// at a time with their row pointers and nonzeros staged in shared memory
// (one coalesced load each), draws G[j, i] for its rows j and every row i,
// and adds G[j, i] A_ih into its shared-memory slice C[j, :] for each
// nonzero.  The row ranges of A are
// split over blocks too (split-K); the partial slices are summed in a fixed
// order.  One Philox call gives four rows of G for one row of A, so the four
// threads of a quad draw for four consecutive rows of A at once and swap the
// values among themselves (a 4 x 4 transpose by shuffles): one call per
// thread per four rows, two independent calls in flight per thread.
#include "lsk_internal.cuh"

namespace {

constexpr int kRowChunk = 128;    // rows of A staged at once (row pointers in shared memory)
constexpr int kNzChunk = 1024;    // their nonzeros staged with them, if they fit

template <int JB>
__global__ void __launch_bounds__(JB) csrjlt_kernel(const float* __restrict__ V, const int32_t* __restrict__ J,
                                                    const int64_t* __restrict__ I, int64_t n, int64_t nnz, int d,
                                                    int m, int64_t rows_per_split, uint32_t k0, uint32_t k1,
                                                    float scale, int bf16, float* __restrict__ part, int* flag) {
    extern __shared__ float cpart[];                         // [d][JB], then the staged rows
    int64_t* s_rp = reinterpret_cast<int64_t*>(cpart + (size_t)d * JB);   // [kRowChunk + 1]
    int32_t* s_j = reinterpret_cast<int32_t*>(s_rp + kRowChunk + 1);      // [kNzChunk]
    float* s_v = reinterpret_cast<float*>(s_j + kNzChunk);                // [kNzChunk]
    const int t = threadIdx.x, e = t & 3;
    const int j0 = blockIdx.x * JB, j = j0 + t;
    const int64_t r0 = (int64_t)blockIdx.y * rows_per_split;
    const int64_t r1 = r0 + rows_per_split < n ? r0 + rows_per_split : n;
    for (int x = t; x < d * JB; x += JB) cpart[x] = 0.f;
    const uint32_t quad = (uint32_t)(j >> 2);
    const int lane = t & 31, base = lane & ~3;
    bool bad = false;
    for (int64_t ra = r0; ra < r1; ra += kRowChunk) {
        const int nr = (int)(r1 - ra < kRowChunk ? r1 - ra : kRowChunk);
        __syncthreads();                                     // previous chunk done with the staging
        for (int x = t; x <= nr; x += JB) s_rp[x] = __ldg(I + ra + x);
        __syncthreads();
        const int64_t nz0 = s_rp[0], nz1 = s_rp[nr];
        const bool bad_span = nz0 < 0 || nz1 < nz0 || nz1 > nnz;
        const bool staged = !bad_span && nz1 - nz0 <= kNzChunk;
        if (staged)
            for (int64_t x = t; x < nz1 - nz0; x += JB) {
                s_j[x] = __ldg(J + nz0 + x);
                s_v[x] = __ldg(V + nz0 + x);
            }
        __syncthreads();
        for (int i = 0; i < nr; i += 8) {
            // this thread draws rows 4 quad .. 4 quad + 3 of G for rows ra + i + e
            // and ra + i + 4 + e of A (two independent chains)
            float4 z0 = make_float4(0.f, 0.f, 0.f, 0.f), z1 = z0;
            if (i + e < nr) z0 = gauss4((uint64_t)(ra + i + e), quad, k0, k1, 3u);
            if (i + 4 + e < nr) z1 = gauss4((uint64_t)(ra + i + 4 + e), quad, k0, k1, 3u);
            float g[8];
#pragma unroll
            for (int rr = 0; rr < 8; ++rr) {
                const float4 z = rr < 4 ? z0 : z1;
                const int src = base + (rr & 3);
                const float a = __shfl_sync(0xffffffffu, z.x, src);
                const float b = __shfl_sync(0xffffffffu, z.y, src);
                const float c = __shfl_sync(0xffffffffu, z.z, src);
                const float w = __shfl_sync(0xffffffffu, z.w, src);
                float v = e == 0 ? a : (e == 1 ? b : (e == 2 ? c : w));   // G[j, row] * sqrt(m)
                v *= scale;
                g[rr] = bf16 ? bf16_round(v) : v;
            }
            if (j >= m || bad_span) continue;
#pragma unroll
            for (int rr = 0; rr < 8; ++rr) {
                if (i + rr >= nr) break;
                const int64_t p0 = s_rp[i + rr], p1 = s_rp[i + rr + 1];
                if (p1 < p0 || p0 < nz0 || p1 > nz1) {
                    bad = true;
                    continue;
                }
                for (int64_t p = p0; p < p1; ++p) {
                    const int32_t col = staged ? s_j[p - nz0] : __ldg(J + p);
                    const float val = staged ? s_v[p - nz0] : __ldg(V + p);
                    if (col < 0 || col >= d) {
                        bad = true;
                        continue;
                    }
                    cpart[col * JB + t] = fmaf(g[rr], val, cpart[col * JB + t]);
                }
            }
        }
        if (bad_span) bad = true;
    }
    if (bad) set_flag(flag, LSK_FLAG_BAD_CSR);
    // part[split][col][j]: consecutive threads, consecutive addresses
    if (j < m)
        for (int col = 0; col < d; ++col) part[((int64_t)blockIdx.y * d + col) * m + j] = cpart[col * JB + t];
}

// C[j][col] = sum over splits of part[split][col][j], in split order
__global__ void csrjlt_reduce_kernel(const float* __restrict__ part, int nsplit, int d, int m, float* __restrict__ C) {
    const int64_t total = (int64_t)d * m;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += (int64_t)gridDim.x * blockDim.x) {
        const int col = (int)(x / m), j = (int)(x % m);
        double s = 0.0;
        for (int b = 0; b < nsplit; ++b) s += (double)part[((int64_t)b * d + col) * m + j];
        C[(int64_t)j * d + col] = (float)s;
    }
}

struct JltPlan {
    int jb, jblocks, nsplit;
    int64_t rows_per_split;
    size_t smem;
};

bool jlt_plan(int64_t n, int64_t d, int64_t m, int sm_count, JltPlan& p) {
    if (d < 1 || m < 1 || m > (1 << 20)) return false;
    // a block's slice of C plus the staged rows; the widest slice (most rows
    // of G a block, i.e. fewest draws shuffled) that still keeps two blocks
    // on an SM
    const size_t stage = (size_t)(kRowChunk + 1) * 8 + (size_t)kNzChunk * 8;
    const size_t smem_sm = 227 * 1024;
    p.jb = 128;
    while (p.jb > 32 && 2 * ((size_t)p.jb * d * 4 + stage) > smem_sm) p.jb >>= 1;
    p.smem = (size_t)p.jb * d * 4 + stage;
    if (p.smem > 200 * 1024) return false;
    p.jblocks = (int)((m + p.jb - 1) / p.jb);
    // one wave: as many row splits as resident blocks allow
    int64_t per_sm = (int64_t)(smem_sm / p.smem);
    if (per_sm > 16) per_sm = 16;
    if (per_sm < 1) per_sm = 1;
    int64_t ns = (int64_t)sm_count * per_sm / p.jblocks;
    const int64_t max_ns = (n + 1023) / 1024;
    if (ns > max_ns) ns = max_ns;
    if (ns < 1) ns = 1;
    p.rows_per_split = ((n + ns - 1) / ns + 7) / 8 * 8;
    if (p.rows_per_split < 8) p.rows_per_split = 8;
    p.nsplit = (int)((n + p.rows_per_split - 1) / p.rows_per_split);
    if (p.nsplit < 1) p.nsplit = 1;
    return true;
}

}  // namespace

bool jlt_supported(int64_t d, int64_t m) {
    JltPlan p;
    return jlt_plan(1024, d, m, 152, p);
}

size_t jlt_workspace_bytes(int64_t n, int64_t d, int64_t m, int sm_count) {
    JltPlan p;
    if (!jlt_plan(n, d, m, sm_count, p)) return 0;
    return ws_round((size_t)p.nsplit * d * m * 4);
}

cudaError_t jlt_launch(const lsk_mat* A, int64_t m, uint64_t seed, int32_t prec, float* C, void* ws, int* flag,
                       int sm_count, cudaStream_t st) {
    const int64_t n = A->n, d = A->d;
    JltPlan p;
    if (!jlt_plan(n, d, m, sm_count, p)) return cudaErrorNotSupported;
    if (n == 0) return cudaMemsetAsync(C, 0, (size_t)m * d * 4, st);
    float* part = (float*)ws;
    const float scale = (float)(1.0 / sqrt((double)m));
    const dim3 grid((unsigned)p.jblocks, (unsigned)p.nsplit);
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const int bf16 = prec == LSK_PREC_BF16 ? 1 : 0;
    cudaError_t e = cudaSuccess;
#define LSK_JLT_LAUNCH(JBV)                                                                                       \
    do {                                                                                                          \
        if (p.smem > 48 * 1024 && (e = allow_dynamic_smem(csrjlt_kernel<JBV>)) != cudaSuccess) return e;         \
        LSK_PROF("csrjlt", st) csrjlt_kernel<JBV><<<grid, JBV, p.smem, st>>>(                                    \
            (const float*)A->values, A->colidx, A->rowptr, n, A->nnz, (int)d, (int)m, p.rows_per_split, k0, k1, \
            scale, bf16, part, flag);                                                                             \
    } while (0)
    switch (p.jb) {
        case 128: LSK_JLT_LAUNCH(128); break;
        case 64: LSK_JLT_LAUNCH(64); break;
        default: LSK_JLT_LAUNCH(32); break;
    }
#undef LSK_JLT_LAUNCH
    const int64_t total = d * m;
    const unsigned rg = (unsigned)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
    LSK_PROF("csrjlt_reduce", st) csrjlt_reduce_kernel<<<rg, 256, 0, st>>>(part, p.nsplit, (int)d, (int)m, C);
    return cudaGetLastError();
}
