// css.cu -- column subset selection (Alg. 9) and the pieces of Alg. 14 / 16.
//
// Alg. 9 asks for a pivoted QR of the sketch B = G S A and keeps the first c
// columns of its permutation.  Here the pivots come from a diagonally pivoted
// Cholesky of C = B^T B (FP64, formed with exact products): the Schur
// complement diagonal at step j holds the squared norms of the columns of B
// reduced against the pivots so far, so taking its largest entry is exactly
// the column-pivoting rule of QR (Businger-Golub) in exact arithmetic, on a
// d x d matrix instead of the m x d sketch.  Ties go to the lowest position.
#include "lsk_internal.cuh"

namespace {

// Left-looking pivoted Cholesky of C (d x d, FP64) for c steps, one block:
// L[t * d + a] = column t of the factor at original index a.
// Stops at the first pivot <= max(16 eps d, rcond^2) times the largest
// diagonal entry: with `flag_rank` that is the deferred rank error, else the
// truncation point; *rank_out (if given) receives the pivots taken.
__global__ void __launch_bounds__(1024) pivchol_kernel(const double* __restrict__ C, int d, int c, double rcond,
                                                        int flag_rank, double* __restrict__ L,
                                                        int32_t* __restrict__ cols, int* rank_out, int* flag) {
    __shared__ double dg[1024];
    __shared__ int perm[1024];
    __shared__ double lp[1024];
    __shared__ double red_v[32];
    __shared__ int red_p[32];
    __shared__ int s_stop;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    double dmax = 0.0;
    for (int a = tid; a < d; a += blockDim.x) {
        dg[a] = C[(int64_t)a * d + a];
        perm[a] = a;
        dmax = fmax(dmax, dg[a]);
    }
    for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    if (lane == 0) red_v[wid] = dmax;
    if (tid == 0) s_stop = 0;
    __syncthreads();
    if (tid == 0) {
        double m = 0.0;
        for (int w = 0; w < nw; ++w) m = fmax(m, red_v[w]);
        red_v[0] = m;
    }
    __syncthreads();
    const double tol = fmax(16.0 * 2.220446049250313e-16 * d, rcond * rcond) * red_v[0];
    __syncthreads();
    int taken = c;
    for (int j = 0; j < c; ++j) {
        // largest remaining diagonal entry, lowest position on ties
        double bv = -INFINITY;
        int bp = d;
        for (int pos = j + tid; pos < d; pos += blockDim.x) {
            const double v = dg[perm[pos]];
            if (v > bv || (v == bv && pos < bp)) {
                bv = v;
                bp = pos;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int op = __shfl_xor_sync(0xffffffffu, bp, o);
            if (ov > bv || (ov == bv && op < bp)) {
                bv = ov;
                bp = op;
            }
        }
        if (lane == 0) {
            red_v[wid] = bv;
            red_p[wid] = bp;
        }
        __syncthreads();
        if (tid == 0) {
            double v = red_v[0];
            int p = red_p[0];
            for (int w = 1; w < nw; ++w)
                if (red_v[w] > v || (red_v[w] == v && red_p[w] < p)) {
                    v = red_v[w];
                    p = red_p[w];
                }
            const int pv = perm[p];
            perm[p] = perm[j];
            perm[j] = pv;
            cols[j] = pv;
            if (!(v > tol)) s_stop = 1;
        }
        __syncthreads();
        if (s_stop) {
            // numerically rank deficient: the remaining columns in their order
            for (int t = j + 1 + tid; t < c; t += blockDim.x) cols[t] = perm[t];
            if (tid == 0 && flag_rank) set_flag(flag, LSK_FLAG_RANK_DEFICIENT);
            taken = j;
            break;
        }
        const int pv = perm[j];
        for (int t = tid; t < j; t += blockDim.x) lp[t] = L[(int64_t)t * d + pv];
        __syncthreads();
        const double piv = dg[pv];
        const double rs = 1.0 / sqrt(piv);
        for (int pos = j + 1 + tid; pos < d; pos += blockDim.x) {
            const int a = perm[pos];
            double v = C[(int64_t)pv * d + a];
            for (int t = 0; t < j; ++t) v = fma(-L[(int64_t)t * d + a], lp[t], v);
            const double l = v * rs;
            L[(int64_t)j * d + a] = l;
            dg[a] -= l * l;
        }
        if (tid == 0) L[(int64_t)j * d + pv] = sqrt(piv);
        __syncthreads();
    }
    if (tid == 0 && rank_out) *rank_out = taken;
}

__global__ void gather_sub_gram_kernel(const double* __restrict__ C, int64_t d, const int32_t* __restrict__ cols,
                                       int64_t c, double* __restrict__ Csub) {
    const int64_t total = c * c;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += (int64_t)gridDim.x * blockDim.x)
        Csub[x] = C[(int64_t)cols[x / c] * d + cols[x % c]];
}

__global__ void gather_cols_kernel(const float* __restrict__ B, int64_t rows, int64_t d,
                                   const int32_t* __restrict__ cols, int64_t c, float* __restrict__ Bk) {
    const int64_t total = rows * c;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += (int64_t)gridDim.x * blockDim.x)
        Bk[x] = B[(x / c) * d + cols[x % c]];
}

// Bf (d x c) = E_K X: row cols[t] of Bf is row t of X (c x c), the rest zero
__global__ void embed_rows_kernel(const float* __restrict__ X, int64_t c, const int32_t* __restrict__ cols, int64_t d,
                                  float* __restrict__ Bf) {
    const int64_t total = c * c;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += (int64_t)gridDim.x * blockDim.x)
        Bf[(int64_t)cols[x / c] * c + x % c] = X[x];
}

unsigned grid_of(int64_t total) {
    const int64_t g = (total + 255) / 256;
    return (unsigned)(g < 1 ? 1 : (g > 4096 ? 4096 : g));
}

}  // namespace

size_t pivchol_workspace_bytes(int64_t d, int64_t c) { return ws_round((size_t)d * c * 8); }

cudaError_t pivchol_launch(const double* C, int64_t d, int64_t c, double rcond, int flag_rank, int32_t* cols,
                           int* rank_out, void* ws, int* flag, cudaStream_t st) {
    if (d < 1 || d > 1024 || c < 1 || c > d) return cudaErrorInvalidValue;
    LSK_PROF("css_pivchol", st) pivchol_kernel<<<1, 1024, 0, st>>>(C, (int)d, (int)c, rcond, flag_rank, (double*)ws,
                                                                    cols, rank_out, flag);
    return cudaGetLastError();
}

cudaError_t gather_sub_gram_launch(const double* C, int64_t d, const int32_t* cols, int64_t c, double* Csub,
                                   cudaStream_t st) {
    LSK_PROF("css_gather", st) gather_sub_gram_kernel<<<grid_of(c * c), 256, 0, st>>>(C, d, cols, c, Csub);
    return cudaGetLastError();
}

cudaError_t gather_cols_launch(const float* B, int64_t rows, int64_t d, const int32_t* cols, int64_t c, float* Bk,
                               cudaStream_t st) {
    LSK_PROF("css_gather", st) gather_cols_kernel<<<grid_of(rows * c), 256, 0, st>>>(B, rows, d, cols, c, Bk);
    return cudaGetLastError();
}

cudaError_t embed_rows_launch(const float* X, int64_t c, const int32_t* cols, int64_t d, float* Bf, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(Bf, 0, (size_t)d * c * 4, st);
    if (e != cudaSuccess) return e;
    LSK_PROF("css_gather", st) embed_rows_kernel<<<grid_of(c * c), 256, 0, st>>>(X, c, cols, d, Bf);
    return cudaGetLastError();
}
