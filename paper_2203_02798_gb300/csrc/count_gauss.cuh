// count_gauss.cuh -- the fused CountSketch + Gaussian stage (G * (S * A) with
// S * A kept on chip) and the pieces of the CountSketch and Gaussian stages it
// shares with them.
#pragma once
#include "lsk_internal.cuh"

// CountSketch steps 1-3 (rank, scan, place) on ws (cs_workspace_bytes(n, r)
// bytes): *off (r + 1 entries, off[r] = n) and *perm (n entries, row index |
// sign bit << 31, grouped by bucket) point into ws when the queued launches
// have run.
// A bounded wait of the scan that runs out sets LSK_FLAG_TIMEOUT in *flag.
cudaError_t cs_prep_launch(int64_t n, int64_t r, uint64_t seed, void* ws, int sm_count, cudaStream_t st,
                           const uint32_t** off, const uint32_t** perm, uint64_t row0, int* flag, bool rx = true);

// out[e] = the slice-order compensated sum of part[z * len + e], z < slices.
cudaError_t gauss_tc_reduce_launch(const float* part, int slices, int64_t len, float* out, int sm_count,
                                   cudaStream_t st);

// G * (S * A) for dense FP32 A in the BF16 mode (G the bf16 rounding of the
// scaled draws, S * A carried as bf16 hi + lo), one pass over A: supported for
// 32 <= d <= 256 with d, ld multiples of 4 and A 16-byte aligned, 1 <= k <= 512.
bool count_gauss_supported(const lsk_mat* A, int64_t r, int64_t k);
// Whether the fused kernel is expected to beat the two stages for this shape:
// each gather lane fully used (d > 192), enough buckets to give every CTA pair
// of the device a slice of >= 8 chunks, and >= 8 rows a bucket on average
// (measured on GB300: 4M x 256, r = 65,536: 0.70 ms against 0.92 ms; at
// d <= 200, few buckets or few rows a bucket the two stages are faster).
bool count_gauss_preferred(const lsk_mat* A, int64_t r, int64_t k, int sm_count);
size_t count_gauss_workspace_bytes(const lsk_mat* A, int64_t r, int64_t k, int sm_count);
// row0: global index of A's first row (A is a block of rows of a larger matrix)
cudaError_t count_gauss_launch(const lsk_mat* A, int64_t r, int64_t k, uint64_t seed, float* GSA, void* ws,
                               int* flag, int sm_count, cudaStream_t st, uint64_t row0 = 0);
