"""Gaussian sketch G and the product G*(S*A) (oracle; test infrastructure).

Alg. 3 (Sec. 2.2.2) multiplies S*A by an m x r matrix G of i.i.d. N(0,1)
entries; the library call csrcgs / rmcgs (Sec. 5) scales G by 1/sqrt(m).
The reading used here keeps that scaling (m is called k below) and makes
every entry a deterministic function of (seed, j, c) through Philox-4x32-10
and the Box-Muller transform (Box & Muller 1958):

    (w0, w1, w2, w3) = Philox4x32_10(ctr = (c mod 2^32, c >> 32, 1, j >> 2),
                                     key = (seed mod 2^32, seed >> 32))
    p = (j >> 1) & 1;  (a, b) = (w_{2p} >> 8, w_{2p+1} >> 8)   (24-bit words)
    u1 = (a + 1) / 2^24 in (0, 1],   u2 = b / 2^24 in [0, 1)
    z  = sqrt(-2 ln u1) * cos(2 pi u2)   if j is even
         sqrt(-2 ln u1) * sin(2 pi u2)   if j is odd
    G[j, c] = z / sqrt(k)

so one Philox call yields the four entries j = 4q..4q+3 of column c.  The
24-bit uniforms are exact in float32, so a float32 evaluation of the same
formula sees exactly the arguments the float64 oracle sees (the paper only
asks for i.i.d. N(0,1) entries; the uniform resolution is part of this
reading, and it caps |z| at sqrt(48 ln 2) = 5.77).
In the BF16 precision mode G is *defined* as the bfloat16 value nearest
(ties to even) to the float32 rounding of z / sqrt(k); that rounding is the
one decision both the oracle and the GPU take in float32.

The same construction, with the third counter word changed, draws the other
Gaussian matrices of the paper: stream 2 the right projection Pi of Alg. 15
(``jl_matrix``), stream 3 the m x n matrix of the Gaussian CSR sketch of
Alg. 4 (``csrjlt``, column index = row index of A, scaled by 1/sqrt(m)).
"""
import numpy as np

from .philox import philox4x32_10, split_seed

STREAM_G = 1
STREAM_PI = 2   # the right JL projection of Alg. 15
STREAM_JLT = 3  # the Gaussian sketch of a CSR matrix (Alg. 4, csrjlt)

PREC_FP32 = 0
PREC_TF32 = 1
PREC_BF16 = 2


def float32_to_bf16_rne(x32):
    """Round float32 values to bfloat16 (nearest, ties to even); returns float64."""
    x32 = np.ascontiguousarray(x32, dtype=np.float32)
    u = x32.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    rounded = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    out = (rounded & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32)
    return out.astype(np.float64)


def gaussian_matrix(k, r, seed, prec=PREC_FP32):
    """G (k x r, float64): z / sqrt(k), bfloat16-rounded in the BF16 mode."""
    return gaussian_columns(k, 0, r, seed, prec)


def gaussian_columns(k, c0, c1, seed, prec=PREC_FP32, stream=STREAM_G):
    """Columns c0..c1-1 of G (k x (c1-c0), float64); ``stream`` is the third
    counter word (STREAM_G for the Gaussian stage of Alg. 3)."""
    j = np.arange(k, dtype=np.uint64)[:, None]
    c = np.arange(c0, c1, dtype=np.uint64)[None, :]
    k0, k1 = split_seed(seed)
    w = philox4x32_10(c & np.uint64(0xFFFFFFFF), c >> np.uint64(32), stream,
                      j >> np.uint64(2), k0, k1)
    p = ((j >> np.uint64(1)) & np.uint64(1)).astype(bool)
    a = (np.where(p, w[2], w[0]) >> np.uint32(8)).astype(np.float64)
    b = (np.where(p, w[3], w[1]) >> np.uint32(8)).astype(np.float64)
    u1 = (a + 1.0) * 2.0**-24
    u2 = b * 2.0**-24
    rho = np.sqrt(-2.0 * np.log(u1))
    even = (np.arange(k)[:, None] % 2) == 0
    z = np.where(even, rho * np.cos(2.0 * np.pi * u2), rho * np.sin(2.0 * np.pi * u2))
    g = z / np.sqrt(float(k))
    if prec == PREC_BF16:
        return float32_to_bf16_rne(g.astype(np.float32))
    return g


def jl_matrix(d, m, seed):
    """Pi (d x m, float64) of Alg. 15: a Gaussian scaled by 1/sqrt(m).

    Pi[i, c] is entry (c, i) of the m x d matrix drawn as G above (column
    index i, row index c) on stream STREAM_PI, i.e. z / sqrt(m) with the same
    Philox-4x32-10 / Box-Muller construction.
    """
    return gaussian_columns(m, 0, d, seed, PREC_FP32, STREAM_PI).T.copy()


def gauss_sketch(SA, k, seed, prec=PREC_FP32, batch=4096):
    """G * SA in float64 (Alg. 3).

    As in Alg. 3, the r columns of G are taken in batches of ``batch``: each
    batch of G is generated and C <- C + G_i B_i is accumulated, so G is never
    held whole.  Batching changes only the float64 summation order.
    """
    SA = np.asarray(SA, dtype=np.float64)
    r = SA.shape[0]
    C = np.zeros((k, SA.shape[1]), dtype=np.float64)
    for c0 in range(0, r, batch):
        c1 = min(r, c0 + batch)
        C += gaussian_columns(k, c0, c1, seed, prec) @ SA[c0:c1]
    return C


def count_gauss_dense(A, r, k, seed, prec=PREC_BF16, block=32):
    """rmcgs(A, m=k, r) in Alg. 3's blocked order (Sec. 2.2.2): G (S A), float64.

    Alg. 3 never holds S*A whole: for each block of rows of S -- here the
    buckets [c0, c1), ``block`` at a time -- it forms B = S_i A from the rows
    of A that hash into those buckets (Def. 3: row i adds sigma_i A[i, :] to
    row h(i)), draws the block's columns of G and accumulates C <- C + G_i B.
    The hash is CountSketch's (same seed, stream 0) and G the one of
    ``gauss_sketch`` (stream 1).  The blocking changes only the float64
    summation order.
    """
    from .countsketch import countsketch_hash
    A = np.asarray(A)
    n, d = A.shape
    bucket, sign = countsketch_hash(n, r, seed)
    order = np.argsort(bucket, kind="stable")            # rows grouped by bucket
    first = np.searchsorted(bucket[order], np.arange(r + 1))   # bucket b: order[first[b]:first[b + 1]]
    sgn = np.asarray(sign, dtype=np.float64)
    C = np.zeros((k, d), dtype=np.float64)
    for c0 in range(0, r, block):
        c1 = min(r, c0 + block)
        rows = order[first[c0]:first[c1]]
        B = np.zeros((c1 - c0, d), dtype=np.float64)
        np.add.at(B, bucket[rows] - c0, sgn[rows, None] * A[rows].astype(np.float64))
        C += gaussian_columns(k, c0, c1, seed, prec) @ B
    return C


def csrjlt(V, J, I, n, d, m, seed, prec=PREC_FP32, batch=4096):
    """C = G A (m x d, float64) for CSR A (Alg. 4, ``csrjlt``).

    G is m x n, drawn like the Gaussian stage's G (z / sqrt(m), bfloat16-
    rounded in the BF16 mode) with column index = row index of A, on counter
    stream STREAM_JLT.  C = G A is a plain product; as in Alg. 4 the rows of A
    are taken in order (here in batches, each with its own columns of G), so
    G is never held whole.
    """
    V = np.asarray(V, dtype=np.float64)
    J = np.asarray(J)
    I = np.asarray(I)
    C = np.zeros((m, d), dtype=np.float64)
    for r0 in range(0, n, batch):
        r1 = min(n, r0 + batch)
        blk = np.zeros((r1 - r0, d), dtype=np.float64)
        for i in range(r0, r1):
            blk[i - r0, J[I[i]:I[i + 1]]] += V[I[i]:I[i + 1]]
        C += gaussian_columns(m, r0, r1, seed, prec, STREAM_JLT) @ blk
    return C
