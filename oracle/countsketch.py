"""CountSketch S in R^{r x n} and the product S*A (oracle; test infrastructure).

Def. 3 (Sec. 1): S is fixed by a hash h:[n]->[r] and signs sigma in {+-1}^n;
column i of S holds sigma_i in row h(i) and zeros elsewhere.  Following
Sec. 1 (after Def. 3) the hash and the signs are treated as fully
independent and uniform.  The paper draws them from STL engines
(Alg. 1, "generate a row index uniformly at random"); the reading used here
makes them a deterministic function of (seed, i) through Philox-4x32-10:

    (w0, w1, w2, w3) = Philox4x32_10(ctr = (i mod 2^32, i >> 32, 0, 0),
                                     key = (seed mod 2^32, seed >> 32))
    h(i)     = floor(w0 * r / 2^32)          (multiply-shift to [0, r))
    sigma_i  = -1 if w1 >= 2^31 else +1

Indices are 0-based here (the paper's [n] is 1-based).  The vector
representation of Sec. 2.1.1 (Fig. 2) stores v_i = sigma_i * (h(i) + 1).

S*A is Alg. 2: every row i of A is added, with sign sigma_i, into row h(i)
of the dense row-major result; the oracle does that scatter directly in
float64 over the stored values of A.
"""
import numpy as np

from .philox import philox4x32_10, split_seed

STREAM_S = 0  # third Philox counter word of every CountSketch draw


def countsketch_hash(n, r, seed):
    """(h, sigma) for columns 0..n-1 of an r x n CountSketch (Def. 3).

    Returns bucket int64[n] in [0, r) and sign int8[n] in {-1, +1}.
    """
    if r <= 0 or r >= 2**32:
        raise ValueError("r must be in [1, 2^32)")
    i = np.arange(n, dtype=np.uint64)
    k0, k1 = split_seed(seed)
    w0, w1, _, _ = philox4x32_10(i & np.uint64(0xFFFFFFFF), i >> np.uint64(32),
                                 STREAM_S, 0, k0, k1)
    bucket = ((w0.astype(np.uint64) * np.uint64(r)) >> np.uint64(32)).astype(np.int64)
    sign = np.where(w1 >= np.uint32(2**31), -1, 1).astype(np.int8)
    return bucket, sign


def countsketch_hash_rows(row0, n, r, seed):
    """(h, sigma) for columns row0 .. row0 + n - 1 of S (Def. 3): the hash of
    a block of rows of a larger matrix, which keeps each row's global index
    (the counter of its Philox draw)."""
    if r <= 0 or r >= 2**32:
        raise ValueError("r must be in [1, 2^32)")
    if row0 < 0:
        raise ValueError("row0 must be >= 0")
    i = np.arange(n, dtype=np.uint64) + np.uint64(row0)
    k0, k1 = split_seed(seed)
    w0, w1, _, _ = philox4x32_10(i & np.uint64(0xFFFFFFFF), i >> np.uint64(32),
                                 STREAM_S, 0, k0, k1)
    bucket = ((w0.astype(np.uint64) * np.uint64(r)) >> np.uint64(32)).astype(np.int64)
    sign = np.where(w1 >= np.uint32(2**31), -1, 1).astype(np.int8)
    return bucket, sign


def countsketch_matrix(bucket, sign, r):
    """Explicit dense S (r x n, float64) with S[h(i), i] = sigma_i (Def. 3)."""
    n = len(bucket)
    S = np.zeros((r, n), dtype=np.float64)
    S[np.asarray(bucket), np.arange(n)] = np.asarray(sign, dtype=np.float64)
    return S


def vector_representation(bucket, sign):
    """Sec. 2.1.1 / Fig. 2: v_i = sigma_i * (h(i) + 1) (1-based row index)."""
    return np.asarray(sign, dtype=np.int64) * (np.asarray(bucket, dtype=np.int64) + 1)


def from_vector_representation(v):
    """Inverse of :func:`vector_representation`: (bucket, sign) from v."""
    v = np.asarray(v, dtype=np.int64)
    if np.any(v == 0):
        raise ValueError("a CountSketch vector has no zero entries")
    return np.abs(v) - 1, np.sign(v).astype(np.int8)


def countsketch_apply_dense(A, bucket, sign, r, chunk=1 << 16):
    """S*A for a dense row-major A (Alg. 2): SA[h(i), :] += sigma_i * A[i, :].

    The rows are visited in chunks only to bound the float64 temporaries
    (the order of the additions is the row order either way).
    """
    A = np.asarray(A)
    bucket = np.asarray(bucket)
    sign = np.asarray(sign, dtype=np.float64)
    SA = np.zeros((r, A.shape[1]), dtype=np.float64)
    for i0 in range(0, A.shape[0], chunk):
        i1 = min(A.shape[0], i0 + chunk)
        np.add.at(SA, bucket[i0:i1], sign[i0:i1, None] * A[i0:i1].astype(np.float64))
    return SA


def countsketch_apply_csr(V, J, I, n, d, bucket, sign, r):
    """S*A for CSR A = (V, J, I), 0-based (Alg. 2 over the nonzeros of A)."""
    V = np.asarray(V, dtype=np.float64)
    I = np.asarray(I, dtype=np.int64)
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(I))
    SA = np.zeros((r, d), dtype=np.float64)
    np.add.at(SA, (np.asarray(bucket)[rows], np.asarray(J, dtype=np.int64)),
              np.asarray(sign, dtype=np.float64)[rows] * V)
    return SA


def cs_sketch_dense(A, r, seed):
    """rmcgs(A, m=0, r): S*A with S from (r, seed) (Sec. 5, Alg. 2)."""
    bucket, sign = countsketch_hash(A.shape[0], r, seed)
    return countsketch_apply_dense(A, bucket, sign, r)


def cs_sketch_csr(V, J, I, n, d, r, seed):
    """csrcgs(A, m=0, r) for CSR A (Sec. 5, Alg. 2)."""
    bucket, sign = countsketch_hash(n, r, seed)
    return countsketch_apply_csr(V, J, I, n, d, bucket, sign, r)
