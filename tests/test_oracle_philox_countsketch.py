"""Pins of the oracle's Philox and CountSketch (CPU only).

Philox: published known-answer vectors.  CountSketch: the paper's printed
6 x 12 example (Fig. 1 / Fig. 2), brute force against an explicit S,
uniformity of the hash, the workload bounds of Lemma 1-3, and the closed
forms E||Sy||^2 = ||y||^2, Var||Sy||^2 = (2/r)(||y||^4 - ||y||_4^4) that
follow from Def. 3.
"""
import numpy as np
import pytest
from scipy import stats

from conftest import golden_path
from oracle import countsketch as cs
from oracle.philox import philox4x32_10


def _read_kat():
    rows = []
    for line in open(golden_path("philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        rows.append([int(x, 16) for x in line.split()])
    return rows


def test_philox_known_answers():
    rows = _read_kat()
    assert len(rows) == 3
    for row in rows:
        c0, c1, c2, c3, k0, k1 = row[:6]
        out = philox4x32_10(c0, c1, c2, c3, k0, k1)
        assert [int(x) for x in out] == row[6:]


def test_philox_vectorised_matches_scalar():
    rng = np.random.default_rng(5)
    c = rng.integers(0, 2**32, size=(4, 50), dtype=np.uint64)
    k = rng.integers(0, 2**32, size=2)
    vec = philox4x32_10(c[0], c[1], c[2], c[3], int(k[0]), int(k[1]))
    for t in range(50):
        one = philox4x32_10(int(c[0, t]), int(c[1, t]), int(c[2, t]), int(c[3, t]),
                            int(k[0]), int(k[1]))
        assert [int(x) for x in one] == [int(v[t]) for v in vec]


def _read_fig():
    lines = [l.strip() for l in open(golden_path("fig1_fig2_countsketch.txt"))
             if l.strip() and not l.startswith("#")]
    v = [int(x) for x in lines[0].split(":")[1].split()]
    S = np.array([[int(x) for x in l.split()] for l in lines[2:8]], dtype=np.float64)
    return np.array(v), S


def test_fig2_vector_gives_fig1_matrix_except_erratum():
    v, S_fig1 = _read_fig()
    bucket, sign = cs.from_vector_representation(v)
    S = cs.countsketch_matrix(bucket, sign, 6)
    assert S.shape == (6, 12)
    # every column of S has exactly one +-1 (Def. 3)
    assert np.all(np.sum(S != 0, axis=0) == 1)
    mismatched = sorted(set(np.nonzero(S != S_fig1)[1] + 1))
    assert mismatched == [5]          # the documented erratum, nothing else
    assert np.array_equal(cs.vector_representation(bucket, sign), v)


def test_scatter_equals_explicit_S_on_paper_example():
    v, _ = _read_fig()
    bucket, sign = cs.from_vector_representation(v)
    A = np.arange(12 * 3, dtype=np.float64).reshape(12, 3) - 7.0
    S = cs.countsketch_matrix(bucket, sign, 6)
    assert np.array_equal(cs.countsketch_apply_dense(A, bucket, sign, 6), S @ A)


@pytest.mark.parametrize("n,d,r,seed", [(50, 4, 7, 0), (300, 9, 40, 11), (1000, 3, 1, 2)])
def test_scatter_brute_force_dense_and_csr(n, d, r, seed):
    rng = np.random.default_rng(seed)
    A = rng.integers(-5, 6, size=(n, d)).astype(np.float64)
    A[rng.random((n, d)) < 0.5] = 0.0
    bucket, sign = cs.countsketch_hash(n, r, seed)
    S = cs.countsketch_matrix(bucket, sign, r)
    ref = S @ A
    assert np.array_equal(cs.countsketch_apply_dense(A, bucket, sign, r), ref)
    I = np.concatenate([[0], np.cumsum(np.sum(A != 0, axis=1))]).astype(np.int64)
    rows, cols = np.nonzero(A)
    got = cs.countsketch_apply_csr(A[rows, cols], cols, I, n, d, bucket, sign, r)
    assert np.array_equal(got, ref)


def test_hash_is_counter_based_and_in_range():
    b1, s1 = cs.countsketch_hash(5000, 97, 42)
    b0, s0 = cs.countsketch_hash(1234, 97, 42)
    assert np.array_equal(b1[:1234], b0) and np.array_equal(s1[:1234], s0)
    assert b1.min() >= 0 and b1.max() < 97
    assert set(np.unique(s1)) == {-1, 1}
    b2, _ = cs.countsketch_hash(5000, 97, 43)
    assert not np.array_equal(b1, b2)


def test_hash_uniform_and_signs_fair():
    n, r = 400_000, 64
    b, s = cs.countsketch_hash(n, r, 7)
    counts = np.bincount(b, minlength=r)
    chi2 = stats.chisquare(counts)
    assert chi2.pvalue > 1e-4
    # signs: fair coin, and independent of the bucket (2 x r table)
    assert abs(np.mean(s)) < 5.0 / np.sqrt(n)
    table = np.stack([np.bincount(b[s > 0], minlength=r), np.bincount(b[s < 0], minlength=r)])
    assert stats.chi2_contingency(table)[1] > 1e-4


def test_workload_concentration_lemma_1_to_3():
    """Lemma 1: E[Y] = q nnz(A), Var = q(1-q) nnz2(A); Lemma 3 tail over p sets."""
    rng = np.random.default_rng(3)
    n, r, p = 200_000, 4096, 16
    w = rng.integers(0, 40, size=n)          # nonzeros per row of a sparse A
    nnz, nnz2 = w.sum(), np.sum(w.astype(np.float64) ** 2)
    q = 1.0 / p
    loads = []
    for seed in range(20):
        b, _ = cs.countsketch_hash(n, r, seed)
        owner = b // (r // p)                  # contiguous ranges of B = r/p rows
        Y = np.bincount(owner, weights=w, minlength=p)
        loads.append(Y)
        bound = (1 - q) * np.sqrt(2 * nnz2 * np.log(n))   # Lemma 2 / Lemma 3
        assert np.all(np.abs(Y - q * nnz) <= bound)
    loads = np.array(loads).ravel()
    assert abs(loads.mean() - q * nnz) < 5 * np.sqrt(q * (1 - q) * nnz2 / len(loads))
    assert 0.5 < loads.var() / (q * (1 - q) * nnz2) < 1.6


def test_sketch_norm_closed_forms():
    """E||Sy||^2 = ||y||^2 and Var = (2/r)(||y||^4 - ||y||_4^4) (from Def. 3)."""
    rng = np.random.default_rng(9)
    n, r = 400, 25
    y = rng.standard_normal(n)
    vals = np.array([np.sum(cs.cs_sketch_dense(y[:, None], r, seed) ** 2)
                     for seed in range(3000)])
    y2, y4 = np.sum(y**2), np.sum(y**4)
    var = 2.0 / r * (y2**2 - y4)
    assert abs(vals.mean() - y2) < 5 * np.sqrt(var / len(vals))
    assert 0.85 < vals.var() / var < 1.15


def test_sketch_subspace_embedding_singular_values():
    """Def. 2: singular values of S Q_A near 1 for r >> d^2."""
    rng = np.random.default_rng(2)
    n, d = 20000, 6
    Q, _ = np.linalg.qr(rng.standard_normal((n, d)))
    sv = np.linalg.svd(cs.cs_sketch_dense(Q, 4000, 5), compute_uv=False)
    assert np.all(np.abs(sv - 1.0) < 0.15)


def test_block_hash_keeps_global_row_index():
    """A block of rows starting at row0 is hashed as columns row0.. of S
    (Def. 3): the block hash is the slice of the whole matrix's hash,
    including across the 2^32 boundary of the counter's low word."""
    r, seed = 1000, 77
    b, s = cs.countsketch_hash(5000, r, seed)
    for row0, n in [(0, 5000), (1234, 2000), (4999, 1)]:
        bb, ss = cs.countsketch_hash_rows(row0, n, r, seed)
        assert np.array_equal(bb, b[row0:row0 + n]) and np.array_equal(ss, s[row0:row0 + n])
    # rows 2^32 - 2 .. 2^32 + 1: the counter's high word takes the carry
    bb, ss = cs.countsketch_hash_rows(2**32 - 2, 4, r, seed)
    for t, i in enumerate(range(2**32 - 2, 2**32 + 2)):
        w = philox4x32_10(i & 0xFFFFFFFF, i >> 32, cs.STREAM_S, 0, seed & 0xFFFFFFFF, seed >> 32)
        assert bb[t] == (int(w[0]) * r) >> 32
        assert ss[t] == (-1 if int(w[1]) >= 2**31 else 1)


def test_row_partition_sketches_sum_to_the_whole():
    """S A = sum_g S_g A_g for a row partition (the exchange of the sharded
    path): brute force with the explicit S of the whole matrix."""
    rng = np.random.default_rng(3)
    n, d, r, seed = 300, 7, 40, 9
    A = rng.standard_normal((n, d))
    b, s = cs.countsketch_hash(n, r, seed)
    whole = cs.countsketch_matrix(b, s, r) @ A
    parts = np.zeros((r, d))
    for row0, rows in [(0, 120), (120, 1), (121, 179)]:
        bb, ss = cs.countsketch_hash_rows(row0, rows, r, seed)
        parts += cs.countsketch_apply_dense(A[row0:row0 + rows], bb, ss, r)
    assert np.allclose(parts, whole, rtol=0, atol=1e-12)
