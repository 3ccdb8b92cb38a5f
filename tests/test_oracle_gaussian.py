"""Pins of the oracle's Gaussian G (CPU only): distribution, JL closed forms
(Def. 1), bfloat16 rounding, and the batching of Alg. 3."""
import numpy as np
from scipy import stats

from oracle import gaussian as ga


def test_entries_standard_normal_after_scaling():
    k, r = 64, 20000
    G = ga.gaussian_matrix(k, r, 3)
    z = (G * np.sqrt(k)).ravel()
    assert abs(z.mean()) < 5 / np.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / z.size)
    assert abs(stats.kurtosis(z, fisher=False) - 3.0) < 0.02
    assert stats.kstest(z, "norm").pvalue > 1e-3


def test_rows_uncorrelated_including_box_muller_pairs():
    k, r = 8, 200000
    z = ga.gaussian_matrix(k, r, 4) * np.sqrt(k)
    C = np.corrcoef(z)
    off = C[~np.eye(k, dtype=bool)]
    assert np.max(np.abs(off)) < 5 / np.sqrt(r)
    # the cos / sin pair of one Box-Muller draw: squares are uncorrelated too
    assert abs(np.corrcoef(z[0] ** 2, z[1] ** 2)[0, 1]) < 5 / np.sqrt(r)


def test_columns_independent_of_r_and_rows_of_k():
    G1 = ga.gaussian_matrix(12, 300, 9) * np.sqrt(12)
    G2 = ga.gaussian_matrix(12, 100, 9) * np.sqrt(12)
    assert np.array_equal(G1[:, :100], G2)
    G3 = ga.gaussian_matrix(5, 100, 9) * np.sqrt(5)
    assert np.allclose(G3, G2[:5], rtol=0, atol=1e-12)


def test_jl_closed_forms():
    """E||Gz||^2 = ||z||^2, Var = 2||z||^4 / k (Def. 1 / scaling 1/sqrt(k))."""
    rng = np.random.default_rng(1)
    r, k = 50, 16
    z = rng.standard_normal(r)
    vals = np.array([np.sum((ga.gaussian_matrix(k, r, s) @ z) ** 2) for s in range(2000)])
    z2 = z @ z
    var = 2 * z2**2 / k
    assert abs(vals.mean() - z2) < 5 * np.sqrt(var / len(vals))
    assert 0.85 < vals.var() / var < 1.15


def test_bf16_round_to_nearest_even():
    one = 1.0
    ulp = 2.0**-7                                   # bf16 spacing in [1, 2)
    cases = {
        one: one,
        one + ulp / 2: one,                          # tie -> even (1.0)
        one + 3 * ulp / 2: one + 2 * ulp,            # tie -> even (1 + 2 ulp)
        one + ulp / 2 + 2.0**-20: one + ulp,         # above the tie -> up
        -(one + ulp / 4): -one,
        3.0e-39: 3.0e-39,                            # checked below as subnormal
    }
    x = np.array(list(cases.keys()), dtype=np.float32)
    got = ga.float32_to_bf16_rne(x)
    for xi, gi, (k, want) in zip(x, got, cases.items()):
        if k == 3.0e-39:
            # bf16 keeps 7 explicit bits: the result is within one bf16 ulp
            assert abs(gi - float(xi)) <= 2.0**-133
        else:
            assert gi == want, (k, gi, want)
    # every output is a bf16 value: low 16 bits of the float32 pattern are zero
    bits = got.astype(np.float32).view(np.uint32)
    assert np.all(bits & 0xFFFF == 0)


def test_bf16_mode_is_rounding_of_fp32_mode():
    G = ga.gaussian_matrix(16, 500, 2, ga.PREC_FP32)
    Gb = ga.gaussian_matrix(16, 500, 2, ga.PREC_BF16)
    rel = np.abs(Gb - G) / np.abs(G)
    assert np.max(rel) <= 2.0**-8 * 1.0001


def test_gauss_sketch_batching_only_changes_rounding():
    rng = np.random.default_rng(0)
    SA = rng.standard_normal((1000, 7))
    a = ga.gauss_sketch(SA, 10, 5, batch=37)
    b = ga.gauss_sketch(SA, 10, 5, batch=4096)
    G = ga.gaussian_matrix(10, 1000, 5)
    assert np.allclose(a, G @ SA, rtol=1e-13, atol=1e-13)
    assert np.allclose(b, G @ SA, rtol=1e-13, atol=1e-13)


def test_jl_projection_scale_distribution_and_stream():
    """Pi of Alg. 15: entries N(0, 1/m) (so E ||x Pi||^2 = ||x||^2), drawn on
    their own counter stream (not the Gaussian stage's G)."""
    d, m, seed = 64, 4000, 17
    P = ga.jl_matrix(d, m, seed)
    assert P.shape == (d, m)
    z = P.ravel() * np.sqrt(m)
    assert abs(z.mean()) < 5 / np.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / z.size)
    rng = np.random.default_rng(3)
    for _ in range(5):
        x = rng.standard_normal(d)
        ratio = np.sum((x @ P) ** 2) / np.sum(x * x)
        assert abs(ratio - 1.0) < 5 * np.sqrt(2.0 / m)        # chi^2_m / m
    G = ga.gaussian_matrix(m, d, seed)                        # stream 1, same shape as Pi^T
    assert abs(np.corrcoef(G.ravel(), P.T.ravel())[0, 1]) < 5 / np.sqrt(G.size)
    # the construction: Pi[i, c] is G's entry (c, i) on the Pi stream
    assert np.array_equal(P[5:9, 40:48], ga.gaussian_columns(m, 5, 9, seed, stream=ga.STREAM_PI)[40:48].T)


def test_count_gauss_blocked_equals_explicit_product():
    """Alg. 3's blocked CountGauss against the plain product G S A with the
    explicit S of Def. 3 (brute force on small inputs), for block sizes that
    split buckets unevenly, one bucket per block and the whole of r; buckets
    that no row hashes to (r > n) add nothing."""
    from oracle import countsketch as cs
    rng = np.random.default_rng(5)
    for n, d, r, k in [(300, 7, 40, 9), (50, 3, 200, 4), (1, 5, 3, 2)]:
        A = rng.standard_normal((n, d))
        bucket, sign = cs.countsketch_hash(n, r, 11)
        S = cs.countsketch_matrix(bucket, sign, r)
        for prec in (ga.PREC_FP32, ga.PREC_BF16):
            ref = ga.gaussian_matrix(k, r, 11, prec) @ (S @ A)
            for block in (1, 7, 32, r):
                got = ga.count_gauss_dense(A, r, k, 11, prec, block=block)
                assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_count_gauss_blocked_equals_the_two_stages():
    """The blocked form equals the separate stages S A, then G (S A)."""
    from oracle import countsketch as cs
    A = np.random.default_rng(6).standard_normal((5000, 16))
    two = ga.gauss_sketch(cs.cs_sketch_dense(A, 700, 3), 48, 3, ga.PREC_BF16)
    got = ga.count_gauss_dense(A, 700, 48, 3, ga.PREC_BF16)
    assert np.allclose(got, two, rtol=1e-12, atol=1e-12 * np.abs(two).max())
    # a sign flip of one row of A changes exactly its bucket's column of G times that row
    A2 = A.copy()
    A2[17] *= -1
    bucket, sign = cs.countsketch_hash(5000, 700, 3)
    g = ga.gaussian_columns(48, int(bucket[17]), int(bucket[17]) + 1, 3, ga.PREC_BF16)[:, 0]
    diff = ga.count_gauss_dense(A2, 700, 48, 3, ga.PREC_BF16) - got
    assert np.allclose(diff, -2 * sign[17] * np.outer(g, A[17]), atol=1e-12)
