"""GPU parity of the fused CountSketch + Gaussian stage (lsk_count_gauss):
G*(S*A) in one pass over A, S*A kept on chip (Alg. 3's blocked CountGauss),
against the FP64 oracle's blocked CountGauss on the same seeds.

Tolerances: the BF16 mode of the Gaussian stage -- G is the bf16 rounding of
the scaled draws on both sides (rare one-ulp disagreements where the float32
evaluations straddle a rounding midpoint, taken into the bound exactly from
the device's G) and S*A is carried as bf16 hi + lo (2^-16 relative); 1e-4
relative Frobenius error, and an element-wise bound from the summation
lengths.
"""
import numpy as np
import pytest
import torch

import workloads
from oracle import countsketch as ocs
from oracle import gaussian as oga
from oracle import leverage as olev

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def lsk():
    from paper_2203_02798_gb300 import build
    build.build()
    import paper_2203_02798_gb300 as p
    return p


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def rel_fro(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


# (n, d, r, k): two 256-row sets (k = 512) and one (k <= 256), a ragged k;
# d = 256 (both 128-column halves full), ragged halves (d = 100, 36, 200);
# r with a partial last chunk and slices of a few buckets; r > n (empty buckets)
CASES = [(20_000, 256, 1000, 512), (20_011, 100, 2500, 300), (5_000, 32, 40, 7),
         (9_000, 64, 700, 256), (3_000, 36, 5000, 257), (30_000, 200, 33, 64)]


@pytest.mark.parametrize("n,d,r,k", CASES)
def test_count_gauss_matches_oracle(lsk, n, d, r, k):
    seed = n + r
    A = workloads.dense_normal(n, d, seed=d + k)
    got = host(lsk.count_gauss(dev(A), r, k, seed)).astype(np.float64)
    A64 = A.astype(np.float64)
    ref = oga.count_gauss_dense(A64, r, k, seed, oga.PREC_BF16)   # Alg. 3's blocked order
    assert rel_fro(got, ref) <= 1e-4
    bucket, sign = ocs.countsketch_hash(n, r, seed)
    absSA = ocs.countsketch_apply_dense(np.abs(A64), bucket, np.ones_like(sign), r)
    G = oga.gaussian_matrix(k, r, seed, oga.PREC_BF16)
    bound = np.abs(G) @ absSA
    maxlen = np.bincount(bucket, minlength=r).max() if n else 0
    # G on the device (the same draws, bf16-rounded): the entries where the two
    # float32 evaluations straddle a bf16 rounding midpoint differ by one bf16
    # ulp; their exact effect on G S A is bounded by |G_gpu - G| |S A|, so every
    # other element keeps the tight bound (FP32 sums of the bucket and of the
    # r columns, and the 2^-16 bf16 hi / lo split of S A)
    Gd = host(lsk.debug_gauss(k, r, seed, "bf16")).astype(np.float64)
    dG = np.abs(Gd - G)
    assert np.count_nonzero(dG) <= max(4, 4e-4 * dG.size)
    tight = (2 * (r + maxlen + 16) * U32 + 2.0**-16) * bound
    assert np.all(np.abs(got - ref) <= tight + 1.01 * (dG @ absSA) + 1e-30)


def test_count_gauss_integer_agrees_with_two_stages(lsk):
    """Integer-valued A: S*A and its bf16 split are exact on both paths, so the
    fused and the two-stage results differ only in FP32 accumulation order."""
    n, d, r, k = 40_000, 128, 3000, 384
    A = workloads.integer_dense(n, d, seed=5, lo=-4, hi=4)
    fused = host(lsk.count_gauss(dev(A), r, k, 7)).astype(np.float64)
    two = host(lsk.gauss_sketch(lsk.cs_sketch(dev(A), r, 7), k, 7, "bf16")).astype(np.float64)
    assert rel_fro(fused, two) <= 1e-6
    SA = ocs.cs_sketch_dense(A.astype(np.float64), r, 7)
    assert rel_fro(fused, oga.gauss_sketch(SA, k, 7, oga.PREC_BF16)) <= 1e-4


def test_count_gauss_empty_matrix_is_zero(lsk):
    A = torch.empty((0, 64), dtype=torch.float32, device="cuda")
    out = lsk.count_gauss(A, 100, 32, 1)
    assert torch.count_nonzero(out).item() == 0


@pytest.mark.parametrize("d,k", [(30, 16), (260, 16), (66, 16), (64, 513), (64, 0)])
def test_count_gauss_rejects_unsupported(lsk, d, k):
    A = torch.zeros((100, d), dtype=torch.float32, device="cuda")
    with pytest.raises(lsk.LskError):
        lsk.count_gauss(A, 64, k, 0)


@pytest.mark.parametrize("d", [64, 256])
def test_leverage_fused_sketch_matches_oracle(lsk, d):
    """The leverage-score pipeline in the BF16 mode forms its sketch with the
    fused kernel; the scores agree with the oracle's estimate on the same
    seeds as those of the two-stage sketch do."""
    n, r, k = 60_000, 4096, 2 * d
    A = workloads.dense_normal(n, d, seed=d)
    A[:3] *= 30.0
    ref, _ = olev.leverage_scores_dense(A.astype(np.float64), r, k, 9, oga.PREC_BF16)
    prev = lsk.set_fused_sketch(True)
    try:
        fused = host(lsk.leverage_scores(dev(A), r, k, 9, "bf16")).astype(np.float64)
        lsk.set_fused_sketch(False)
        two = host(lsk.leverage_scores(dev(A), r, k, 9, "bf16")).astype(np.float64)
    finally:
        lsk.set_fused_sketch(prev)
    assert np.max(np.abs(fused - ref) / ref) <= 1e-3
    assert np.max(np.abs(two - ref) / ref) <= 1e-3
    assert np.max(np.abs(fused - two) / two) <= 1e-4
