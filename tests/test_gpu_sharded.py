"""GPU parity of the row-partitioned path (lsk_sketch_rows +
lsk_leverage_scores_from_sketch): the blocks of a row partition run one
after the other on one GPU and their partial sketches are summed on the
device, standing in for the all-reduce of a multi-GPU run.

- integer-valued data: the summed CountSketch partials equal the sketch of
  the whole matrix bit for bit (every sum is exact);
- a block far from row 0 (across the 2^32 boundary of the hash counter)
  against the oracle's block hash;
- the fused BF16 partial of a block against the oracle (1e-4 relative
  Frobenius, as the fused-kernel tests);
- leverage scores from the summed sketch against lsk_leverage_scores of the
  whole matrix (1e-4 relative: FP32 summation order of the sketch) and the
  oracle's estimate on the same seeds (1e-3).
"""
import numpy as np
import pytest
import torch

import workloads
from oracle import countsketch as ocs
from oracle import gaussian as oga
from oracle import leverage as olev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lsk():
    from paper_2203_02798_gb300 import build
    build.build()
    import paper_2203_02798_gb300 as p
    return p


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def rel_fro(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("parts", [[50_000], [20_000, 30_000], [1, 9_999, 17_000, 23_000]])
def test_countsketch_partials_sum_to_the_whole_integer_exact(lsk, parts):
    n, d, r, seed = sum(parts), 64, 3000, 17
    A = workloads.integer_dense(n, d, seed=4)
    whole = lsk.cs_sketch(dev(A), r, seed)
    acc = torch.zeros_like(whole)
    row0 = 0
    for rows in parts:
        acc += lsk.sketch_rows(dev(A[row0:row0 + rows]), r, 0, seed, "fp32", row0=row0)
        row0 += rows
    lsk.context().sync()
    assert torch.equal(acc, whole)


def test_block_across_the_counter_boundary_matches_the_oracle_hash(lsk):
    n, d, r, seed = 4000, 32, 500, 3
    row0 = 2**32 - 1500
    A = workloads.integer_dense(n, d, seed=6)
    got = lsk.sketch_rows(dev(A), r, 0, seed, "fp32", row0=row0).cpu().numpy().astype(np.float64)
    b, s = ocs.countsketch_hash_rows(row0, n, r, seed)
    assert np.array_equal(got, ocs.countsketch_apply_dense(A.astype(np.float64), b, s, r))


@pytest.mark.parametrize("fused", [0, 2])
def test_gaussian_partial_of_a_block_matches_the_oracle(lsk, fused):
    n, d, r, k, seed = 30_000, 256, 2048, 512, 8
    row0 = 123_457
    A = workloads.dense_normal(n, d, seed=2)
    prev = lsk.set_fused_sketch(fused)
    try:
        got = lsk.sketch_rows(dev(A), r, k, seed, "bf16", row0=row0).cpu().numpy().astype(np.float64)
    finally:
        lsk.set_fused_sketch(prev)
    b, s = ocs.countsketch_hash_rows(row0, n, r, seed)
    SA = ocs.countsketch_apply_dense(A.astype(np.float64), b, s, r)
    assert rel_fro(got, oga.gauss_sketch(SA, k, seed, oga.PREC_BF16)) <= 1e-4


@pytest.mark.parametrize("n,d,r,k,parts,prec", [
    (60_000, 64, 4096, 128, [25_000, 35_000], "bf16"),
    (40_000, 50, 2500, 100, [10_000, 10_000, 20_000], "fp32"),
    (1_000_000, 256, 65_536, 512, [500_000, 500_000], "bf16"),
])
def test_scores_from_the_summed_sketch(lsk, n, d, r, k, parts, prec):
    seed = 21
    A = workloads.dense_normal(n, d, seed=d)
    A[:3] *= 40.0
    Ad = dev(A)
    whole = lsk.leverage_scores(Ad, r, k, seed, prec).cpu().numpy().astype(np.float64)
    sk = None
    row0 = 0
    for rows in parts:
        p = lsk.sketch_rows(Ad[row0:row0 + rows], r, k, seed, prec, row0=row0)
        sk = p if sk is None else sk + p
        row0 += rows
    got = []
    row0 = 0
    for rows in parts:
        got.append(lsk.leverage_scores_from_sketch(Ad[row0:row0 + rows], sk, prec).cpu().numpy())
        row0 += rows
    lsk.context().sync()
    got = np.concatenate(got).astype(np.float64)
    assert np.max(np.abs(got - whole) / whole) <= 1e-4
    if n <= 60_000:
        ref, _ = olev.leverage_scores_dense(A.astype(np.float64), r, k, seed,
                                            oga.PREC_BF16 if prec == "bf16" else oga.PREC_FP32)
        assert np.max(np.abs(got - ref) / ref) <= 1e-3


def test_driver_on_one_rank_is_the_plain_call(lsk):
    from paper_2203_02798_gb300 import sharded
    n, d, r, k, seed = 30_000, 32, 1024, 64, 4
    A = dev(workloads.dense_normal(n, d, seed=1))
    a = sharded.leverage_scores_sharded(A, 0, r, k, seed, "bf16")
    b = lsk.leverage_scores(A, r, k, seed, "bf16")
    lsk.context().sync()
    assert torch.allclose(a, b, rtol=1e-5, atol=0)


def test_sketch_rows_rejects_bad_arguments(lsk):
    A = torch.zeros((10, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(lsk.LskError):
        lsk.sketch_rows(A, 16, 0, 1, "fp32", row0=-1)
    with pytest.raises(lsk.LskError):
        lsk.sketch_rows(A, 0, 0, 1, "fp32")
    with pytest.raises(lsk.LskError):
        lsk.leverage_scores_from_sketch(A, torch.zeros((4, 8), dtype=torch.float32, device="cuda"))


def test_accumulated_blocks_equal_the_whole_sketch(lsk):
    """lsk_sketch_rows with accumulate: one buffer summing the blocks' sketches
    (integer data: exact), for k = 0 (added by the gather itself) and k > 0."""
    n, d, r, k, seed = 40_000, 48, 2000, 96, 13
    A = workloads.integer_dense(n, d, seed=8)
    Ad = dev(A)
    whole = lsk.cs_sketch(Ad, r, seed)
    acc = torch.full_like(whole, float("nan"))
    for i, (c0, c1) in enumerate([(0, 7_000), (7_000, 7_001), (7_001, 40_000)]):
        lsk.sketch_rows(Ad[c0:c1], r, 0, seed, "fp32", row0=c0, out=acc, accumulate=i > 0)
    lsk.context().sync()
    assert torch.equal(acc, whole)
    g_whole = lsk.sketch_rows(Ad, r, k, seed, "fp32")
    g_acc = torch.zeros_like(g_whole)
    for c0, c1 in [(0, 25_000), (25_000, 40_000)]:
        lsk.sketch_rows(Ad[c0:c1], r, k, seed, "fp32", row0=c0, out=g_acc, accumulate=True)
    lsk.context().sync()
    assert rel_fro(g_acc.cpu().numpy().astype(np.float64), g_whole.cpu().numpy().astype(np.float64)) <= 1e-6


@pytest.mark.parametrize("n,chunk", [(300_001, 65_536), (50_000, 1 << 19)])
def test_leverage_scores_from_host_memory(lsk, n, chunk):
    """The end-to-end call (copy of block c + 1 overlapping the sketch of block
    c) gives the scores of the device call with the two-stage sketch, to FP32
    summation order."""
    d, r, k, seed = 64, 4096, 128, 3
    A = workloads.dense_normal(n, d, seed=12)
    A[:2] *= 30.0
    A_host = torch.from_numpy(A).pin_memory()
    got = lsk.leverage_scores_host(A_host, r, k, seed, "bf16", chunk_rows=chunk)
    torch.cuda.synchronize()
    prev = lsk.set_fused_sketch(0)
    try:
        ref = lsk.leverage_scores(dev(A), r, k, seed, "bf16").cpu()
    finally:
        lsk.set_fused_sketch(prev)
    assert torch.allclose(got, ref, rtol=2e-5, atol=0)
