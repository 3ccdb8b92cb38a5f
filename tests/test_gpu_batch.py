"""Batched leverage scores: every problem of a mixed batch (dense / CSR,
d in {32, 64, 128, 256}, uneven n) equals its single-problem result and the
oracle's estimate (<= 1e-3), with and without CUDA-graph capture and with
the stream-count autotuner.

Two BF16 computations of the same problem agree to CONSISTENT = 1e-4
relative, not to the last FP32 bit: the row norms split A and R^-1 into
bfloat16 pairs (about 2^-16 relative), so R^-1 values that differ in their
last bits (the grouped Gaussian stage adds its partial sums in other groups;
CountSketch adds the rows of a bucket in the order the atomic ranking gave
them) can round to different pairs."""
import numpy as np
import pytest
import torch

import workloads
from oracle import gaussian as oga
from oracle import leverage as olev

pytestmark = pytest.mark.gpu

CONSISTENT = 1e-4


@pytest.fixture(scope="module")
def lsk():
    from paper_2203_02798_gb300 import build
    build.build()
    import paper_2203_02798_gb300 as p
    return p


def make_batch(lsk, count=16, seed=11):
    rng = np.random.default_rng(seed)
    probs, host = [], []
    for p in range(count):
        d = int(rng.choice([32, 64, 128, 256]))
        n = int(10 ** rng.uniform(3.7, 4.6))
        r, k = max(d * d // 4, 4 * d), 2 * d
        if p % 2 == 0:
            A = workloads.dense_normal(n, d, seed=1000 + p)
            probs.append((torch.from_numpy(A).cuda(), r, k, 77 + p))
            host.append(("dense", A, n, d, r, k, 77 + p))
        else:
            V, J, I = workloads.csr_bernoulli(n, d, float(rng.uniform(0.05, 0.15)), seed=1000 + p)
            probs.append((lsk.csr_from_numpy(V, J, I, d), r, k, 77 + p))
            host.append(("csr", (V, J, I), n, d, r, k, 77 + p))
    return probs, host


@pytest.mark.parametrize("graph", [False, True])
def test_batch_matches_single_and_oracle(lsk, graph):
    probs, host = make_batch(lsk)
    outs = lsk.batch_leverage_scores(probs, prec="bf16", graph=graph, streams=4)
    lsk.context().sync()
    if graph:   # replay of the cached graph gives the same answer
        again = lsk.batch_leverage_scores(probs, prec="bf16", graph=True, streams=4)
        lsk.context().sync()
        for a, b in zip(outs, again):
            assert torch.allclose(a, b, rtol=CONSISTENT, atol=0)
    for (A, r, k, seed), ell, h in zip(probs, outs, host):
        single = lsk.leverage_scores(A, r, k, seed, "bf16")
        lsk.context().sync()
        nz = single > 0
        assert torch.all((ell[~nz] == 0))
        assert torch.max(torch.abs(ell[nz] - single[nz]) / single[nz]).item() <= CONSISTENT
    for (A, r, k, seed), ell, h in list(zip(probs, outs, host))[:6]:
        kind, data, n, d, r, k, seed = h
        if kind == "dense":
            ref, _ = olev.leverage_scores_dense(data.astype(np.float64), r, k, seed, oga.PREC_BF16)
        else:
            V, J, I = data
            ref, _ = olev.leverage_scores_csr(V, J, I, n, d, r, k, seed, oga.PREC_BF16)
        got = ell.cpu().numpy().astype(np.float64)
        nz = ref > 0
        assert np.max(np.abs(got[nz] - ref[nz]) / ref[nz]) <= 1e-3


def test_batch_autotune_chooses_streams(lsk):
    probs, _ = make_batch(lsk, count=10, seed=5)
    outs = lsk.batch_leverage_scores(probs, prec="bf16", autotune=True)
    lsk.context().sync()
    s = lsk.batch_streams(probs, prec="bf16")
    assert s in (1, 4, 8, 16, 32)
    single = lsk.leverage_scores(probs[0][0], *probs[0][1:], "bf16")
    lsk.context().sync()
    assert torch.allclose(outs[0], single, rtol=CONSISTENT, atol=1e-30)


def test_batch_empty_and_single(lsk):
    assert lsk.batch_leverage_scores([], prec="bf16") == []
    A = torch.from_numpy(workloads.dense_normal(5000, 32, seed=3)).cuda()
    out = lsk.batch_leverage_scores([(A, 1024, 64, 9)], prec="fp32")
    lsk.context().sync()
    ref = lsk.leverage_scores(A, 1024, 64, 9, "fp32")
    lsk.context().sync()
    assert torch.allclose(out[0], ref, rtol=1e-5, atol=1e-30)


def test_grouped_stages_match_per_problem_pipelines(lsk):
    """The grouped Gaussian / R^-1 stages give each problem the result of its
    own pipeline (the Gaussian partial sums are grouped differently, so
    agreement is to rounding), in a batch that also holds problems the grouped
    path does not take (d > 256, k = 0)."""
    probs, host = make_batch(lsk, count=12, seed=21)
    A300 = torch.from_numpy(workloads.dense_normal(6000, 300, seed=4)).cuda()
    probs.append((A300, 90_000, 600, 5))                       # d > 256: per-problem FP64 path
    A64 = torch.from_numpy(workloads.dense_normal(9000, 64, seed=6)).cuda()
    probs.append((A64, 4096, 0, 8))                            # k = 0: CountSketch only
    grouped = lsk.batch_leverage_scores(probs, prec="bf16", streams=4)
    lsk.context().sync()
    ref = lsk.batch_leverage_scores(probs, prec="bf16", streams=4, per_problem=True)
    lsk.context().sync()
    for a, b in zip(grouped, ref):
        assert a.shape == b.shape
        if b.numel() == 0:
            continue
        nz = b > 0
        assert torch.all(a[~nz] == 0)
        assert torch.max(torch.abs(a[nz] - b[nz]) / b[nz]).item() <= CONSISTENT
    # and against the oracle for two of the grouped problems
    for (A, r, k, seed), ell, h in list(zip(probs, grouped, host))[:2]:
        kind, data, n, d, r, k, seed = h
        if kind == "dense":
            o, _ = olev.leverage_scores_dense(data.astype(np.float64), r, k, seed, oga.PREC_BF16)
        else:
            V, J, I = data
            o, _ = olev.leverage_scores_csr(V, J, I, n, d, r, k, seed, oga.PREC_BF16)
        got = ell.cpu().numpy().astype(np.float64)
        nz = o > 0
        assert np.max(np.abs(got[nz] - o[nz]) / o[nz]) <= 1e-3


def test_grouped_compacted_sketches_match_per_problem_pipelines(lsk):
    """Problems with n < 4r take a sketch compacted to their non-empty buckets
    (most buckets empty here: n / r from 0.05 to 0.5), and the grouped
    Gaussian stage draws G only for those columns; each result equals the
    problem's own uncompacted pipeline to rounding and the oracle's estimate
    to 1e-3."""
    specs = [("dense", 3000, 128, 16384), ("csr", 5000, 128, 16384), ("dense", 9000, 256, 65536),
             ("dense", 33000, 256, 65536), ("csr", 2000, 64, 4096), ("dense", 1500, 32, 1024)]
    probs, host = [], []
    for i, (kind, n, d, r) in enumerate(specs):
        k = 2 * d
        if kind == "dense":
            A = workloads.dense_normal(n, d, seed=300 + i)
            A[: 2] *= 20.0
            probs.append((torch.from_numpy(A).cuda(), r, k, 500 + i))
            host.append((kind, A, n, d, r, k, 500 + i))
        else:
            V, J, I = workloads.csr_bernoulli(n, d, 0.1, seed=300 + i)
            probs.append((lsk.csr_from_numpy(V, J, I, d), r, k, 500 + i))
            host.append((kind, (V, J, I), n, d, r, k, 500 + i))
    grouped = lsk.batch_leverage_scores(probs, prec="bf16", streams=3)
    lsk.context().sync()
    ref = lsk.batch_leverage_scores(probs, prec="bf16", streams=3, per_problem=True)
    lsk.context().sync()
    for a, b in zip(grouped, ref):
        nz = b > 0
        assert torch.all(a[~nz] == 0)
        assert torch.max(torch.abs(a[nz] - b[nz]) / b[nz]).item() <= CONSISTENT
    for ell, h in list(zip(grouped, host))[:3]:
        kind, data, n, d, r, k, seed = h
        if kind == "dense":
            o, _ = olev.leverage_scores_dense(data.astype(np.float64), r, k, seed, oga.PREC_BF16)
        else:
            V, J, I = data
            o, _ = olev.leverage_scores_csr(V, J, I, n, d, r, k, seed, oga.PREC_BF16)
        got = ell.cpu().numpy().astype(np.float64)
        nz = o > 0
        assert np.all(got[~nz] == 0)
        assert np.max(np.abs(got[nz] - o[nz]) / o[nz]) <= 1e-3


def test_grouped_batch_graph_replay_and_rank_deficiency(lsk):
    """A graph-captured grouped batch replays to the same answer; a rank-
    deficient member raises the context's deferred error."""
    probs, _ = make_batch(lsk, count=6, seed=31)
    first = lsk.batch_leverage_scores(probs, prec="bf16", graph=True, streams=2)
    lsk.context().sync()
    again = lsk.batch_leverage_scores(probs, prec="bf16", graph=True, streams=2)
    lsk.context().sync()
    for a, b in zip(first, again):
        assert torch.allclose(a, b, rtol=CONSISTENT, atol=0)
    A = torch.from_numpy(workloads.dense_normal(5000, 64, seed=2)).cuda()
    A[:, 7] = A[:, 3]                                          # rank 63
    bad = probs[:2] + [(A, 4096, 128, 3)]
    lsk.batch_leverage_scores(bad, prec="bf16", streams=2)
    with pytest.raises(lsk.LskError) as ei:
        lsk.context().sync()
    assert ei.value.name == "RANK_DEFICIENT"
