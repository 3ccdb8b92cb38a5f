"""The row-partitioned (sharded) leverage-score path on the CPU: world size
2 and 3 over gloo, each rank holding a block of rows.  The compute calls run
the FP64 oracle (standing in for the CUDA library, which needs a GPU), so
this checks what the driver itself does -- the row partition, the global
row offsets handed to the sketch, the one all-reduce of the partial
sketches, the redundant R and the local scores -- against the oracle's
scores of the whole matrix.  The GPU calls behind the same driver are
checked in test_gpu_sharded.py."""
import json
import os
import socket
import sys
import tempfile

import numpy as np
import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2203_02798_gb300.sharded import shard_rows  # noqa: E402


class OracleOps:
    """The three compute calls of the driver, from the FP64 oracle."""

    def sketch_rows(self, A, r, k, seed, prec, row0=0, ctx=None):
        from oracle import countsketch as ocs
        from oracle import gaussian as oga
        A = A.numpy()
        b, s = ocs.countsketch_hash_rows(row0, A.shape[0], r, seed)
        SA = ocs.countsketch_apply_dense(A, b, s, r)
        out = SA if k == 0 else oga.gauss_sketch(SA, k, seed, oga.PREC_BF16 if prec == "bf16" else oga.PREC_FP32)
        return torch.from_numpy(np.ascontiguousarray(out))

    def leverage_scores_from_sketch(self, A, sk, prec, out=None, ctx=None):
        from oracle import leverage as olev
        from oracle import qr as oqr
        from oracle import rownorms as orn
        R = olev.sketch_R(sk.numpy())
        return torch.from_numpy(orn.rownorms_prod_dense(A.numpy(), oqr.upper_triangular_inverse(R)))

    def gram(self, A, prec="fp32", ctx=None):
        from oracle import gram as og
        return torch.from_numpy(og.gram_dense(A.numpy()))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


N, D, R, K, SEED = 3001, 12, 300, 40, 5


def _matrix():
    rng = np.random.default_rng(11)
    A = rng.standard_normal((N, D))
    A[:4] *= 50.0
    return A


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    from paper_2203_02798_gb300 import sharded
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    A = _matrix()
    row0, rows = shard_rows(N, world, rank)
    A_local = torch.from_numpy(A[row0:row0 + rows].copy())
    ell = sharded.leverage_scores_sharded(A_local, row0, R, K, SEED, "bf16", ops=OracleOps())
    C = sharded.gram_sharded(A_local, ops=OracleOps())
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"row0": row0, "ell": ell.tolist(), "C": C.numpy().tolist()}, f)


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_scores_equal_the_whole_matrix_scores(world):
    import torch.multiprocessing as mp
    from oracle import gaussian as oga
    from oracle import leverage as olev
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_rank_main, args=(world, _free_port(), d), nprocs=world, join=True)
        res = [json.load(open(os.path.join(d, f"r{r}.json"))) for r in range(world)]
    A = _matrix()
    ref, _ = olev.leverage_scores_dense(A, R, K, SEED, oga.PREC_BF16)
    got = np.concatenate([np.array(r["ell"]) for r in sorted(res, key=lambda r: r["row0"])])
    assert got.shape == ref.shape
    # the sketch is summed in another order than the whole-matrix scatter: FP64 rounding only
    assert np.max(np.abs(got - ref) / ref) <= 1e-10
    for r in res:
        assert np.allclose(np.array(r["C"]), A.T @ A, rtol=1e-12, atol=1e-9)


def test_row_partition_covers_every_row_once():
    for n in [0, 1, 7, 3001]:
        for world in [1, 2, 3, 8]:
            spans = [shard_rows(n, world, g) for g in range(world)]
            assert spans[0][0] == 0
            for (a0, an), (b0, _) in zip(spans, spans[1:]):
                assert a0 + an == b0
            assert spans[-1][0] + spans[-1][1] == n
            assert max(s[1] for s in spans) - min(s[1] for s in spans) <= 1
    with pytest.raises(ValueError):
        shard_rows(10, 2, 2)
