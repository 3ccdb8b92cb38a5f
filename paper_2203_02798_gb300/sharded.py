"""Leverage scores and Gram matrices of a matrix split by rows over ranks.

One process per GPU, each holding a contiguous block of rows of A.  The
sketch is linear in A and the CountSketch hashes a row by its index in the
whole matrix (Def. 3), so with blocks A_g starting at row row0_g

    G S A = sum_g G S_g A_g,        A^T A = sum_g A_g^T A_g.

Each rank forms its partial sketch (``sketch_rows``), one sum all-reduce of
k x d floats makes the whole sketch on every rank (the only exchange: the
reason Def. 4 asks for a small sketch), every rank forms the same R from it,
and scores its own rows (``leverage_scores_from_sketch``).  The Gram matrix
takes one all-reduce of d x d floats.

The compute calls go through ``ops`` (by default the CUDA library's
binding), so the exchange and the row bookkeeping are the only work here.
"""
import torch
import torch.distributed as dist


def shard_rows(n, world, rank):
    """(row0, rows) of rank's block of a contiguous row partition of n rows:
    the first n % world ranks take one row more."""
    if world < 1 or not (0 <= rank < world) or n < 0:
        raise ValueError("bad partition arguments")
    base, extra = divmod(n, world)
    rows = base + (1 if rank < extra else 0)
    row0 = rank * base + min(rank, extra)
    return row0, rows


def _ops(ops):
    if ops is not None:
        return ops
    import paper_2203_02798_gb300 as lsk
    return lsk


def leverage_scores_sharded(A_local, row0, r, k, seed, prec="bf16", out=None, group=None, ops=None, ctx=None):
    """ell for the rows of A_local (rows row0.. of the whole matrix) in the
    leverage scores of the whole matrix; every rank of `group` calls it with
    its own block and the same r, k, seed and prec."""
    ops = _ops(ops)
    sk = ops.sketch_rows(A_local, r, k, seed, prec, row0=row0, ctx=ctx)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(sk, op=dist.ReduceOp.SUM, group=group)
    return ops.leverage_scores_from_sketch(A_local, sk, prec, out=out, ctx=ctx)


def gram_sharded(A_local, prec="fp32", group=None, ops=None, ctx=None):
    """A^T A of the whole matrix on every rank (d x d float32)."""
    ops = _ops(ops)
    C = ops.gram(A_local, prec=prec, ctx=ctx)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(C, op=dist.ReduceOp.SUM, group=group)
    return C
