"""The N > 1 path of bench.py on the CPU: two gloo ranks (replicas, no data-
path collective).  The job time is the slowest rank's, the whole-job rate
counts every rank's bytes, and the reference arm runs on rank 0 only."""
import io
import json
import os
import socket
import sys
import tempfile
import types
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(10.0 + 5.0 * rank)          # rank 1 is the slow one
    rate = bench.whole_job_rate(1e9, world, ms)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"ms": ms, "rate": rate}, f)


def test_two_gloo_ranks_take_the_slowest_time_and_count_all_bytes():
    import torch.multiprocessing as mp
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_rank_main, args=(2, _free_port(), d), nprocs=2, join=True)
        res = [json.load(open(os.path.join(d, f"r{r}.json"))) for r in range(2)]
    for r in res:
        assert r["ms"] == 15.0
        assert r["rate"] == pytest.approx(2 * 1e9 / 15e-3 / 1e9)


def test_single_process_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_rate(4.096e9, 1, 2.0) == pytest.approx(2048.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import bench
    args = types.SimpleNamespace(ref_rows=2000, warmup=1, steps=1, gpus=2, prec="bf16")
    calls = []
    monkeypatch.setattr(bench, "oracle_sample", lambda n: (calls.append(n), (n * 256 * 4, 0.01))[1])
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args)
    assert buf.getvalue() == "" and calls == []             # no work on rank 1
    monkeypatch.setenv("RANK", "0")
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args)
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
