"""Multi-process host logic of bench.py on CPU (world_size 2, gloo over 127.0.0.1): the
barrier and max-over-ranks timing reduction, the sharding of independent units across
ranks, and the reference arm printing only on rank 0."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    import bench
    bench._barrier(world)
    out[rank] = {
        "max": bench._max_over_ranks(world, 10.0 * (rank + 1)),
        "shard": bench.shard(range(7), rank, world),
    }
    bench._barrier(world)
    dist.destroy_process_group()


def test_gloo_two_ranks_reduce_and_shard():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert out[0]["max"] == out[1]["max"] == 20.0
    assert out[0]["shard"] == [0, 2, 4, 6] and out[1]["shard"] == [1, 3, 5]
    assert sorted(out[0]["shard"] + out[1]["shard"]) == list(range(7))


def test_reference_arm_prints_on_rank_zero_only(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = type("A", (), {"steps": 1, "warmup": 0, "gpus": 2, "ref_sample_steps": 1})()
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args)
    assert buf.getvalue() == ""
