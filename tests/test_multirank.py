"""Multi-process host logic of bench.py on CPU (world_size 2, gloo over 127.0.0.1): the
barrier and max-over-ranks timing reduction, the router that shards independent units
(the 512 ensembles of the batched workload, the requests of the serving stream) across
ranks so that each runs exactly once, the aggregation of the ranks' records on rank 0,
and the reference arm printing only on rank 0."""
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
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert out[0]["max"] == out[1]["max"] == 20.0
    assert out[0]["shard"] == [0, 2, 4, 6] and out[1]["shard"] == [1, 3, 5]
    assert sorted(out[0]["shard"] + out[1]["shard"]) == list(range(7))


def _serve_record(rank, n):
    # a rank's serving record as serve_measurement builds it (latencies in s)
    lat = [0.01 * (rank + 1) * (k + 1) for k in range(n)]
    return {"lat": lat, "wall": 2.0 + rank, "lat07": [l / 2 for l in lat], "wall07": 3.0 + rank,
            "arr07": [0.1 * k for k in range(n)], "lat64": [0.5] + [None] * (n - 1), "wall64": 4.0,
            "arrivals": [0.01 * k for k in range(n)], "pairs": 1000 * (rank + 1), "ion_steps": 100 * (rank + 1),
            "errs": [{"request": rank, "n": 8, "force_rel_rms_vs_oracle": 1e-7}], "redraws": rank, "n": n,
            "ns": [(100, 1000, 5000)[k % 3] for k in range(n)]}


def _router_worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    import bench
    units = bench._gather(world, {"ensembles": bench.shard(range(512), rank, world),
                                  "requests": bench.shard(range(100), rank, world)})
    b = bench._gather(world, {"ensembles": len(units[rank]["ensembles"]), "ions": 10 * (rank + 1),
                              "pairs": 90 * (rank + 1), "ms": 5.0 + rank, "steps": 2000,
                              "errs": [1e-7 * (rank + 1)], "redraws": rank, "tuned": {}})
    sv = bench._gather(world, _serve_record(rank, len(units[rank]["requests"])))
    out[rank] = {"units": units, "batched": bench.aggregate_batched(b),
                 "serve": bench.aggregate_serve(sv, {"requests": 100, "step_scale": 20.0, "mem_budget_bytes": 1 << 30,
                                                     "full_stream_requests": 20000,
                                                     "full_stream_offered_pairs_per_s": 1e15, "arrival_span_s": 0.5,
                                                     "fp64_cap_s": 30.0})}
    dist.destroy_process_group()


def test_gloo_two_ranks_route_ensembles_and_requests():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_router_worker, args=(world, port, out), nprocs=world, join=True)
    units = out[0]["units"]
    assert units == out[1]["units"]
    for kind, count in (("ensembles", 512), ("requests", 100)):
        got = [u for r in range(world) for u in units[r][kind]]
        assert sorted(got) == list(range(count)), kind  # every unit on exactly one rank
        assert abs(len(units[0][kind]) - len(units[1][kind])) <= 1
    b = out[0]["batched"]
    assert b["ensembles"] == 512 and b["ions"] == 30 and b["ranks"] == 2
    assert b["ms"] == 6.0  # the slowest rank's time
    assert b["ion_steps_per_s"] == 30 * 2000 / 6e-3
    assert b["force_rel_rms_vs_oracle_max"] == 2e-7 and b["unstable_trap_redraws"] == 1
    sv = out[0]["serve"]
    assert sv["requests_per_rank"] == [50, 50] and sv["unstable_trap_redraws"] == 1
    prim = sv["at_generated_arrivals"]
    assert prim["wall_s"] == 3.0 and prim["pair_interactions_per_s"] == 3000 / 3.0
    lat = sorted([0.01 * (r + 1) * (k + 1) for r in range(2) for k in range(50)])
    assert abs(prim["p50_ms"] - 1e3 * (lat[49] + lat[50]) / 2) < 1e-9
    by = prim["by_size"]
    assert [by[k]["requests"] for k in ("n_le_256", "n_257_2048", "n_gt_2048")] == [34, 34, 32]
    small = sorted(0.01 * (r + 1) * (k + 1) for r in range(2) for k in range(0, 50, 3))
    assert abs(by["n_le_256"]["p50_ms"] - 1e3 * (small[16] + small[17]) / 2) < 1e-9
    assert sv["at_0.7_capacity"]["by_size"]["n_gt_2048"]["requests"] == 32
    fifo = sv["fp64_fifo_same_requests"]
    assert fifo["served"] == 2 and fifo["not_served"] == 98 and fifo["percentiles_are_lower_bounds"]
    assert len(sv["per_result_error"]) == 2


def test_reference_arm_prints_on_rank_zero_only(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = type("A", (), {"steps": 1, "warmup": 0, "gpus": 2, "ref_sample_steps": 1})()
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args)
    assert buf.getvalue() == ""
