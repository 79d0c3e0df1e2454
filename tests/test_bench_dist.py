"""The multi-process side of bench.py on CPU: two gloo ranks on 127.0.0.1.

The benchmark runs one independent IMM replica per GPU (the method's RR
sampling would shard by rr_id, but one GPU per machine leaves replicas only).
Whole-job throughput is the units summed over ranks divided by the slowest
rank's seconds; these tests check that reduction, the barrier, and that only
rank 0 prints a line, without a GPU.
"""
import json
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        # rank r did 100*(r+1) units in (r+1) seconds
        units, secs = bench.aggregate(100.0 * (rank + 1), float(rank + 1))
        bench.barrier()
        e2e_units, e2e_secs = bench.aggregate(7.0, 0.5 + rank)
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"units": units, "secs": secs, "e2e_units": e2e_units, "e2e_secs": e2e_secs,
                       "env": list(bench.dist_env())}, f)
    finally:
        dist.destroy_process_group()


def test_aggregate_two_gloo_ranks(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r, x in enumerate(res):
        assert x["units"] == 300.0            # sum over ranks
        assert x["secs"] == 2.0               # the slowest rank
        assert x["e2e_units"] == 14.0
        assert x["e2e_secs"] == 1.5
        assert x["env"] == [r, world, r]


def test_aggregate_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(12.0, 3.5) == (12.0, 3.5)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    """Under torchrun only rank 0 times the oracle; the others return 0 at once."""
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    called = []
    monkeypatch.setattr(bench, "load_workload", lambda: called.append(1))
    ns = type("A", (), dict(warmup=3, steps=2, ref_budget=0.1))()
    assert bench.run_reference(ns) == 0
    assert called == []
    assert capsys.readouterr().out == ""
