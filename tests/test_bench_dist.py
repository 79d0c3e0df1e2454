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


def test_reference_arm_rank0_line(monkeypatch, capsys):
    """Rank 0 times the oracle for warmup + steps bounded samples and prints one line whose value is
    the timed steps' RR sets over their seconds, with the reference arm's keys."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2009_07325_gb300 import inputs as I
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    g = I.wc_weights(I.er(2000, 20000, 1))
    monkeypatch.setattr(bench, "load_workload", lambda: g)
    monkeypatch.setattr(bench, "WORKLOAD", dict(bench.WORKLOAD, k=10))
    seen = []
    real = bench.cpu_baseline

    def spy(graph, budget_s):
        r = real(graph, budget_s=budget_s)
        seen.append(r)
        return r

    monkeypatch.setattr(bench, "cpu_baseline", spy)
    ns = type("A", (), dict(warmup=1, steps=2, ref_budget=0.05))()
    assert bench.run_reference(ns) == 0
    out = capsys.readouterr().out.strip().splitlines()
    assert len(out) == 1
    line = json.loads(out[0])
    assert len(seen) == 3
    timed = seen[1:]
    want = sum(r["rr_sets"] for r in timed) / sum(r["seconds"] for r in timed)
    assert line["impl"] == "reference" and line["value"] == pytest.approx(want)
    assert line["steps"] == 2 and line["warmup"] == 1 and line["n_gpus"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "RR-sets/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["ms_per_step"] == pytest.approx(1e3 * sum(r["seconds"] for r in timed) / 2)
