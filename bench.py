"""Benchmark: IMM end to end on R-MAT scale 22, IC weighted cascade, k=50, eps=0.1.

One step is one full IMM run through the C ABI (lower-bound search with its
RR sampling and greedy rounds, then sampling up to theta and the final
greedy) on a graph resident in HBM. The JSON line reports RR sets per second
(value), the IMM seconds per run (ms_per_step), an end-to-end figure through
host buffers (graph upload from pinned memory + IMM + seed readback), the
roofline position of the dominant kernel (the RR-sampling kernel) against the
measured HBM copy bandwidth, and the CPU oracle timed on a bounded sample of
the same workload on this machine's host cores.

Multi-GPU (torchrun, one process per GPU): each rank runs its own
independent IMM replica (replicas only); value = RR sets over all ranks / the
slowest rank's time.

--impl reference times the CPU oracle (the only reference implementation this
method has here) on a bounded sample per step.
"""
from __future__ import annotations

import argparse
import hashlib
import gc
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "IMM end-to-end s & RR-sets/s (IC, R-MAT-22, k=50, ε=0.1); % HBM peak"
_RMAT = "R-MAT scale {s} (16*2^{s} draws, a,b,c,d=.57/.19/.19/.05, dedup, seed {seed})"
WORKLOADS = {
    # the headline: IC weighted cascade on the R-MAT scale-22 graph
    "imm-ic-wc-rmat22": dict(graph=_RMAT.format(s=22, seed=3), weights="weighted cascade 1/indeg(v) fp32",
                             model="IC", k=50, eps=0.1, ell=1.0, philox_seed=7),
    # the same graph under LT (in-weights 1/indeg(v)), k=100, eps=0.05
    "imm-lt-wc-rmat22": dict(graph=_RMAT.format(s=22, seed=3), weights="LT 1/indeg(v) fp32",
                             model="LT", k=100, eps=0.05, ell=1.0, philox_seed=7),
    # R-MAT scale 20, IC weighted cascade, k=50, eps=0.1
    "imm-ic-wc-rmat20": dict(graph=_RMAT.format(s=20, seed=2), weights="weighted cascade 1/indeg(v) fp32",
                             model="IC", k=50, eps=0.1, ell=1.0, philox_seed=7),
    # the same graph under IC with uniform p = 0.01 (supercritical: ~5% of the RR sets reach a
    # giant component of ~205K vertices), k = 100. eps = 0.2: at eps = 0.05 the collection
    # (theta ~1.4e7 sets, ~9.5K members each) would need ~540 GB, beyond the GPU's memory
    "imm-ic-p001-rmat22": dict(graph=_RMAT.format(s=22, seed=3), weights="uniform p=0.01 fp32",
                               model="IC", k=100, eps=0.2, ell=1.0, philox_seed=7),
    # the stated eps = 0.05 on that graph: compact collection (the sets drawn after the first
    # selection that hold its first pick keep only their size; all giant sets hold it)
    "imm-ic-p001-rmat22-eps005-compact": dict(graph=_RMAT.format(s=22, seed=3), weights="uniform p=0.01 fp32",
                                              model="IC", k=100, eps=0.05, ell=1.0, philox_seed=7, compact=True),
    # directed Erdos-Renyi n=2000, m=20000, IC weighted cascade, k=10, eps=0.5
    "imm-ic-wc-er2000": dict(graph="directed Erdos-Renyi n=2000 m=20000 seed 1",
                             weights="weighted cascade 1/indeg(v) fp32", model="IC", k=10, eps=0.5, ell=1.0,
                             philox_seed=7),
    # the headline with IMM's final phase on theta fresh RR sets (rr_ids 2^63 + j)
    "imm-ic-wc-rmat22-fresh": dict(graph=_RMAT.format(s=22, seed=3), weights="weighted cascade 1/indeg(v) fp32",
                                   model="IC", k=50, eps=0.1, ell=1.0, philox_seed=7, fresh_final=True),
}
# multi-round IM (Sec. IV-H, CR-NAIMM) with the paper's T = 5 rounds, k = 10 per round, eps = 0.1
WORKLOADS["mrim-ic-wc-rmat22-T5"] = dict(graph=_RMAT.format(s=22, seed=3), weights="weighted cascade 1/indeg(v) fp32",
                                         model="IC", k=10, eps=0.1, ell=1.0, philox_seed=7, rounds=5)
# Barabasi-Albert density sweep (Sec. IV-F): n = 10^6, r = 2 .. 32 undirected edges per new vertex
# (both directions stored), clique of r0 = r vertices, IC weighted cascade, k = 50, eps = 0.05
for _r in (2, 4, 8, 16, 32):
    WORKLOADS[f"imm-ic-wc-ba1m-r{_r}"] = dict(
        graph=f"Barabasi-Albert n=10^6 r={_r} (clique r0={_r}, degree-proportional attachment, seed 6)",
        weights="weighted cascade 1/indeg(v) fp32", model="IC", k=50, eps=0.05, ell=1.0, philox_seed=7)
WORKLOADS["batch-chunglu-256"] = dict(
    graph="256 Chung-Lu graphs (degree exponent 2.1, 8n draws, dedup), n = round(10^(4+2U)), graph seed 1000+i",
    weights="weighted cascade 1/indeg(v) fp32", model="IC", k="from {10,25,50}", eps="from {0.1,0.2,0.5}", ell=1.0,
    philox_seed="1000+i", instances=256)
WORKLOAD = dict(workload="imm-ic-wc-rmat22", **WORKLOADS["imm-ic-wc-rmat22"])


def batch_instances(count=256):
    """The batched workload: per instance (graph, (model, k, eps, ell, seed))."""
    from paper_2009_07325_gb300 import GIM_IC
    from paper_2009_07325_gb300 import inputs as I
    r = I.u64_stream(4, 900, 3 * count)
    out = []
    for i in range(count):
        u = float(r[3 * i] >> np.uint64(11)) * 2.0 ** -53
        n = int(round(10 ** (4 + 2 * u)))
        k = (10, 25, 50)[int(r[3 * i + 1] % np.uint64(3))]
        eps = (0.1, 0.2, 0.5)[int(r[3 * i + 2] % np.uint64(3))]
        out.append((n, (GIM_IC, k, eps, 1.0, 1000 + i)))
    return out


WORKLOADS["serve-rmat24"] = dict(
    graph=_RMAT.format(s=24, seed=4), weights="weighted cascade 1/indeg(v) fp32 (also the LT weights)",
    model="IC or LT 50/50", k="uniform in [10,200]", eps="log-uniform in [0.05,0.5]", ell=1.0, philox_seed=7,
    arrivals="Poisson, 50 queries/s", queries=60)


def serve_trace(count, rate=50.0, seed=5, distinct=False):
    """Arrival times (s) and query parameters of the serving workload. Every
    query draws its RR sets with the workload's Philox seed, so queries of one
    model share them; distinct=True gives query i the Philox seed 2000 + i
    instead, so no two queries share an RR set."""
    from paper_2009_07325_gb300 import GIM_IC, GIM_LT
    from paper_2009_07325_gb300 import inputs as I
    r = I.u64_stream(seed, 950, 4 * count)
    u = (r >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    t, out = 0.0, []
    for i in range(count):
        t += -np.log(max(1.0 - u[4 * i], 1e-300)) / rate
        k = 10 + int(u[4 * i + 1] * 191)
        eps = float(0.05 * 10.0 ** u[4 * i + 2])
        model = GIM_IC if u[4 * i + 3] < 0.5 else GIM_LT
        out.append((t, (model, k, eps, 1.0, 2000 + i if distinct else WORKLOAD["philox_seed"])))
    return out


SERVE_SLOTS = 8    # queries the server advances together


def run_serve(args):
    """Serving: the arrival trace against the query server (continuous
    batching, resident RR pools) and against one gim_imm at a time (FIFO)."""
    import threading
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2009_07325_gb300 import Context, binding
    from paper_2009_07325_gb300 import inputs as I
    t0 = time.perf_counter()
    g = I.wc_weights(I.rmat(24, 4))
    t_gen = time.perf_counter() - t0
    ctx = Context(local)
    ctx.load(g)
    trace = serve_trace(WORKLOAD["queries"])
    warm = serve_trace(20, seed=6)                 # earlier traffic: a disjoint trace of the same mix

    def served(srv, tr):
        done = {}
        tickets = []
        start = time.perf_counter()
        for arr, p in tr:
            d = start + arr - time.perf_counter()
            if d > 0:
                time.sleep(d)
            tickets.append((srv.submit(*p), arr))
        for tk, arr in tickets:
            done[tk] = srv.wait(tk, 1800)
        lat = [done[tk]["latency_ms"] for tk, _ in tickets]
        finish = max(arr * 1e3 + done[tk]["latency_ms"] for tk, arr in tickets)
        return [done[tk] for tk, _ in tickets], lat, finish / 1e3

    def plain(tr):
        start = time.perf_counter()
        res, lat = [], []
        for arr, p in tr:
            d = start + arr - time.perf_counter()
            if d > 0:
                time.sleep(d)
            r = ctx.imm(*p)
            now = time.perf_counter() - start
            res.append(r)
            lat.append((now - arr) * 1e3)
        return res, lat, time.perf_counter() - start

    # steady state: a server whose resident pools hold the RR sets of earlier, different queries
    srv = binding.Server(ctx, max_active=SERVE_SLOTS, max_k=200)
    served(srv, warm)
    with ClockSampler(local) as clk:
        s_res, s_lat, s_span = served(srv, trace)
    st = srv.stats()
    srv.stop()
    # cold start: a fresh server, empty pools
    srv = binding.Server(ctx, max_active=SERVE_SLOTS, max_k=200)
    c_res, c_lat, c_span = served(srv, trace)
    srv.stop()
    plain(warm[:2])
    p_res, p_lat, p_span = plain(trace)
    same_res = lambda xs, ys: all(a["seeds"].tolist() == b["seeds"].tolist() and a["theta"] == b["theta"]
                                  for a, b in zip(xs, ys))
    same = same_res(s_res, p_res)
    same_c = same_res(c_res, p_res)
    # distinct Philox seeds: no query shares an RR set with another, so the
    # served speed-up is the overlap of continuous batching alone; against
    # one query at a time through gim_imm and through a one-slot server
    dtrace = serve_trace(WORKLOAD["queries"], distinct=True)
    srv = binding.Server(ctx, max_active=SERVE_SLOTS, max_k=200)
    with ClockSampler(local) as dclk:
        d_res, d_lat, d_span = served(srv, dtrace)
    d_st = srv.stats()
    srv.stop()
    srv = binding.Server(ctx, max_active=1, max_k=200)
    o_res, o_lat, o_span = served(srv, dtrace)
    srv.stop()
    dp_res, dp_lat, dp_span = plain(dtrace)
    same_d = same_res(d_res, dp_res) and same_res(o_res, dp_res)
    q = len(trace)
    pct = lambda x, p: float(np.percentile(np.array(x), p))
    line = {"metric": "served IMM queries/s with p50/p99 latency (R-MAT-24, Poisson 50 q/s, IC/LT mix)",
            "value": q / s_span, "unit": "queries/s", "n_gpus": 1, "steps": q, "warmup": len(warm),
            "ms_per_step": 1e3 * s_span / q, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic", "config": dict(WORKLOAD),
            "served": {"queries_per_s": q / s_span, "p50_ms": pct(s_lat, 50), "p99_ms": pct(s_lat, 99),
                       "makespan_s": s_span,
                       "pools": f"resident from {len(warm)} earlier queries of a disjoint trace (seed 6)",
                       "rounds": st["rounds"], "peak_active": st["peak_active"], "sample_ms": st["sample_ms"],
                       "select_ms": st["select_ms"], "pool_sets": st["pool_sets"]},
            "served_cold": {"queries_per_s": q / c_span, "p50_ms": pct(c_lat, 50), "p99_ms": pct(c_lat, 99),
                            "makespan_s": c_span, "pools": "empty at start (fresh server)",
                            "throughput_vs_plain": (q / c_span) / (q / p_span)},
            "plain_one_at_a_time": {"queries_per_s": q / p_span, "p50_ms": pct(p_lat, 50), "p99_ms": pct(p_lat, 99),
                                    "makespan_s": p_span},
            "throughput_vs_plain": (q / s_span) / (q / p_span),
            "shared_seed_note": "every query above uses Philox seed 7, so queries of one model share RR sets "
                                "(resident pools); distinct_seeds below shares none",
            "distinct_seeds": {
                "philox_seeds": "2000 + query index", "queries": len(dtrace),
                "served": {"queries_per_s": q / d_span, "p50_ms": pct(d_lat, 50), "p99_ms": pct(d_lat, 99),
                           "makespan_s": d_span, "pools": "empty at start (fresh server)",
                           "rounds": d_st["rounds"], "peak_active": d_st["peak_active"],
                           "sample_ms": d_st["sample_ms"], "select_ms": d_st["select_ms"]},
                "one_slot_server": {"queries_per_s": q / o_span, "p50_ms": pct(o_lat, 50),
                                    "p99_ms": pct(o_lat, 99), "makespan_s": o_span},
                "plain_one_at_a_time": {"queries_per_s": q / dp_span, "p50_ms": pct(dp_lat, 50),
                                        "p99_ms": pct(dp_lat, 99), "makespan_s": dp_span},
                "throughput_vs_plain": (q / d_span) / (q / dp_span),
                "throughput_vs_one_slot": (q / d_span) / (q / o_span),
                "identical_seed_sets": bool(same_d), "clocks": dclk.summary()},
            "identical_seed_sets": bool(same and same_c), "graph_generation_s": t_gen, "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def batch_measure(local, steps, warmup, count=256):
    """Batched IMM (gim_batch_imm over the instances of the batch workload)
    against the same instances run one after another with gim_imm, graphs
    resident: batch seconds (median of `steps` timed batches), plain seconds,
    identical seed sets, and the split of the time."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2009_07325_gb300 import Context, binding
    from paper_2009_07325_gb300 import inputs as I
    specs = batch_instances(count)
    t0 = time.perf_counter()
    graphs = [I.wc_weights(I.chung_lu(n, 1000 + i)) for i, (n, _) in enumerate(specs)]
    t_gen = time.perf_counter() - t0
    stream = torch.cuda.Stream(device=local)
    ctxs = []
    for g in graphs:
        c = Context(local, stream=stream.cuda_stream)
        c.load(g)
        ctxs.append(c)
    del graphs
    params = [p for _, p in specs]
    batch_budget, _ = binding.autotune(ctxs, params, 2000)        # schedule for the batch as a whole
    batch_schedule = ctxs[0].schedule()
    for _ in range(max(1, warmup)):
        res = binding.batch_imm(ctxs, params)
    ctxs[0].reset_timings()
    launches0 = ctxs[0].launch_count()
    torch.cuda.synchronize()
    bt = []
    with ClockSampler(local) as clk:
        for _ in range(steps):
            t1 = time.perf_counter()
            res = binding.batch_imm(ctxs, params)
            torch.cuda.synchronize()
            bt.append(time.perf_counter() - t1)
    launches = ctxs[0].launch_count() - launches0
    tb = ctxs[0].timings()                        # host-side phase split of the last batch
    batched_seeds = [r["seeds"].tolist() for r in res]
    # the plain path: one gim_imm per instance, back to back, each instance
    # with the schedule the autotuner picks for it alone (one warm-up pass)
    plain_schedules = []
    for c, p in zip(ctxs, params):
        binding.autotune([c], [p], 2000)
        plain_schedules.append(c.schedule())
    plain_budgets = [x["group_budget"] for x in plain_schedules]
    for c, p in zip(ctxs, params):
        c.imm(*p)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for c in ctxs:
        c.reset_timings()
    plain, p_sample, p_select = [], 0.0, 0.0
    for c, p in zip(ctxs, params):
        plain.append(c.imm(*p))
        tp = c.timings()
        p_sample += tp["sample_ms"]
        p_select += tp["select_ms"]
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t1
    same = all(a == b["seeds"].tolist() and r["theta"] == b["theta"]
               for a, r, b in zip(batched_seeds, res, plain))
    t_b = float(np.median(bt))
    out = {"instances": len(ctxs), "batched_s": t_b, "batch_times_s": bt, "plain_sequential_s": t_plain,
           "speedup_vs_plain": t_plain / t_b, "instances_per_s": len(ctxs) / t_b,
           "plain_instances_per_s": len(ctxs) / t_plain, "identical_seed_sets": same,
           "rr_sets": sum(r["rr_count"] for r in res),
           "batched_split_ms": {"sample": tb["sample_ms"], "select": tb["select_ms"], "wall": tb["wall_ms"]},
           "plain_split_ms": {"sample": p_sample, "select": p_select,
                              "common_kernel": sum(c.timings()["kernel_ms"] for c in ctxs),
                              "large_kernel": sum(c.timings()["large_ms"] for c in ctxs)},
           "batched_kernel_ms_per_batch": {"common": tb["kernel_ms"] / max(1, steps),
                                           "large": tb["large_ms"] / max(1, steps)},
           "rounds": max(r["lb_rounds"] for r in res) + 1,
           "tuning": {"batch_group_budget": batch_budget, "batch_schedule": batch_schedule,
                      "plain_group_budgets": sorted(set(plain_budgets)),
                      "plain_schedules": sorted({tuple(sorted(x.items())) for x in plain_schedules}),
                      "by": "gim_autotune"},
           "gpu_launches": launches, "graph_generation_s": t_gen, "clocks": clk.summary()}
    for c in ctxs:
        c.close()
    return out


def run_batch(args):
    """The batched workload on its own line (see batch_measure)."""
    rank, world, local = dist_env()
    import torch
    torch.cuda.set_device(local)
    b = batch_measure(local, args.steps, args.warmup, WORKLOAD["instances"])
    units, secs = aggregate(float(b["instances"]) * args.steps, sum(b["batch_times_s"]))
    line = {"metric": "batched IMM queries/s (256 Chung-Lu instances, IC-WC)", "value": units / secs,
            "unit": "IMM-instances/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic", "config": dict(WORKLOAD), **b}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


L2_FLUSH_BYTES = 512 << 20


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def aggregate(units: float, seconds: float):
    """Whole-job totals over ranks: sum of units, max of seconds."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return units, seconds
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    u = torch.tensor([units], dtype=torch.float64, device=dev)
    s = torch.tensor([seconds], dtype=torch.float64, device=dev)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(s, op=dist.ReduceOp.MAX)
    return float(u.item()), float(s.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def traffic_record(kernel: str):
    """DRAM bytes per unit from the committed ncu summary, if the kernel source is unchanged
    (the key hashes sample.cu followed by gim_internal.cuh, which holds the launch shapes)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    csrc = os.path.join(ROOT, "paper_2009_07325_gb300", "csrc")
    if not os.path.exists(path):
        return None
    blob = b"".join(open(os.path.join(csrc, f), "rb").read() for f in ("sample.cu", "gim_internal.cuh"))
    h = hashlib.sha256(blob).hexdigest()[:16]
    for line in open(path):
        parts = line.split()
        if len(parts) >= 4 and parts[0] == kernel and parts[1] == h:
            return float(parts[2]), parts[3]          # bytes per unit, unit name
    return None


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


_GRAPH_CACHE = {}


def load_workload():
    from paper_2009_07325_gb300 import inputs as I
    name = WORKLOAD["workload"]
    key = WORKLOAD["graph"] + WORKLOAD["weights"]
    if key in _GRAPH_CACHE:
        return _GRAPH_CACHE[key]
    if name.startswith("imm-ic-p001-rmat22"):
        g = I.uniform_weights(I.rmat(22, 3), 0.01)
    elif "-ba1m-r" in name:
        g = I.wc_weights(I.barabasi_albert(10 ** 6, int(name.rsplit("-r", 1)[1]), 6))
    elif "rmat22" in name:
        g = I.wc_weights(I.rmat(22, 3))
    elif name.endswith("rmat20"):
        g = I.wc_weights(I.rmat(20, 2))
    else:
        g = I.wc_weights(I.er(2000, 20000, 1))
    _GRAPH_CACHE.clear()
    _GRAPH_CACHE[key] = g
    return g


def model_id():
    from paper_2009_07325_gb300 import GIM_IC, GIM_LT
    return GIM_LT if WORKLOAD["model"] == "LT" else GIM_IC


def coin_count(cnt: np.ndarray, indeg: np.ndarray) -> float:
    """IC sampling work: one coin per in-edge of every expanded vertex, i.e.
    sum over RR-set members v of indeg(v) (four coins per Philox call)."""
    return float(np.dot(cnt.astype(np.float64), indeg.astype(np.float64)))


def philox_calls(cnt: np.ndarray, indeg: np.ndarray, row_p: np.ndarray) -> float:
    """IC sampling ALU work in Philox4x32-10 calls: a row with probability
    p > 2^-8 costs one call per 4 in-edges; a row with p <= 2^-8 one call per
    16 in-edges for the top bytes plus, on average, one per 256 in-edges for
    the residuals of the edges whose byte is zero."""
    d = indeg.astype(np.float64)
    per = np.where(row_p <= 2.0 ** -8, d / 16.0 + d / 256.0, d / 4.0)
    return float(np.dot(cnt.astype(np.float64), per))


def row_probability(g) -> np.ndarray:
    """The in-edge probability of each row (rows of these workloads share one; 1 for empty rows)."""
    d = g.indegree()
    p = np.ones(g.n, np.float64)
    nz = d > 0
    p[nz] = g.weights[g.offsets[:-1][nz].astype(np.int64)].astype(np.float64)
    return p


def algorithmic_bytes(cnt: np.ndarray, indeg: np.ndarray) -> float:
    """IC sampling memory per member v on a row with a common threshold:
    8 B offsets + 4 B row threshold + 4 B store write + 4 B count update
    (sources of live edges, about one per row under weighted cascade, add 4 B)."""
    return float(cnt.astype(np.float64).sum() * 24.0)


def issue_slots(calls, kern_s, inst_per_call, sms, sm_mhz):
    """Issue-slot view of the IC sampler: warp instructions issued per second
    (the Philox calls of the timed runs times the warp instructions per call
    that one ncu capture of both sampling kernels counted) against the SMs'
    issue rate, one warp instruction per cycle in each of 4 schedulers."""
    if not (kern_s > 0 and inst_per_call and sms and sm_mhz):
        return None
    achieved = calls * inst_per_call / kern_s / 1e9          # G warp instructions / s
    peak = sms * 4 * sm_mhz * 1e6 / 1e9
    return {"achieved": achieved, "peak": peak, "unit": "G warp-instructions/s", "frac": achieved / peak,
            "warp_instructions_per_philox_call": inst_per_call, "sms": sms, "sm_mhz": sm_mhz,
            "peak_kind": "4 issue slots per SM per cycle at the sampled SM clock"}


def roofline(kname, coins, calls, alg_bytes, members, kern_s, n_launch, philox_calls_per_s, hbm_peak, peak_kind,
             traffic, large_launches, issue=None):
    """Roofline position of the dominant sampling kernel.

    IC (weighted cascade): the in-edge scans read no edge data; the work is
    the Philox calls that decide the coins of every expanded vertex's
    in-edges (philox_calls), so the bound is the integer ALU and the peak is
    the measured pure-Philox call rate.
    LT: a chain of dependent loads per walk step; reported against HBM with
    36 algorithmic bytes per member (8 B offsets, 16 B bracketing thresholds,
    4 B source, 4 B store write, 4 B count)."""
    base = {"kernel": kname, "traffic": traffic, "avg_launch_ms": 1e3 * kern_s / n_launch, "launches": n_launch,
            "large_pass_launches": large_launches}
    if kname == "sample_lt_kernel":
        achieved = 36.0 * members / kern_s / 1e9 if kern_s > 0 else 0.0
        base.update(bound="hbm", achieved=achieved, peak=hbm_peak, unit="GB/s", frac=achieved / hbm_peak,
                    peak_kind=peak_kind, algorithmic_bytes_per_launch=36.0 * members / n_launch)
        return base
    achieved = calls / kern_s / 1e9 if kern_s > 0 else 0.0          # G Philox calls / s
    peak = philox_calls_per_s / 1e9                                  # G calls / s, measured
    base.update(bound="alu", achieved=achieved, peak=peak, unit="G Philox calls/s", frac=achieved / peak,
                peak_kind="measured: pure Philox4x32-10 kernel on this GPU",
                calls_per_launch=calls / n_launch, coins_per_launch=coins / n_launch,
                gcoins_per_s=coins / kern_s / 1e9 if kern_s > 0 else 0.0,
                hbm_view={"algorithmic_gbs": alg_bytes / kern_s / 1e9 if kern_s > 0 else 0.0, "peak_gbs": hbm_peak,
                          "peak_kind": peak_kind})
    if issue is not None:
        base["issue_slots"] = issue
    return base


def select_roofline(sel: dict, hbm_peak: float, peak_kind: str):
    """Greedy selection (index build + k rounds) against HBM: its algorithmic bytes
    (counted by the library per selection) over the device time of its kernels."""
    secs = sel["kernel_ms"] / 1e3
    if secs <= 0 or sel["calls"] == 0:
        return None
    gbs = sel["bytes"] / secs / 1e9
    return {"kernels": "bsel_* + greedy_kernel", "bound": "hbm", "achieved": gbs, "peak": hbm_peak,
            "unit": "GB/s", "frac": gbs / hbm_peak, "peak_kind": peak_kind,
            "ms_per_selection": sel["kernel_ms"] / sel["calls"], "selections": sel["calls"],
            "bytes_per_selection": sel["bytes"] / sel["calls"], "traffic": None}


def _oracle_sample(O, graph, threads: int, budget_s: float):
    """RR sets of the workload drawn by the oracle for about budget_s seconds, then the greedy over them."""
    o = O.Oracle(graph)
    T = WORKLOAD.get("rounds", 0)
    if T:
        o.set_rounds(T)
    t0 = time.perf_counter()
    chunk = (4000 if not T else 500) if threads > 1 else (500 if not T else 100)
    while time.perf_counter() - t0 < budget_s:
        o.sample(O.LT if WORKLOAD["model"] == "LT" else O.IC, WORKLOAD["philox_seed"], chunk, threads)
    o.greedy(WORKLOAD["k"])
    dt = time.perf_counter() - t0
    n = o.rr_count
    kind = f"{T}-round {WORKLOAD['model']}" if T else WORKLOAD["model"]
    return n, dt, (f"{n} {kind} RR sets of the workload (rr_ids 0..{n - 1}) + greedy k={WORKLOAD['k']} over them; "
                   f"{dt:.1f} s")


def cpu_baseline(graph, budget_s: float = 12.0, single_core_s: float = 0.0):
    """The oracle, as it stands, on a bounded sample of the workload on all host cores; with
    single_core_s > 0 also on one core (the experiment setup of Sec. V runs sequential IMM on one core)."""
    import oracle as O
    O.build()
    th = max(1, O.max_threads())
    n, dt, sample = _oracle_sample(O, graph, th, budget_s)
    r = {"value": n / dt, "unit": "RR-sets/s", "cores": th, "kind": "oracle", "sample": sample,
         "rr_sets": n, "seconds": dt}
    if single_core_s > 0:
        n1, dt1, sample1 = _oracle_sample(O, graph, 1, single_core_s)
        r["single_core"] = {"value": n1 / dt1, "unit": "RR-sets/s", "cores": 1, "sample": sample1}
    return r


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    g = load_workload()
    steps = []
    for i in range(args.warmup + args.steps):
        r = cpu_baseline(g, budget_s=args.ref_budget)
        if i >= args.warmup:
            steps.append(r)
    units = float(sum(r["rr_sets"] for r in steps))
    secs = sum(r["seconds"] for r in steps)
    value = units / secs
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "RR-sets/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": dict(WORKLOAD, l2="n/a (CPU)"),
            "cpu_baseline": {"value": value, "unit": "RR-sets/s", "cores": steps[0]["cores"], "kind": "oracle",
                             "sample": steps[0]["sample"]},
            "e2e": {"value": value, "unit": "RR-sets/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2009_07325_gb300 import GIM_IC, Context

    g = load_workload()
    indeg = g.indegree()
    row_p = row_probability(g)
    stream = torch.cuda.Stream(device=local)
    ctx = Context(local, stream=stream.cuda_stream)
    ctx.load(g)
    k, eps, ell, seed = WORKLOAD["k"], WORKLOAD["eps"], WORKLOAD["ell"], WORKLOAD["philox_seed"]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=f"cuda:{local}")

    mdl = model_id()
    from paper_2009_07325_gb300 import binding
    if WORKLOAD.get("fresh_final"):
        ctx.set_option(binding.GIM_OPT_FRESH_FINAL, 1)
    if WORKLOAD.get("compact"):
        ctx.set_option(binding.GIM_OPT_COMPACT_FIRST_PICK, 1)
    if args.group_budget:   # a fixed schedule (profiler runs: timings under a profiler mislead the tuner)
        ctx.set_option(binding.GIM_OPT_GROUP_BUDGET, args.group_budget)
        budget, tuned_by = args.group_budget, "--group-budget"
    else:
        budget, _ = binding.autotune([ctx], [(mdl, k, eps, ell, seed)], 20000)   # schedule for this profile
        tuned_by = "gim_autotune"
    ctx_schedule = ctx.schedule()
    T = WORKLOAD.get("rounds", 0)

    def run_once():
        return ctx.mrim(mdl, T, k, eps, ell, seed) if T else ctx.imm(mdl, k, eps, ell, seed)

    def vertex_counts():   # occurrences per vertex (a multi-round collection counts per (vertex, round))
        c = ctx.coverage()
        return c.reshape(T, -1).sum(axis=0) if T else c

    for _ in range(args.warmup):
        run_once()

    ctx.reset_timings()
    launches0 = ctx.launch_count()
    step_ms, rr_sets, alg_bytes, coins, sample_ms, select_ms, thetas = [], 0, 0.0, 0.0, 0.0, 0.0, []
    calls = 0.0
    members_total = 0
    barrier()
    torch.cuda.synchronize()
    gc.collect()
    gc.disable()   # no interpreter garbage-collection pauses inside the timed steps
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(1)                       # evict L2 between steps (not timed)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = run_once()
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            t = ctx.timings()
            sample_ms += t["sample_ms"]
            select_ms += t["select_ms"]
            rr_sets += r["rr_count"]
            thetas.append(r["theta"])
            members_total += ctx.rr_count()[1]
            cov = vertex_counts()
            alg_bytes += algorithmic_bytes(cov, indeg)
            coins += coin_count(cov, indeg)
            calls += philox_calls(cov, indeg, row_p)
    torch.cuda.synchronize()
    gc.enable()
    barrier()
    tk = ctx.timings()
    sel = ctx.selection_stats()
    launches = ctx.launch_count() - launches0
    philox_calls_per_s = ctx.philox_rate()       # measured ALU ceiling (after the timed region)
    local_s = sum(step_ms) / 1e3
    units, secs = aggregate(float(rr_sets), local_s)

    # end to end through host buffers: graph upload from pinned memory, IMM, seeds back
    pinned = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (g.offsets, g.sources, g.weights)]
    off_p, src_p, w_p = (t.numpy() for t in pinned)   # the tensors stay referenced: the memory stays pinned
    h2d = off_p.nbytes + src_p.nbytes + w_p.nbytes
    e2e_t, e2e_units = 0.0, 0
    for _ in range(2):   # untimed warm-up: the first two loads allocate both sets of graph arrays
        ctx.graph_load(g.n, off_p, src_p, w_p)
        run_once()
    e2e_load, e2e_run = [], []
    gc.collect()
    gc.disable()   # as timeit does: no interpreter garbage-collection pauses inside the timed iterations
    for _ in range(max(1, min(args.steps, 5))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.graph_load(g.n, off_p, src_p, w_p)
        t1 = time.perf_counter()
        r = run_once()
        t2 = time.perf_counter()
        e2e_t += t2 - t0
        e2e_load.append(1e3 * (t1 - t0))
        e2e_run.append(1e3 * (t2 - t1))
        e2e_units += r["rr_count"]
    gc.enable()
    e2e_u, e2e_s = aggregate(float(e2e_units), e2e_t)
    d2h = 4 * k * max(T, 1) + 8 + 8

    if rank == 0:
        hbm_peak, peak_kind = measured_peaks()
        kern_s = (tk["kernel_ms"] + tk["large_ms"]) / 1e3
        n_launch = max(tk["kernel_launches"] + tk["large_launches"], 1)
        kname = "sample_lt_kernel" if WORKLOAD["model"] == "LT" else "sample_ic_kernel"
        # the recorded DRAM bytes per RR set hold for the headline graph and weights only
        same_sets = WORKLOAD["workload"].startswith("imm-ic-wc-rmat22") and "sweep" not in WORKLOAD
        tr = traffic_record(kname) if same_sets else None
        traffic = None
        if tr is not None:
            per_unit, unit = tr
            traffic = per_unit * (rr_sets / n_launch) if unit == "rr_set" else None
        clocks = clk.summary()
        issue = None
        ir = traffic_record("sample_ic_issue") if kname == "sample_ic_kernel" else None
        if ir is not None and ir[1] == "warp_inst_per_philox_call" and clocks:
            sms = torch.cuda.get_device_properties(local).multi_processor_count
            issue = issue_slots(calls, kern_s, ir[0], sms, clocks["sm_mhz"])
        line = {
            "metric": METRIC, "value": units / secs, "unit": "RR-sets/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": dict(WORKLOAD, parallelism=f"replicas{world}", l2="flushed between steps (512 MiB write)"),
            "imm_s": secs / args.steps, "theta": thetas[-1], "rr_sets_per_step": rr_sets / args.steps,
            "tuning": dict(ctx_schedule, by=tuned_by),
            "sample_ms_per_step": sample_ms / args.steps, "select_ms_per_step": select_ms / args.steps,
            "e2e": {"value": e2e_u / e2e_s, "unit": "RR-sets/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "imm_s": e2e_s / max(1, min(args.steps, 5)),
                    "load_ms": e2e_load, "run_ms": e2e_run},
            "gpu_launches": launches,
            "roofline": roofline(kname, coins, calls, alg_bytes, members_total, kern_s, n_launch, philox_calls_per_s,
                                 hbm_peak, peak_kind, traffic, tk["large_launches"], issue),
            "select_roofline": select_roofline(sel, hbm_peak, peak_kind),
            "clocks": clocks,
        }
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(g, budget_s=args.cpu_budget, single_core_s=args.cpu_single_budget)
    ctx.close()
    if rank == 0:
        if world == 1 and not args.no_batch and WORKLOAD["workload"] == "imm-ic-wc-rmat22" \
                and "sweep" not in WORKLOAD:
            # the batched workload (256 Chung-Lu IMM instances in lockstep against
            # 256 sequential gim_imm runs), one timed batch after one warm-up
            line["batch"] = dict(workload="batch-chunglu-256", **batch_measure(local, 1, 1))
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_case(args):
    """Small single-call cases for profiling: one gim_sample_rr / gim_select_seeds on the workload graph."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2009_07325_gb300 import GIM_IC, GIM_LT, Context
    from paper_2009_07325_gb300 import inputs as I
    base = I.rmat(22, 3)
    g = I.uniform_weights(base, 0.01) if args.case == "sample-ic-p001" else I.wc_weights(base)
    model = GIM_LT if args.case == "sample-lt" else GIM_IC
    ctx = Context(0)
    from paper_2009_07325_gb300 import binding
    if args.large_bytes:
        ctx.set_option(binding.GIM_OPT_LARGE_PASS_BYTES, int(args.large_bytes))
    if args.group_budget:
        ctx.set_option(binding.GIM_OPT_GROUP_BUDGET, args.group_budget)
    ctx.load(g)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.sample_rr(model, args.count, WORKLOAD["philox_seed"])
    t_s = time.perf_counter() - t0
    out = {"case": args.case, "count": args.count, "sample_s": t_s, "timings": ctx.timings(),
           "members": ctx.rr_count()[1]}
    if model == GIM_IC:   # the Philox calls the sampled collection needed (see philox_calls)
        out["philox_calls"] = philox_calls(ctx.coverage(), g.indegree(), row_probability(g))
    if args.case == "select":
        t0 = time.perf_counter()
        s, gains, cov = ctx.select_seeds(WORKLOAD["k"])
        out.update(select_s=time.perf_counter() - t0, covered=cov, timings_select=ctx.timings())
    print(json.dumps(out), flush=True)
    ctx.close()
    return 0


SWEEPS = {
    # runtime against k and against eps on the headline graph (the shapes of Figs. 4-6)
    "k": [("imm-ic-wc-rmat22", dict(k=k)) for k in (1, 10, 25, 50, 100, 200)],
    "eps": [("imm-ic-wc-rmat22", dict(eps=e)) for e in (0.5, 0.3, 0.2, 0.1, 0.05)],
    # density: Barabasi-Albert n = 10^6, r = 2 .. 32 (Fig. 7)
    "ba": [(f"imm-ic-wc-ba1m-r{r}", {}) for r in (2, 4, 8, 16, 32)],
}


def run_sweep(args):
    """One benchmark line per point of a sweep (no CPU baseline); single GPU only."""
    rank, world, _ = dist_env()
    if world > 1:
        print("--sweep runs on one GPU", file=sys.stderr)
        return 2
    args.no_cpu_baseline = True
    rc = 0
    for name, over in SWEEPS[args.sweep]:
        WORKLOAD.clear()
        WORKLOAD.update(workload=name, **WORKLOADS[name])
        WORKLOAD.update(over, sweep=args.sweep)
        rc = rc or run_ours(args)
    return rc


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=12.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--cpu-single-budget", type=float, default=4.0,
                    help="seconds of one-core oracle work for cpu_baseline.single_core (0: skip)")
    ap.add_argument("--ref-budget", type=float, default=4.0, help="seconds of oracle work per reference step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true",
                    help="leave the batched-workload object out of the headline line")
    ap.add_argument("--case", default=None, choices=["sample-ic", "sample-lt", "sample-ic-p001", "select"],
                    help="run one small profiling case instead of the benchmark")
    ap.add_argument("--count", type=int, default=20000, help="RR sets for --case")
    ap.add_argument("--group-budget", type=int, default=0,
                    help="fix GIM_OPT_GROUP_BUDGET instead of autotuning (for profiler runs)")
    ap.add_argument("--large-bytes", type=float, default=0,
                    help="--case: device bytes for the block-per-set pass scratch (keeps profiler captures small)")
    ap.add_argument("--workload", default="imm-ic-wc-rmat22", choices=sorted(WORKLOADS),
                    help="IMM workload (default: the headline)")
    ap.add_argument("--sweep", default=None, choices=sorted(SWEEPS),
                    help="print one line per point of a k, eps or Barabasi-Albert density sweep")
    args = ap.parse_args()
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps; the timing rules want at least 3", file=sys.stderr)
    WORKLOAD.clear()
    WORKLOAD.update(workload=args.workload, **WORKLOADS[args.workload])
    if args.case:
        return run_case(args)
    if args.sweep and args.impl == "ours":
        return run_sweep(args)
    if args.workload.startswith("batch-") and args.impl == "ours":
        return run_batch(args)
    if args.workload.startswith("serve-") and args.impl == "ours":
        return run_serve(args)
    return run_reference(args) if args.impl == "reference" else run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
