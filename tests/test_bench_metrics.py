"""CPU checks of the benchmark's work accounting (the roofline numerators).

* Philox calls per expanded vertex: indeg/4 for a row with p > 2^-8, and
  indeg/16 + indeg/256 for a row with p <= 2^-8 (the boundary p = 2^-8 is a
  16-coin row, as in the coin reading), weighted by occurrence counts.
* The row probability of a weighted-cascade graph is 1/indeg(v) in fp32, 1
  for rows without in-edges.
* The roofline line: achieved = work / time, frac = achieved / peak, in the
  stated units; the selection roofline divides the library's byte count by
  the selection kernels' time.
* Every workload name resolves to a graph recipe and every sweep point to a
  workload.
* The CPU baseline runs the oracle on all host cores and, when asked, on one
  core, each over a bounded sample it describes.
* The served query trace (Poisson arrivals at 50 q/s, k uniform on [10, 200],
  eps log-uniform on [0.05, 0.5], IC or LT half each) and the batch recipe
  (n = round(10^(4+2U)), k and eps from fixed sets, seed 1000 + i).
* The clock record: median SM clock, maximum, and the throttle reasons seen
  active, parsed from nvidia-smi's CSV samples.
"""
import math

import numpy as np
import pytest

import bench
from paper_2009_07325_gb300 import inputs as I


def test_philox_calls_per_row_kind():
    indeg = np.array([4, 255, 256, 1024, 0], np.int64)
    p = np.array([0.25, 1 / 255, 2.0 ** -8, 1 / 1024, 1.0])
    cnt = np.array([1, 1, 1, 1, 1], np.uint32)
    want = 4 / 4 + 255 / 4 + (256 / 16 + 256 / 256) + (1024 / 16 + 1024 / 256) + 0
    assert bench.philox_calls(cnt, indeg, p) == pytest.approx(want)
    cnt = np.array([3, 0, 2, 0, 7], np.uint32)
    assert bench.philox_calls(cnt, indeg, p) == pytest.approx(3 * 1 + 2 * 17)
    assert bench.coin_count(cnt, indeg) == 3 * 4 + 2 * 256


def test_row_probability_weighted_cascade():
    g = I.wc_weights(I.er(300, 2000, 3))
    p = bench.row_probability(g)
    d = g.indegree()
    nz = d > 0
    assert np.array_equal(p[nz].astype(np.float32), (np.float32(1.0) / d[nz].astype(np.float32)))
    assert np.all(p[~nz] == 1.0)


def test_roofline_lines():
    r = bench.roofline("sample_ic_kernel", coins=8e9, calls=6e8, alg_bytes=1e9, members=5e7, kern_s=0.01,
                       n_launch=4, philox_calls_per_s=4.9e11, hbm_peak=6644.1, peak_kind="measured",
                       traffic=1.0e8, large_launches=2)
    assert r["bound"] == "alu" and r["unit"] == "G Philox calls/s"
    assert r["achieved"] == pytest.approx(60.0) and r["peak"] == pytest.approx(490.0)
    assert r["frac"] == pytest.approx(60.0 / 490.0)
    assert r["calls_per_launch"] == pytest.approx(1.5e8) and r["avg_launch_ms"] == pytest.approx(2.5)
    lt = bench.roofline("sample_lt_kernel", coins=0, calls=0, alg_bytes=0, members=1e8, kern_s=0.02, n_launch=2,
                        philox_calls_per_s=4.9e11, hbm_peak=6644.1, peak_kind="measured", traffic=None,
                        large_launches=1)
    assert lt["bound"] == "hbm" and lt["unit"] == "GB/s"
    assert lt["achieved"] == pytest.approx(36.0 * 1e8 / 0.02 / 1e9)
    iss = bench.issue_slots(calls=6e8, kern_s=0.01, inst_per_call=7.0, sms=152, sm_mhz=2070.0)
    assert iss["achieved"] == pytest.approx(6e8 * 7.0 / 0.01 / 1e9)
    assert iss["peak"] == pytest.approx(152 * 4 * 2.07) and iss["frac"] == pytest.approx(420.0 / (152 * 4 * 2.07))
    assert bench.issue_slots(6e8, 0.0, 7.0, 152, 2070.0) is None
    with_issue = bench.roofline("sample_ic_kernel", coins=8e9, calls=6e8, alg_bytes=1e9, members=5e7, kern_s=0.01,
                                n_launch=4, philox_calls_per_s=4.8e11, hbm_peak=6644.1, peak_kind="measured",
                                traffic=None, large_launches=1, issue=iss)
    assert with_issue["issue_slots"] is iss and with_issue["unit"] == "G Philox calls/s"
    sel = bench.select_roofline({"kernel_ms": 5.0, "bytes": 6.6441e9, "calls": 4}, 6644.1, "measured")
    assert sel["achieved"] == pytest.approx(1328.82) and sel["frac"] == pytest.approx(0.2)
    assert sel["ms_per_selection"] == pytest.approx(1.25)
    assert bench.select_roofline({"kernel_ms": 0.0, "bytes": 0.0, "calls": 0}, 6644.1, "measured") is None


def test_workloads_and_sweeps_resolve():
    for name, spec in bench.WORKLOADS.items():
        assert {"graph", "weights", "model"} <= set(spec), name
    for sweep, points in bench.SWEEPS.items():
        for name, over in points:
            assert name in bench.WORKLOADS, (sweep, name)
            assert set(over) <= {"k", "eps"}
    assert bench.WORKLOADS["mrim-ic-wc-rmat22-T5"]["rounds"] == 5
    assert bench.WORKLOADS["imm-ic-wc-rmat22-fresh"]["fresh_final"] is True
    assert math.isclose(bench.WORKLOADS["imm-ic-wc-rmat22"]["eps"], 0.1)


def test_cpu_baseline_all_cores_and_one_core(monkeypatch):
    g = I.wc_weights(I.er(2000, 20000, 1))
    monkeypatch.setattr(bench, "WORKLOAD", dict(bench.WORKLOAD, k=10))
    r = bench.cpu_baseline(g, budget_s=0.05, single_core_s=0.05)
    assert r["kind"] == "oracle" and r["unit"] == "RR-sets/s" and r["cores"] >= 1 and r["value"] > 0
    assert int(r["sample"].split()[0]) > 0 and "greedy k=10" in r["sample"]
    one = r["single_core"]
    assert one["cores"] == 1 and one["value"] > 0 and int(one["sample"].split()[0]) > 0
    assert "single_core" not in bench.cpu_baseline(g, budget_s=0.05)


def test_serve_trace_distributions():
    N = 20000
    tr = bench.serve_trace(N)
    t = np.array([x[0] for x in tr])
    gaps = np.diff(np.r_[0.0, t])
    assert np.all(gaps > 0)
    rate = 50.0
    assert abs(gaps.mean() - 1 / rate) < 5 * (1 / rate) / math.sqrt(N)          # Poisson at 50 q/s
    frac = float(np.mean(gaps > 1 / rate))
    assert abs(frac - math.exp(-1)) < 5 * math.sqrt(math.exp(-1) * (1 - math.exp(-1)) / N)   # exponential gaps
    k = np.array([x[1][1] for x in tr])
    assert k.min() >= 10 and k.max() <= 200
    cnt = np.bincount(k - 10, minlength=191)
    chi2 = float(((cnt - N / 191) ** 2 / (N / 191)).sum())
    assert abs(chi2 - 190) < 6 * math.sqrt(2 * 190)                              # k uniform on [10, 200]
    eps = np.array([x[1][2] for x in tr])
    z = np.log10(eps / 0.05)
    assert z.min() >= 0 and z.max() < 1 and abs(z.mean() - 0.5) < 5 * math.sqrt(1 / 12 / N)   # log-uniform
    lt = np.mean([x[1][0] == 1 for x in tr])
    assert abs(lt - 0.5) < 5 * math.sqrt(0.25 / N)
    assert all(x[1][3] == 1.0 for x in tr)
    assert bench.serve_trace(60) == tr[:60]


def test_batch_instances_recipe():
    inst = bench.batch_instances(256)
    assert len(inst) == 256 and inst == bench.batch_instances(256)
    ns = np.array([x[0] for x in inst])
    assert ns.min() >= 10 ** 4 and ns.max() <= 10 ** 6
    z = np.log10(ns) - 4
    assert abs(z.mean() - 1.0) < 5 * math.sqrt(4 / 12 / 256)                    # n = round(10^(4 + 2U))
    assert {x[1][1] for x in inst} == {10, 25, 50} and {x[1][2] for x in inst} == {0.1, 0.2, 0.5}
    assert [x[1][4] for x in inst] == [1000 + i for i in range(256)]


def test_clock_summary_parses_nvidia_smi_lines(tmp_path):
    rows = [
        "0, 2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2040, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, [N/A], 2070, 10.0, 0x0, Not Active, Not Active, Not Active, Not Active",   # skipped sample
        "0, 1980, 2070, 1400.0, 0x0000000000000008, Active, Not Active, Not Active, Not Active",
        "garbage",
    ]
    path = tmp_path / "clocks.csv"
    path.write_text("\n".join(rows) + "\n")
    s = bench.ClockSampler(0)
    s.path = str(path)
    out = s.summary()
    assert out == {"sm_mhz": 2040.0, "sm_max_mhz": 2070.0, "reasons": ["hw_slowdown", "sw_power_cap"], "samples": 3}
    assert not path.exists()                 # the sample file is removed after reading
    assert s.summary() is None
    empty = tmp_path / "empty.csv"
    empty.write_text("")
    s.path = str(empty)
    assert s.summary() is None
