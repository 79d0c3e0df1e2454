"""GPU parity at full size, in the launch configuration the benchmark times.

IMM on R-MAT scale 22 (seed 3, weighted-cascade weights 1/indeg(v) in fp32):
IC with k = 50, eps = 0.1 and LT with k = 100, eps = 0.05; and IC on
Barabasi-Albert graphs of 10^6 vertices (r = 2 and 32, k = 50, eps = 0.05).
All with l = 1 and Philox seed 7, after the same schedule autotuning the benchmark
runs. The oracle cannot redraw a million RR sets in a test's time, so:

* RR sets: every set of a prefix of rr_ids (tens of thousands, drawn by the
  oracle on all host cores), plus a seeded sample of rr_ids over the whole
  collection and the largest sets, each redrawn by the oracle one by one, all
  compared as sorted vertex lists;
* occurrence counts: equal to the member histogram of the exported store;
* IMM: the oracle runs Alg. 2 and Alg. 1 over the GPU's collection (each
  "sample until |R| >= t" served by its first t sets), which must give the
  same seeds, theta, LB and |R|.
"""
import numpy as np
import pytest

import oracle as O
from paper_2009_07325_gb300 import GIM_IC, GIM_LT, Context, binding
from paper_2009_07325_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2009_07325_gb300 import build
    build.build()
    O.build()
    I.build()


@pytest.fixture(scope="module")
def rmat22_wc():
    return I.wc_weights(I.rmat(22, 3))


def _keyed(off, mem, count):
    """The first `count` sets of a collection as sorted (set << 32 | vertex) keys."""
    off = np.asarray(off, dtype=np.int64)
    end = int(off[count])
    sets = np.repeat(np.arange(count, dtype=np.uint64), np.diff(off[:count + 1]))
    return np.sort((sets << np.uint64(32)) | np.asarray(mem[:end], dtype=np.uint64))


def _prefix_matches(g, model, seed, off, mem, count):
    """Every one of the first `count` RR sets equals the oracle's (a sampling fault
    that spares a random sample still shows up here)."""
    count = min(count, len(off) - 1)
    o = O.Oracle(g)
    o.sample(model, seed, count, max(1, O.max_threads()))
    ooff, omem = o.export()
    assert len(ooff) - 1 == count
    assert np.array_equal(_keyed(off, mem, count), _keyed(ooff, omem, count)), "a prefix RR set differs"
    o.close()


def _sampled_sets_match(ctx, orc, model, seed, off, mem, n_sample=256):
    R = len(off) - 1
    rng = np.random.default_rng(12345)
    sizes = np.diff(off)
    ids = set(rng.choice(R, size=min(n_sample, R), replace=False).tolist())
    ids |= set(np.argsort(sizes)[-16:].tolist()) | {0, R - 1}
    for j in sorted(ids):
        got = np.sort(mem[off[j]:off[j + 1]])
        want = np.sort(orc.rr_one(model, seed, int(j)))
        assert np.array_equal(got, want), f"RR set {j} differs"
    cnt = np.bincount(mem, minlength=ctx.n).astype(np.uint32)
    assert np.array_equal(ctx.coverage(), cnt)


@pytest.mark.parametrize("model,k,eps", [(GIM_IC, 50, 0.1), (GIM_LT, 100, 0.05)])
def test_imm_rmat22_full_size(rmat22_wc, model, k, eps):
    g = rmat22_wc
    ctx = Context(0)
    ctx.load(g)
    binding.autotune([ctx], [(model, k, eps, 1.0, 7)], 20000)
    r = ctx.imm(model, k, eps, 1.0, 7)
    off, mem = ctx.rr_export()
    assert len(off) - 1 == r["rr_count"] >= r["theta"]
    orc = O.Oracle(g)
    _sampled_sets_match(ctx, orc, model, 7, off, mem)
    _prefix_matches(g, model, 7, off, mem, 50000)
    orc.load_csr(off, mem)
    o = orc.imm_replay(k, eps, 1.0)
    assert r["seeds"].tolist() == o["seeds"].tolist()
    assert (r["theta"], r["lb"], r["rr_count"]) == (o["theta"], o["lb"], o["rr_count"])
    ctx.close()


def test_imm_rmat22_ic_p001_full_size():
    """IC with uniform p = 0.01 on R-MAT-22, k = 100, eps = 0.2 (about 10^10 members:
    too many to export or replay), checked on sampled RR sets and through
    properties that hold at any size."""
    g = I.uniform_weights(I.rmat(22, 3), 0.01)
    k, eps = 100, 0.2
    ctx = Context(0)
    ctx.load(g)
    binding.autotune([ctx], [(GIM_IC, k, eps, 1.0, 7)], 5000)
    r = ctx.imm(GIM_IC, k, eps, 1.0, 7)
    R, Z = ctx.rr_count()
    assert R == r["rr_count"] >= r["theta"]
    # theta from the oracle's constants and the LB the run found
    c = O.imm_constants(g.n, k, eps, 1.0)
    assert r["lb"] >= 1.0 and r["theta"] == int(np.ceil(c["lambda_star"] / r["lb"]))
    # sampled RR sets, redrawn by the oracle one by one
    orc = O.Oracle(g)
    rng = np.random.default_rng(99)
    for j in sorted(set(rng.choice(R, 48, replace=False).tolist()) | {0, R - 1}):
        assert np.array_equal(ctx.rr_get(j), np.sort(orc.rr_one(GIM_IC, 7, j))), f"RR set {j} differs"
    # counts sum to the store; the first seed is the lowest-id argmax of the counts
    cnt = ctx.coverage().astype(np.int64)
    assert int(cnt.sum()) == Z
    s, gains, cov = ctx.select_seeds(k)
    assert s.tolist() == r["seeds"].tolist()
    assert s[0] == int(np.argmax(cnt)) and gains[0] == cnt.max()
    assert len(set(s.tolist())) == k and all(a >= b for a, b in zip(gains[:-1], gains[1:]))
    assert int(gains.astype(np.int64).sum()) == cov <= R
    ctx.close()


@pytest.mark.parametrize("r", [2, 32])
def test_imm_barabasi_albert_full_size(r):
    """The density sweep's end points: Barabasi-Albert n = 10^6 with r = 2 (about 10^7
    RR sets of a few members) and r = 32 (64 M arcs, sets of tens of members and a few
    of ten thousand), IC weighted cascade, k = 50, eps = 0.05, as the benchmark runs them."""
    g = I.wc_weights(I.barabasi_albert(10 ** 6, r, 6))
    k, eps = 50, 0.05
    ctx = Context(0)
    ctx.load(g)
    binding.autotune([ctx], [(GIM_IC, k, eps, 1.0, 7)], 20000)
    res = ctx.imm(GIM_IC, k, eps, 1.0, 7)
    off, mem = ctx.rr_export()
    assert len(off) - 1 == res["rr_count"] >= res["theta"]
    orc = O.Oracle(g)
    _sampled_sets_match(ctx, orc, GIM_IC, 7, off, mem)
    _prefix_matches(g, GIM_IC, 7, off, mem, 20000)
    orc.load_csr(off, mem)
    o = orc.imm_replay(k, eps, 1.0)
    assert res["seeds"].tolist() == o["seeds"].tolist()
    assert (res["theta"], res["lb"], res["rr_count"]) == (o["theta"], o["lb"], o["rr_count"])
    ctx.close()
