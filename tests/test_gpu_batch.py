"""Batched IMM (gim_batch_imm) against one-at-a-time gim_imm and the oracle.

A batch of instances with different graphs (Erdos-Renyi, Chung-Lu power
law, a 3-vertex graph whose lower-bound search has no round), diffusion
models (IC and LT), k, eps and seeds must give every instance exactly the
seeds, theta, LB and RR collection it gets alone.
"""
import numpy as np
import pytest

import oracle as O
from paper_2009_07325_gb300 import GIM_IC, GIM_LT, Context, GimError
from paper_2009_07325_gb300 import binding
from paper_2009_07325_gb300 import inputs as I

pytestmark = pytest.mark.gpu
THREADS = max(1, O.max_threads())


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2009_07325_gb300 import build
    build.build()


def _graphs():
    three = I.from_edges(3, [0, 1, 2, 0], [1, 2, 0, 2]).with_weights(np.array([0.5, 0.5, 0.5, 0.4], np.float32), "three")
    return [
        (I.wc_weights(I.er(2000, 20000, 1)), (GIM_IC, 10, 0.5, 1.0, 7)),
        (I.wc_weights(I.chung_lu(12000, 11)), (GIM_IC, 25, 0.2, 1.0, 1011)),
        (I.wc_weights(I.chung_lu(30000, 12)), (GIM_LT, 10, 0.3, 1.0, 1012)),
        (I.wc_weights(I.er(500, 3000, 4)), (GIM_LT, 50, 0.5, 1.0, 3)),
        (I.wc_weights(I.chung_lu(20000, 13)), (GIM_IC, 50, 0.5, 1.0, 1013)),
        (three, (GIM_IC, 1, 0.5, 1.0, 9)),
    ]


def test_batch_matches_single_runs_and_oracle():
    cases = _graphs()
    ctxs = []
    for g, _ in cases:
        c = Context(0)
        c.load(g)
        ctxs.append(c)
    res = binding.batch_imm(ctxs, [p for _, p in cases])
    for (g, p), c, r in zip(cases, ctxs, res):
        alone = Context(0)
        alone.load(g)
        a = alone.imm(*p)
        assert r["seeds"].tolist() == a["seeds"].tolist(), p
        assert (r["theta"], r["lb"], r["rr_count"]) == (a["theta"], a["lb"], a["rr_count"]), p
        ob, mb = c.rr_export()
        oa, ma = alone.rr_export()
        assert np.array_equal(ob, oa) and np.array_equal(mb, ma)
        o = O.Oracle(g).imm(p[0], p[1], p[2], p[3], p[4], THREADS)
        assert r["seeds"].tolist() == o["seeds"].tolist() and r["theta"] == o["theta"] and r["lb"] == o["lb"]
        assert r["lb_rounds"] == len(o["rounds"])


def test_batch_twice_in_a_row_and_errors():
    g = I.wc_weights(I.er(1000, 8000, 2))
    a, b = Context(0), Context(0)
    a.load(g)
    b.load(g)
    p = [(GIM_IC, 5, 0.4, 1.0, 1), (GIM_LT, 7, 0.4, 1.0, 2)]
    r1 = binding.batch_imm([a, b], p)
    r2 = binding.batch_imm([a, b], p)
    for x, y in zip(r1, r2):
        assert x["seeds"].tolist() == y["seeds"].tolist() and x["theta"] == y["theta"]
    # the contexts stay usable for the single-query calls after a batch
    assert a.imm(*p[0])["seeds"].tolist() == r1[0]["seeds"].tolist()
    assert b.select_seeds(7)[0].tolist() == r1[1]["seeds"].tolist()
    with pytest.raises(GimError):
        binding.batch_imm([a, a], p)                   # repeated context
    with pytest.raises(GimError):
        binding.batch_imm([a, b], [(GIM_IC, 5, 1.5, 1.0, 1), p[1]])   # bad eps
    bad = Context(0)
    bad.load(I.uniform_weights(I.er(100, 900, 1), 0.9))   # not LT-valid
    with pytest.raises(GimError):
        binding.batch_imm([a, bad], [p[0], (GIM_LT, 3, 0.5, 1.0, 1)])


def test_schedule_never_changes_results():
    """Every schedule knob changes speed only: the group budget (warps per
    heavy RR set), the block pass's chunk and frontier batch, the warp
    pass's queue capacity."""
    g = I.wc_weights(I.rmat(16, 8))
    ref = None
    schedules = [dict(group_budget=b) for b in (1, 64, 4096, 1 << 30)]
    schedules += [dict(group_budget=64, chunk_groups=cg, frontier_batch=fb)
                  for cg, fb in ((64, 32), (256, 96), (4096, 256), (1024, 64))]
    schedules += [dict(group_budget=1 << 30, queue_cap=qc) for qc in (256, 1024)]
    for sched in schedules:
        c = Context(0)
        c.load(g)
        for name, value in sched.items():
            c.set_option(binding.SCHEDULE_OPTIONS[name], value)
        assert {k: c.schedule()[k] for k in sched} == sched
        c.sample_rr(GIM_IC, 8000, 5)
        got = c.rr_export(), c.coverage(), c.select_seeds(20)
        if ref is None:
            ref = got
        else:
            assert np.array_equal(got[0][0], ref[0][0]) and np.array_equal(got[0][1], ref[0][1])
            assert np.array_equal(got[1], ref[1])
            assert [x.tolist() if hasattr(x, "tolist") else x for x in got[2]] == \
                   [x.tolist() if hasattr(x, "tolist") else x for x in ref[2]]


def test_schedule_options_reject_values_out_of_range():
    c = Context(0)
    c.load(I.wc_weights(I.er(200, 1000, 3)))
    for opt, bad in ((binding.GIM_OPT_FRONTIER_BATCH, 16), (binding.GIM_OPT_FRONTIER_BATCH, 257),
                     (binding.GIM_OPT_FRONTIER_BATCH, 100), (binding.GIM_OPT_CHUNK_GROUPS, 32),
                     (binding.GIM_OPT_CHUNK_GROUPS, 100), (binding.GIM_OPT_CHUNK_GROUPS, 8192),
                     (binding.GIM_OPT_QUEUE_CAP, 128), (binding.GIM_OPT_QUEUE_CAP, 8192),
                     (binding.GIM_OPT_QUEUE_CAP, 1000)):
        before = c.get_option(opt)
        with pytest.raises(GimError):
            c.set_option(opt, bad)
        assert c.get_option(opt) == before


def test_autotune_picks_a_candidate_and_caches_it():
    g = I.wc_weights(I.chung_lu(20000, 5))
    cs = [Context(0) for _ in range(3)]
    for c in cs:
        c.load(g)
    params = [(GIM_IC, 10, 0.5, 1.0, s) for s in (1, 2, 3)]
    b1, m1 = binding.autotune(cs, params, 500)
    b2, m2 = binding.autotune(cs, params, 500)
    assert b1 in (1 << 12, 1 << 14, 1 << 16, 1 << 18, 1 << 30) and m1 and b1 == b2 and not m2
    assert all(c.get_option(binding.GIM_OPT_GROUP_BUDGET) == b1 and c.rr_count() == (0, 0) for c in cs)
    sched = cs[0].schedule()
    assert sched["chunk_groups"] in (256, 512, 1024, 2048) and sched["frontier_batch"] in (32, 64, 128)
    assert sched["queue_cap"] in (1024, 2048, 4096) and all(c.schedule() == sched for c in cs)
    r = binding.batch_imm(cs, params)
    for c, p, x in zip(cs, params, r):
        alone = Context(0)
        alone.load(g)
        assert alone.imm(*p)["seeds"].tolist() == x["seeds"].tolist()
