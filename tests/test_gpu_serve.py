"""Query server (gim_server_*): every result equals the query run alone.

Queries with mixed models, k, eps and seeds are submitted in two waves, the
second while the first is on the GPU (continuous batching over resident RR
pools). Each query's seeds, theta, LB and |R| must equal gim_imm on a fresh
context with the same parameters, and the oracle's IMM.
"""
import numpy as np
import pytest

import oracle as O
from paper_2009_07325_gb300 import GIM_IC, GIM_LT, Context, GimError
from paper_2009_07325_gb300 import binding
from paper_2009_07325_gb300 import inputs as I

pytestmark = pytest.mark.gpu
THREADS = max(1, O.max_threads())


@pytest.fixture(scope="module")
def graph():
    from paper_2009_07325_gb300 import build
    build.build()
    return I.wc_weights(I.rmat(14, 6))


def _alone(g, p):
    c = Context(0)
    c.load(g)
    return c.imm(*p)


def test_server_results_equal_lone_runs(graph):
    ctx = Context(0)
    ctx.load(graph)
    srv = binding.Server(ctx, max_active=4, max_k=64)
    wave1 = [(GIM_IC, 10, 0.3, 1.0, 7), (GIM_LT, 20, 0.2, 1.0, 7), (GIM_IC, 40, 0.15, 1.0, 7),
             (GIM_IC, 5, 0.5, 1.0, 11), (GIM_LT, 64, 0.3, 1.0, 7), (GIM_IC, 25, 0.1, 1.0, 7)]
    wave2 = [(GIM_IC, 30, 0.2, 1.0, 7), (GIM_LT, 8, 0.4, 1.0, 7), (GIM_IC, 12, 0.25, 1.0, 11)]
    t1 = [(srv.submit(*p), p) for p in wave1]
    first = srv.wait(t1[0][0])          # the second wave arrives while others run
    t2 = [(srv.submit(*p), p) for p in wave2]
    got = {t: srv.wait(t) for t, _ in t1 + t2}
    st = srv.stats()
    srv.stop()
    assert st["completed"] == len(wave1) + len(wave2) and st["peak_active"] > 1
    assert got[t1[0][0]]["seeds"].tolist() == first["seeds"].tolist()
    for t, p in t1 + t2:
        a = _alone(graph, p)
        r = got[t]
        assert r["seeds"].tolist() == a["seeds"].tolist(), p
        assert (r["theta"], r["lb"], r["rr_count"]) == (a["theta"], a["lb"], a["rr_count"]), p
        assert r["latency_ms"] > 0
    # one query against the oracle as well
    o = O.Oracle(graph).imm(*wave1[1][:4], wave1[1][4], THREADS)
    assert got[t1[1][0]]["seeds"].tolist() == o["seeds"].tolist() and got[t1[1][0]]["theta"] == o["theta"]


def test_server_rejects_bad_queries_and_stops_cleanly(graph):
    ctx = Context(0)
    ctx.load(graph)
    srv = binding.Server(ctx, max_active=2, max_k=16)
    with pytest.raises(GimError):
        srv.submit(GIM_IC, 17, 0.3, 1.0, 1)          # k above max_k
    with pytest.raises(GimError):
        srv.submit(GIM_IC, 5, 1.2, 1.0, 1)           # eps outside (0, 1)
    t = srv.submit(GIM_IC, 5, 0.5, 1.0, 1)
    r = srv.wait(t)
    assert r["seeds"].tolist() == _alone(graph, (GIM_IC, 5, 0.5, 1.0, 1))["seeds"].tolist()
    srv.stop()
    # the graph context stays usable
    assert ctx.imm(GIM_IC, 3, 0.5, 1.0, 2)["seeds"].size == 3
