"""GPU parity of multi-round IM (Sec. IV-H; CR-NAIMM) against the oracle.

Multi-round collections (T rounds, elements t*n + v) must equal the oracle's
set by set after several appends, with the same element counts; the greedy
with k seeds per round must give the same seeds, gains and coverage; gim_mrim
must give the oracle's seeds, theta, LB and |R| (T = 1: gim_imm exactly). At
full size (R-MAT scale 22, IC weighted cascade, T = 5, k = 10, eps = 0.1, the
paper's setting) sampled multi-round sets are redrawn one by one and the
oracle replays the run over the GPU's collection.
"""
import numpy as np
import pytest

import oracle as O
from paper_2009_07325_gb300 import GIM_IC, GIM_LT, Context, GimError, binding
from paper_2009_07325_gb300 import inputs as I

pytestmark = pytest.mark.gpu
THREADS = max(1, O.max_threads())


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2009_07325_gb300 import build
    build.build()
    O.build()
    I.build()


@pytest.fixture(scope="module")
def er_wc():
    return I.wc_weights(I.er(2000, 20000, 1))


def _same_collection(ctx, orc):
    off_g, mem_g = ctx.rr_export()
    off_o, mem_o = orc.export()
    assert off_g.shape == off_o.shape
    if not np.array_equal(off_g, off_o):
        bad = int(np.nonzero(off_g != off_o)[0][0])
        raise AssertionError(f"first differing multi-round set near {bad - 1}")
    assert np.array_equal(mem_g, mem_o)
    assert np.array_equal(ctx.coverage(), orc.counts())


@pytest.mark.parametrize("model,T", [(GIM_IC, 3), (GIM_LT, 3), (GIM_IC, 32)])
def test_multi_round_collection_and_greedy(er_wc, model, T):
    ctx = Context(0)
    ctx.load(er_wc)
    ctx.set_rounds(T)
    assert ctx.rounds() == T
    orc = O.Oracle(er_wc)
    orc.set_rounds(T)
    for count in (1, 999, 3000):
        ctx.sample_rr(model, count, 7)
        orc.sample(model, 7, count, THREADS)
    _same_collection(ctx, orc)
    for k in (1, 10, 40):
        gs, gg, gc = ctx.select_seeds(k)
        os_, og, oc = orc.greedy(k)
        assert gs.tolist() == os_.tolist() and gg.tolist() == og.tolist() and gc == oc
        assert all(int(np.sum(gs // er_wc.n == t)) == k for t in range(T))
    ctx.reset_rr()
    assert ctx.rounds() == 1
    ctx.close()


@pytest.mark.parametrize("gname,model,T,k,eps", [
    ("er", GIM_IC, 5, 10, 0.5), ("er", GIM_LT, 3, 10, 0.5), ("er", GIM_IC, 2, 25, 0.3),
    ("rmat18", GIM_IC, 5, 10, 0.2)])
def test_mrim_bit_exact(er_wc, gname, model, T, k, eps):
    g = er_wc if gname == "er" else I.wc_weights(I.rmat(18, 5))
    ctx = Context(0)
    ctx.load(g)
    r = ctx.mrim(model, T, k, eps, 1.0, 7)
    orc = O.Oracle(g)
    o = orc.mrim(model, T, k, eps, 1.0, 7, THREADS)
    assert r["seeds"].tolist() == o["seeds"].tolist()
    assert (r["theta"], r["lb"], r["rr_count"]) == (o["theta"], o["lb"], o["rr_count"])
    _same_collection(ctx, orc)
    ctx.close()


def test_mrim_one_round_is_imm(er_wc):
    a = Context(0)
    a.load(er_wc)
    b = Context(0)
    b.load(er_wc)
    ra = a.mrim(GIM_IC, 1, 10, 0.5, 1.0, 7)
    rb = b.imm(GIM_IC, 10, 0.5, 1.0, 7)
    assert ra["seeds"].tolist() == rb["seeds"].tolist()
    assert (ra["theta"], ra["lb"], ra["rr_count"]) == (rb["theta"], rb["lb"], rb["rr_count"])
    # a multi-round run, then a plain IMM on the same context: the context returns to plain sets
    a.mrim(GIM_IC, 4, 5, 0.5, 1.0, 7)
    assert a.rounds() == 4
    rc = a.imm(GIM_IC, 10, 0.5, 1.0, 7)
    assert a.rounds() == 1 and rc["seeds"].tolist() == rb["seeds"].tolist()
    a.close()
    b.close()


def test_rounds_errors(er_wc):
    ctx = Context(0)
    ctx.load(er_wc)
    for T in (0, 33):
        with pytest.raises(GimError):
            ctx.set_rounds(T)
    ctx.sample_rr(GIM_IC, 10, 7)
    with pytest.raises(GimError):        # the collection is not empty
        ctx.set_rounds(2)
    with pytest.raises(GimError):
        ctx.mrim(GIM_IC, 0, 5, 0.5, 1.0, 7)
    ctx.close()


def test_mrim_rmat22_full_size():
    g = I.wc_weights(I.rmat(22, 3))
    T, k, eps = 5, 10, 0.1
    ctx = Context(0)
    ctx.load(g)
    binding.autotune([ctx], [(GIM_IC, k, eps, 1.0, 7)], 20000)
    r = ctx.mrim(GIM_IC, T, k, eps, 1.0, 7)
    off, mem = ctx.rr_export()
    R = len(off) - 1
    assert R == r["rr_count"] >= r["theta"]
    orc = O.Oracle(g)
    rng = np.random.default_rng(777)
    sizes = np.diff(off)
    ids = set(rng.choice(R, size=min(192, R), replace=False).tolist())
    ids |= set(np.argsort(sizes)[-8:].tolist()) | {0, R - 1}
    for j in sorted(ids):
        assert np.array_equal(mem[off[j]:off[j + 1]], orc.mrim_one(GIM_IC, T, 7, int(j))), f"set {j} differs"
    assert np.array_equal(ctx.coverage(), np.bincount(mem, minlength=g.n * T).astype(np.uint32))
    orc.set_rounds(T)
    orc.load_csr(off, mem)
    o = orc.imm_replay(k, eps, 1.0)
    assert r["seeds"].tolist() == o["seeds"].tolist()
    assert (r["theta"], r["lb"], r["rr_count"]) == (o["theta"], o["lb"], o["rr_count"])
    ctx.close()
