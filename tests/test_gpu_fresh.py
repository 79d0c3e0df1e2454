"""GPU parity of IMM with a fresh final phase (GIM_OPT_FRESH_FINAL = 1).

After the lower-bound search (Alg. 2), theta new RR sets with rr_ids
2^63 + j replace the collection and the greedy (Alg. 1) runs over them.
Against the oracle's imm_fresh: seeds, theta, LB, |R| and the whole RR
collection bit-exact on an Erdos-Renyi graph (n = 2000, m = 20000) and
R-MAT scale 18; in a batch that mixes fresh and reusing instances; and at
full size (R-MAT scale 22, IC, k = 50, eps = 0.1) on sampled RR sets
redrawn one by one plus the oracle's greedy over the GPU's collection.
"""
import numpy as np
import pytest

import oracle as O
from paper_2009_07325_gb300 import GIM_IC, GIM_LT, Context, GimError, binding
from paper_2009_07325_gb300 import inputs as I
from paper_2009_07325_gb300.binding import GIM_OPT_FRESH_FINAL

pytestmark = pytest.mark.gpu
THREADS = max(1, O.max_threads())
BASE = 1 << 63


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2009_07325_gb300 import build
    build.build()
    O.build()
    I.build()


def _fresh_ctx(g, on=True):
    c = Context(0)
    c.load(g)
    c.set_option(GIM_OPT_FRESH_FINAL, 1 if on else 0)
    return c


def _same_collection(ctx, orc):
    off_g, mem_g = ctx.rr_export()
    off_o, mem_o = orc.export()
    assert np.array_equal(off_g, off_o)
    assert np.array_equal(mem_g, mem_o)
    assert np.array_equal(ctx.coverage(), orc.counts())


@pytest.mark.parametrize("gname,model,k,eps", [
    ("er", GIM_IC, 10, 0.5), ("er", GIM_LT, 10, 0.5), ("er", GIM_IC, 25, 0.3),
    ("rmat18", GIM_IC, 50, 0.2), ("rmat18", GIM_LT, 50, 0.2)])
def test_fresh_imm_bit_exact(gname, model, k, eps):
    g = I.wc_weights(I.er(2000, 20000, 1) if gname == "er" else I.rmat(18, 5))
    ctx = _fresh_ctx(g)
    r = ctx.imm(model, k, eps, 1.0, 7)
    orc = O.Oracle(g)
    o = orc.imm_fresh(model, k, eps, 1.0, 7, THREADS)
    assert r["seeds"].tolist() == o["seeds"].tolist()
    assert (r["theta"], r["lb"], r["rr_count"]) == (o["theta"], o["lb"], o["rr_count"])
    assert r["rr_count"] == r["theta"]
    _same_collection(ctx, orc)
    # the collection keeps its counter base: appended sets continue at 2^63 + theta
    ctx.sample_rr(model, 50, 7)
    off, mem = ctx.rr_export()
    for j in (r["theta"], r["theta"] + 49):
        assert np.array_equal(np.sort(mem[off[j]:off[j + 1]]), np.sort(orc.rr_one(model, 7, BASE + j)))
    # a reset returns to rr_ids 0, 1, ...
    ctx.reset_rr()
    ctx.sample_rr(model, 300, 7)
    plain = O.Oracle(g)
    plain.sample(model, 7, 300, THREADS)
    _same_collection(ctx, plain)
    ctx.close()


def test_fresh_option_values():
    g = I.wc_weights(I.er(200, 1000, 2))
    ctx = _fresh_ctx(g, on=False)
    assert ctx.get_option(GIM_OPT_FRESH_FINAL) == 0
    ctx.set_option(GIM_OPT_FRESH_FINAL, 1)
    assert ctx.get_option(GIM_OPT_FRESH_FINAL) == 1
    with pytest.raises(GimError):
        ctx.set_option(GIM_OPT_FRESH_FINAL, 2)
    assert ctx.get_option(GIM_OPT_FRESH_FINAL) == 1
    ctx.close()


def test_batch_mixes_fresh_and_reusing_instances():
    three = I.from_edges(3, [0, 1, 2, 0], [1, 2, 0, 2]).with_weights(np.array([0.5, 0.5, 0.5, 0.4], np.float32),
                                                                    "three")
    cases = [
        (I.wc_weights(I.er(2000, 20000, 1)), (GIM_IC, 10, 0.5, 1.0, 7), True),
        (I.wc_weights(I.er(2000, 20000, 1)), (GIM_IC, 10, 0.5, 1.0, 7), False),
        (I.wc_weights(I.chung_lu(12000, 11)), (GIM_IC, 25, 0.2, 1.0, 1011), True),
        (I.wc_weights(I.chung_lu(30000, 12)), (GIM_LT, 10, 0.3, 1.0, 1012), True),
        (I.wc_weights(I.er(500, 3000, 4)), (GIM_LT, 50, 0.5, 1.0, 3), False),
        (three, (GIM_IC, 1, 0.5, 1.0, 9), True),
    ]
    ctxs = [_fresh_ctx(g, on) for g, _, on in cases]
    res = binding.batch_imm(ctxs, [p for _, p, _ in cases])
    for (g, p, on), c, r in zip(cases, ctxs, res):
        orc = O.Oracle(g)
        o = orc.imm_fresh(*p, THREADS) if on else orc.imm(*p, THREADS)
        assert r["seeds"].tolist() == o["seeds"].tolist(), p
        assert (r["theta"], r["lb"], r["rr_count"]) == (o["theta"], o["lb"], o["rr_count"]), p
        assert r["lb_rounds"] == len(o["rounds"])
        _same_collection(c, orc)
    for c in ctxs:
        c.close()


def test_fresh_imm_rmat22_full_size():
    g = I.wc_weights(I.rmat(22, 3))
    k, eps = 50, 0.1
    ctx = Context(0)
    ctx.load(g)
    binding.autotune([ctx], [(GIM_IC, k, eps, 1.0, 7)], 20000)
    r0 = ctx.imm(GIM_IC, k, eps, 1.0, 7)
    ctx.set_option(GIM_OPT_FRESH_FINAL, 1)
    r = ctx.imm(GIM_IC, k, eps, 1.0, 7)
    assert (r["theta"], r["lb"]) == (r0["theta"], r0["lb"])
    assert r["rr_count"] == r["theta"]
    off, mem = ctx.rr_export()
    assert len(off) - 1 == r["theta"]
    orc = O.Oracle(g)
    rng = np.random.default_rng(2468)
    sizes = np.diff(off)
    ids = set(rng.choice(r["theta"], size=256, replace=False).tolist())
    ids |= set(np.argsort(sizes)[-16:].tolist()) | {0, r["theta"] - 1}
    for j in sorted(ids):
        got = np.sort(mem[off[j]:off[j + 1]])
        assert np.array_equal(got, np.sort(orc.rr_one(GIM_IC, 7, BASE + int(j)))), f"RR set {j} differs"
    assert np.array_equal(ctx.coverage(), np.bincount(mem, minlength=ctx.n).astype(np.uint32))
    orc.load_csr(off, mem)
    os_, _, _ = orc.greedy(k)
    assert r["seeds"].tolist() == os_.tolist()
    ctx.close()
