"""GPU parity: libgim (through the C ABI) against the CPU oracle, bit-exact.

RR sets (as sorted vertex lists per rr_id), occurrence counts, seed lists,
marginal gains, covered counts, theta and LB must be identical. Inputs are
seeded synthetic graphs of the paper's kind (Sec. IV-B weighting): a directed
Erdos-Renyi graph (n = 2000, m = 20000), R-MAT scale 20 and 22 with
(a, b, c, d) = (0.57, 0.19, 0.19, 0.05), weighted-cascade probabilities and
uniform p = 0.01. Edge cases: p = 0 and p = 1, n = 2, k = n, empty
collection, RR sets larger than a worker's queue (the large-set pass) and a
store that must grow mid-call.
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


@pytest.fixture(scope="module")
def rmat20_wc():
    return I.wc_weights(I.rmat(20, 2))


@pytest.fixture(scope="module")
def rmat22():
    return I.rmat(22, 3)


def _ctx(g):
    c = Context(0)
    c.load(g)
    return c


def _same_collection(ctx, orc):
    off_g, mem_g = ctx.rr_export()
    off_o, mem_o = orc.export()
    assert off_g.shape == off_o.shape
    if not np.array_equal(off_g, off_o):
        bad = int(np.nonzero(off_g != off_o)[0][0])
        raise AssertionError(f"first differing RR set near rr_id {bad - 1}")
    assert np.array_equal(mem_g, mem_o)
    assert np.array_equal(ctx.coverage(), orc.counts())


@pytest.mark.parametrize("model", [GIM_IC, GIM_LT])
def test_er_sample_select_bit_exact(er_wc, model):
    ctx = _ctx(er_wc)
    orc = O.Oracle(er_wc)
    for count in (1, 999, 4000):       # several appends: ids continue across calls
        ctx.sample_rr(model, count, 7)
        orc.sample(model, 7, count, THREADS)
    _same_collection(ctx, orc)
    for k in (1, 10, 64):
        assert [a.tolist() if hasattr(a, "tolist") else a for a in ctx.select_seeds(k)] == \
               [a.tolist() if hasattr(a, "tolist") else a for a in orc.greedy(k)]


@pytest.mark.parametrize("model,k,eps", [(GIM_IC, 10, 0.5), (GIM_LT, 10, 0.5), (GIM_IC, 25, 0.3)])
def test_er_imm_bit_exact(er_wc, model, k, eps):
    ctx = _ctx(er_wc)
    orc = O.Oracle(er_wc)
    g = ctx.imm(model, k, eps, 1.0, 7)
    o = orc.imm(model, k, eps, 1.0, 7, THREADS)
    assert g["seeds"].tolist() == o["seeds"].tolist()
    assert g["theta"] == o["theta"] and g["lb"] == o["lb"] and g["rr_count"] == o["rr_count"]
    _same_collection(ctx, orc)


def test_rmat20_ic_wc_bit_exact(rmat20_wc):
    ctx = _ctx(rmat20_wc)
    orc = O.Oracle(rmat20_wc)
    ctx.sample_rr(GIM_IC, 30000, 7)
    orc.sample(GIM_IC, 7, 30000, THREADS)
    _same_collection(ctx, orc)
    gs, gg, gc = ctx.select_seeds(50)
    os_, og, oc = orc.greedy(50)
    assert gs.tolist() == os_.tolist() and gg.tolist() == og.tolist() and gc == oc


def test_rmat22_lt_bit_exact(rmat22):
    g = I.wc_weights(rmat22)
    ctx = _ctx(g)
    assert ctx.lt_valid
    orc = O.Oracle(g)
    ctx.sample_rr(GIM_LT, 50000, 7)
    orc.sample(GIM_LT, 7, 50000, THREADS)
    _same_collection(ctx, orc)
    gs, gg, gc = ctx.select_seeds(100)
    os_, og, oc = orc.greedy(100)
    assert gs.tolist() == os_.tolist() and gg.tolist() == og.tolist() and gc == oc


def test_rmat22_ic_p001_giant_sets_bit_exact(rmat22):
    """Uniform p = 0.01: ~5% of RR sets reach a giant component (> queue capacity)."""
    g = I.uniform_weights(rmat22, 0.01)
    ctx = _ctx(g)
    assert not ctx.lt_valid
    orc = O.Oracle(g)
    ctx.sample_rr(GIM_IC, 1500, 7)
    orc.sample(GIM_IC, 7, 1500, THREADS)
    _same_collection(ctx, orc)
    gs, gg, gc = ctx.select_seeds(20)
    os_, og, oc = orc.greedy(20)
    assert gs.tolist() == os_.tolist() and gg.tolist() == og.tolist() and gc == oc


def test_lt_thresholds_exact_and_sequential_rows_bit_exact():
    """LT thresholds: rows whose fp64 prefix sums are exact (parallel path), rows
    whose weights span more than 2^39 (sequential fp64 path), zero weights."""
    base = I.er(3000, 24000, 17)
    rng = np.random.default_rng(5)
    d = base.indegree()
    w = np.zeros(base.m, np.float64)
    off = base.offsets.astype(np.int64)
    for v in range(base.n):
        row = slice(off[v], off[v + 1])
        kind = v % 4
        if kind == 0:      # weighted cascade
            w[row] = 1.0 / max(d[v], 1)
        elif kind == 1:    # random, scaled to sum 0.9
            x = rng.random(d[v])
            w[row] = 0.9 * x / max(x.sum(), 1e-300)
        elif kind == 2:    # tiny and large weights in one row: fp64 sums round
            x = np.where(rng.random(d[v]) < 0.5, 1e-30, rng.random(d[v]) * 0.2)
            w[row] = x * (0.95 / max(x.sum(), 1e-300))
        else:              # zero weights mixed in, or an all-zero row
            x = np.where(rng.random(d[v]) < 0.4, 0.0, rng.random(d[v]))
            w[row] = (0.0 if v % 8 == 3 else 0.7) * x / max(x.sum(), 1e-300)
    g = base.with_weights(w.astype(np.float32), "mixed")
    ctx = _ctx(g)
    orc = O.Oracle(g)
    assert ctx.lt_valid and orc.lt_valid
    ctx.sample_rr(GIM_LT, 30000, 21)
    orc.sample(GIM_LT, 21, 30000, THREADS)
    _same_collection(ctx, orc)


def test_store_growth_and_large_sets():
    """p = 1 on a strongly connected ER graph: every RR set is ~n vertices, so each
    set overflows the worker queue and the store (64M entries) must grow."""
    g = I.uniform_weights(I.er(20000, 200000, 5), 1.0)
    ctx = _ctx(g)
    orc = O.Oracle(g)
    ctx.sample_rr(GIM_IC, 4000, 3)
    orc.sample(GIM_IC, 3, 4000, THREADS)
    _same_collection(ctx, orc)
    assert ctx.rr_count()[1] > (1 << 26)
    # one heavy set in flight at a time (the smallest block-pass scratch): same sets
    from paper_2009_07325_gb300 import binding
    one = _ctx(g)
    one.set_option(binding.GIM_OPT_LARGE_PASS_BYTES, 1)
    assert one.get_option(binding.GIM_OPT_LARGE_PASS_BYTES) == 1
    one.sample_rr(GIM_IC, 300, 3)
    off1, mem1 = one.rr_export()
    off0, mem0 = orc.export()
    assert np.array_equal(off1, off0[:301]) and np.array_equal(mem1, mem0[: off0[300]])
    one.set_option(binding.GIM_OPT_LARGE_PASS_BYTES, 16 << 30)   # back to the default


def test_sets_beyond_the_capped_queue():
    """p = 1 on ER n = 1.2M: every RR set (~the whole giant component) exceeds the
    first large-set pass's 2^20-entry queue, is abandoned there and finished by
    the pass with n-entry queues."""
    g = I.uniform_weights(I.er(1_200_000, 6_000_000, 8), 1.0)
    ctx = _ctx(g)
    orc = O.Oracle(g)
    ctx.sample_rr(GIM_IC, 12, 5)
    orc.sample(GIM_IC, 5, 12, THREADS)
    off, _ = orc.export()
    assert np.diff(off).min() > (1 << 20)
    _same_collection(ctx, orc)


@pytest.mark.parametrize("budget", [0, 1])
def test_screened_coins_bit_exact(budget):
    """In-edges with p <= 2^-8 (16 coins per Philox call, residual draws for
    zero bytes): common-probability rows (a complete fan-in graph, weighted
    cascade 1/1000) and rows whose per-edge weights straddle 2^-8
    (log-uniform in [2^-12, 2^-3]); budget 1 sends every set to the
    block-per-set pass."""
    K, S = 2000, 1000
    fan = I.wc_weights(I.from_edges(K + S, np.tile(np.arange(K, K + S, dtype=np.uint32), K),
                                    np.repeat(np.arange(K, dtype=np.uint32), S), "fanin"))
    base = I.er(3000, 90000, 21)
    r = I.u64_stream(21, 5, base.m)
    w = np.exp2(-3.0 - 9.0 * (r >> np.uint64(11)).astype(np.float64) * 2.0 ** -53).astype(np.float32)
    mixed = base.with_weights(w, "mixed")
    for g in (fan, mixed):
        ctx = _ctx(g)
        if budget:
            ctx.set_option(binding.GIM_OPT_GROUP_BUDGET, budget)
        orc = O.Oracle(g)
        for count in (7000, 13000):
            ctx.sample_rr(GIM_IC, count, 9)
            orc.sample(GIM_IC, 9, count, THREADS)
        _same_collection(ctx, orc)
        gs, gg, gc = ctx.select_seeds(20)
        os_, og, oc = orc.greedy(20)
        assert gs.tolist() == os_.tolist() and gg.tolist() == og.tolist() and gc == oc
        ctx.close()


def test_graph_reloads_lazy_lt_and_offset_errors():
    """Graphs loaded one after another reuse the previous graph's arrays (a
    smaller graph, then the first again); the LT thresholds are built on the
    first LT use, after IC work on the same graph; decreasing offsets are
    rejected with their row and leave the context as it was."""
    a = I.wc_weights(I.er(2000, 20000, 1))
    b = I.wc_weights(I.er(500, 3000, 4))
    ctx = Context(0)
    for g in (a, b, a, b, a):
        ctx.load(g)
        ctx.sample_rr(GIM_IC, 3000, 5)
        orc = O.Oracle(g)
        orc.sample(GIM_IC, 5, 3000, THREADS)
        _same_collection(ctx, orc)
        # LT after IC work: thresholds built now, from the weights kept on the device
        ctx.reset_rr()
        ctx.sample_rr(GIM_LT, 2000, 6)
        olt = O.Oracle(g)
        olt.sample(GIM_LT, 6, 2000, THREADS)
        _same_collection(ctx, olt)
        assert ctx.lt_valid
    off = a.offsets.copy()
    off[7], off[8] = off[8], off[7]          # row 7 now ends before it starts
    assert off[7] > off[8]
    bad_row = 7
    with pytest.raises(GimError, match=f"row {bad_row}"):
        ctx.graph_load(a.n, off, a.sources, a.weights)
    olt = O.Oracle(a)
    olt.sample(GIM_LT, 6, 2000, THREADS)
    _same_collection(ctx, olt)               # the previous graph and collection are intact
    ctx.close()


def test_degenerate_weights_and_sizes():
    base = I.er(300, 1500, 2)
    for p in (0.0, 1.0):
        g = I.uniform_weights(base, p)
        ctx = _ctx(g)
        orc = O.Oracle(g)
        for model in ((GIM_IC, GIM_LT) if p == 0.0 else (GIM_IC,)):
            ctx.reset_rr()
            orc.reset()
            ctx.sample_rr(model, 2000, 11)
            orc.sample(model, 11, 2000, THREADS)
            _same_collection(ctx, orc)
            assert ctx.select_seeds(300)[0].tolist() == orc.greedy(300)[0].tolist()   # k = n
    # n = 2, a single edge
    two = I.from_edges(2, [0], [1]).with_weights(np.array([0.5], np.float32), "two")
    ctx = _ctx(two)
    orc = O.Oracle(two)
    ctx.sample_rr(GIM_IC, 100, 1)
    orc.sample(GIM_IC, 1, 100)
    _same_collection(ctx, orc)
    r = ctx.imm(GIM_IC, 1, 0.5, 1.0, 1)
    o = O.Oracle(two).imm(GIM_IC, 1, 0.5, 1.0, 1)
    assert r["seeds"].tolist() == o["seeds"].tolist() and r["theta"] == o["theta"] and r["lb"] == o["lb"]


def test_empty_collection_selection(er_wc):
    ctx = _ctx(er_wc)
    s, gains, cov = ctx.select_seeds(5)
    assert s.tolist() == [0, 1, 2, 3, 4] and gains.tolist() == [0] * 5 and cov == 0


def test_state_and_argument_errors(er_wc):
    ctx = Context(0)
    with pytest.raises(GimError):
        ctx.sample_rr(GIM_IC, 10, 1)            # no graph
    ctx.load(er_wc)
    ctx.sample_rr(GIM_IC, 10, 1)
    with pytest.raises(GimError):
        ctx.sample_rr(GIM_LT, 10, 1)            # model change needs reset
    with pytest.raises(GimError):
        ctx.sample_rr(GIM_IC, 10, 2)            # seed change needs reset
    assert ctx.rr_count()[0] == 10
    with pytest.raises(GimError):
        ctx.select_seeds(2001)
    with pytest.raises(GimError):
        ctx.imm(GIM_IC, 5, 1.5, 1.0, 1)
    bad = I.er(50, 100, 1)
    with pytest.raises(GimError):            # weight outside [0, 1]
        ctx.graph_load(50, bad.offsets, bad.sources, np.full(bad.m, 1.5, np.float32))
    with pytest.raises(GimError):            # source out of range
        src = bad.sources.copy()
        src[0] = 50
        ctx.graph_load(50, bad.offsets, src, np.full(bad.m, 0.5, np.float32))
    # the failed loads left the previous graph and collection in place
    assert ctx.rr_count()[0] == 10
    ctx.reset_rr()
    assert ctx.rr_count() == (0, 0)
    ic = I.uniform_weights(I.er(50, 400, 1), 0.9)   # rows sum above 1: not LT-valid
    ctx.load(ic)
    assert not ctx.lt_valid
    with pytest.raises(GimError):
        ctx.sample_rr(GIM_LT, 10, 1)
    assert ctx.launch_count() > 0
