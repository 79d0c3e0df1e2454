"""Pins of the oracle's RR-set sampling (IC and LT) and LT thresholds.

* Exhaustive live-edge enumeration on tiny random graphs gives the exact
  probability that u lies in the RR set of root v (Sec. II-E definition);
  the oracle's empirical frequencies must sit within a 5-sigma binomial band.
* Eq. 3: n * Pr[S meets a random RR set] equals the exact expected spread
  E[I(S)], computed by forward reachability in every world.
* Per-world exactness: each IC RR set equals networkx's ancestor set of the
  root in the live-edge graph fixed by the oracle's own per-edge coins.
* Special cases: p = 1 gives plain reverse reachability, p = 0 gives the
  root alone, a weight-1 LT chain walks back deterministically.
* LT thresholds equal the exactly rounded rational prefix sums.
"""
from fractions import Fraction

import networkx as nx
import numpy as np
import pytest

SEED = 7


from exact_enum import edges as _edges, exact_ic as _exact_ic, exact_lt as _exact_lt


def _empirical(oracle_mod, g, model, N):
    o = oracle_mod.Oracle(g)
    o.sample(model, SEED, N, threads=4)
    off, mem = o.export()
    roots = np.array([oracle_mod.root(SEED, j, g.n) for j in range(N)])
    member = np.zeros((N, g.n), bool)
    rows = np.repeat(np.arange(N), np.diff(off).astype(np.int64))
    member[rows, mem] = True
    return roots, member, off, mem


def _check_freq(exact, roots, member, n):
    worst = 0.0
    for v in range(n):
        sel = roots == v
        Nv = int(sel.sum())
        assert Nv > 1000
        freq = member[sel].mean(axis=0)
        for u in range(n):
            pe = exact[u, v]
            sd = np.sqrt(max(pe * (1 - pe), 1e-12) / Nv)
            z = abs(freq[u] - pe) / sd if pe not in (0.0, 1.0) else (0.0 if freq[u] == pe else np.inf)
            worst = max(worst, z)
    assert worst < 5.0, worst


@pytest.mark.parametrize("gseed", [1, 2, 3])
def test_ic_rr_matches_exhaustive_enumeration(oracle_mod, inputs_mod, gseed):
    g = inputs_mod.tiny_graph(6, 13, gseed)
    exact, _, _ = _exact_ic(g)
    roots, member, _, _ = _empirical(oracle_mod, g, oracle_mod.IC, 60000)
    _check_freq(exact, roots, member, g.n)


@pytest.mark.parametrize("gseed", [4, 5])
def test_lt_rr_matches_exhaustive_enumeration(oracle_mod, inputs_mod, gseed):
    g = inputs_mod.tiny_graph(6, 12, gseed, weights="lt", max_indeg_sum=0.9)
    o = oracle_mod.Oracle(g)
    assert o.lt_valid
    exact, _, _ = _exact_lt(g)
    roots, member, _, _ = _empirical(oracle_mod, g, oracle_mod.LT, 60000)
    _check_freq(exact, roots, member, g.n)


def test_lt_normalised_rows_match_enumeration(oracle_mod, inputs_mod):
    """Rows summing to exactly 1 (LT weighted cascade) always pick an edge."""
    g = inputs_mod.wc_weights(inputs_mod.er(6, 12, 9))
    exact, _, _ = _exact_lt(g)
    roots, member, _, _ = _empirical(oracle_mod, g, oracle_mod.LT, 60000)
    _check_freq(exact, roots, member, g.n)


@pytest.mark.parametrize("model", ["ic", "lt"])
def test_eq3_unbiased_spread(oracle_mod, inputs_mod, model):
    """Eq. 3: E[I(S)] = n Pr[S intersects RR], with E[I(S)] by forward reachability."""
    if model == "ic":
        g = inputs_mod.tiny_graph(6, 12, 21)
        _, R, prob = _exact_ic(g)
        mdl = oracle_mod.IC
    else:
        g = inputs_mod.tiny_graph(6, 12, 22, weights="lt", max_indeg_sum=1.0)
        _, R, prob = _exact_lt(g)
        mdl = oracle_mod.LT
    N = 60000
    _, member, _, _ = _empirical(oracle_mod, g, mdl, N)
    for S in ([0], [3], [1, 4], [0, 2, 5]):
        spread = float(np.einsum("w,w->", prob, R[:, S, :].any(axis=1).sum(axis=1).astype(np.float64)))
        hit = member[:, S].any(axis=1)
        phat = hit.mean()
        pe = spread / g.n
        sd = np.sqrt(pe * (1 - pe) / N)
        assert abs(phat - pe) < 5 * sd, (S, g.n * phat, spread)


def test_ic_rr_equals_reachability_in_live_world(oracle_mod, inputs_mod):
    """Each RR set is exactly the ancestor set of its root in the world its coins define."""
    g = inputs_mod.tiny_graph(40, 160, 31)
    src, dst, _ = _edges(g)
    o = oracle_mod.Oracle(g)
    for j in range(200):
        root = oracle_mod.root(SEED, j, g.n)
        G = nx.DiGraph()
        G.add_nodes_from(range(g.n))
        for e in range(g.m):
            if oracle_mod.ic_live(SEED, j, e, float(g.weights[e])):
                G.add_edge(int(src[e]), int(dst[e]))
        want = sorted(nx.ancestors(G, root) | {root})
        assert o.rr_one(oracle_mod.IC, SEED, j).tolist() == want


def test_ic_p1_is_reverse_reachability_and_p0_is_root(oracle_mod, inputs_mod):
    base = inputs_mod.er(50, 120, 3)
    src, dst = base.sources.astype(np.int64), np.repeat(np.arange(base.n), base.indegree())
    G = nx.DiGraph()
    G.add_nodes_from(range(base.n))
    G.add_edges_from(zip(src.tolist(), dst.tolist()))
    o1 = oracle_mod.Oracle(inputs_mod.uniform_weights(base, 1.0))
    o0 = oracle_mod.Oracle(inputs_mod.uniform_weights(base, 0.0))
    for j in range(100):
        root = oracle_mod.root(SEED, j, base.n)
        assert o1.rr_one(oracle_mod.IC, SEED, j).tolist() == sorted(nx.ancestors(G, root) | {root})
        assert o0.rr_one(oracle_mod.IC, SEED, j).tolist() == [root]
        assert o0.rr_one(oracle_mod.LT, SEED, j).tolist() == [root]


def test_lt_weight_one_chain(oracle_mod, inputs_mod):
    """v_i's only in-edge comes from v_{i-1} with weight 1: the walk goes back to v_0."""
    n = 30
    g = inputs_mod.from_edges(n, np.arange(n - 1), np.arange(1, n))
    g = g.with_weights(np.ones(g.m, np.float32), "chain")
    o = oracle_mod.Oracle(g)
    for j in range(50):
        root = oracle_mod.root(SEED, j, n)
        assert o.rr_one(oracle_mod.LT, SEED, j).tolist() == list(range(root + 1))
    # a cycle stops the walk at the first repeat: members are the whole cycle
    cyc = inputs_mod.from_edges(n, np.arange(n), (np.arange(n) + 1) % n)
    o2 = oracle_mod.Oracle(cyc.with_weights(np.ones(n, np.float32), "cycle"))
    for j in range(20):
        assert o2.rr_one(oracle_mod.LT, SEED, j).tolist() == list(range(n))


def test_lt_thresholds_exact_rational(oracle_mod, inputs_mod):
    g = inputs_mod.tiny_graph(60, 400, 41, weights="lt", max_indeg_sum=1.0)
    o = oracle_mod.Oracle(g)
    cum = o.lt_thresholds()
    off = g.offsets.astype(np.int64)
    for v in range(g.n):
        acc = Fraction(0)
        row_total = sum(Fraction(float(x)) for x in g.weights[off[v]:off[v + 1]])
        for e in range(off[v], off[v + 1]):
            acc += Fraction(float(g.weights[e]))
            x = acc * (1 << 32)
            want = int(x) + (1 if x - int(x) >= Fraction(1, 2) else 0)   # half away from zero, x >= 0
            want = min(want, 1 << 32)
            if e == off[v + 1] - 1 and abs(row_total - 1) <= Fraction(1, 10**6):
                want = 1 << 32
            assert int(cum[e]) == want, (v, e)


def test_lt_thresholds_wc_within_rounding(oracle_mod, inputs_mod):
    """Weighted-cascade rows: every threshold is within 1/2 (+ fp64 error) of the exact value."""
    g = inputs_mod.wc_weights(inputs_mod.rmat(10, 5))
    o = oracle_mod.Oracle(g)
    assert o.lt_valid
    cum = o.lt_thresholds().astype(np.float64)
    off = g.offsets.astype(np.int64)
    for v in np.nonzero(g.indegree())[0][:300]:
        ws = [Fraction(float(x)) for x in g.weights[off[v]:off[v + 1]]]
        acc = Fraction(0)
        for i, e in enumerate(range(off[v], off[v + 1])):
            acc += ws[i]
            if e == off[v + 1] - 1:
                assert cum[e] == 2.0 ** 32
            else:
                assert abs(cum[e] - float(acc * (1 << 32))) <= 0.5 + 1e-3


def test_rr_invariants_on_rmat(oracle_mod, inputs_mod):
    """Root in its own set, sorted without repeats, counts equal set membership."""
    g = inputs_mod.wc_weights(inputs_mod.rmat(12, 2))
    for model in (oracle_mod.IC, oracle_mod.LT):
        o = oracle_mod.Oracle(g)
        o.sample(model, SEED, 3000, threads=4)
        off, mem = o.export()
        for j in range(3000):
            s = mem[off[j]:off[j + 1]]
            assert oracle_mod.root(SEED, j, g.n) in s
            assert np.all(np.diff(s.astype(np.int64)) > 0)
        cnt = o.counts()
        assert np.array_equal(cnt, np.bincount(mem, minlength=g.n).astype(np.uint32))
        assert int(cnt.sum()) == o.store_size
        if model == oracle_mod.LT:
            # a walk back from the root: inside the set, every member reaches the root
            src = g.sources.astype(np.int64)
            dst = np.repeat(np.arange(g.n), g.indegree())
            G = nx.DiGraph()
            G.add_edges_from(zip(src.tolist(), dst.tolist()))
            for j in range(0, 3000, 10):
                s = mem[off[j]:off[j + 1]].tolist()
                r = oracle_mod.root(SEED, j, g.n)
                H = G.subgraph(s)
                assert set(s) == (nx.ancestors(H, r) | {r}) if r in H else s == [r]


def test_threads_do_not_change_collection(oracle_mod, inputs_mod):
    g = inputs_mod.wc_weights(inputs_mod.rmat(12, 3))
    a = oracle_mod.Oracle(g)
    b = oracle_mod.Oracle(g)
    a.sample(oracle_mod.IC, 99, 2000, threads=1)
    a.sample(oracle_mod.IC, 99, 777, threads=1)
    b.sample(oracle_mod.IC, 99, 2777, threads=8)
    oa, ma = a.export()
    ob, mb = b.export()
    assert np.array_equal(oa, ob) and np.array_equal(ma, mb)


def test_model_or_seed_change_needs_reset(oracle_mod, inputs_mod):
    g = inputs_mod.wc_weights(inputs_mod.er(100, 400, 2))
    o = oracle_mod.Oracle(g)
    o.sample(oracle_mod.IC, 1, 10)
    with pytest.raises(RuntimeError):
        o.sample(oracle_mod.LT, 1, 10)
    with pytest.raises(RuntimeError):
        o.sample(oracle_mod.IC, 2, 10)
    o.reset()
    o.sample(oracle_mod.LT, 2, 10)
    assert o.rr_count == 10
