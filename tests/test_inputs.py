"""Pins of the seeded synthetic input generators (the stand-ins for the
paper's SNAP graphs, Table 1, and its Barabasi-Albert graphs, Sec. IV-F).

They hold none of the method's arithmetic, but every parity case and every
benchmark line runs on them, so their recipes are checked here against
independent statements:

* the in-edge CSR equals a numpy deduplication of the edge list (rows by
  target, sources ascending, self-loops and duplicates dropped);
* Erdos-Renyi: exactly m distinct edges, no self-loops, uniform endpoints;
* R-MAT: per-level (source bit, target bit) frequencies are (a, b, c, d) at
  every level, independently of the other levels;
* Chung-Lu: endpoint frequencies proportional to (i+1)^(-1/(gamma-1));
* Barabasi-Albert: undirected, a clique on r0 vertices, then r distinct
  earlier neighbours per new vertex, earlier vertices favoured;
* weighted cascade: fp32 1/indeg(v) on every in-edge of v;
* every generator is a pure function of its seed.
"""
import math

import numpy as np
import pytest


def _csr_from_numpy(n, src, dst):
    keep = src != dst
    key = np.unique(dst[keep].astype(np.uint64) << np.uint64(32) | src[keep].astype(np.uint64))
    d = (key >> np.uint64(32)).astype(np.int64)
    s = (key & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    off = np.zeros(n + 1, np.uint64)
    off[1:] = np.cumsum(np.bincount(d, minlength=n))
    return off, s


def _edges(g):
    dst = np.repeat(np.arange(g.n, dtype=np.uint32), g.indegree())
    return g.sources, dst


def _raw(inputs_mod, fn, D, *args):
    src = np.empty(D, np.uint32)
    dst = np.empty(D, np.uint32)
    rc = getattr(inputs_mod._l(), fn)(*args, src, dst)
    assert rc is None or rc >= 0
    return src, dst


def test_csr_equals_numpy_dedup(inputs_mod):
    rng = np.random.default_rng(5)
    n = 300
    src = rng.integers(0, n, 5000).astype(np.uint32)
    dst = rng.integers(0, n, 5000).astype(np.uint32)
    src[:40] = dst[:40]                                  # self-loops
    src[40:80], dst[40:80] = src[80:120], dst[80:120]    # duplicates
    g = inputs_mod.from_edges(n, src, dst)
    off, s = _csr_from_numpy(n, src, dst)
    assert np.array_equal(g.offsets, off) and np.array_equal(g.sources, s)
    for v in range(n):
        row = g.sources[int(g.offsets[v]):int(g.offsets[v + 1])]
        assert np.all(np.diff(row.astype(np.int64)) > 0) and not np.any(row == v)
    e = inputs_mod.from_edges(7, np.zeros(0, np.uint32), np.zeros(0, np.uint32))
    assert e.m == 0 and np.array_equal(e.offsets, np.zeros(8, np.uint64))
    with pytest.raises(ValueError):
        inputs_mod.from_edges(3, np.array([3], np.uint32), np.array([0], np.uint32))


def test_er_exact_edges_uniform(inputs_mod):
    n, m = 2000, 20000
    g = inputs_mod.er(n, m, 1)
    assert g.m == m
    src, dst = _edges(g)
    assert not np.any(src == dst)
    assert np.unique(dst.astype(np.uint64) * n + src).size == m
    # endpoints uniform: in- and out-degrees are Binomial(m, 1/n) up to the dedup
    for deg in (g.indegree(), np.bincount(src, minlength=n)):
        chi2 = float(((deg - m / n) ** 2 / (m / n)).sum())
        assert abs(chi2 - (n - 1)) < 6 * math.sqrt(2 * (n - 1)), chi2
    h = inputs_mod.er(n, m, 1)
    assert np.array_equal(g.sources, h.sources) and np.array_equal(g.offsets, h.offsets)
    assert not np.array_equal(g.sources, inputs_mod.er(n, m, 2).sources)
    full = inputs_mod.er(5, 20, 3)                      # m = n(n-1): the complete digraph
    assert full.m == 20 and np.array_equal(full.indegree(), np.full(5, 4))
    with pytest.raises(ValueError):
        inputs_mod.er(5, 21, 3)


def test_rmat_level_frequencies(inputs_mod):
    scale, D = 12, 400000
    a, b, c = 0.57, 0.19, 0.19
    src, dst = _raw(inputs_mod, "gg_rmat_edges", D, scale, D, a, b, c, 2)
    assert int(src.max()) < (1 << scale) and int(dst.max()) < (1 << scale)
    probs = np.array([a, b, c, 1 - a - b - c])
    for lvl in range(scale):
        sh = scale - 1 - lvl                       # most significant bit first
        q = ((src >> sh) & 1).astype(np.int64) * 2 + ((dst >> sh) & 1).astype(np.int64)
        cnt = np.bincount(q, minlength=4)
        assert np.all(np.abs(cnt - D * probs) < 5 * np.sqrt(D * probs * (1 - probs))), (lvl, cnt)
    # levels are independent: the joint frequency of two levels' quadrants is the product
    q0 = ((src >> (scale - 1)) & 1) * 2 + ((dst >> (scale - 1)) & 1)
    q5 = ((src >> (scale - 6)) & 1) * 2 + ((dst >> (scale - 6)) & 1)
    joint = np.bincount(q0.astype(np.int64) * 4 + q5.astype(np.int64), minlength=16)
    pj = np.outer(probs, probs).ravel()
    assert np.all(np.abs(joint - D * pj) < 5 * np.sqrt(D * pj * (1 - pj)) + 1)
    g = inputs_mod.rmat(scale, 2)
    off, s = _csr_from_numpy(1 << scale, src[:16 << scale], dst[:16 << scale])
    assert np.array_equal(g.offsets, off) and np.array_equal(g.sources, s)   # 16 n draws, then dedup
    assert g.m < 16 << scale


def test_chung_lu_endpoint_weights(inputs_mod):
    n, gamma = 5000, 2.1
    D = 8 * n
    src, dst = _raw(inputs_mod, "gg_chung_lu_edges", D, n, D, gamma, 4)
    w = (np.arange(n) + 1.0) ** (-1.0 / (gamma - 1.0))
    p = w / w.sum()
    for ends in (src, dst):
        cnt = np.bincount(ends, minlength=n)
        head = slice(0, 20)                        # the heaviest vertices one by one
        assert np.all(np.abs(cnt[head] - D * p[head]) < 5 * np.sqrt(D * p[head]) + 1)
        # the rest in 20 bins of equal expected mass
        cut = np.searchsorted(np.cumsum(p[20:]) / p[20:].sum(), np.linspace(0, 1, 21)[1:-1])
        bins = np.add.reduceat(cnt[20:], np.r_[0, cut])
        mass = np.add.reduceat(p[20:], np.r_[0, cut]) * D
        assert np.all(np.abs(bins - mass) < 5 * np.sqrt(mass)), (bins, mass)
    g = inputs_mod.chung_lu(n, 4)
    off, s = _csr_from_numpy(n, src, dst)
    assert np.array_equal(g.offsets, off) and np.array_equal(g.sources, s)


@pytest.mark.parametrize("n,r", [(3000, 2), (3000, 8), (500, 32)])
def test_barabasi_albert_structure(inputs_mod, n, r):
    g = inputs_mod.barabasi_albert(n, r, 9)
    r0 = max(r, 2)
    assert g.m == r0 * (r0 - 1) + 2 * (n - r0) * r
    src, dst = _edges(g)
    fwd = set(zip(src.tolist(), dst.tolist()))
    assert all((v, u) in fwd for u, v in fwd)                      # undirected
    for v in range(r0):                                           # the starting clique
        row = set(g.sources[int(g.offsets[v]):int(g.offsets[v + 1])].tolist())
        assert set(range(r0)) - {v} <= row
    for v in range(r0, n):                                        # r distinct earlier neighbours
        row = g.sources[int(g.offsets[v]):int(g.offsets[v + 1])]
        assert int(np.sum(row < v)) == r
    deg = g.indegree()
    assert deg[: n // 100 + r0].mean() > 3 * deg[n // 2:].mean()   # preferential attachment
    h = inputs_mod.barabasi_albert(n, r, 9)
    assert np.array_equal(g.sources, h.sources)


def test_wc_weights_are_fp32_reciprocal_indegree(inputs_mod):
    g = inputs_mod.wc_weights(inputs_mod.rmat(10, 3))
    d = g.indegree()
    for v in np.nonzero(d)[0][:200]:
        row = g.weights[int(g.offsets[v]):int(g.offsets[v + 1])]
        assert np.all(row == np.float32(1.0) / np.float32(d[v]))
    assert g.weights.dtype == np.float32 and g.weights.size == g.m


def test_u64_stream_seeded_and_uniform(inputs_mod):
    a = inputs_mod.u64_stream(11, 3, 50000)
    assert np.array_equal(a, inputs_mod.u64_stream(11, 3, 50000))
    assert not np.array_equal(a, inputs_mod.u64_stream(11, 4, 50000))
    assert np.array_equal(a[:100], inputs_mod.u64_stream(11, 3, 100))   # index-addressed, not sequential state
    top = np.bincount((a >> np.uint64(60)).astype(np.int64), minlength=16)
    chi2 = float(((top - a.size / 16) ** 2 / (a.size / 16)).sum())
    assert chi2 < 50.0
