"""Pins of the oracle's multi-round IM (Sec. IV-H, CR-NAIMM of Sun et al.).

* T = 1 reduces to IMM: same seeds, theta, LB, lower-bound trace and
  collection as orc_imm, and the constants equal IMM's exactly.
* A multi-round RR set rebuilt from the Philox primitives alone (one root,
  T reverse traversals in the worlds of rr_ids t * 2^32 + j, written here as a
  plain BFS / walk) equals the oracle's, for IC and LT; round 0 is RR set j.
* The partition-constrained greedy equals a brute-force statement of its
  definition on random small set systems (k per round, lowest id on ties,
  gain-0 picks once everything is covered).
* Exact multi-round spreads from live-edge enumeration (rounds are
  independent worlds): n Pr[S meets a random multi-round RR set] matches the
  exact spread within a 5-sigma band, and the seeds reach (1/2 - eps) OPT
  over every feasible seed set.
"""
import itertools
import math

import numpy as np
import pytest

from exact_enum import exact_ic, exact_lt

SEED = 7


def _bfs_ic(oracle_mod, g, seed, root, rr_id):
    seen = {root}
    q = [root]
    h = 0
    off, src, w = g.offsets, g.sources, g.weights
    while h < len(q):
        v = q[h]
        h += 1
        for e in range(int(off[v]), int(off[v + 1])):
            u = int(src[e])
            if u not in seen and oracle_mod.ic_live(seed, rr_id, e, float(w[e])):
                seen.add(u)
                q.append(u)
    return seen


def _walk_lt(oracle_mod, g, cum, seed, root, rr_id):
    seen = [root]
    x = root
    while True:
        U = oracle_mod.lt_draw(seed, rr_id, x)
        chosen = next((e for e in range(int(g.offsets[x]), int(g.offsets[x + 1])) if U < int(cum[e])), None)
        if chosen is None:
            break
        u = int(g.sources[chosen])
        if u in seen:
            break
        seen.append(u)
        x = u
    return set(seen)


@pytest.mark.parametrize("model", [0, 1])
def test_t1_reduces_to_imm(oracle_mod, inputs_mod, model):
    g = inputs_mod.wc_weights(inputs_mod.er(2000, 20000, 1))
    a = oracle_mod.Oracle(g)
    r1 = a.mrim(model, 1, 10, 0.5, 1.0, 7)
    b = oracle_mod.Oracle(g)
    r0 = b.imm(model, 10, 0.5, 1.0, 7)
    assert r1["seeds"].tolist() == r0["seeds"].tolist()
    assert (r1["theta"], r1["lb"], r1["rr_count"]) == (r0["theta"], r0["lb"], r0["rr_count"])
    assert r1["rounds"] == r0["rounds"]
    oa, ma = a.export()
    ob, mb = b.export()
    assert np.array_equal(oa, ob) and np.array_equal(ma, mb)
    for n, k in [(2000, 10), (1 << 22, 50)]:
        assert oracle_mod.mrim_constants(n, k, 1, 0.1, 1.0) == oracle_mod.imm_constants(n, k, 0.1, 1.0)


def test_constants_grow_with_rounds(oracle_mod):
    n, k, eps = 1 << 20, 10, 0.1
    c = [oracle_mod.mrim_constants(n, k, T, eps, 1.0) for T in (1, 2, 3, 5, 8)]
    lnC = oracle_mod.log_binom(n, k)
    ep = c[0]["eps_prime"]
    unit = (2 + 2 * ep / 3) * n / ep ** 2   # lambda' is affine in the ln C term with this slope
    for T, ct in zip((2, 3, 5, 8), c[1:]):
        assert ct["lambda_prime"] - c[0]["lambda_prime"] == pytest.approx((T - 1) * lnC * unit, rel=1e-9)
        assert ct["i_max"] == c[0]["i_max"] and ct["eps_prime"] == ep
    assert all(a["lambda_star"] < b["lambda_star"] for a, b in zip(c[1:], c[2:]))


@pytest.mark.parametrize("model,T", [(0, 3), (1, 3), (0, 5)])
def test_multi_round_sets_from_primitives(oracle_mod, inputs_mod, model, T):
    g = inputs_mod.wc_weights(inputs_mod.er(40, 200, 9))
    o = oracle_mod.Oracle(g)
    cum = o.lt_thresholds()
    o.set_rounds(T)
    o.sample(model, SEED, 60, threads=3)
    off, mem = o.export()
    for j in range(60):
        root = oracle_mod.root(SEED, j, g.n)
        want = []
        for t in range(T):
            rid = (t << 32) | j
            part = _bfs_ic(oracle_mod, g, SEED, root, rid) if model == 0 else _walk_lt(oracle_mod, g, cum, SEED, root, rid)
            want += sorted(t * g.n + v for v in part)
        assert mem[off[j]:off[j + 1]].tolist() == want
        assert o.mrim_one(model, T, SEED, j).tolist() == want
        round0 = [x for x in want if x < g.n]
        assert round0 == sorted(o.rr_one(model, SEED, j).tolist())
    cnt = o.counts()
    assert cnt.shape == (g.n * T,) and np.array_equal(cnt, np.bincount(mem, minlength=g.n * T))


def _greedy_brute(sets, U, n, k):
    T = U // n
    covered = [False] * len(sets)
    chosen, gains, per = [], [], [0] * T
    for _ in range(k * T):
        best, bg = None, -1
        for x in range(U):
            if x in chosen or per[x // n] == k:
                continue
            gain = sum(1 for j, s in enumerate(sets) if not covered[j] and x in s)
            if gain > bg:
                best, bg = x, gain
        chosen.append(best)
        gains.append(bg)
        per[best // n] += 1
        for j, s in enumerate(sets):
            if best in s:
                covered[j] = True
    return chosen, gains, sum(covered)


@pytest.mark.parametrize("n,T,k,R,trial", [(6, 3, 2, 40, 0), (5, 2, 1, 25, 1), (4, 4, 4, 30, 2), (7, 2, 3, 3, 3)])
def test_partition_greedy_matches_brute_force(oracle_mod, inputs_mod, n, T, k, R, trial):
    g = inputs_mod.er(n, 2 * n, 100 + trial).with_weights(np.ones(2 * n, np.float32), "ones")
    rng = np.random.default_rng(trial)
    U = n * T
    sets = [sorted(set(rng.choice(U, size=int(rng.integers(1, 5)), replace=False).tolist())) for _ in range(R)]
    o = oracle_mod.Oracle(g)
    o.set_rounds(T)
    o.load_collection(sets)
    s, gains, cov = o.greedy(k)
    bs, bg, bc = _greedy_brute([set(x) for x in sets], U, n, k)
    assert s.tolist() == bs and gains.tolist() == bg and cov == bc
    assert all(sum(1 for x in s if x // n == t) == k for t in range(T))


def _round_reach(R, prob, S_t, n):
    """Pr[u reachable from S_t] for every u, exactly (0 for an empty S_t)."""
    if not S_t:
        return np.zeros(n)
    return np.einsum("w,wu->u", prob, R[:, list(S_t), :].any(axis=1).astype(np.float64))


def _mr_spread(R, prob, seeds, n, T):
    miss = np.ones(n)
    for t in range(T):
        miss *= 1.0 - _round_reach(R, prob, [x - t * n for x in seeds if x // n == t], n)
    return float((1.0 - miss).sum())


@pytest.mark.parametrize("model,gseed", [(0, 51), (1, 53)])
def test_estimate_is_the_exact_multi_round_spread(oracle_mod, inputs_mod, model, gseed):
    if model == 0:
        g = inputs_mod.tiny_graph(7, 13, gseed)
        _, R, prob = exact_ic(g)
    else:
        g = inputs_mod.tiny_graph(7, 12, gseed, weights="lt", max_indeg_sum=1.0)
        _, R, prob = exact_lt(g)
    T, N = 3, 60000
    o = oracle_mod.Oracle(g)
    o.set_rounds(T)
    o.sample(model, SEED, N, threads=4)
    off, mem = o.export()
    rows = np.repeat(np.arange(N), np.diff(off).astype(np.int64))
    for seeds in ([0, g.n + 1, 2 * g.n + 2], [3, 4], [2 * g.n + 5], [1, g.n + 1]):
        hit = np.zeros(N, bool)
        hit[rows[np.isin(mem, seeds)]] = True
        est = g.n * hit.mean()
        exact = _mr_spread(R, prob, seeds, g.n, T)
        p = exact / g.n
        band = 5 * g.n * math.sqrt(max(p * (1 - p), 1e-12) / N)
        assert abs(est - exact) <= band, (seeds, est, exact)


@pytest.mark.parametrize("model,gseed,T,k", [(0, 51, 2, 1), (0, 52, 2, 2), (1, 53, 3, 1)])
def test_quality_against_exact_opt(oracle_mod, inputs_mod, model, gseed, T, k):
    if model == 0:
        g = inputs_mod.tiny_graph(7, 13, gseed)
        _, R, prob = exact_ic(g)
    else:
        g = inputs_mod.tiny_graph(7, 12, gseed, weights="lt", max_indeg_sum=1.0)
        _, R, prob = exact_lt(g)
    eps = 0.3
    n = g.n
    per_round = list(itertools.combinations(range(n), k))
    opt = max(_mr_spread(R, prob, [t * n + v for t, S in enumerate(choice) for v in S], n, T)
              for choice in itertools.product(per_round, repeat=T))
    for s in range(3):
        res = oracle_mod.Oracle(g).mrim(model, T, k, eps, 1.0, 300 + s)
        seeds = res["seeds"].tolist()
        assert len(seeds) == k * T and len(set(seeds)) == k * T
        assert all(sum(1 for x in seeds if x // n == t) == k for t in range(T))
        assert _mr_spread(R, prob, seeds, n, T) >= (0.5 - eps) * opt


def test_mrim_rejects_bad_arguments(oracle_mod, inputs_mod):
    g = inputs_mod.wc_weights(inputs_mod.er(50, 200, 1))
    o = oracle_mod.Oracle(g)
    with pytest.raises(RuntimeError):
        o.mrim(0, 0, 5, 0.5, 1.0, 1)
    with pytest.raises(RuntimeError):
        o.mrim(0, 2, 51, 0.5, 1.0, 1)
    o.sample(0, 1, 10)
    with pytest.raises(RuntimeError):   # the store must start empty
        o.mrim(0, 2, 5, 0.5, 1.0, 1)
