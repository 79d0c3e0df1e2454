"""Pins of the oracle's IMM driver (Alg. 2 then Alg. 1, IMM's constants).

* ln C(n, k) against the library's lgamma and the exact integer binomial.
* Scaling facts of the constants: lambda* is proportional to eps^-2,
  lambda' to (2 + 2 eps'/3) / eps'^2; both grow with k and with ell.
* The lower-bound loop's trace obeys its own definition: x_i = n / 2^i,
  the collection reaches ceil(lambda'/x_i), the stop test fires exactly at
  the first round with n F_R(S) >= (1 + eps') x_i, theta = ceil(lambda*/LB).
* Solution quality: on tiny graphs, with exact expected spreads from
  exhaustive enumeration, IMM's seeds reach (1 - 1/e - eps) OPT.
"""
import itertools
import math

import numpy as np
import pytest

from exact_enum import exact_ic, exact_lt, spread


@pytest.mark.parametrize("n,k", [(2000, 10), (1 << 20, 50), (1 << 22, 100), (7, 3), (10, 10)])
def test_log_binom_matches_library(oracle_mod, n, k):
    got = oracle_mod.log_binom(n, k)
    via_lgamma = math.lgamma(n + 1) - math.lgamma(k + 1) - math.lgamma(n - k + 1)
    assert got == pytest.approx(via_lgamma, rel=1e-11, abs=1e-9)
    if n < 100000:
        assert got == pytest.approx(math.log(math.comb(n, k)), rel=1e-12, abs=1e-12)


def test_constants_scaling(oracle_mod):
    a = oracle_mod.imm_constants(1 << 20, 50, 0.1, 1.0)
    b = oracle_mod.imm_constants(1 << 20, 50, 0.05, 1.0)
    assert b["lambda_star"] / a["lambda_star"] == pytest.approx(4.0, rel=1e-14)
    ea, eb = a["eps_prime"], b["eps_prime"]
    assert ea == pytest.approx(math.sqrt(2) * 0.1, rel=1e-15)
    ratio = ((2 + 2 * eb / 3) / eb ** 2) / ((2 + 2 * ea / 3) / ea ** 2)
    assert b["lambda_prime"] / a["lambda_prime"] == pytest.approx(ratio, rel=1e-13)
    assert a["ell_prime"] == pytest.approx(1 + math.log(2) / math.log(1 << 20), rel=1e-15)
    for key in ("lambda_prime", "lambda_star"):
        lo = oracle_mod.imm_constants(1 << 20, 10, 0.1, 1.0)[key]
        hi = oracle_mod.imm_constants(1 << 20, 100, 0.1, 1.0)[key]
        assert lo < a[key] < hi
        assert oracle_mod.imm_constants(1 << 20, 50, 0.1, 2.0)[key] > a[key]


@pytest.mark.parametrize("n", [2, 3, 4, 7, 8, 2000, 2047, 2048, (1 << 22), (1 << 32) - 2])
def test_i_max_is_floor_log2_minus_one(oracle_mod, n):
    assert oracle_mod.imm_constants(n, 1, 0.5, 1.0)["i_max"] == n.bit_length() - 2


def _check_trace(oracle_mod, g, res, k, eps, ell):
    c = oracle_mod.imm_constants(g.n, k, eps, ell)
    rounds = res["rounds"]
    prev = 0
    passed = False
    for i, r in enumerate(rounds, start=1):
        assert r["x"] == g.n / 2 ** i
        assert r["theta_i"] == math.ceil(c["lambda_prime"] / r["x"])
        assert r["rr_count"] == max(prev, r["theta_i"])
        prev = r["rr_count"]
        est = (g.n * r["covered"]) / r["rr_count"]
        passed = est >= (1 + c["eps_prime"]) * r["x"]
        if i < len(rounds):
            assert not passed
    if passed:
        assert res["lb"] == est / (1 + c["eps_prime"])
    else:
        assert len(rounds) == c["i_max"] and res["lb"] == 1.0
    assert res["theta"] == math.ceil(c["lambda_star"] / res["lb"])
    assert res["rr_count"] == max(res["theta"], prev)


def test_imm_trace_follows_alg2(oracle_mod, inputs_mod):
    g = inputs_mod.wc_weights(inputs_mod.er(2000, 20000, 1))
    o = oracle_mod.Oracle(g)
    res = o.imm(oracle_mod.IC, 10, 0.5, 1.0, 7)
    assert len(res["rounds"]) >= 1
    _check_trace(oracle_mod, g, res, 10, 0.5, 1.0)


def test_imm_trace_lt_and_no_early_stop(oracle_mod, inputs_mod):
    g = inputs_mod.wc_weights(inputs_mod.er(300, 900, 4))
    o = oracle_mod.Oracle(g)
    res = o.imm(oracle_mod.LT, 3, 0.4, 1.0, 11)
    _check_trace(oracle_mod, g, res, 3, 0.4, 1.0)
    # p = 0: every RR set is its root, so coverage stays tiny and the search never stops early
    z = oracle_mod.Oracle(inputs_mod.uniform_weights(inputs_mod.er(64, 128, 4), 0.0))
    rz = z.imm(oracle_mod.IC, 2, 0.5, 1.0, 3)
    _check_trace(oracle_mod, inputs_mod.er(64, 128, 4), rz, 2, 0.5, 1.0)


@pytest.mark.parametrize("model,gseed", [("ic", 51), ("ic", 52), ("lt", 53)])
def test_imm_quality_against_exact_opt(oracle_mod, inputs_mod, model, gseed):
    """E[I(S_IMM)] >= (1 - 1/e - eps) OPT, with every expectation computed exactly."""
    if model == "ic":
        g = inputs_mod.tiny_graph(7, 13, gseed)
        _, R, prob = exact_ic(g)
        mdl = oracle_mod.IC
    else:
        g = inputs_mod.tiny_graph(7, 12, gseed, weights="lt", max_indeg_sum=1.0)
        _, R, prob = exact_lt(g)
        mdl = oracle_mod.LT
    k, eps = 2, 0.3
    opt = max(spread(R, prob, S) for S in itertools.combinations(range(g.n), k))
    for s in range(4):
        o = oracle_mod.Oracle(g)
        res = o.imm(mdl, k, eps, 1.0, 100 + s)
        got = spread(R, prob, res["seeds"].tolist())
        assert got >= (1 - math.exp(-1) - eps) * opt, (got, opt)
        assert len(set(res["seeds"].tolist())) == k


def test_imm_rejects_bad_arguments(oracle_mod, inputs_mod):
    g = inputs_mod.wc_weights(inputs_mod.er(50, 200, 1))
    o = oracle_mod.Oracle(g)
    for k, eps, ell in [(0, 0.5, 1.0), (51, 0.5, 1.0), (5, 0.0, 1.0), (5, 1.0, 1.0), (5, 0.5, 0.0)]:
        with pytest.raises(RuntimeError):
            o.imm(oracle_mod.IC, k, eps, ell, 1)


@pytest.mark.parametrize("model", ["ic", "lt"])
def test_imm_replay_equals_fresh_imm(oracle_mod, inputs_mod, model):
    """IMM over a preloaded collection of RR sets 0, 1, ... (what the full-size
    GPU checks use) takes the same steps as IMM that samples them itself."""
    g = inputs_mod.wc_weights(inputs_mod.er(2000, 20000, 1))
    mdl = oracle_mod.IC if model == "ic" else oracle_mod.LT
    fresh = oracle_mod.Oracle(g).imm(mdl, 10, 0.5, 1.0, 7)
    pool = oracle_mod.Oracle(g)
    pool.sample(mdl, 7, fresh["rr_count"] + 5000, 1)
    off, mem = pool.export()
    rep = oracle_mod.Oracle(g)
    rep.load_csr(off, mem)
    r = rep.imm_replay(10, 0.5, 1.0)
    assert r["seeds"].tolist() == fresh["seeds"].tolist()
    assert (r["theta"], r["lb"], r["rr_count"]) == (fresh["theta"], fresh["lb"], fresh["rr_count"])
    assert r["rounds"] == fresh["rounds"]
    _check_trace(oracle_mod, g, r, 10, 0.5, 1.0)
    # a collection shorter than the theta IMM needs is an error, not a silent answer
    short = oracle_mod.Oracle(g)
    short.load_csr(off[: fresh["rr_count"]], mem[: int(off[fresh["rr_count"] - 1])])
    with pytest.raises(RuntimeError):
        short.imm_replay(10, 0.5, 1.0)


@pytest.mark.parametrize("model", ["ic", "lt"])
def test_imm_fresh_final_phase(oracle_mod, inputs_mod, model):
    """IMM with a fresh final phase: the lower-bound search is IMM's own, and the
    final greedy runs over exactly theta new RR sets whose rr_ids are 2^63 + j."""
    g = inputs_mod.wc_weights(inputs_mod.er(2000, 20000, 1))
    mdl = oracle_mod.IC if model == "ic" else oracle_mod.LT
    base = oracle_mod.Oracle(g).imm(mdl, 10, 0.5, 1.0, 7)
    o = oracle_mod.Oracle(g)
    fr = o.imm_fresh(mdl, 10, 0.5, 1.0, 7)
    assert fr["rounds"] == base["rounds"]
    assert (fr["theta"], fr["lb"]) == (base["theta"], base["lb"])
    assert fr["rr_count"] == fr["theta"]
    off, mem = o.export()
    for j in list(range(0, 40)) + list(range(fr["theta"] - 40, fr["theta"])):
        want = sorted(o.rr_one(mdl, 7, (1 << 63) + j).tolist())
        assert sorted(mem[int(off[j]):int(off[j + 1])].tolist()) == want
    # rr_id 2^63 + j is not rr_id j: the collection is not the search's
    same = sum(sorted(o.rr_one(mdl, 7, j).tolist()) == sorted(o.rr_one(mdl, 7, (1 << 63) + j).tolist())
               for j in range(200))
    assert same < 200
    # the greedy over the fresh sets, rerun from a copy of them, picks the same seeds
    chk = oracle_mod.Oracle(g)
    chk.load_csr(off, mem)
    assert chk.greedy(10)[0].tolist() == fr["seeds"].tolist()


@pytest.mark.parametrize("model,gseed", [("ic", 51), ("lt", 53)])
def test_imm_fresh_quality_against_exact_opt(oracle_mod, inputs_mod, model, gseed):
    """The fresh variant's seeds also reach (1 - 1/e - eps) OPT, with exact spreads."""
    if model == "ic":
        g = inputs_mod.tiny_graph(7, 13, gseed)
        _, R, prob = exact_ic(g)
        mdl = oracle_mod.IC
    else:
        g = inputs_mod.tiny_graph(7, 12, gseed, weights="lt", max_indeg_sum=1.0)
        _, R, prob = exact_lt(g)
        mdl = oracle_mod.LT
    k, eps = 2, 0.3
    opt = max(spread(R, prob, S) for S in itertools.combinations(range(g.n), k))
    for s in range(4):
        res = oracle_mod.Oracle(g).imm_fresh(mdl, k, eps, 1.0, 200 + s)
        assert spread(R, prob, res["seeds"].tolist()) >= (1 - math.exp(-1) - eps) * opt
        assert len(set(res["seeds"].tolist())) == k
