"""Pins of the oracle's greedy maximum coverage (the maximum-coverage step of Alg. 1).

Checked against brute force on small hand-made and random set systems: each
round's pick maximises the marginal coverage (lowest id on ties), coverage
is at least (1 - 1/e) of the exhaustive optimum (and equal to it for k = 1),
gains never increase and sum to the covered count, and the degenerate cases
(nothing left to cover, empty collection, k = n) behave as stated.
"""
import itertools
import math

import numpy as np
import pytest


def _oracle_for(oracle_mod, inputs_mod, n, sets):
    g = inputs_mod.er(max(n, 2), 1, 0) if n >= 2 else None
    o = oracle_mod.Oracle(g.with_weights(np.zeros(g.m, np.float32), "z"))
    o.load_collection(sets)
    return o


def _brute_greedy(n, sets, k):
    sets = [set(s) for s in sets]
    alive = list(range(len(sets)))
    S, gains = [], []
    for _ in range(k):
        best, bg = None, -1
        for x in range(n):
            if x in S:
                continue
            gain = sum(1 for j in alive if x in sets[j])
            if gain > bg:
                best, bg = x, gain
        S.append(best)
        gains.append(bg)
        alive = [j for j in alive if best not in sets[j]]
    return S, gains, len(sets) - len(alive)


def _random_sets(rng, n, R, pmax=0.5):
    out = []
    for _ in range(R):
        size = int(rng.integers(1, max(2, int(n * pmax)) + 1))
        out.append(sorted(rng.choice(n, size=size, replace=False).tolist()))
    return out


@pytest.mark.parametrize("trial", range(8))
def test_greedy_matches_brute_force_rounds(oracle_mod, inputs_mod, trial):
    rng = np.random.default_rng(100 + trial)
    n, R = 9, 40
    sets = _random_sets(rng, n, R)
    o = _oracle_for(oracle_mod, inputs_mod, n, sets)
    for k in (1, 2, 3, 5, n):
        seeds, gains, cov = o.greedy(k)
        bs, bg, bc = _brute_greedy(n, sets, k)
        assert seeds.tolist() == bs and gains.tolist() == bg and cov == bc


@pytest.mark.parametrize("trial", range(6))
def test_greedy_approximation_ratio(oracle_mod, inputs_mod, trial):
    rng = np.random.default_rng(200 + trial)
    n, R = 10, 30
    sets = _random_sets(rng, n, R, pmax=0.3)
    o = _oracle_for(oracle_mod, inputs_mod, n, sets)
    ss = [set(s) for s in sets]
    for k in (1, 2, 3, 4):
        opt = max(sum(1 for s in ss if s & set(c)) for c in itertools.combinations(range(n), k))
        _, gains, cov = o.greedy(k)
        assert cov >= (1 - math.exp(-1)) * opt - 1e-9
        if k == 1:
            assert cov == opt
        assert all(gains[i] >= gains[i + 1] for i in range(k - 1))
        assert int(gains.sum()) == cov


def test_greedy_lowest_id_on_ties(oracle_mod, inputs_mod):
    o = _oracle_for(oracle_mod, inputs_mod, 6, [[4, 5], [4, 5], [1, 2], [1, 2], [3]])
    seeds, gains, cov = o.greedy(3)
    assert seeds.tolist() == [1, 4, 3] and gains.tolist() == [2, 2, 1] and cov == 5


def test_greedy_zero_gain_rounds(oracle_mod, inputs_mod):
    """Once all sets are covered, the lowest unselected ids follow with gain 0."""
    o = _oracle_for(oracle_mod, inputs_mod, 5, [[3], [3, 4]])
    seeds, gains, cov = o.greedy(4)
    assert seeds.tolist() == [3, 0, 1, 2] and gains.tolist() == [2, 0, 0, 0] and cov == 2


def test_greedy_empty_collection_and_k_equals_n(oracle_mod, inputs_mod):
    o = _oracle_for(oracle_mod, inputs_mod, 4, [])
    seeds, gains, cov = o.greedy(4)
    assert seeds.tolist() == [0, 1, 2, 3] and gains.tolist() == [0, 0, 0, 0] and cov == 0
    with pytest.raises(ValueError):
        o.greedy(5)
    with pytest.raises(ValueError):
        o.greedy(0)


def test_greedy_on_sampled_rr_sets_matches_brute_force(oracle_mod, inputs_mod):
    g = inputs_mod.wc_weights(inputs_mod.er(60, 300, 8))
    o = oracle_mod.Oracle(g)
    o.sample(oracle_mod.IC, 3, 500)
    off, mem = o.export()
    sets = [mem[off[j]:off[j + 1]].tolist() for j in range(500)]
    seeds, gains, cov = o.greedy(6)
    bs, bg, bc = _brute_greedy(g.n, sets, 6)
    assert seeds.tolist() == bs and gains.tolist() == bg and cov == bc
