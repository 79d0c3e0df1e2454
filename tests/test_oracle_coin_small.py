"""Pins of the IC coin for in-edges with p <= 2^-8 (a zero-test byte, 16 per
Philox draw, then a 16-bit residual).

On complete bipartite fan-in graphs (every target vertex has in-edges from
all S source vertices, the sources have none; weighted cascade p = 1/S) an
RR set rooted at a target is the root plus each source independently with
probability P = ceil(p 2^24) / 2^24, the exact coin probability of the
reading. Checked: the number of live in-edges against its binomial mean
(5 sigma), their spread over the 16 byte positions of a draw (chi-square),
and pairs inside one draw being live together at rate P^2 (a shared byte
would make them P).
"""
import math

import numpy as np
import pytest

from paper_2009_07325_gb300 import inputs as I


def _fan_in(K, S):
    src = np.tile(np.arange(K, K + S, dtype=np.uint32), K)
    dst = np.repeat(np.arange(K, dtype=np.uint32), S)
    return I.wc_weights(I.from_edges(K + S, src, dst, f"fanin-{K}-{S}"))


def _target_sets(oracle_mod, g, K, N, seed):
    o = oracle_mod.Oracle(g)
    o.sample(oracle_mod.IC, seed, N, threads=4)
    off, mem = o.export()
    roots = np.array([oracle_mod.root(seed, j, g.n) for j in range(N)])
    keep = roots < K
    sets = [mem[off[j]:off[j + 1]] for j in np.nonzero(keep)[0]]
    return [s[s >= K] - K for s in sets]   # live sources, as in-edge positions 0..S-1 of the row


@pytest.mark.parametrize("K,S,N", [(2000, 256, 6000), (1500, 1000, 8000), (500, 4096, 20000)])
def test_small_p_coin_rate(oracle_mod, inputs_mod, K, S, N):
    g = _fan_in(K, S)
    p = float(np.float32(1.0) / np.float32(S))
    assert p <= 2.0 ** -8
    P = math.ceil(p * 2 ** 24) / 2 ** 24
    live = _target_sets(oracle_mod, g, K, N, 13)
    trials = len(live) * S
    hits = sum(len(x) for x in live)
    assert abs(hits - trials * P) < 5 * math.sqrt(trials * P * (1 - P)), (hits, trials * P)
    # every byte position of a draw is used: live edges spread evenly over e mod 16
    pos = np.bincount(np.concatenate(live) % 16, minlength=16) if hits else np.zeros(16)
    exp = hits / 16
    chi2 = float(((pos - exp) ** 2 / exp).sum())
    assert chi2 < 50.0, pos


def test_small_p_edges_of_one_draw_independent(oracle_mod, inputs_mod):
    K, S, N = 2000, 256, 30000
    g = _fan_in(K, S)
    P = math.ceil(float(np.float32(1.0) / np.float32(S)) * 2 ** 24) / 2 ** 24
    live = _target_sets(oracle_mod, g, K, N, 17)
    # each row starts at a multiple of 256, so in-edge position x lies in draw x // 16
    together = 0
    for x in live:
        if len(x) > 1:
            grp = np.bincount(x // 16, minlength=S // 16)
            together += int((grp * (grp - 1) // 2).sum())
    pairs = len(live) * (S // 16) * (16 * 15 // 2)
    mean = pairs * P * P
    assert abs(together - mean) < 5 * math.sqrt(mean) + 1, (together, mean)
