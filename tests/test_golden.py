"""Stored values from tests/golden/oracle_er64.json (written by
tests/golden/make_golden.py, which calls only the oracle).

CPU: the oracle reproduces them on this machine (a regression pin: the same
values must come out of the x86 host and the Arm GPU host). GPU: the library
reproduces them through the C ABI.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2009_07325_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = json.load(open(os.path.join(HERE, "golden", "oracle_er64.json")))
SEED = GOLDEN["philox_seed"]
MODELS = {"IC": O.IC, "LT": O.LT}


def _graph(inputs_mod):
    return inputs_mod.wc_weights(inputs_mod.er(64, 256, 9))


@pytest.mark.parametrize("name", ["IC", "LT"])
def test_oracle_reproduces_golden(oracle_mod, inputs_mod, name):
    g = _graph(inputs_mod)
    want = GOLDEN["models"][name]
    o = oracle_mod.Oracle(g)
    o.sample(MODELS[name], SEED, 100, 1)
    off, mem = o.export()
    assert [sorted(mem[off[j]:off[j + 1]].tolist()) for j in range(100)] == want["rr_sets"]
    s, gains, cov = o.greedy(5)
    assert (s.tolist(), gains.tolist(), cov) == (want["greedy_k5"]["seeds"], want["greedy_k5"]["gains"],
                                                 want["greedy_k5"]["covered"])
    r = oracle_mod.Oracle(g).imm(MODELS[name], 3, 0.5, 1.0, SEED)
    w = want["imm_k3_eps05"]
    assert (r["seeds"].tolist(), r["theta"], r["lb"], r["rr_count"]) == (w["seeds"], w["theta"], w["lb"],
                                                                        w["rr_count"])


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["IC", "LT"])
def test_library_reproduces_golden(name):
    from paper_2009_07325_gb300 import Context, build
    build.build()
    I.build()
    g = I.wc_weights(I.er(64, 256, 9))
    want = GOLDEN["models"][name]
    ctx = Context(0)
    ctx.load(g)
    ctx.sample_rr(MODELS[name], 100, SEED)
    off, mem = ctx.rr_export()
    assert [mem[off[j]:off[j + 1]].tolist() for j in range(100)] == want["rr_sets"]
    s, gains, cov = ctx.select_seeds(5)
    assert (s.tolist(), gains.tolist(), cov) == (want["greedy_k5"]["seeds"], want["greedy_k5"]["gains"],
                                                 want["greedy_k5"]["covered"])
    r = ctx.imm(MODELS[name], 3, 0.5, 1.0, SEED)
    w = want["imm_k3_eps05"]
    assert (r["seeds"].tolist(), r["theta"], r["lb"], r["rr_count"]) == (w["seeds"], w["theta"], w["lb"],
                                                                        w["rr_count"])
    ctx.close()
