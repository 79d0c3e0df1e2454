"""Compact collections (GIM_OPT_COMPACT_FIRST_PICK) against the oracle.

After its first selection gim_imm keeps only the size and the occurrence
counts of every later set that holds the first pick. The greedy never reads
those members again (the first pick covers those sets), so the seeds, theta
and LB must equal the oracle's plain IMM, and a run whose first pick changes
after the first selection must fail with GIM_ERR_STATE instead of answering
differently.
"""
import numpy as np
import pytest

import oracle as O
from paper_2009_07325_gb300 import GIM_IC, Context, GimError
from paper_2009_07325_gb300 import binding
from paper_2009_07325_gb300 import inputs as I

pytestmark = pytest.mark.gpu
THREADS = max(1, O.max_threads())


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2009_07325_gb300 import build
    build.build()


def _first_picks(g, seed, res):
    """The oracle's first greedy pick over every prefix the IMM run selects on."""
    picks = []
    for r in res["rounds"] + [dict(rr_count=res["rr_count"])]:
        o = O.Oracle(g)
        o.sample(O.IC, seed, r["rr_count"], THREADS)
        picks.append(int(o.greedy(1)[0][0]))
    return picks


def test_compact_imm_equals_oracle_on_a_supercritical_graph():
    # uniform p = 0.15 on a directed ER graph of mean in-degree 10: mean live
    # in-degree 1.5, so a giant component holds most large RR sets
    g = I.uniform_weights(I.er(3000, 30000, 21), 0.15)
    for seed in range(7, 40):   # a seed whose first pick is the same over every prefix
        want = O.Oracle(g).imm(O.IC, 10, 0.3, 1.0, seed, THREADS)
        if len(want["rounds"]) >= 1 and len(set(_first_picks(g, seed, want))) == 1:
            break
    else:
        pytest.fail("no seed keeps its first pick")
    params = (GIM_IC, 10, 0.3, 1.0, seed)
    plain = Context(0)
    plain.load(g)
    p = plain.imm(*params)
    comp = Context(0)
    comp.load(g)
    comp.set_option(binding.GIM_OPT_COMPACT_FIRST_PICK, 1)
    assert comp.get_option(binding.GIM_OPT_COMPACT_FIRST_PICK) == 1
    c = comp.imm(*params)
    for r in (p, c):
        assert r["seeds"].tolist() == want["seeds"].tolist()
        assert r["theta"] == want["theta"] and r["lb"] == want["lb"] and r["rr_count"] == want["rr_count"]
    # occurrence counts are kept for every set
    assert np.array_equal(comp.coverage(), plain.coverage())
    # sets drawn after the first selection that hold the first pick keep only their size
    off_p, mem_p = plain.rr_export()
    off_c, mem_c, flags = comp.rr_export_compact()
    u1 = int(c["seeds"][0])
    first_R = want["rounds"][0]["rr_count"]
    R = len(off_p) - 1
    assert flags.shape == (R,) and not flags[:first_R].any() and flags.any()
    assert comp.rr_count()[1] < plain.rr_count()[1]
    for j in range(R):
        full = mem_p[off_p[j]:off_p[j + 1]]
        if flags[j]:
            assert j >= first_R and u1 in full and off_c[j + 1] == off_c[j]
            assert comp.rr_info(j) == (len(full), False)
        else:
            assert np.array_equal(mem_c[off_c[j]:off_c[j + 1]], full)
            assert j < first_R or u1 not in full
    with pytest.raises(GimError):
        comp.rr_export()
    j = int(np.nonzero(flags)[0][0])
    with pytest.raises(GimError):
        comp.rr_get(j)
    # a later selection over the same collection (first pick unchanged) still works
    s, gains, cov = comp.select_seeds(10)
    assert s.tolist() == want["seeds"].tolist()


def test_compact_imm_fails_when_the_first_pick_changes():
    # vertices 0 and 1 both reach 2 and 3 with p = 1; 4..7 are isolated, so
    # which of 0 and 1 lies in more sets flips with the roots drawn
    g = I.from_edges(8, [0, 1, 0, 1], [2, 2, 3, 3]).with_weights(np.ones(4, np.float32), "ab")
    changed = kept = None
    for seed in range(1, 200):
        want = O.Oracle(g).imm(O.IC, 1, 0.5, 1.0, seed, 1)
        picks = _first_picks(g, seed, want)
        if len(set(picks)) > 1 and changed is None:
            changed = (seed, want)
        if len(set(picks)) == 1 and kept is None:
            kept = (seed, want)
        if changed and kept:
            break
    assert changed and kept
    for (seed, want), must_fail in ((changed, True), (kept, False)):
        c = Context(0)
        c.load(g)
        c.set_option(binding.GIM_OPT_COMPACT_FIRST_PICK, 1)
        if must_fail:
            with pytest.raises(GimError) as e:
                c.imm(GIM_IC, 1, 0.5, 1.0, seed)
            assert e.value.status == 5   # GIM_ERR_STATE
            # the plain run on the same context gives the oracle's answer
            c.set_option(binding.GIM_OPT_COMPACT_FIRST_PICK, 0)
        r = c.imm(GIM_IC, 1, 0.5, 1.0, seed)
        assert r["seeds"].tolist() == want["seeds"].tolist() and r["theta"] == want["theta"]
