"""Failure handling on the GPU without a fault.

The persistent greedy kernel's group barriers are bounded waits. A
diagnostic launches it with a block group declared as two blocks while only
one runs, so the barrier can never be met: the wait must give up (about
2 s), the call must report GIM_ERR_TIMEOUT, and the context must keep
working (a selection afterwards still matches the oracle).
"""
import numpy as np
import pytest

import oracle as O
from paper_2009_07325_gb300 import GIM_IC, Context
from paper_2009_07325_gb300 import inputs as I

pytestmark = pytest.mark.gpu
GIM_ERR_TIMEOUT = 4


def test_greedy_barrier_wait_gives_up_and_the_context_survives():
    from paper_2009_07325_gb300 import build
    build.build()
    O.build()
    I.build()
    g = I.wc_weights(I.er(2000, 20000, 1))
    ctx = Context(0)
    ctx.load(g)
    status, ms = ctx.diag_barrier_timeout()
    assert status == GIM_ERR_TIMEOUT
    assert 100.0 < ms < 30000.0
    ctx.sample_rr(GIM_IC, 3000, 7)
    orc = O.Oracle(g)
    orc.sample(GIM_IC, 7, 3000, 1)
    s, gains, cov = ctx.select_seeds(10)
    os_, og, oc = orc.greedy(10)
    assert s.tolist() == os_.tolist() and gains.tolist() == og.tolist() and cov == oc
    ctx.close()
