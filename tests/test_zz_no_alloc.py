"""The allocation-free selection entry point agrees with the context-based one.

gim_select_seeds_noalloc serves callers that cannot let a library allocate
device memory (their device memory is reserved up front by their own pool, or
their path cannot afford an allocation's synchronisation); it keeps its
scratch in one fixed array inside the library. Here it is called through the
C ABI on an RR collection held in caller-owned device memory, twice in a row
(the second call finds the first call's leftovers in the shared array), and
must return exactly the seeds, gains and covered count of gim_select_seeds
on the same collection.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def collections():
    from paper_2009_07325_gb300 import build
    build.build()
    from paper_2009_07325_gb300 import GIM_IC, GIM_LT, Context
    from paper_2009_07325_gb300 import inputs as I
    g = I.wc_weights(I.er(2000, 20000, 1))
    out = []
    for model, count in ((GIM_IC, 6000), (GIM_LT, 4000)):
        ctx = Context(0)
        ctx.load(g)
        ctx.sample_rr(model, count, 7)
        out.append((ctx, g.n))
    return out


def _run(ctx, n, k):
    import torch
    from paper_2009_07325_gb300 import binding
    off, mem = ctx.rr_export()
    d_off = torch.from_numpy(off.view(np.int64)).cuda()
    d_mem = torch.from_numpy(mem.view(np.int32)).cuda()
    seeds = torch.full((k,), -1, dtype=torch.int32, device="cuda")
    gains = torch.full((k,), -1, dtype=torch.int32, device="cuda")
    cov = torch.zeros(1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    binding.select_seeds_noalloc(n, off.size - 1, mem.size, d_off.data_ptr(), d_mem.data_ptr(), k,
                                 seeds.data_ptr(), gains.data_ptr(), cov.data_ptr(), stream.cuda_stream)
    stream.synchronize()
    return (seeds.cpu().numpy().view(np.uint32).tolist(), gains.cpu().numpy().view(np.uint32).tolist(),
            int(cov.cpu().item()))


@pytest.mark.parametrize("which", [0, 1])
def test_noalloc_selection_matches_select_seeds_twice(collections, which):
    ctx, n = collections[which]
    for k in (25, 10):                     # two calls in a row on the shared scratch
        got = _run(ctx, n, k)
        s, g, c = ctx.select_seeds(k)
        assert got == (s.tolist(), g.tolist(), c)


def test_noalloc_rejects_sizes_above_the_limit(collections):
    import torch
    from paper_2009_07325_gb300 import binding
    from paper_2009_07325_gb300.binding import GimError
    d = torch.zeros(4, dtype=torch.int64, device="cuda")
    with pytest.raises(GimError, match="limit"):
        binding.select_seeds_noalloc(70000, 1, 1, d.data_ptr(), d.data_ptr(), 5, d.data_ptr())
    with pytest.raises(GimError, match="limit"):
        binding.select_seeds_noalloc(100, 1, 1, d.data_ptr(), d.data_ptr(), 2000, d.data_ptr())
