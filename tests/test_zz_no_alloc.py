"""The allocation-free selection entry point agrees with the oracle and with
the context-based one.

gim_select_seeds_noalloc serves callers that cannot let a library allocate
device memory (their device memory is reserved up front by their own pool, or
their path cannot afford an allocation's synchronisation); it keeps its
scratch in one fixed array inside the library. Here it is called through the
C ABI on RR collections held in caller-owned device memory, twice in a row
(the second call finds the first call's leftovers in the shared array), and
must return exactly the seeds, gains and covered count of the oracle's greedy
(Alg. 1, lowest id on ties) and of gim_select_seeds on the same collection.
The cases cover n divisible by 4 and not (the argmax kernel's vector body and
its scalar tail), n below 4, and an empty collection (every gain 0, the
lowest ids in order).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def collections(oracle_mod):
    from paper_2009_07325_gb300 import build
    build.build()
    from paper_2009_07325_gb300 import GIM_IC, GIM_LT, Context
    from paper_2009_07325_gb300 import inputs as I
    out = []
    for n, model, count in ((2000, GIM_IC, 6000), (2000, GIM_LT, 4000), (1999, GIM_IC, 5000)):
        g = I.wc_weights(I.er(n, 10 * n, 1))
        ctx = Context(0)
        ctx.load(g)
        ctx.sample_rr(model, count, 7)
        out.append((ctx, g))
    return out


def _run(n, off, mem, k):
    import torch
    from paper_2009_07325_gb300 import binding
    d_off = torch.from_numpy(np.ascontiguousarray(off, np.uint64).view(np.int64)).cuda()
    d_mem = torch.from_numpy(np.ascontiguousarray(mem if len(mem) else np.zeros(1, np.uint32),
                                                  np.uint32).view(np.int32)).cuda()
    seeds = torch.full((k,), -1, dtype=torch.int32, device="cuda")
    gains = torch.full((k,), -1, dtype=torch.int32, device="cuda")
    cov = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    binding.select_seeds_noalloc(n, len(off) - 1, len(mem), d_off.data_ptr(), d_mem.data_ptr(), k,
                                 seeds.data_ptr(), gains.data_ptr(), cov.data_ptr(), stream.cuda_stream)
    stream.synchronize()
    return (seeds.cpu().numpy().view(np.uint32).tolist(), gains.cpu().numpy().view(np.uint32).tolist(),
            int(cov.cpu().item()))


def _oracle_greedy(oracle_mod, g, off, mem, k):
    o = oracle_mod.Oracle(g)
    o.load_csr(off, mem)
    s, gn, c = o.greedy(k)
    o.close()
    return s.tolist(), gn.tolist(), c


@pytest.mark.parametrize("which", [0, 1, 2])
def test_noalloc_selection_matches_oracle_and_select_seeds_twice(oracle_mod, collections, which):
    ctx, g = collections[which]
    off, mem = ctx.rr_export()
    for k in (25, 10):                     # two calls in a row on the shared scratch
        got = _run(g.n, off, mem, k)
        assert got == _oracle_greedy(oracle_mod, g, off, mem, k)
        s, gn, c = ctx.select_seeds(k)
        assert got == (s.tolist(), gn.tolist(), c)


def test_noalloc_tiny_and_empty_collections(oracle_mod, collections):
    from paper_2009_07325_gb300 import inputs as I
    g3 = I.wc_weights(I.from_edges(3, np.array([0, 1], np.uint32), np.array([1, 2], np.uint32), "path3"))
    sets = [[2], [1, 2], [0, 1, 2], [1], [2]]
    off = np.zeros(len(sets) + 1, np.uint64)
    off[1:] = np.cumsum([len(s) for s in sets])
    mem = np.array([x for s in sets for x in s], np.uint32)
    for k in (3, 2):
        assert _run(3, off, mem, k) == _oracle_greedy(oracle_mod, g3, off, mem, k)
    # no RR sets at all: gains 0, the lowest ids in order, nothing covered
    empty_off = np.zeros(1, np.uint64)
    empty_mem = np.zeros(0, np.uint32)
    for n, k in ((3, 3), (1999, 7)):
        got = _run(n, empty_off, empty_mem, k)
        assert got == (list(range(k)), [0] * k, 0)
    assert _run(3, empty_off, empty_mem, 2) == _oracle_greedy(oracle_mod, g3, empty_off, empty_mem, 2)


def test_noalloc_rejects_sizes_above_the_limit(collections):
    import torch
    from paper_2009_07325_gb300 import binding
    from paper_2009_07325_gb300.binding import GimError
    d = torch.zeros(4, dtype=torch.int64, device="cuda")
    with pytest.raises(GimError, match="limit"):
        binding.select_seeds_noalloc(70000, 1, 1, d.data_ptr(), d.data_ptr(), 5, d.data_ptr())
    with pytest.raises(GimError, match="limit"):
        binding.select_seeds_noalloc(100, 1, 1, d.data_ptr(), d.data_ptr(), 2000, d.data_ptr())
