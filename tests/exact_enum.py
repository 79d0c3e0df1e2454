"""Exhaustive live-edge enumeration on tiny graphs (shared by the CPU pins).

IC: all 2^m worlds, each edge kept with its probability. LT: every vertex
keeps at most one in-edge, edge e with probability w[e] and none with
1 - (row sum). In each world the reflexive-transitive closure gives who
reaches whom; weighting by the world probabilities gives exact reach
probabilities and exact expected spreads E[I(S)].
"""
import itertools

import numpy as np


def edges(g):
    d = g.indegree()
    dst = np.repeat(np.arange(g.n), d)
    return g.sources.astype(np.int64), dst, g.weights.astype(np.float64)


def closure(A):
    """Reflexive-transitive closure of a batch of boolean adjacency matrices."""
    W, n, _ = A.shape
    R = (A | np.eye(n, dtype=bool)[None]).astype(np.int32)
    for _ in range(int(np.ceil(np.log2(max(n, 2)))) + 1):
        R = (np.matmul(R, R) > 0).astype(np.int32)
    return R.astype(bool)


def exact_ic(g):
    """Pr[u reaches v] over all 2^m live-edge worlds, and per-world closures + probs."""
    src, dst, p = edges(g)
    m, n = len(src), g.n
    masks = np.arange(1 << m, dtype=np.int64)
    live = ((masks[:, None] >> np.arange(m)) & 1).astype(bool)
    prob = np.prod(np.where(live, p[None], 1.0 - p[None]), axis=1)
    A = np.zeros((len(masks), n, n), bool)
    for e in range(m):
        A[:, src[e], dst[e]] |= live[:, e]
    R = closure(A)
    return np.einsum("w,wuv->uv", prob, R.astype(np.float64)), R, prob


def exact_lt(g):
    """Exact Pr[u reaches v] in the LT live-edge model: each vertex keeps at most one in-edge."""
    src, dst, p = edges(g)
    n = g.n
    off = g.offsets.astype(np.int64)
    choices = []
    for v in range(n):
        opts = [(-1, 1.0 - float(p[off[v]:off[v + 1]].sum()))]
        opts += [(e, float(p[e])) for e in range(off[v], off[v + 1])]
        choices.append(opts)
    worlds = list(itertools.product(*choices))
    A = np.zeros((len(worlds), n, n), bool)
    prob = np.zeros(len(worlds))
    for wi, world in enumerate(worlds):
        pr = 1.0
        for v, (e, q) in enumerate(world):
            pr *= q
            if e >= 0:
                A[wi, src[e], v] = True
        prob[wi] = pr
    R = closure(A)
    return np.einsum("w,wuv->uv", prob, R.astype(np.float64)), R, prob



def spread(R, prob, S):
    """Exact E[I(S)]: expected number of vertices reachable from S."""
    return float(np.einsum("w,w->", prob, R[:, list(S), :].any(axis=1).sum(axis=1).astype(np.float64)))
