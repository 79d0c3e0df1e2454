"""Seeded synthetic inputs: graphs, edge weights and query mixes.

This module holds no part of the influence-maximisation method. It builds the
graphs the method runs on (in-edge CSR by target vertex, sources ascending
within a row, duplicates and self-loops dropped) and their edge probabilities,
and it is shared by the tests, the benchmark and the CPU oracle so that every
side reads identical bytes.

Workload recipes (stand-ins for the SNAP social graphs of the paper's
Table 1, which are not available here):

* ``er(n, m, seed)``: directed Erdos-Renyi, exactly m distinct edges.
* ``rmat(scale, seed)``: R-MAT with 16 * 2^scale quadrant draws and
  (a, b, c, d) = (0.57, 0.19, 0.19, 0.05); the kept edge count is smaller.
* ``chung_lu(n, seed)``: power law with degree exponent 2.1, mean degree 8
  before duplicate removal.
* ``barabasi_albert(n, r, seed)``: the paper's Sec. IV-F scalability graphs.
* ``wc_weights``: weighted cascade p(u,v) = 1/indeg(v) in fp32 (Sec. IV-B),
  usable under both IC and LT; ``uniform_weights``: a constant p.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_SO = os.path.join(_HERE, "libgimgen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the generator library in-tree with gcc (OpenMP when available)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-shared", "-fPIC", "-std=c11", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:2] + ["-fopenmp"] + base[2:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _SO)
    return _SO


def _l():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
            u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
            lib.gg_build_in_csr.restype = ctypes.c_int64
            lib.gg_build_in_csr.argtypes = [ctypes.c_uint32, ctypes.c_uint64, u32p, u32p, u64p, u32p]
            lib.gg_rmat_edges.restype = None
            lib.gg_rmat_edges.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_uint64, u32p, u32p]
            lib.gg_er_edges.restype = ctypes.c_int
            lib.gg_er_edges.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, u32p, u32p]
            lib.gg_chung_lu_edges.restype = ctypes.c_int
            lib.gg_chung_lu_edges.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double,
                                              ctypes.c_uint64, u32p, u32p]
            lib.gg_barabasi_albert_edges.restype = ctypes.c_int64
            lib.gg_barabasi_albert_edges.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                                     ctypes.c_uint64, u32p, u32p]
            lib.gg_u64.restype = None
            lib.gg_u64.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, u64p]
            _lib = lib
    return _lib


@dataclasses.dataclass
class Graph:
    """Directed graph as an in-edge CSR: row v holds the sources u of edges u->v."""

    n: int
    offsets: np.ndarray          # uint64[n+1]
    sources: np.ndarray          # uint32[m], ascending within each row
    weights: np.ndarray | None = None   # float32[m], p(u,v) on the in-edge
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.offsets[-1])

    def indegree(self) -> np.ndarray:
        return np.diff(self.offsets).astype(np.int64)

    def with_weights(self, w: np.ndarray, suffix: str) -> "Graph":
        return Graph(self.n, self.offsets, self.sources, np.ascontiguousarray(w, dtype=np.float32),
                     f"{self.name}/{suffix}")


def from_edges(n: int, src, dst, name: str = "") -> Graph:
    """Deduplicated in-edge CSR of the directed edges src[i] -> dst[i]."""
    src = np.ascontiguousarray(src, dtype=np.uint32)
    dst = np.ascontiguousarray(dst, dtype=np.uint32)
    assert src.shape == dst.shape
    if src.size and (int(src.max()) >= n or int(dst.max()) >= n):
        raise ValueError("edge endpoint out of range")
    off = np.zeros(n + 1, dtype=np.uint64)
    out = np.zeros(max(src.size, 1), dtype=np.uint32)
    m = _l().gg_build_in_csr(n, src.size, src if src.size else np.zeros(1, np.uint32),
                             dst if dst.size else np.zeros(1, np.uint32), off, out)
    if m < 0:
        raise MemoryError("graph build failed")
    return Graph(n, off, out[:m].copy(), None, name)


def er(n: int, m: int, seed: int) -> Graph:
    src = np.zeros(m, np.uint32)
    dst = np.zeros(m, np.uint32)
    if _l().gg_er_edges(n, m, seed, src, dst) != 0:
        raise ValueError("bad Erdos-Renyi arguments")
    return from_edges(n, src, dst, f"er-n{n}-m{m}-s{seed}")


def rmat(scale: int, seed: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19,
         c: float = 0.19) -> Graph:
    n = 1 << scale
    D = edge_factor * n
    src = np.empty(D, np.uint32)
    dst = np.empty(D, np.uint32)
    _l().gg_rmat_edges(scale, D, a, b, c, seed, src, dst)
    g = from_edges(n, src, dst, f"rmat{scale}-s{seed}")
    return g


def chung_lu(n: int, seed: int, gamma: float = 2.1, mean_degree: float = 8.0) -> Graph:
    D = int(round(mean_degree * n))
    src = np.empty(D, np.uint32)
    dst = np.empty(D, np.uint32)
    if _l().gg_chung_lu_edges(n, D, gamma, seed, src, dst) != 0:
        raise MemoryError("Chung-Lu draw failed")
    return from_edges(n, src, dst, f"chunglu-n{n}-s{seed}")


def barabasi_albert(n: int, r: int, seed: int, r0: int | None = None) -> Graph:
    r0 = max(r, 2) if r0 is None else r0
    E = r0 * (r0 - 1) + 2 * (n - r0) * r
    src = np.empty(E, np.uint32)
    dst = np.empty(E, np.uint32)
    got = _l().gg_barabasi_albert_edges(n, r0, r, seed, src, dst)
    if got < 0:
        raise ValueError("bad Barabasi-Albert arguments")
    return from_edges(n, src[:got], dst[:got], f"ba-n{n}-r{r}-s{seed}")


def wc_weights(g: Graph) -> Graph:
    """Weighted cascade: every in-edge of v gets 1/indeg(v), rounded to fp32."""
    d = g.indegree()
    per_row = np.zeros(g.n, np.float32)
    nz = d > 0
    per_row[nz] = np.float32(1.0) / d[nz].astype(np.float32)
    return g.with_weights(np.repeat(per_row, d), "wc")


def uniform_weights(g: Graph, p: float) -> Graph:
    return g.with_weights(np.full(g.m, p, np.float32), f"p{p}")


def u64_stream(seed: int, stream: int, count: int) -> np.ndarray:
    out = np.zeros(max(count, 1), np.uint64)
    _l().gg_u64(seed, stream, count, out)
    return out[:count]


def tiny_graph(n: int, m: int, seed: int, weights: str = "random", max_indeg_sum: float = 1.0) -> Graph:
    """Small random graph for exhaustive checks.

    weights="random" draws p(u,v) on a 1/16 grid in (0, 1]; "lt" draws weights
    on the same grid and scales each row so its sum is at most max_indeg_sum.
    """
    g = er(n, m, seed)
    r = u64_stream(seed, 77, g.m)
    grid = ((r >> np.uint64(60)).astype(np.int64) + 1).astype(np.float32) / np.float32(16.0)
    if weights == "lt":
        d = g.indegree()
        rows = np.repeat(np.arange(g.n), d)
        sums = np.bincount(rows, weights=grid.astype(np.float64), minlength=g.n)
        scale = np.where(sums > max_indeg_sum, max_indeg_sum / np.maximum(sums, 1e-300), 1.0)
        # round down the scaled weights onto a 1/64 grid so row sums stay <= the bound exactly
        w = np.floor(grid.astype(np.float64) * scale[rows] * 64.0) / 64.0
        grid = w.astype(np.float32)
    return g.with_weights(grid, weights)
