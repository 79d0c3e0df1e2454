"""CPU oracle for IMM RR-set sampling and greedy max coverage.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only code that may load or run this
package. The library path never imports it. The arithmetic lives in
``gim_oracle.c`` (plain sequential C, each function citing the paper passage
it follows); this module only compiles it with gcc and marshals arguments.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gim_oracle.c")
_SO = os.path.join(_HERE, "libgim_oracle.so")
_lock = threading.Lock()
_lib = None

IC, LT = 0, 1


def build(force: bool = False) -> str:
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    # -ffp-contract=off keeps every fp64 operation a separately rounded IEEE op
    base = ["gcc", "-O2", "-ffp-contract=off", "-shared", "-fPIC", "-std=c11", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:3] + ["-fopenmp"] + base[3:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _SO)
    return _SO


def _lib_():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
            u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
            f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
            f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
            vp = ctypes.c_void_p
            L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.orc_philox4x32_10.restype = None
            L.orc_root.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32]
            L.orc_root.restype = ctypes.c_uint32
            L.orc_ic_live.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_float]
            L.orc_ic_live.restype = ctypes.c_int
            L.orc_lt_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32]
            L.orc_lt_draw.restype = ctypes.c_uint32
            L.orc_create.argtypes = [ctypes.c_uint32, ctypes.c_uint64, u64p, u32p, f32p]
            L.orc_create.restype = vp
            L.orc_destroy.argtypes = [vp]
            L.orc_destroy.restype = None
            L.orc_lt_valid.argtypes = [vp]
            L.orc_lt_valid.restype = ctypes.c_int
            L.orc_lt_export.argtypes = [vp, u64p]
            L.orc_lt_export.restype = None
            L.orc_rr_one.argtypes = [vp, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, u32p]
            L.orc_rr_one.restype = ctypes.c_int64
            L.orc_sample.argtypes = [vp, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int]
            L.orc_sample.restype = ctypes.c_int
            L.orc_load_collection.argtypes = [vp, ctypes.c_uint64, u64p, u32p]
            L.orc_load_collection.restype = ctypes.c_int
            L.orc_reset.argtypes = [vp]
            L.orc_reset.restype = None
            L.orc_rr_count.argtypes = [vp]
            L.orc_rr_count.restype = ctypes.c_uint64
            L.orc_store_size.argtypes = [vp]
            L.orc_store_size.restype = ctypes.c_uint64
            L.orc_export.argtypes = [vp, u64p, u32p]
            L.orc_export.restype = None
            L.orc_counts.argtypes = [vp, u32p]
            L.orc_counts.restype = None
            L.orc_greedy.argtypes = [vp, ctypes.c_uint32, u32p, u32p]
            L.orc_greedy.restype = ctypes.c_int64
            L.orc_log_binom.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
            L.orc_log_binom.restype = ctypes.c_double
            L.orc_imm_constants.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double, ctypes.c_double,
                                            f64p]
            L.orc_imm_constants.restype = None
            L.orc_imm.argtypes = [vp, ctypes.c_int, ctypes.c_uint32, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_uint64, ctypes.c_int, u32p, u64p, f64p, f64p]
            L.orc_imm.restype = ctypes.c_int
            L.orc_imm_fresh.argtypes = [vp, ctypes.c_int, ctypes.c_uint32, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_uint64, ctypes.c_int, u32p, u64p, f64p, f64p]
            L.orc_imm_fresh.restype = ctypes.c_int
            L.orc_mrim.argtypes = [vp, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_uint64, ctypes.c_int, u32p, u64p, f64p, f64p]
            L.orc_mrim.restype = ctypes.c_int
            L.orc_mrim_one.argtypes = [vp, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, u32p]
            L.orc_mrim_one.restype = ctypes.c_int64
            L.orc_mrim_constants.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double,
                                             ctypes.c_double, f64p]
            L.orc_mrim_constants.restype = None
            L.orc_set_rounds.argtypes = [vp, ctypes.c_uint32]
            L.orc_set_rounds.restype = ctypes.c_int
            L.orc_rounds.argtypes = [vp]
            L.orc_rounds.restype = ctypes.c_uint32
            L.orc_imm_replay.argtypes = [vp, ctypes.c_uint32, ctypes.c_double, ctypes.c_double, u32p, u64p, f64p,
                                         f64p]
            L.orc_imm_replay.restype = ctypes.c_int
            L.orc_max_threads.argtypes = []
            L.orc_max_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def philox4x32_10(ctr, key) -> np.ndarray:
    out = np.zeros(4, np.uint32)
    _lib_().orc_philox4x32_10(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


def root(seed: int, j: int, n: int) -> int:
    return int(_lib_().orc_root(seed, j, n))


def ic_live(seed: int, j: int, e: int, p: float) -> bool:
    return bool(_lib_().orc_ic_live(seed, j, e, p))


def lt_draw(seed: int, j: int, x: int) -> int:
    return int(_lib_().orc_lt_draw(seed, j, x))


def log_binom(n: int, k: int) -> float:
    return float(_lib_().orc_log_binom(n, k))


def imm_constants(n: int, k: int, eps: float, ell: float) -> dict:
    out = np.zeros(5, np.float64)
    _lib_().orc_imm_constants(n, k, eps, ell, out)
    return dict(ell_prime=out[0], eps_prime=out[1], lambda_prime=out[2], lambda_star=out[3], i_max=int(out[4]))


def mrim_constants(n: int, k: int, T: int, eps: float, ell: float) -> dict:
    out = np.zeros(5, np.float64)
    _lib_().orc_mrim_constants(n, k, T, eps, ell, out)
    return dict(ell_prime=out[0], eps_prime=out[1], lambda_prime=out[2], lambda_star=out[3], i_max=int(out[4]))


def max_threads() -> int:
    return int(_lib_().orc_max_threads())


class Oracle:
    """One graph plus an RR collection, mirroring the library's context."""

    def __init__(self, graph):
        self.L = _lib_()
        self.n = int(graph.n)
        self.m = int(graph.m)
        off = np.ascontiguousarray(graph.offsets, np.uint64)
        src = np.ascontiguousarray(graph.sources, np.uint32) if self.m else np.zeros(1, np.uint32)
        w = np.ascontiguousarray(graph.weights, np.float32) if self.m else np.zeros(1, np.float32)
        self.h = self.L.orc_create(self.n, self.m, off, src, w)
        if not self.h:
            raise MemoryError("oracle allocation failed")

    def close(self):
        if self.h:
            self.L.orc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def lt_valid(self) -> bool:
        return bool(self.L.orc_lt_valid(self.h))

    def lt_thresholds(self) -> np.ndarray:
        out = np.zeros(max(self.m, 1), np.uint64)
        self.L.orc_lt_export(self.h, out)
        return out[: self.m]

    def rr_one(self, model: int, seed: int, j: int) -> np.ndarray:
        out = np.zeros(self.n, np.uint32)
        s = self.L.orc_rr_one(self.h, model, seed, j, out)
        if s < 0:
            raise ValueError(f"rr_one failed ({s})")
        return out[:s].copy()

    def sample(self, model: int, seed: int, count: int, threads: int = 1) -> None:
        rc = self.L.orc_sample(self.h, model, seed, count, threads)
        if rc:
            raise RuntimeError(f"oracle sample failed ({rc})")

    def load_collection(self, sets) -> None:
        """Replace R with hand-built RR sets (a list of vertex lists)."""
        sizes = np.array([len(s) for s in sets], np.uint64)
        off = np.zeros(len(sets) + 1, np.uint64)
        off[1:] = np.cumsum(sizes)
        mem = np.array([x for s in sets for x in s] or [0], np.uint32)
        if self.L.orc_load_collection(self.h, len(sets), off, mem) != 0:
            raise ValueError("bad collection")

    def load_csr(self, offsets, members) -> None:
        """Replace R with the collection given as CSR arrays (offsets: |R|+1, members)."""
        off = np.ascontiguousarray(offsets, np.uint64)
        mem = np.ascontiguousarray(members, np.uint32) if len(members) else np.zeros(1, np.uint32)
        if self.L.orc_load_collection(self.h, len(off) - 1, off, mem) != 0:
            raise ValueError("bad collection")

    def imm_fresh(self, model: int, k: int, eps: float, ell: float, seed: int, threads: int = 1):
        """IMM whose final greedy runs over theta fresh RR sets (rr_ids 2^63 + j)."""
        seeds = np.zeros(k, np.uint32)
        theta = np.zeros(1, np.uint64)
        lb = np.zeros(1, np.float64)
        trace = np.zeros(4 * 64, np.float64)
        rc = self.L.orc_imm_fresh(self.h, model, k, eps, ell, seed, threads, seeds, theta, lb, trace)
        if rc < 0:
            raise RuntimeError(f"oracle fresh imm failed ({rc})")
        tr = trace[: 4 * min(rc, 64)].reshape(-1, 4)
        rounds = [dict(x=r[0], theta_i=int(r[1]), covered=int(r[2]), rr_count=int(r[3])) for r in tr]
        return dict(seeds=seeds, theta=int(theta[0]), lb=float(lb[0]), rounds=rounds, rr_count=self.rr_count)

    def mrim(self, model: int, T: int, k: int, eps: float, ell: float, seed: int, threads: int = 1):
        """Multi-round IM (CR-NAIMM): k*T seeds t*n + v in pick order."""
        seeds = np.zeros(k * T, np.uint32)
        theta = np.zeros(1, np.uint64)
        lb = np.zeros(1, np.float64)
        trace = np.zeros(4 * 64, np.float64)
        rc = self.L.orc_mrim(self.h, model, T, k, eps, ell, seed, threads, seeds, theta, lb, trace)
        if rc < 0:
            raise RuntimeError(f"oracle mrim failed ({rc})")
        tr = trace[: 4 * min(rc, 64)].reshape(-1, 4)
        rounds = [dict(x=r[0], theta_i=int(r[1]), covered=int(r[2]), rr_count=int(r[3])) for r in tr]
        return dict(seeds=seeds, theta=int(theta[0]), lb=float(lb[0]), rounds=rounds, rr_count=self.rr_count)

    def mrim_one(self, model: int, T: int, seed: int, j: int) -> np.ndarray:
        out = np.zeros(self.n * T, np.uint32)
        s = self.L.orc_mrim_one(self.h, model, T, seed, j, out)
        if s < 0:
            raise ValueError(f"mrim_one failed ({s})")
        return out[:s].copy()

    def imm_replay(self, k: int, eps: float, ell: float):
        """IMM (Alg. 2 then Alg. 1) with every sampling step served by a prefix of
        the loaded collection; |R| is left at the prefix IMM used."""
        seeds = np.zeros(k * self.rounds, np.uint32)
        theta = np.zeros(1, np.uint64)
        lb = np.zeros(1, np.float64)
        trace = np.zeros(4 * 64, np.float64)
        rc = self.L.orc_imm_replay(self.h, k, eps, ell, seeds, theta, lb, trace)
        if rc < 0:
            raise RuntimeError(f"oracle imm replay failed ({rc})")
        tr = trace[: 4 * min(rc, 64)].reshape(-1, 4)
        rounds = [dict(x=r[0], theta_i=int(r[1]), covered=int(r[2]), rr_count=int(r[3])) for r in tr]
        return dict(seeds=seeds, theta=int(theta[0]), lb=float(lb[0]), rounds=rounds, rr_count=self.rr_count)

    def reset(self) -> None:
        self.L.orc_reset(self.h)

    @property
    def rr_count(self) -> int:
        return int(self.L.orc_rr_count(self.h))

    @property
    def store_size(self) -> int:
        return int(self.L.orc_store_size(self.h))

    def export(self):
        R = self.rr_count
        off = np.zeros(R + 1, np.uint64)
        mem = np.zeros(max(self.store_size, 1), np.uint32)
        self.L.orc_export(self.h, off, mem)
        return off, mem[: self.store_size]

    @property
    def rounds(self) -> int:
        return int(self.L.orc_rounds(self.h))

    def set_rounds(self, T: int) -> None:
        """T rounds for an empty collection (multi-round sets, or before loading one)."""
        if self.L.orc_set_rounds(self.h, T) != 0:
            raise ValueError("set_rounds needs an empty collection and n*T < 2^32 - 1")

    def counts(self) -> np.ndarray:
        out = np.zeros(self.n * self.rounds, np.uint32)
        self.L.orc_counts(self.h, out)
        return out

    def greedy(self, k: int):
        """k seeds (k per round, k*T picks, when the collection has T > 1 rounds)."""
        kt = k * self.rounds
        seeds = np.zeros(kt, np.uint32)
        gains = np.zeros(kt, np.uint32)
        cov = self.L.orc_greedy(self.h, k, seeds, gains)
        if cov < 0:
            raise ValueError("greedy failed")
        return seeds, gains, int(cov)

    def imm(self, model: int, k: int, eps: float, ell: float, seed: int, threads: int = 1):
        seeds = np.zeros(k, np.uint32)
        theta = np.zeros(1, np.uint64)
        lb = np.zeros(1, np.float64)
        trace = np.zeros(4 * 64, np.float64)
        rc = self.L.orc_imm(self.h, model, k, eps, ell, seed, threads, seeds, theta, lb, trace)
        if rc < 0:
            raise RuntimeError(f"oracle imm failed ({rc})")
        tr = trace[: 4 * min(rc, 64)].reshape(-1, 4)
        rounds = [dict(x=r[0], theta_i=int(r[1]), covered=int(r[2]), rr_count=int(r[3])) for r in tr]
        return dict(seeds=seeds, theta=int(theta[0]), lb=float(lb[0]), rounds=rounds, rr_count=self.rr_count)
