"""Thin ctypes binding of libgim's C ABI (include/gim.h).

Argument marshalling only: every step of sampling, selection and IMM runs in
libgim's CUDA kernels. There is no fallback: if libgim.so has not been built
(``__graft_entry__.build()`` or ``python -m paper_2009_07325_gb300.build``)
or no CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgim.so")

GIM_IC, GIM_LT = 0, 1
GIM_OPT_GROUP_BUDGET = 0
GIM_OPT_LARGE_PASS_BYTES = 1
GIM_OPT_FRESH_FINAL = 2
GIM_OPT_FRONTIER_BATCH = 3
GIM_OPT_CHUNK_GROUPS = 4
GIM_OPT_QUEUE_CAP = 5
GIM_OPT_COMPACT_FIRST_PICK = 6
SCHEDULE_OPTIONS = {"group_budget": GIM_OPT_GROUP_BUDGET, "chunk_groups": GIM_OPT_CHUNK_GROUPS,
                    "frontier_batch": GIM_OPT_FRONTIER_BATCH, "queue_cap": GIM_OPT_QUEUE_CAP}
STATUS = {0: "GIM_OK", 1: "GIM_ERR_ARG", 2: "GIM_ERR_OOM", 3: "GIM_ERR_CUDA", 4: "GIM_ERR_TIMEOUT",
          5: "GIM_ERR_STATE"}

_lock = threading.Lock()
_lib = None

_c_u32p = ctypes.POINTER(ctypes.c_uint32)
_c_u64p = ctypes.POINTER(ctypes.c_uint64)
_c_f32p = ctypes.POINTER(ctypes.c_float)
_c_f64p = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p

class ImmParams(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int), ("k", ctypes.c_uint32), ("eps", ctypes.c_double), ("ell", ctypes.c_double),
                ("seed", ctypes.c_uint64)]


class ImmResult(ctypes.Structure):
    _fields_ = [("theta", ctypes.c_uint64), ("lb", ctypes.c_double), ("rr_count", ctypes.c_uint64),
                ("lb_rounds", ctypes.c_uint32), ("status", ctypes.c_int)]


# name -> (restype, argtypes), mirroring include/gim.h
SIGNATURES = {
    "gim_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, _vp]),
    "gim_destroy": (None, [_vp]),
    "gim_graph_load": (ctypes.c_int, [_vp, ctypes.c_uint32, ctypes.c_uint64, _c_u64p, _c_u32p, _c_f32p]),
    "gim_graph_lt_valid": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int)]),
    "gim_sample_rr": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64]),
    "gim_reset_rr": (ctypes.c_int, [_vp]),
    "gim_rr_set_rounds": (ctypes.c_int, [_vp, ctypes.c_uint32]),
    "gim_rr_rounds": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_uint32)]),
    "gim_mrim": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double,
                                ctypes.c_double, ctypes.c_uint64, _c_u32p, _c_u64p, _c_f64p]),
    "gim_select_seeds": (ctypes.c_int, [_vp, ctypes.c_uint32, _c_u32p, _c_u64p, _c_u32p]),
    "gim_imm": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_uint32, ctypes.c_double, ctypes.c_double,
                               ctypes.c_uint64, _c_u32p, _c_u64p, _c_f64p]),
    "gim_batch_imm": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_uint32, ctypes.POINTER(ImmParams),
                                     ctypes.POINTER(_c_u32p), ctypes.POINTER(ImmResult)]),
    "gim_set_option": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_uint64]),
    "gim_get_option": (ctypes.c_int, [_vp, ctypes.c_int, _c_u64p]),
    "gim_autotune": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_uint32, ctypes.POINTER(ImmParams),
                                    ctypes.c_uint64, _c_u64p, ctypes.POINTER(ctypes.c_int)]),
    "gim_server_start": (ctypes.c_int, [ctypes.POINTER(_vp), _vp, ctypes.c_uint32, ctypes.c_uint32,
                                        ctypes.c_uint64]),
    "gim_server_submit": (ctypes.c_int, [_vp, ctypes.POINTER(ImmParams), _c_u64p]),
    "gim_server_poll": (ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.c_uint32, ctypes.POINTER(ctypes.c_int), _c_u32p,
                                       ctypes.POINTER(ImmResult), _c_f64p]),
    "gim_server_stats": (ctypes.c_int, [_vp, _c_f64p]),
    "gim_server_stop": (None, [_vp]),
    "gim_rr_count": (ctypes.c_int, [_vp, _c_u64p, _c_u64p]),
    "gim_rr_export": (ctypes.c_int, [_vp, _c_u64p, _c_u32p]),
    "gim_rr_export_compact": (ctypes.c_int, [_vp, _c_u64p, _c_u32p, ctypes.POINTER(ctypes.c_uint8)]),
    "gim_rr_info": (ctypes.c_int, [_vp, ctypes.c_uint64, _c_u32p, ctypes.POINTER(ctypes.c_int)]),
    "gim_coverage_export": (ctypes.c_int, [_vp, _c_u32p]),
    "gim_last_timings": (ctypes.c_int, [_vp, _c_f64p]),
    "gim_reset_timings": (ctypes.c_int, [_vp]),
    "gim_selection_stats": (ctypes.c_int, [_vp, _c_f64p]),
    "gim_rr_get": (ctypes.c_int, [_vp, ctypes.c_uint64, _vp, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32)]),
    "gim_diag_philox_rate": (ctypes.c_int, [_vp, _c_f64p]),
    "gim_diag_barrier_timeout": (ctypes.c_int, [_vp, _c_f64p]),
    "gim_launch_count": (ctypes.c_int, [_vp, _c_u64p]),
    "gim_last_error_string": (ctypes.c_char_p, [_vp]),
    "gim_select_seeds_noalloc": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, _vp, _vp,
                                                ctypes.c_uint32, _vp, _vp, _vp, _vp, ctypes.c_char_p,
                                                ctypes.c_size_t]),
}


class GimError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def load_library(path: str = LIB_PATH):
    """Loads libgim.so (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"libgim.so not found at {path}: build it first "
                                   "(python -m paper_2009_07325_gb300.build)")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(ct)


class Context:
    """One libgim context: a graph, an RR collection and device scratch on one GPU."""

    def __init__(self, device: int = 0, stream: int | None = None):
        self.L = load_library()
        h = _vp()
        st = self.L.gim_create(ctypes.byref(h), device, _vp(stream) if stream else None)
        if st != 0:
            raise GimError(st, f"gim_create(device={device}) failed")
        self.h = h
        self.n = 0

    def close(self):
        if getattr(self, "h", None):
            self.L.gim_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int, what: str):
        if st != 0:
            msg = self.L.gim_last_error_string(self.h)
            raise GimError(st, f"{what}: {msg.decode() if msg else ''}")

    # --- API ---------------------------------------------------------------
    def graph_load(self, n: int, offsets, sources, weights):
        off = np.ascontiguousarray(offsets, np.uint64)
        src = np.ascontiguousarray(sources, np.uint32)
        w = np.ascontiguousarray(weights, np.float32)
        m = int(off[-1]) if off.size else 0
        if off.size != n + 1:
            raise ValueError("offsets must have n+1 entries")
        if src.size < m or w.size < m:
            raise ValueError("sources/weights shorter than m")
        self._check(self.L.gim_graph_load(self.h, n, m, _p(off, _c_u64p), _p(src, _c_u32p), _p(w, _c_f32p)),
                    "gim_graph_load")
        self.n = n

    def load(self, graph):
        self.graph_load(graph.n, graph.offsets, graph.sources, graph.weights)

    @property
    def lt_valid(self) -> bool:
        v = ctypes.c_int(0)
        self._check(self.L.gim_graph_lt_valid(self.h, ctypes.byref(v)), "gim_graph_lt_valid")
        return bool(v.value)

    def sample_rr(self, model: int, count: int, seed: int):
        self._check(self.L.gim_sample_rr(self.h, model, count, seed), "gim_sample_rr")

    def reset_rr(self):
        self._check(self.L.gim_reset_rr(self.h), "gim_reset_rr")

    def set_rounds(self, T: int):
        """Makes the empty collection a multi-round collection of T rounds."""
        self._check(self.L.gim_rr_set_rounds(self.h, T), "gim_rr_set_rounds")

    def rounds(self) -> int:
        t = ctypes.c_uint32(0)
        self._check(self.L.gim_rr_rounds(self.h, ctypes.byref(t)), "gim_rr_rounds")
        return int(t.value)

    def select_seeds(self, k: int):
        """k seeds (k per round, k*T entries, on a multi-round collection)."""
        kt = k * self.rounds()
        seeds = np.zeros(kt, np.uint32)
        gains = np.zeros(kt, np.uint32)
        cov = ctypes.c_uint64(0)
        self._check(self.L.gim_select_seeds(self.h, k, _p(seeds, _c_u32p), ctypes.byref(cov), _p(gains, _c_u32p)),
                    "gim_select_seeds")
        return seeds, gains, int(cov.value)

    def imm(self, model: int, k: int, eps: float, ell: float, seed: int):
        seeds = np.zeros(k, np.uint32)
        theta = ctypes.c_uint64(0)
        lb = ctypes.c_double(0)
        self._check(self.L.gim_imm(self.h, model, k, eps, ell, seed, _p(seeds, _c_u32p), ctypes.byref(theta),
                                   ctypes.byref(lb)), "gim_imm")
        return dict(seeds=seeds, theta=int(theta.value), lb=float(lb.value), rr_count=self.rr_count()[0])

    def mrim(self, model: int, T: int, k: int, eps: float, ell: float, seed: int):
        """Multi-round IM (CR-NAIMM): k*T seeds as element ids t*n + v, in pick order."""
        seeds = np.zeros(k * T, np.uint32)
        theta = ctypes.c_uint64(0)
        lb = ctypes.c_double(0)
        self._check(self.L.gim_mrim(self.h, model, T, k, eps, ell, seed, _p(seeds, _c_u32p), ctypes.byref(theta),
                                    ctypes.byref(lb)), "gim_mrim")
        return dict(seeds=seeds, theta=int(theta.value), lb=float(lb.value), rr_count=self.rr_count()[0])

    def rr_count(self):
        c = ctypes.c_uint64(0)
        z = ctypes.c_uint64(0)
        self._check(self.L.gim_rr_count(self.h, ctypes.byref(c), ctypes.byref(z)), "gim_rr_count")
        return int(c.value), int(z.value)

    def rr_export(self):
        R, Z = self.rr_count()
        off = np.zeros(R + 1, np.uint64)
        mem = np.zeros(max(Z, 1), np.uint32)
        self._check(self.L.gim_rr_export(self.h, _p(off, _c_u64p), _p(mem, _c_u32p)), "gim_rr_export")
        return off, mem[:Z]

    def rr_export_compact(self):
        """(offsets, members, compact): a compact collection as a CSR; the sets
        kept without members export none and have compact[j] = 1."""
        R, Z = self.rr_count()
        off = np.zeros(R + 1, np.uint64)
        mem = np.zeros(max(Z, 1), np.uint32)
        flags = np.zeros(max(R, 1), np.uint8)
        self._check(self.L.gim_rr_export_compact(self.h, _p(off, _c_u64p), _p(mem, _c_u32p),
                                                 flags.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))),
                    "gim_rr_export_compact")
        return off, mem[:Z], flags[:R]

    def rr_info(self, rr_id: int):
        """(size, stored) of RR set rr_id."""
        n = ctypes.c_uint32(0)
        stored = ctypes.c_int(0)
        self._check(self.L.gim_rr_info(self.h, rr_id, ctypes.byref(n), ctypes.byref(stored)), "gim_rr_info")
        return int(n.value), bool(stored.value)

    def coverage(self) -> np.ndarray:
        """Occurrence counts: n entries, or T*n for a multi-round collection."""
        u = self.n * self.rounds()
        out = np.zeros(max(u, 1), np.uint32)
        self._check(self.L.gim_coverage_export(self.h, _p(out, _c_u32p)), "gim_coverage_export")
        return out[:u]

    def timings(self) -> dict:
        out = np.zeros(8, np.float64)
        self._check(self.L.gim_last_timings(self.h, _p(out, _c_f64p)), "gim_last_timings")
        return dict(sample_ms=out[0], select_ms=out[1], wall_ms=out[2], lb_rounds=int(out[3]),
                    kernel_ms=out[4], kernel_launches=int(out[5]), large_ms=out[6], large_launches=int(out[7]))

    def reset_timings(self):
        self._check(self.L.gim_reset_timings(self.h), "gim_reset_timings")

    def rr_get(self, rr_id: int) -> np.ndarray:
        """RR set rr_id as an ascending vertex array."""
        n = ctypes.c_uint32(0)
        cap = 1024
        while True:
            out = np.zeros(cap, np.uint32)
            st = self.L.gim_rr_get(self.h, int(rr_id), out.ctypes.data, cap, ctypes.byref(n))
            if st == 0:
                return out[: n.value].copy()
            if n.value > cap:
                cap = int(n.value)
                continue
            self._check(st, "gim_rr_get")

    def selection_stats(self) -> dict:
        """Selections since reset_timings: device ms, algorithmic bytes, calls, covered-set members."""
        out = np.zeros(4, np.float64)
        self._check(self.L.gim_selection_stats(self.h, _p(out, _c_f64p)), "gim_selection_stats")
        return dict(kernel_ms=out[0], bytes=out[1], calls=int(out[2]), covered_members=out[3])

    def diag_barrier_timeout(self):
        """Runs the greedy kernel with a barrier that can never be met; returns
        (status, ms): GIM_ERR_TIMEOUT (4) and the time the bounded wait took."""
        out = ctypes.c_double(0)
        st = self.L.gim_diag_barrier_timeout(self.h, ctypes.byref(out))
        return int(st), float(out.value)

    def philox_rate(self) -> float:
        """Measured Philox4x32-10 calls per second of this device (ALU ceiling of the coins)."""
        out = ctypes.c_double(0)
        self._check(self.L.gim_diag_philox_rate(self.h, ctypes.byref(out)), "gim_diag_philox_rate")
        return float(out.value)

    def set_option(self, opt: int, value: int):
        self._check(self.L.gim_set_option(self.h, opt, value), "gim_set_option")

    def schedule(self) -> dict:
        """The sampling schedule's knobs (gim_get_option of each)."""
        return {name: self.get_option(opt) for name, opt in SCHEDULE_OPTIONS.items()}

    def get_option(self, opt: int) -> int:
        v = ctypes.c_uint64(0)
        self._check(self.L.gim_get_option(self.h, opt, ctypes.byref(v)), "gim_get_option")
        return int(v.value)

    def launch_count(self) -> int:
        c = ctypes.c_uint64(0)
        self._check(self.L.gim_launch_count(self.h, ctypes.byref(c)), "gim_launch_count")
        return int(c.value)


def select_seeds_noalloc(n: int, num_sets: int, num_members: int, d_offsets: int, d_members: int, k: int,
                         d_seeds: int, d_gains: int = 0, d_covered: int = 0, stream: int = 0) -> None:
    """gim_select_seeds_noalloc on caller-owned device buffers (raw device addresses).

    For callers that cannot let the library allocate device memory; see the
    declaration in include/gim.h for limits and the shared-scratch contract.
    """
    L = load_library()
    buf = ctypes.create_string_buffer(256)
    st = L.gim_select_seeds_noalloc(n, num_sets, num_members, _vp(d_offsets), _vp(d_members), k, _vp(d_seeds),
                                    _vp(d_gains) if d_gains else None, _vp(d_covered) if d_covered else None,
                                    _vp(stream) if stream else None, buf, 256)
    if st != 0:
        raise GimError(st, "gim_select_seeds_noalloc: " + buf.value.decode())


def batch_imm(contexts, params):
    """gim_batch_imm over Context objects; params: list of (model, k, eps, ell, seed).

    Returns one dict per instance (seeds, theta, lb, rr_count, lb_rounds)."""
    L = load_library()
    n = len(contexts)
    hs = (_vp * n)(*[c.h for c in contexts])
    ps = (ImmParams * n)(*[ImmParams(int(m), int(k), float(e), float(l), int(sd)) for (m, k, e, l, sd) in params])
    seeds = [np.zeros(int(p[1]), np.uint32) for p in params]
    sp = (_c_u32p * n)(*[_p(a, _c_u32p) for a in seeds])
    rs = (ImmResult * n)()
    st = L.gim_batch_imm(hs, n, ps, sp, rs)
    if st != 0:
        msg = L.gim_last_error_string(contexts[0].h)
        raise GimError(st, "gim_batch_imm: " + (msg.decode() if msg else ""))
    return [dict(seeds=seeds[i], theta=int(rs[i].theta), lb=float(rs[i].lb), rr_count=int(rs[i].rr_count),
                 lb_rounds=int(rs[i].lb_rounds)) for i in range(n)]


def autotune(contexts, params, sample_sets: int = 2000):
    """gim_autotune: choose the sampling schedule for these contexts; returns (budget, measured)."""
    L = load_library()
    n = len(contexts)
    hs = (_vp * n)(*[c.h for c in contexts])
    ps = (ImmParams * n)(*[ImmParams(int(m), int(k), float(e), float(l), int(sd)) for (m, k, e, l, sd) in params])
    budget = ctypes.c_uint64(0)
    measured = ctypes.c_int(0)
    st = L.gim_autotune(hs, n, ps, sample_sets, ctypes.byref(budget), ctypes.byref(measured))
    if st != 0:
        msg = L.gim_last_error_string(contexts[0].h)
        raise GimError(st, "gim_autotune: " + (msg.decode() if msg else ""))
    return int(budget.value), bool(measured.value)


class Server:
    """IMM query server over the graph resident in a Context (gim_server_*)."""

    def __init__(self, graph_ctx: Context, max_active: int = 8, max_k: int = 256, mem_budget_bytes: int = 0):
        self.L = load_library()
        self.ctx = graph_ctx
        h = _vp()
        st = self.L.gim_server_start(ctypes.byref(h), graph_ctx.h, max_active, max_k, mem_budget_bytes)
        if st != 0:
            msg = self.L.gim_last_error_string(graph_ctx.h)
            raise GimError(st, "gim_server_start: " + (msg.decode() if msg else ""))
        self.h = h
        self.k = {}

    def submit(self, model: int, k: int, eps: float, ell: float, seed: int) -> int:
        t = ctypes.c_uint64(0)
        p = ImmParams(int(model), int(k), float(eps), float(ell), int(seed))
        st = self.L.gim_server_submit(self.h, ctypes.byref(p), ctypes.byref(t))
        if st != 0:
            raise GimError(st, "gim_server_submit")
        self.k[int(t.value)] = int(k)
        return int(t.value)

    def poll(self, ticket: int, timeout_ms: int = 0):
        """None while running, else dict(seeds, theta, lb, rr_count, lb_rounds, latency_ms)."""
        done = ctypes.c_int(0)
        seeds = np.zeros(self.k[ticket], np.uint32)
        res = ImmResult()
        lat = ctypes.c_double(0)
        st = self.L.gim_server_poll(self.h, ticket, timeout_ms, ctypes.byref(done), _p(seeds, _c_u32p),
                                    ctypes.byref(res), ctypes.byref(lat))
        if st != 0:
            raise GimError(st, f"gim_server_poll({ticket})")
        if not done.value:
            return None
        return dict(seeds=seeds, theta=int(res.theta), lb=float(res.lb), rr_count=int(res.rr_count),
                    lb_rounds=int(res.lb_rounds), latency_ms=float(lat.value))

    def wait(self, ticket: int, timeout_s: float = 600.0):
        import time
        t0 = time.time()
        while time.time() - t0 < timeout_s:
            r = self.poll(ticket, 100)
            if r is not None:
                return r
        raise TimeoutError(f"query {ticket} did not finish in {timeout_s} s")

    def stats(self) -> dict:
        out = np.zeros(8, np.float64)
        if self.L.gim_server_stats(self.h, _p(out, _c_f64p)) != 0:
            raise GimError(1, "gim_server_stats")
        keys = ["completed", "rounds", "busy_ms", "sample_ms", "select_ms", "peak_active", "waiting", "pool_sets"]
        return dict(zip(keys, out.tolist()))

    def stop(self):
        if getattr(self, "h", None):
            self.L.gim_server_stop(self.h)
            self.h = None

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass
