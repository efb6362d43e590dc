"""ctypes binding of the C ABI in include/mapa.h (argument marshalling only).

Every function named ``mapa_*`` here forwards to the C function of the same
name in ``_build/libmapa.so``; all enumeration, scoring and selection runs in
that library's CUDA kernels.  Importing this module raises if the library has
not been built (``python -m paper_2110_03214_gb300.build``): there is no
fallback path.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

MAPA_OK = 0
MAPA_NO_FIT = 1
MAPA_INEXACT = 2
MAPA_E_INVALID = -1
MAPA_E_RANGE = -2
MAPA_E_NOMEM = -3
MAPA_E_CUDA = -4
MAPA_E_BUDGET = -5
MAPA_E_TIMEOUT = -6
MAPA_E_STATE = -7

MAPA_RING, MAPA_TREE, MAPA_CLIQUE, MAPA_PATH = 0, 1, 2, 3
MAPA_MODE_EXHAUSTIVE, MAPA_MODE_BOUNDED = 0, 1
MAPA_POLICY_BW_SENSITIVE = 1
MAPA_POLICY_ANYTIME = 2
KIND = {"ring": MAPA_RING, "tree": MAPA_TREE, "clique": MAPA_CLIQUE, "path": MAPA_PATH}

MAPA_BATCH_INDEPENDENT = 0
MAPA_BATCH_SEQUENTIAL = 1
MAPA_BATCH_DEVICE = 2

MAX_K = 32

REQUEST_DTYPE = np.dtype(
    {
        "names": ["pattern_id", "root_lo", "root_hi", "alpha", "beta", "mode", "flags", "max_embeddings", "busy"],
        "formats": ["<i4", "<u2", "<u2", "<i4", "<i4", "<i4", "<i4", "<u8", ("<u4", (8,))],
        "offsets": [0, 4, 6, 8, 12, 16, 20, 24, 32],
        "itemsize": 64,
    }
)

RESULT_DTYPE = np.dtype(
    {
        "names": ["status", "score", "agg", "pres", "count", "job_id", "k", "reserved", "verts", "reserved2"],
        "formats": ["<i4", "<i4", "<i4", "<i4", "<u8", "<i8", "<i4", "<i4", ("u1", (32,)), "<u8"],
        "offsets": [0, 4, 8, 12, 16, 24, 32, 36, 40, 72],
        "itemsize": 80,
    }
)


MAPA_EVENT_ARRIVE = 0
MAPA_EVENT_DEPART = 1

EVENT_DTYPE = np.dtype(
    {
        "names": ["request_id", "at_ns", "lifetime_ns", "job_id", "kind", "pattern_id", "alpha", "beta", "mode",
                  "flags", "max_embeddings"],
        "formats": ["<i8", "<i8", "<i8", "<i8", "<i4", "<i4", "<i4", "<i4", "<i4", "<i4", "<u8"],
        "offsets": [0, 8, 16, 24, 32, 36, 40, 44, 48, 52, 56],
        "itemsize": 64,
    }
)

MAPA_SIM_BASELINE, MAPA_SIM_GREEDY, MAPA_SIM_PRESERVE, MAPA_SIM_EFFBW = 0, 1, 2, 3

SIM_JOB_DTYPE = np.dtype(
    {
        "names": ["job_id", "arrive", "duration", "pattern_id", "sensitive"],
        "formats": ["<i8", "<i8", "<i8", "<i4", "<i4"],
        "offsets": [0, 8, 16, 24, 28],
        "itemsize": 32,
    }
)

SIM_RECORD_DTYPE = np.dtype(
    {
        "names": ["job_id", "start", "end", "status", "effbw_milli", "agg", "pres", "k", "reserved", "verts"],
        "formats": ["<i8", "<i8", "<i8", "<i4", "<i4", "<i4", "<i4", "<i4", "<i4", ("u1", (32,))],
        "offsets": [0, 8, 16, 24, 28, 32, 36, 40, 44, 48],
        "itemsize": 80,
    }
)

SERVED_DTYPE = np.dtype(
    {
        "names": ["request_id", "arrive_ns", "done_ns", "kind", "rounds", "snapshot", "result"],
        "formats": ["<i8", "<i8", "<i8", "<i4", "<i4", ("<u4", (8,)), RESULT_DTYPE],
        "offsets": [0, 8, 16, 24, 28, 32, 64],
        "itemsize": 144,
    }
)


class Stats(ctypes.Structure):
    """mirror of mapa_stats"""

    _fields_ = [
        ("kernel_launches", ctypes.c_uint64),
        ("tail_launches", ctypes.c_uint64),
        ("tail_ms", ctypes.c_double),
        ("tail_parents", ctypes.c_uint64),
        ("tail_nodes", ctypes.c_uint64),
        ("tail_leaves", ctypes.c_uint64),
        ("tail_int_ops", ctypes.c_uint64),
        ("spill_entries", ctypes.c_uint64),
        ("spill_bytes", ctypes.c_uint64),
        ("requests", ctypes.c_uint64),
        ("embeddings", ctypes.c_uint64),
        ("expand_launches", ctypes.c_uint64),
        ("expand_ms", ctypes.c_double),
        ("expand_bytes", ctypes.c_uint64),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class MapaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"mapa error {code}: {msg}")
        self.code = code


def _load() -> ctypes.CDLL:
    if not os.path.exists(_build.LIB):
        raise ImportError(f"{_build.LIB} is missing: build it with `python -m paper_2110_03214_gb300.build`")
    lib = ctypes.CDLL(_build.LIB)
    vp, i32, u32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_int64, ctypes.c_uint64
    i32p = ctypes.POINTER(ctypes.c_int32)
    sig = {
        "mapa_version": ([], ctypes.c_char_p),
        "mapa_ctx_create": ([ctypes.c_int, u64, ctypes.POINTER(vp)], ctypes.c_int),
        "mapa_ctx_destroy": ([vp], None),
        "mapa_ctx_set_stream": ([vp, vp], ctypes.c_int),
        "mapa_last_error": ([vp], ctypes.c_char_p),
        "mapa_topology_load": ([vp, i32, i32, i32p, i32p, i32p, i32, i32p], ctypes.c_int),
        "mapa_pattern_load": ([vp, i32, i32, i32p, i32p, i32p], ctypes.c_int),
        "mapa_pattern_builtin": ([vp, i32, i32, i32p], ctypes.c_int),
        "mapa_allocate": ([vp, i32, i32, vp, vp], ctypes.c_int),
        "mapa_release": ([vp, i32, i64], ctypes.c_int),
        "mapa_allocate_batch": ([vp, i32, i32, vp, vp, u32], ctypes.c_int),
        "mapa_allocate_batch_noalloc": ([vp, i32, i32, i32, vp, vp], ctypes.c_int),
        "mapa_occupancy_get": ([vp, i32, ctypes.POINTER(ctypes.c_uint32)], ctypes.c_int),
        "mapa_stats_get": ([vp, ctypes.POINTER(Stats)], ctypes.c_int),
        "mapa_autotune": ([vp, i32, i32, vp, i32p], ctypes.c_int),
        "mapa_stats_reset": ([vp], ctypes.c_int),
        "mapa_ctx_set_timing": ([vp, ctypes.c_int], ctypes.c_int),
        "mapa_ctx_set_work_budget": ([vp, u64], ctypes.c_int),
        "mapa_measure_int_peak": ([vp, i32, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "mapa_result_merge": ([i32, vp, vp], ctypes.c_int),
        "mapa_autotune_level_limit": ([vp, i32, i32, ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
        "mapa_serve_open": ([vp, i32, i32, u32, ctypes.POINTER(vp)], ctypes.c_int),
        "mapa_serve_submit": ([vp, vp, i32], ctypes.c_int),
        "mapa_serve_poll": ([vp, vp, i32, ctypes.POINTER(ctypes.c_int32), i32], ctypes.c_int),
        "mapa_serve_drain": ([vp, i32], ctypes.c_int),
        "mapa_serve_counters": ([vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                 ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
        "mapa_serve_close": ([vp], ctypes.c_int),
        "mapa_pattern_analyze": ([i32, i32, i32p, i32p, ctypes.POINTER(ctypes.c_uint64),
                                  ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32)], ctypes.c_int),
        "mapa_effbw_predict": ([i32, i32, i32, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "mapa_simulate": ([vp, i32, i32, i32, vp, vp], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


lib = _load()

#: C symbols the header declares; tests check the library exports each one.
SYMBOLS = (
    "mapa_ctx_create", "mapa_ctx_destroy", "mapa_ctx_set_stream", "mapa_last_error", "mapa_topology_load",
    "mapa_pattern_load", "mapa_pattern_builtin", "mapa_allocate", "mapa_release", "mapa_allocate_batch",
    "mapa_occupancy_get", "mapa_pattern_analyze", "mapa_version", "mapa_stats_get", "mapa_stats_reset",
    "mapa_ctx_set_timing", "mapa_allocate_batch_noalloc", "mapa_serve_open", "mapa_serve_submit",
    "mapa_serve_poll", "mapa_serve_drain", "mapa_serve_counters", "mapa_serve_close", "mapa_autotune",
    "mapa_effbw_predict", "mapa_simulate", "mapa_ctx_set_work_budget", "mapa_measure_int_peak",
    "mapa_result_merge", "mapa_autotune_level_limit",
)


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _check(ctx, rc: int, ok=(MAPA_OK,)):
    if rc not in ok:
        raise MapaError(rc, lib.mapa_last_error(ctx).decode())
    return rc


# ---- functions with the C names ---------------------------------------------


def mapa_version() -> str:
    return lib.mapa_version().decode()


def mapa_ctx_create(device: int = 0, frontier_mem_cap: int = 0):
    h = ctypes.c_void_p()
    rc = lib.mapa_ctx_create(device, frontier_mem_cap, ctypes.byref(h))
    if rc != MAPA_OK:
        raise MapaError(rc, lib.mapa_last_error(None).decode())
    return h


def mapa_ctx_destroy(ctx) -> None:
    lib.mapa_ctx_destroy(ctx)


def mapa_ctx_set_stream(ctx, stream_ptr: int) -> None:
    _check(ctx, lib.mapa_ctx_set_stream(ctx, ctypes.c_void_p(stream_ptr or None)))


def mapa_last_error(ctx) -> str:
    return lib.mapa_last_error(ctx).decode()


def mapa_topology_load(ctx, n: int, u, v, w, fill_weight: int = 0) -> int:
    ua, up = _i32(u)
    va, vp_ = _i32(v)
    wa, wp = _i32(w)
    out = ctypes.c_int32()
    _check(ctx, lib.mapa_topology_load(ctx, n, len(ua), up, vp_, wp, fill_weight, ctypes.byref(out)))
    return out.value


def mapa_pattern_load(ctx, k: int, a, b) -> int:
    aa, ap = _i32(a)
    ba, bp = _i32(b)
    out = ctypes.c_int32()
    _check(ctx, lib.mapa_pattern_load(ctx, k, len(aa), ap, bp, ctypes.byref(out)))
    return out.value


def mapa_pattern_builtin(ctx, kind, k: int) -> int:
    kind = KIND.get(kind, kind)
    out = ctypes.c_int32()
    _check(ctx, lib.mapa_pattern_builtin(ctx, int(kind), k, ctypes.byref(out)))
    return out.value


def mapa_allocate(ctx, topo_id: int, pattern_id: int, alpha: int = 1, beta: int = 1, max_embeddings: int = 0,
                  mode: int = MAPA_MODE_EXHAUSTIVE):
    pol = np.zeros(1, dtype=np.dtype([("alpha", "<i4"), ("beta", "<i4"), ("mode", "<i4"), ("r", "<i4"),
                                       ("max_embeddings", "<u8")]))
    pol["alpha"], pol["beta"], pol["mode"], pol["max_embeddings"] = alpha, beta, mode, max_embeddings
    res = np.zeros(1, RESULT_DTYPE)
    rc = lib.mapa_allocate(ctx, topo_id, pattern_id, pol.ctypes.data, res.ctypes.data)
    if rc < 0 and res["status"][0] == rc and rc not in (MAPA_E_BUDGET, MAPA_E_RANGE):
        raise MapaError(rc, lib.mapa_last_error(ctx).decode())
    return res[0]


def mapa_release(ctx, topo_id: int, job_id: int) -> None:
    _check(ctx, lib.mapa_release(ctx, topo_id, int(job_id)))


def mapa_allocate_batch(ctx, topo_id: int, reqs, flags: int = MAPA_BATCH_INDEPENDENT, out=None):
    """Host batch: reqs is a REQUEST_DTYPE array; returns a RESULT_DTYPE array."""
    reqs = np.ascontiguousarray(reqs, dtype=REQUEST_DTYPE)
    if out is None:
        out = np.zeros(reqs.shape[0], RESULT_DTYPE)
    _check(ctx, lib.mapa_allocate_batch(ctx, topo_id, reqs.shape[0], reqs.ctypes.data, out.ctypes.data, flags))
    return out


def mapa_allocate_batch_device(ctx, topo_id: int, nreq: int, reqs_ptr: int, out_ptr: int,
                               flags: int = MAPA_BATCH_INDEPENDENT) -> None:
    """Device batch: reqs_ptr / out_ptr are device addresses (e.g. torch data_ptr())."""
    _check(ctx, lib.mapa_allocate_batch(ctx, topo_id, nreq, ctypes.c_void_p(reqs_ptr), ctypes.c_void_p(out_ptr),
                                        flags | MAPA_BATCH_DEVICE))


def mapa_allocate_batch_noalloc(ctx, topo_id: int, pattern_id: int, nreq: int, reqs_ptr: int, out_ptr: int) -> None:
    """Allocation-free decision of up to 4096 requests of one pattern (device
    pointers; see mapa.h for the limits and the shared-scratch rules)."""
    _check(ctx, lib.mapa_allocate_batch_noalloc(ctx, topo_id, pattern_id, nreq, ctypes.c_void_p(reqs_ptr),
                                                ctypes.c_void_p(out_ptr)))


def mapa_occupancy_get(ctx, topo_id: int) -> np.ndarray:
    busy = np.zeros(8, np.uint32)
    _check(ctx, lib.mapa_occupancy_get(ctx, topo_id, busy.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))))
    return busy


def mapa_autotune(ctx, topo_id: int, reqs, num_patterns: int) -> np.ndarray:
    """Times every fused tail depth per pattern on the host batch `reqs` and
    keeps the fastest; returns the chosen depth per pattern id (0 = absent)."""
    reqs = np.ascontiguousarray(reqs, dtype=REQUEST_DTYPE)
    chosen = np.zeros(max(num_patterns, 1), np.int32)
    _check(ctx, lib.mapa_autotune(ctx, topo_id, reqs.shape[0], reqs.ctypes.data,
                                  chosen.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
    return chosen[:num_patterns]


def mapa_stats_get(ctx) -> dict:
    st = Stats()
    _check(ctx, lib.mapa_stats_get(ctx, ctypes.byref(st)))
    return st.as_dict()


def mapa_stats_reset(ctx) -> None:
    _check(ctx, lib.mapa_stats_reset(ctx))


def mapa_ctx_set_timing(ctx, on: bool) -> None:
    _check(ctx, lib.mapa_ctx_set_timing(ctx, 1 if on else 0))


def mapa_autotune_level_limit(ctx, topo_id: int, pattern_id: int) -> int:
    out = ctypes.c_uint64()
    _check(ctx, lib.mapa_autotune_level_limit(ctx, topo_id, pattern_id, ctypes.byref(out)))
    return int(out.value)


def mapa_result_merge(parts) -> np.ndarray:
    """Reduces the results of the shares of one split request (RESULT_DTYPE
    array) to one result."""
    parts = np.ascontiguousarray(parts, dtype=RESULT_DTYPE)
    out = np.zeros(1, RESULT_DTYPE)
    rc = lib.mapa_result_merge(parts.shape[0], parts.ctypes.data, out.ctypes.data)
    if rc != MAPA_OK:
        raise MapaError(rc, "mapa_result_merge failed")
    return out[0]


def mapa_measure_int_peak(ctx, kind: int) -> float:
    out = ctypes.c_double()
    _check(ctx, lib.mapa_measure_int_peak(ctx, int(kind), ctypes.byref(out)))
    return out.value


def mapa_ctx_set_work_budget(ctx, max_partials: int) -> None:
    _check(ctx, lib.mapa_ctx_set_work_budget(ctx, int(max_partials)))


MAPA_SERVE_REJECT = 1


_SERVER_CTX: dict = {}  # server handle -> its context (for the error text at close)


def mapa_serve_open(ctx, topo_id: int, max_batch: int, flags: int = 0):
    h = ctypes.c_void_p()
    _check(ctx, lib.mapa_serve_open(ctx, topo_id, max_batch, flags, ctypes.byref(h)))
    _SERVER_CTX[h.value] = ctx
    return h


def mapa_serve_submit(srv, events) -> None:
    events = np.ascontiguousarray(events, dtype=EVENT_DTYPE)
    rc = lib.mapa_serve_submit(srv, events.ctypes.data, events.shape[0])
    if rc != MAPA_OK:
        raise MapaError(rc, "mapa_serve_submit failed")


def mapa_serve_poll(srv, max_events: int = 1 << 16, timeout_ms: int = 0) -> np.ndarray:
    out = np.zeros(max_events, SERVED_DTYPE)
    got = ctypes.c_int32()
    rc = lib.mapa_serve_poll(srv, out.ctypes.data, max_events, ctypes.byref(got), timeout_ms)
    if rc != MAPA_OK:
        raise MapaError(rc, "serving loop failed")
    return out[: got.value]


def mapa_serve_drain(srv, timeout_ms: int = 0) -> None:
    rc = lib.mapa_serve_drain(srv, timeout_ms)
    if rc != MAPA_OK:
        raise MapaError(rc, "mapa_serve_drain failed")


def mapa_serve_counters(srv):
    r, d, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    lib.mapa_serve_counters(srv, ctypes.byref(r), ctypes.byref(d), ctypes.byref(c))
    return {"rounds": r.value, "decisions": d.value, "conflicts": c.value}


def mapa_serve_close(srv) -> None:
    ctx = _SERVER_CTX.pop(srv.value, None)
    rc = lib.mapa_serve_close(srv)
    if rc != MAPA_OK:
        why = lib.mapa_last_error(ctx).decode() if ctx is not None else ""
        raise MapaError(rc, f"serving loop ended with an error: {why}")


def make_events(pattern_ids, at_ns, lifetime_ns=0, alpha=1, beta=1, request_ids=None, mode=0, flags=0) -> np.ndarray:
    pattern_ids = np.asarray(pattern_ids, np.int32)
    ev = np.zeros(pattern_ids.shape[0], EVENT_DTYPE)
    ev["request_id"] = np.arange(pattern_ids.shape[0]) if request_ids is None else request_ids
    ev["at_ns"] = at_ns
    ev["lifetime_ns"] = lifetime_ns
    ev["kind"] = MAPA_EVENT_ARRIVE
    ev["pattern_id"] = pattern_ids
    ev["alpha"] = alpha
    ev["beta"] = beta
    ev["mode"] = mode
    ev["flags"] = flags
    return ev


def mapa_simulate(ctx, topo_id: int, policy: int, jobs: np.ndarray) -> np.ndarray:
    """Runs a job file (SIM_JOB_DTYPE) through the simulator; one record per job."""
    jobs = np.ascontiguousarray(jobs, dtype=SIM_JOB_DTYPE)
    out = np.zeros(len(jobs), SIM_RECORD_DTYPE)
    _check(ctx, lib.mapa_simulate(ctx, topo_id, policy, len(jobs), jobs.ctypes.data, out.ctypes.data))
    return out


def make_sim_jobs(pattern_ids, arrive, duration, sensitive, job_ids=None) -> np.ndarray:
    pattern_ids = np.asarray(pattern_ids, np.int32)
    j = np.zeros(pattern_ids.shape[0], SIM_JOB_DTYPE)
    j["job_id"] = np.arange(pattern_ids.shape[0]) if job_ids is None else job_ids
    j["arrive"] = arrive
    j["duration"] = duration
    j["pattern_id"] = pattern_ids
    j["sensitive"] = sensitive
    return j


def mapa_effbw_predict(x: int, y: int, z: int) -> float:
    """Host-only: Predicted Effective Bandwidth (Eq. 2) as the library ranks it."""
    out = ctypes.c_double()
    rc = lib.mapa_effbw_predict(int(x), int(y), int(z), ctypes.byref(out))
    if rc != MAPA_OK:
        raise MapaError(rc, "link counts out of range")
    return out.value


def mapa_pattern_analyze(k: int, a, b):
    """Host-only: (|Aut(P)|, back_masks[k], lo_masks[k])."""
    aa, ap = _i32(a)
    ba, bp = _i32(b)
    aut = ctypes.c_uint64()
    back = np.zeros(max(k, 1), np.uint32)
    lo = np.zeros(max(k, 1), np.uint32)
    rc = lib.mapa_pattern_analyze(k, len(aa), ap, bp, ctypes.byref(aut),
                                  back.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                  lo.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    if rc != MAPA_OK:
        raise MapaError(rc, "pattern analysis failed")
    return aut.value, back[:k], lo[:k]


# ---- convenience ----------------------------------------------------------------


def make_requests(pattern_ids, alpha, beta, busy, max_embeddings=0, mode=0, flags=0) -> np.ndarray:
    pattern_ids = np.asarray(pattern_ids, np.int32)
    r = np.zeros(pattern_ids.shape[0], REQUEST_DTYPE)
    r["pattern_id"] = pattern_ids
    r["alpha"] = alpha
    r["beta"] = beta
    r["mode"] = mode
    r["flags"] = flags
    r["max_embeddings"] = max_embeddings
    r["busy"] = np.asarray(busy, np.uint32).reshape(-1, 8)
    return r


class Context:
    """Owns one mapa_ctx; the methods forward to the mapa_* functions."""

    def __init__(self, device: int = 0, frontier_mem_cap: int = 0):
        self.h = mapa_ctx_create(device, frontier_mem_cap)

    def close(self):
        if self.h:
            mapa_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def topology_load(self, topo) -> int:
        return mapa_topology_load(self.h, topo.n, topo.u, topo.v, topo.w, topo.fill_weight)

    def pattern_load(self, pattern) -> int:
        if pattern.kind in KIND:
            return mapa_pattern_builtin(self.h, pattern.kind, pattern.k)
        return mapa_pattern_load(self.h, pattern.k, pattern.a, pattern.b)

    def requests(self, workload_requests, pattern_ids, mode=MAPA_MODE_EXHAUSTIVE) -> np.ndarray:
        ids = np.asarray(pattern_ids, np.int32)[workload_requests.pattern_index]
        return make_requests(ids, workload_requests.alpha, workload_requests.beta, workload_requests.busy, mode=mode)

    def set_stream(self, stream_ptr: int):
        mapa_ctx_set_stream(self.h, stream_ptr)

    def allocate(self, topo_id, pattern_id, alpha=1, beta=1, max_embeddings=0, mode=MAPA_MODE_EXHAUSTIVE):
        return mapa_allocate(self.h, topo_id, pattern_id, alpha, beta, max_embeddings, mode)

    def release(self, topo_id, job_id):
        mapa_release(self.h, topo_id, job_id)

    def allocate_batch(self, topo_id, reqs, flags=MAPA_BATCH_INDEPENDENT):
        return mapa_allocate_batch(self.h, topo_id, reqs, flags)

    def allocate_batch_device(self, topo_id, nreq, reqs_ptr, out_ptr, flags=MAPA_BATCH_INDEPENDENT):
        mapa_allocate_batch_device(self.h, topo_id, nreq, reqs_ptr, out_ptr, flags)

    def occupancy(self, topo_id):
        return mapa_occupancy_get(self.h, topo_id)

    def stats(self) -> dict:
        return mapa_stats_get(self.h)

    def stats_reset(self):
        mapa_stats_reset(self.h)

    def set_timing(self, on: bool):
        mapa_ctx_set_timing(self.h, on)

    def set_work_budget(self, max_partials: int):
        mapa_ctx_set_work_budget(self.h, max_partials)
