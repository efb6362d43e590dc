"""Python face of the MAPA allocation oracle -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
import this module.  The product path (the CUDA library behind
include/mapa.h) never imports it.

Two independent restatements of the allocation problem of Sec. 3.3-3.5
(arXiv 2110.03214):

* ``decide`` calls the plain C backtracking oracle in ``mapa_oracle.c``
  (tier 2: any size it can finish); ``decide_bounded`` runs the same
  lexicographic enumeration with branch-and-bound cut-offs (same decision,
  no count) to reach larger instances;
* ``brute_force`` is a pure-Python enumeration of every k-permutation of the
  free vertices (tier 1: tiny graphs only), scoring each with Eq. 1 and Eq. 3
  written out again from the paper.

Both take plain inputs (vertex count, edge lists, weights, busy flags,
pattern edges); neither touches the CUDA library.
"""

from __future__ import annotations

import ctypes
import dataclasses
import itertools
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mapa_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAX_K = 32

STATUS_OK = 0
STATUS_NO_MATCH = 1
STATUS_INVALID = -1
STATUS_NOT_DIVISIBLE = -2
STATUS_BUDGET = -5


class _Result(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32),
        ("k", ctypes.c_int32),
        ("score", ctypes.c_int64),
        ("agg", ctypes.c_int64),
        ("pres", ctypes.c_int64),
        ("maps", ctypes.c_uint64),
        ("aut", ctypes.c_uint64),
        ("classes", ctypes.c_uint64),
        ("tuple", ctypes.c_uint8 * MAX_K),
    ]


def build(force: bool = False, extra_flags: tuple = (), out: str | None = None) -> str:
    """Compile mapa_oracle.c with gcc into oracle/_build/ (plain -O2, no vector ISA flags)."""
    target = out or _LIB
    os.makedirs(os.path.dirname(target), exist_ok=True)
    if force or not os.path.exists(target) or os.path.getmtime(target) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", *extra_flags, "-o", target + ".tmp", _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(target + ".tmp", target)
    return target


def load(path: str | None = None):
    """Load (building first if needed) the oracle library."""
    global _lib
    with _lock:
        if path is None and _lib is not None:
            return _lib
        lib = ctypes.CDLL(path or build())
        i32p = ctypes.POINTER(ctypes.c_int32)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.oracle_weight_matrix.argtypes = [ctypes.c_int32, ctypes.c_int32, i32p, i32p, i32p, ctypes.c_int32, i32p]
        lib.oracle_weight_matrix.restype = ctypes.c_int
        lib.oracle_aut_count.argtypes = [ctypes.c_int32, ctypes.c_int32, i32p, i32p]
        lib.oracle_aut_count.restype = ctypes.c_uint64
        lib.oracle_score_tuple.argtypes = [ctypes.c_int32, i32p, u8p, ctypes.c_int32, ctypes.c_int32, i32p, i32p,
                                           ctypes.c_int64, ctypes.c_int64, u8p, i64p, i64p, i64p]
        lib.oracle_score_tuple.restype = ctypes.c_int
        lib.oracle_decide.argtypes = [ctypes.c_int32, i32p, u8p, ctypes.c_int32, ctypes.c_int32, i32p, i32p,
                                      ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64, ctypes.POINTER(_Result)]
        lib.oracle_decide.restype = ctypes.c_int
        lib.oracle_decide_capped.argtypes = lib.oracle_decide.argtypes[:10] + [ctypes.c_uint64,
                                                                                ctypes.POINTER(_Result)]
        lib.oracle_decide_capped.restype = ctypes.c_int
        lib.oracle_decide_rooted.argtypes = lib.oracle_decide.argtypes[:9] + [ctypes.c_int32, ctypes.c_int32,
                                                                               ctypes.POINTER(_Result)]
        lib.oracle_decide_rooted.restype = ctypes.c_int
        lib.oracle_decide_bounded.argtypes = lib.oracle_decide.argtypes
        lib.oracle_decide_bounded.restype = ctypes.c_int
        lib.oracle_effbw.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64]
        lib.oracle_effbw.restype = ctypes.c_double
        lib.oracle_decide_effbw.argtypes = [ctypes.c_int32, i32p, u8p, ctypes.c_int32, ctypes.c_int32, i32p, i32p,
                                            ctypes.c_uint64, ctypes.POINTER(_Result), i64p]
        lib.oracle_decide_effbw.restype = ctypes.c_int
        if path is None:
            _lib = lib
        return lib


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _u8(a):
    a = np.ascontiguousarray(a, dtype=np.uint8)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


@dataclasses.dataclass
class Decision:
    status: int
    score: int
    agg: int
    pres: int
    maps: int
    aut: int
    classes: int
    tuple: tuple


class Instance:
    """A hardware graph prepared for repeated oracle calls."""

    def __init__(self, n: int, u, v, w, fill_weight: int = 0, lib=None):
        self.lib = lib or load()
        self.n = int(n)
        self._keep = [_i32(u), _i32(v), _i32(w)]
        self.wmat = np.zeros(self.n * self.n, np.int32)
        rc = self.lib.oracle_weight_matrix(self.n, len(self._keep[0][0]), self._keep[0][1], self._keep[1][1],
                                           self._keep[2][1], int(fill_weight),
                                           self.wmat.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        if rc != 0:
            raise ValueError("invalid hardware graph")
        self._wp = self.wmat.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))

    @classmethod
    def from_topology(cls, topo, lib=None) -> "Instance":
        return cls(topo.n, topo.u, topo.v, topo.w, topo.fill_weight, lib=lib)

    def decide(self, busy, k: int, pa, pb, alpha: int = 1, beta: int = 1, max_maps: int = 0,
               max_nodes: int = 0) -> Decision:
        """Exhaustive decision; past max_maps matches or max_nodes search nodes
        (0 = no cap) the status is STATUS_BUDGET."""
        busy_a, busy_p = _u8(np.asarray(busy, dtype=bool))
        pa_a, pa_p = _i32(pa)
        pb_a, pb_p = _i32(pb)
        res = _Result()
        self.lib.oracle_decide_capped(self.n, self._wp, busy_p, int(k), len(pa_a), pa_p, pb_p, int(alpha), int(beta),
                                      int(max_maps), int(max_nodes), ctypes.byref(res))
        return Decision(res.status, res.score, res.agg, res.pres, res.maps, res.aut, res.classes,
                        tuple(res.tuple[:k]) if res.status == STATUS_OK else ())

    def decide_rooted(self, busy, k: int, pa, pb, alpha: int, beta: int, root_lo: int, root_hi: int) -> Decision:
        """One share of a split request: only the maps with phi(0) in
        [root_lo, root_hi).  ``maps`` counts the share's maps; ``classes``
        and ``aut`` stay 0 (a share need not hold whole classes)."""
        busy_a, busy_p = _u8(np.asarray(busy, dtype=bool))
        pa_a, pa_p = _i32(pa)
        pb_a, pb_p = _i32(pb)
        res = _Result()
        self.lib.oracle_decide_rooted(self.n, self._wp, busy_p, int(k), len(pa_a), pa_p, pb_p, int(alpha), int(beta),
                                      int(root_lo), int(root_hi), ctypes.byref(res))
        return Decision(res.status, res.score, res.agg, res.pres, res.maps, 0, 0,
                        tuple(res.tuple[:k]) if res.status == STATUS_OK else ())

    def decide_bounded(self, busy, k: int, pa, pb, alpha: int = 1, beta: int = 1, max_nodes: int = 0) -> Decision:
        """Branch and bound over the same lexicographic enumeration: the same
        status, score, agg, pres and tuple as ``decide``; ``maps`` holds the
        search nodes visited and ``aut``/``classes`` stay 0 (no count)."""
        busy_a, busy_p = _u8(np.asarray(busy, dtype=bool))
        pa_a, pa_p = _i32(pa)
        pb_a, pb_p = _i32(pb)
        res = _Result()
        self.lib.oracle_decide_bounded(self.n, self._wp, busy_p, int(k), len(pa_a), pa_p, pb_p, int(alpha),
                                       int(beta), int(max_nodes), ctypes.byref(res))
        return Decision(res.status, res.score, res.agg, res.pres, res.maps, 0, 0,
                        tuple(res.tuple[:k]) if res.status == STATUS_OK else ())

    def decide_effbw(self, busy, k: int, pa, pb, max_maps: int = 0):
        """Decision for a bandwidth-sensitive job (Algorithm 1's first branch):
        the match with the largest Predicted EffBW (Eq. 2).  ``score`` is
        round(1000 * EffBW); returns (Decision, (x, y, z))."""
        busy_a, busy_p = _u8(np.asarray(busy, dtype=bool))
        pa_a, pa_p = _i32(pa)
        pb_a, pb_p = _i32(pb)
        res = _Result()
        xyz = (ctypes.c_int64 * 3)()
        self.lib.oracle_decide_effbw(self.n, self._wp, busy_p, int(k), len(pa_a), pa_p, pb_p, int(max_maps),
                                     ctypes.byref(res), xyz)
        dec = Decision(res.status, res.score, res.agg, res.pres, res.maps, res.aut, res.classes,
                       tuple(res.tuple[:k]) if res.status == STATUS_OK else ())
        return dec, tuple(int(v) for v in xyz)

    def score_tuple(self, busy, k: int, pa, pb, alpha: int, beta: int, tup):
        """(status, agg, pres, score) of one given tuple; status 0 when it is a match."""
        busy_a, busy_p = _u8(np.asarray(busy, dtype=bool))
        pa_a, pa_p = _i32(pa)
        pb_a, pb_p = _i32(pb)
        t_a, t_p = _u8(np.asarray(tup, dtype=np.uint8))
        agg, pres, score = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        st = self.lib.oracle_score_tuple(self.n, self._wp, busy_p, int(k), len(pa_a), pa_p, pb_p, int(alpha),
                                         int(beta), t_p, ctypes.byref(agg), ctypes.byref(pres), ctypes.byref(score))
        return st, agg.value, pres.value, score.value


def effbw(x: int, y: int, z: int, lib=None) -> float:
    """Predicted Effective Bandwidth (Eq. 2, Table 2) of link counts (x, y, z)."""
    lib = lib or load()
    return float(lib.oracle_effbw(int(x), int(y), int(z)))


def aut_count(k: int, pa, pb, lib=None) -> int:
    lib = lib or load()
    pa_a, pa_p = _i32(pa)
    pb_a, pb_p = _i32(pb)
    return int(lib.oracle_aut_count(int(k), len(pa_a), pa_p, pb_p))


# --------------------------------------------------------------------------
# Tier 1: pure-Python brute force over all k-permutations (tiny inputs)


def brute_force(n: int, u, v, w, fill_weight: int, busy, k: int, pa, pb, alpha: int, beta: int) -> Decision:
    """Every k-permutation of the free vertices, in lexicographic order.

    Weight lookup, Eq. 1 and Eq. 3 are written out again here, independently
    of mapa_oracle.c.  The automorphism count comes from all k! permutations
    of the pattern (so k <= 8 in practice).
    """
    weight = {}
    for a, b, x in zip(u, v, w):
        weight[(int(a), int(b))] = int(x)
        weight[(int(b), int(a))] = int(x)

    def wt(a, b):
        if a == b:
            return 0
        return weight.get((a, b), fill_weight if fill_weight > 0 else 0)

    pedges = [(int(a), int(b)) for a, b in zip(pa, pb)]
    free = [x for x in range(n) if not busy[x]]
    best = None
    maps = 0
    for perm in itertools.permutations(free, k):
        if any(wt(perm[a], perm[b]) <= 0 for a, b in pedges):
            continue
        maps += 1
        agg = sum(wt(perm[a], perm[b]) for a, b in pedges)
        rest = [x for x in free if x not in perm]
        pres = sum(wt(rest[i], rest[j]) for i in range(len(rest)) for j in range(i + 1, len(rest)))
        score = alpha * agg + beta * pres
        if best is None or score > best[0]:
            best = (score, agg, pres, perm)
    eset = {frozenset(e) for e in pedges}
    aut = sum(1 for s in itertools.permutations(range(k)) if {frozenset((s[a], s[b])) for a, b in pedges} == eset)
    if best is None:
        return Decision(STATUS_NO_MATCH, 0, 0, 0, 0, 0, 0, ())
    return Decision(STATUS_OK, best[0], best[1], best[2], maps, aut, maps // aut, tuple(best[3]))
