"""Pins of the oracle's bandwidth-sensitive decision (Algorithm 1, first branch).

* Eq. 2 with Table 2's coefficients reproduces the effective bandwidths the
  paper prints (tests/golden/effbw_pins.json);
* the argmax over matches agrees with a pure-Python enumeration of all
  k-permutations on tiny random graphs (link types from Table 1's peak
  bandwidths, counted over pattern-edge images);
* the worked example's ideal 3-GPU allocation (Sec. 2.2) is the one the
  sensitive branch picks on the idle DGX fixture;
* planted mistakes in the formula or the link typing are caught.
"""

import itertools
import json
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import oracle as O
from paper_2110_03214_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "effbw_pins.json")


def _pins(lib):
    with open(GOLDEN) as f:
        g = json.load(f)
    return all(abs(O.effbw(*p["xyz"], lib=lib) - p["value"]) <= p["tol"] for p in g["pins"])


def test_effbw_matches_printed_values():
    with open(GOLDEN) as f:
        g = json.load(f)
    for p in g["pins"]:
        got = O.effbw(*p["xyz"])
        assert abs(got - p["value"]) <= p["tol"], (p["xyz"], got, p["value"])


def _brute_effbw(n, wm, busy, k, pa, pb, lib):
    kind = {50: 0, 25: 1, 20: 1, 12: 2}
    free = [v for v in range(n) if not busy[v]]
    best = None
    count = 0
    for phi in itertools.permutations(free, k):
        if any(wm[phi[a], phi[b]] <= 0 for a, b in zip(pa, pb)):
            continue
        count += 1
        c = [0, 0, 0]
        for a, b in zip(pa, pb):
            t = kind.get(int(wm[phi[a], phi[b]]))
            if t is not None:
                c[t] += 1
        f = O.effbw(*c, lib=lib)
        if best is None or f > best[0]:
            best = (f, phi, tuple(c))
    return best, count


def _argmax_agrees(lib, trials=80) -> bool:
    rng = W.Rng(1203, 5)
    for _ in range(trials):
        n = int(rng.integers(3, 7, 1)[0])
        u, v, w = [], [], []
        for a in range(n):
            for b in range(a + 1, n):
                if rng.uniform(1)[0] < 0.7:
                    u.append(a)
                    v.append(b)
                    w.append(int((50, 25, 12, 20, 10)[int(rng.integers(0, 4, 1)[0])]))
        if not u:
            continue
        inst = O.Instance(n, u, v, w, 0, lib=lib)
        wm = inst.wmat.reshape(n, n)
        busy = rng.uniform(n) < 0.15
        kind = ("ring", "tree", "clique", "path")[int(rng.integers(0, 3, 1)[0])]
        k = int(rng.integers(1, min(n, 5), 1)[0])
        p = W.pattern(kind, k)
        dec, xyz = inst.decide_effbw(busy, k, p.a, p.b)
        best, count = _brute_effbw(n, wm, busy, k, list(p.a), list(p.b), lib)
        if best is None:
            if dec.status != O.STATUS_NO_MATCH:
                return False
            continue
        if dec.status != O.STATUS_OK or dec.tuple != tuple(best[1]) or xyz != best[2]:
            return False
        if dec.score != int(round(1000.0 * best[0])):
            return False
        if dec.classes * O.aut_count(k, p.a, p.b, lib=lib) != count:
            return False
    return True


def test_effbw_argmax_agrees_with_brute_force():
    assert _argmax_agrees(O.load())


def test_effbw_worked_example_ideal_allocation():
    # Sec. 2.2: on the DGX-V, the ideal 3-GPU allocation uses two double
    # NVLinks and one single NVLink: (x, y, z) = (2, 1, 0).
    topo = W.dgx_fixture()
    inst = O.Instance.from_topology(topo)
    p = W.pattern("clique", 3)
    dec, xyz = inst.decide_effbw(np.zeros(8, bool), 3, p.a, p.b)
    assert dec.status == O.STATUS_OK
    assert xyz == (2, 1, 0)
    assert dec.score == int(round(1000.0 * O.effbw(2, 1, 0))) == 57857
    assert dec.agg == 125


_MUTANTS = {
    "theta4_sign": ("-20.694", "20.694"),
    "inverse_without_plus_one": ("theta[4] / (X + 1.0)", "theta[4] / (X + 0.5)"),
    "swap_double_single": ("if (w == 50) return 0;", "if (w == 50) return 1;"),
    "pcie_not_counted": ("if (w == 12) return 2;", "if (w == 12) return -1;"),
    "first_max_lost": ("if (!s->have_best || f > b->best_f) {", "if (!s->have_best || f >= b->best_f) {"),
}


@pytest.mark.parametrize("name", sorted(_MUTANTS))
def test_effbw_pins_catch_planted_mistake(name, tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc missing")
    src = open(O._SRC).read()
    old, new = _MUTANTS[name]
    assert old in src, name
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-o", str(so), str(path), "-lm"])
    lib = O.load(str(so))
    caught = not _pins(lib) or not _argmax_agrees(lib, trials=60)
    if not caught:
        topo = W.dgx_fixture()
        inst = O.Instance.from_topology(topo, lib=lib)
        p = W.pattern("clique", 3)
        dec, xyz = inst.decide_effbw(np.zeros(8, bool), 3, p.a, p.b)
        caught = xyz != (2, 1, 0)
    assert caught, f"planted mistake {name} not caught"
