"""Pins of the oracle's bounded (branch-and-bound) decision.

The bounded search must return exactly the exhaustive decision: the same
status, score, AggBW, PreservedBW and tuple (ties included).  That is pinned
here against the exhaustive oracle -- itself pinned by test_oracle_pins.py --
on random small graphs with every sign of alpha and beta, and on samples of
the benchmark workloads.  A bound that is too tight (not admissible) cuts off
the optimum somewhere; the last test plants such mistakes in copies of the
oracle source and checks that these pins catch each of them.
"""

import shutil
import subprocess

import numpy as np
import pytest

from oracle import oracle as O
from paper_2110_03214_gb300 import workloads as W


def _random_case(rng):
    n = int(rng.integers(4, 10, 1)[0])
    dens = float(rng.uniform(1)[0]) * 0.6 + 0.3
    u, v, w = [], [], []
    for a in range(n):
        for b in range(a + 1, n):
            if rng.uniform(1)[0] < dens:
                u.append(a)
                v.append(b)
                w.append(int((10, 25, 50, 100)[int(rng.integers(0, 3, 1)[0])]))
    if not u:
        u, v, w = [0], [1], [25]
    busy = rng.uniform(n) < 0.25
    kind = ("ring", "tree", "clique", "path")[int(rng.integers(0, 3, 1)[0])]
    k = int(rng.integers(1, min(n, 6), 1)[0])  # Rng.integers is inclusive
    return n, u, v, w, busy, W.pattern(kind, k)


def _same(d, b):
    return (d.status, d.score, d.agg, d.pres, d.tuple) == (b.status, b.score, b.agg, b.pres, b.tuple)


def _bounded_pins_pass(lib, trials=250) -> bool:
    try:
        rng = W.Rng(2110, 7)
        for trial in range(trials):
            n, u, v, w, busy, p = _random_case(rng)
            inst = O.Instance(n, u, v, w, 0, lib=lib)
            al, be = (int(x) for x in rng.integers(0, 3, 2))
            if trial % 10 == 9:
                al, be = -al - 1, be  # a negative weight: nothing may be cut
            d = inst.decide(busy, p.k, p.a, p.b, al, be)
            b = inst.decide_bounded(busy, p.k, p.a, p.b, al, be)
            if not _same(d, b):
                return False
        wl = W.workload("regular32", num_requests=24, seed=5)
        inst = O.Instance.from_topology(wl.topology, lib=lib)
        for i in range(len(wl.requests)):
            p = wl.requests.patterns[wl.requests.pattern_index[i]]
            if p.k > 7:
                continue
            busy = W.busy_to_bool(wl.requests.busy[i], wl.topology.n)
            d = inst.decide(busy, p.k, p.a, p.b, 1, 1)
            b = inst.decide_bounded(busy, p.k, p.a, p.b, 1, 1)
            if not _same(d, b):
                return False
        return True
    except Exception:
        return False


def test_bounded_equals_exhaustive():
    assert _bounded_pins_pass(O.load())


@pytest.mark.parametrize("alpha,beta", [(1, 1), (1, 0), (0, 1), (3, 1), (1, 3)])
def test_bounded_equals_exhaustive_cube_mesh(alpha, beta):
    wl = W.workload("cube_mesh8", num_requests=200, seed=3)
    inst = O.Instance.from_topology(wl.topology)
    for i in range(len(wl.requests)):
        p = wl.requests.patterns[wl.requests.pattern_index[i]]
        busy = W.busy_to_bool(wl.requests.busy[i], wl.topology.n)
        d = inst.decide(busy, p.k, p.a, p.b, alpha, beta)
        b = inst.decide_bounded(busy, p.k, p.a, p.b, alpha, beta)
        assert _same(d, b), (i, d, b)
        assert b.aut == 0 and b.classes == 0  # no count in bounded mode


def test_bounded_cuts_nodes():
    # Idle 4x4x4 torus, ring-8: the bounded search visits (internal nodes
    # included) far fewer nodes than the exhaustive one has complete maps,
    # and agrees with it.
    topo = W.torus3d(4)
    inst = O.Instance.from_topology(topo)
    p = W.pattern("ring", 8)
    idle = np.zeros(64, bool)
    d = inst.decide(idle, 8, p.a, p.b, 1, 1)
    b = inst.decide_bounded(idle, 8, p.a, p.b, 1, 1)
    assert _same(d, b)
    assert d.maps == 637440  # ring-8 maps in the idle torus
    assert b.maps < d.maps // 3


def test_bounded_budget_and_no_match():
    topo = W.torus3d(4)
    inst = O.Instance.from_topology(topo)
    p = W.pattern("ring", 8)
    idle = np.zeros(64, bool)
    assert inst.decide_bounded(idle, 8, p.a, p.b, 1, 1, max_nodes=100).status == O.STATUS_BUDGET
    c = W.pattern("clique", 3)  # the torus has no triangles
    assert inst.decide_bounded(idle, 3, c.a, c.b, 1, 1).status == O.STATUS_NO_MATCH


# ----------------------------------------------------------------- planted mistakes

_MUTANTS = {
    "no_cross_gain": ("const int64_t b1 = s->alpha * b->wmax * e_cross + e_in * in_w;",
                      "const int64_t b1 = e_in * in_w;",
                      "s->alpha * b->wmax * (e_cross + e_in)", "s->alpha * b->wmax * e_in"),
    "gain_at_wmin": ("const int64_t b1 = s->alpha * b->wmax * e_cross + e_in * in_w;",
                     "const int64_t b1 = s->alpha * b->wmin * e_cross + e_in * in_w;",
                     "s->alpha * b->wmax * (e_cross + e_in)", "s->alpha * b->wmin * (e_cross + e_in)"),
    "loss_not_halved": ("(s->beta * dm + 1) / 2", "s->beta * dm"),
    "largest_degrees": ("dm += deg[j];", "dm += deg[r - 1 - j];"),
    "cross_edges_miss_next": ("else if (hi >= i) e_cross += 1;", "else if (hi > i) e_cross += 1;"),
}


def test_bounded_pins_pass_on_oracle():
    assert _bounded_pins_pass(O.load(), trials=60)


@pytest.mark.parametrize("name", sorted(_MUTANTS))
def test_bounded_pins_catch_planted_mistake(name, tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc missing")
    src = open(O._SRC).read()
    subs = _MUTANTS[name]
    changed = src
    for i in range(0, len(subs), 2):
        assert subs[i] in changed, (name, subs[i])
        changed = changed.replace(subs[i], subs[i + 1])
    path = tmp_path / "mutant.c"
    path.write_text(changed)
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O1", "-shared", "-fPIC", "-o", str(so), str(path)])
    lib = O.load(str(so))
    assert not _bounded_pins_pass(lib), f"planted mistake {name} not caught"
