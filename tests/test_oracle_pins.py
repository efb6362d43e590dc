"""Pins of the CPU oracle against facts fixed outside the oracle itself.

* values the paper prints for its worked example (Sec. 2.2, tests/golden/);
* closed-form counts in complete graphs and hand-derived counts on the
  8-vertex hybrid cube-mesh and the 4x4x4 torus (tests/golden/);
* automorphism group orders of the built-in shapes;
* a pure-Python brute force over all k-permutations on tiny random graphs;
* the preserved-bandwidth identity pres = W(F) - sum wdeg_F(phi) + W(G[phi]),
  invariance of the score under Aut(P), and lexicographic minimality of the
  chosen tuple within its automorphism orbit.

A last test plants mistakes in copies of the oracle source and checks that
these pins catch each of them.
"""

import itertools
import json
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import oracle as O
from paper_2110_03214_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _idle(n):
    return np.zeros(n, bool)


def _complete_graph_instance(n, fill=7):
    # K_n through the fill rule on an edgeless graph (Sec. 3.2).
    e = np.zeros(0, np.int32)
    return O.Instance(n, e, e, e, fill_weight=fill)


# ----------------------------------------------------------------- worked example


def test_dgx_worked_example_agg_87():
    g = _golden("dgx_worked_example.json")
    topo = W.dgx_fixture()
    inst = O.Instance.from_topology(topo)
    busy = np.ones(8, bool)
    busy[g["only_free_0indexed"]] = False
    p = W.pattern("clique", 3)
    d = inst.decide(busy, 3, p.a, p.b, g["policy_greedy"]["alpha"], g["policy_greedy"]["beta"])
    assert d.status == O.STATUS_OK
    assert d.agg == g["agg_of_1_2_5"] == 87
    assert d.classes == 1 and d.maps == 6


def test_dgx_worked_example_greedy_ideal_125():
    g = _golden("dgx_worked_example.json")
    topo = W.dgx_fixture()
    inst = O.Instance.from_topology(topo)
    p = W.pattern("clique", 3)
    d = inst.decide(_idle(8), 3, p.a, p.b, 1, 0)
    assert d.status == O.STATUS_OK
    assert d.agg == d.score == g["greedy_best_agg"] == 125
    assert list(d.tuple) == g["greedy_best_0indexed"]
    # fully connected through the fill: every 3-subset is a triangle
    assert d.classes == math.comb(8, 3)


# ----------------------------------------------------------------- closed forms


@pytest.mark.parametrize("f_busy", [(7, 0), (7, 2), (6, 1)])
def test_complete_graph_closed_forms(f_busy):
    n, nbusy = f_busy
    inst = _complete_graph_instance(n)
    busy = _idle(n)
    busy[:nbusy] = True
    f = n - nbusy
    for kind, k in [("ring", 3), ("ring", 4), ("ring", 5), ("path", 2), ("path", 4), ("clique", 3),
                    ("clique", 4), ("tree", 3), ("tree", 4), ("tree", 5)]:
        p = W.pattern(kind, k)
        d = inst.decide(busy, k, p.a, p.b)
        if k > f:
            assert d.status == O.STATUS_NO_MATCH
            continue
        ff = math.perm(f, k)
        if kind == "ring":
            want = ff // (2 * k)
        elif kind == "path":
            want = ff // 2
        elif kind == "clique":
            want = math.comb(f, k)
        else:
            want = ff // d.aut
        assert d.status == O.STATUS_OK
        assert d.maps == ff, (kind, k)
        assert d.classes == want, (kind, k)


def test_aut_sizes():
    g = _golden("closed_form_counts.json")["aut_sizes"]
    for kind in ("ring", "path", "clique", "tree"):
        for k, want in g[kind].items():
            p = W.pattern(kind, int(k))
            assert O.aut_count(p.k, p.a, p.b) == want, (kind, k)


def test_hybrid_cube_mesh_idle_counts():
    g = _golden("closed_form_counts.json")["hybrid_cube_mesh_8_idle"]
    topo = W.hybrid_cube_mesh8(W.Rng(1, 1))
    inst = O.Instance.from_topology(topo)
    for name, want in g.items():
        if name == "note":
            continue
        kind, k = name.split("-")
        p = W.pattern(kind, int(k))
        d = inst.decide(_idle(8), p.k, p.a, p.b)
        assert d.classes == want, name
        assert d.status == (O.STATUS_OK if want else O.STATUS_NO_MATCH)


def test_torus_idle_counts():
    g = _golden("closed_form_counts.json")["torus_4x4x4_idle"]
    inst = O.Instance.from_topology(W.torus3d(4))
    for name, want in g.items():
        if name == "note":
            continue
        kind, k = name.split("-")
        p = W.pattern(kind, int(k))
        d = inst.decide(_idle(64), p.k, p.a, p.b)
        assert d.classes == want, name


# ----------------------------------------------------------------- brute force


def _random_instance(rng, n):
    pairs = [(a, b) for a in range(n) for b in range(a + 1, n)]
    keep = rng.uniform(len(pairs)) < 0.6
    ws = rng.integers(1, 60, len(pairs))
    u = np.asarray([p[0] for p, k in zip(pairs, keep) if k], np.int32)
    v = np.asarray([p[1] for p, k in zip(pairs, keep) if k], np.int32)
    w = np.asarray([x for x, k in zip(ws, keep) if k], np.int32)
    fill = int(rng.integers(0, 1, 1)[0]) * 12
    return u, v, w, fill


def test_brute_force_agrees_on_tiny_random_graphs():
    rng = W.Rng(2024, 7)
    checked = 0
    for trial in range(160):
        n = int(rng.integers(2, 7, 1)[0])
        u, v, w, fill = _random_instance(rng, n)
        inst = O.Instance(n, u, v, w, fill)
        busy = rng.uniform(n) < 0.25
        k = int(rng.integers(1, min(5, n + 1), 1)[0])
        p = W.random_pattern(rng, k, p_edge=0.4, connected=bool(trial % 3))
        alpha, beta = (int(x) for x in rng.integers(-3, 3, 2))
        d = inst.decide(busy, k, p.a, p.b, alpha, beta)
        b = O.brute_force(n, u, v, w, fill, busy, k, p.a, p.b, alpha, beta)
        assert d.status == b.status, trial
        if b.status == O.STATUS_OK:
            checked += 1
            assert (d.score, d.agg, d.pres, d.maps, d.aut, d.classes, d.tuple) == (
                b.score, b.agg, b.pres, b.maps, b.aut, b.classes, b.tuple), trial
    assert checked > 60


# ----------------------------------------------------------------- identities


def _pres_identity(n, wm, busy, tup):
    free = ~busy
    total = sum(int(wm[a, b]) for a in range(n) for b in range(a + 1, n) if free[a] and free[b])
    wdeg = sum(int(wm[x, free].sum()) for x in tup)
    induced = sum(int(wm[tup[i], tup[j]]) for i in range(len(tup)) for j in range(i + 1, len(tup)))
    return total - wdeg + induced


def test_preserved_identity_and_aut_invariance():
    rng = W.Rng(99, 3)
    wl = W.workload("regular32", num_requests=12)
    topo = wl.topology
    inst = O.Instance.from_topology(topo)
    wm = inst.wmat.reshape(topo.n, topo.n)
    for r in range(len(wl.requests)):
        p = wl.requests.patterns[wl.requests.pattern_index[r]]
        if p.kind == "clique":
            p = W.pattern("ring", 5)
        busy = W.busy_to_bool(wl.requests.busy[r], topo.n)
        alpha, beta = (int(x) for x in rng.integers(-2, 3, 2))
        d = inst.decide(busy, p.k, p.a, p.b, alpha, beta)
        if d.status != O.STATUS_OK:
            continue
        assert d.pres == _pres_identity(topo.n, wm, busy, d.tuple)
        assert d.score == alpha * d.agg + beta * d.pres
        # every automorphic image scores the same and is lexicographically >= the choice
        pedges = {frozenset((int(a), int(b))) for a, b in zip(p.a, p.b)}
        seen = 0
        for sigma in itertools.islice(itertools.permutations(range(p.k)), 6000):
            if {frozenset((sigma[int(a)], sigma[int(b)])) for a, b in zip(p.a, p.b)} != pedges:
                continue
            img = tuple(d.tuple[sigma[i]] for i in range(p.k))
            st, agg, pres, score = inst.score_tuple(busy, p.k, p.a, p.b, alpha, beta, img)
            assert st == 0 and score == d.score and agg == d.agg and pres == d.pres
            assert img >= d.tuple
            seen += 1
        assert seen >= 1


def test_pres_zero_when_all_free_taken():
    topo = W.hybrid_cube_mesh8(W.Rng(5, 1))
    inst = O.Instance.from_topology(topo)
    busy = _idle(8)
    busy[4:] = True  # free = one K4
    p = W.pattern("ring", 4)
    d = inst.decide(busy, 4, p.a, p.b, 0, 1)
    assert d.status == O.STATUS_OK and d.pres == 0 and d.classes == 3


def test_k_larger_than_free_is_no_match():
    inst = _complete_graph_instance(6)
    busy = _idle(6)
    busy[:3] = True
    p = W.pattern("path", 4)
    assert inst.decide(busy, 4, p.a, p.b).status == O.STATUS_NO_MATCH


def test_single_vertex_pattern_scores_preserved_only():
    topo = W.hybrid_cube_mesh8(W.Rng(3, 1))
    inst = O.Instance.from_topology(topo)
    wm = inst.wmat.reshape(8, 8)
    p = W.pattern("ring", 1)
    d = inst.decide(_idle(8), 1, p.a, p.b, 1, 1)
    total = int(wm.sum()) // 2
    want = max(range(8), key=lambda x: (total - int(wm[x].sum()), -x))
    assert d.status == O.STATUS_OK and d.agg == 0 and d.classes == 8
    assert d.tuple == (want,) and d.pres == total - int(wm[want].sum())


# ----------------------------------------------------------------- planted mistakes

_MUTANTS = {
    "drop_pres_term": ("*score_out = alpha * agg + beta * pres;", "*score_out = alpha * agg;",
                       "int64_t score = s->alpha * agg + s->beta * pres;", "int64_t score = s->alpha * agg;"),
    "pres_skips_last_vertex": ("for (int32_t b = a + 1; b < n; ++b)", "for (int32_t b = a + 1; b < n - 1; ++b)"),
    "tie_break_last_max": ("score > s->best_score", "score >= s->best_score"),
    "agg_counts_one_endpoint_twice": ("s += wmat[phi[pa[e]] * n + phi[pb[e]]];", "s += wmat[phi[pa[e]] * n + phi[pa[e]]];"),
    "adjacency_not_checked": ("if (s->padj[a][i] && s->wmat[s->phi[a] * s->n + x] <= 0) ok = 0;", "(void)a;"),
    "busy_ignored": ("for (int32_t v = 0; v < n; ++v) s->free_v[v] = busy[v] ? 0 : 1;",
                     "for (int32_t v = 0; v < n; ++v) s->free_v[v] = 1;"),
    "aut_ignores_adjacency": ("if (s->padj[a][i] != s->padj[s->sigma[a]][j]) ok = 0;", "(void)a;"),
    "candidates_skip_vertex_zero": ("for (int32_t x = 0; x < s->n; ++x) {", "for (int32_t x = 1; x < s->n; ++x) {"),
}


def _pins_pass(lib) -> bool:
    """Reduced pin set run against a (possibly mutated) oracle library."""
    try:
        topo = W.dgx_fixture()
        inst = O.Instance.from_topology(topo, lib=lib)
        p = W.pattern("clique", 3)
        busy = np.ones(8, bool)
        busy[[0, 1, 4]] = False
        if inst.decide(busy, 3, p.a, p.b, 1, 0).agg != 87:
            return False
        d = inst.decide(_idle(8), 3, p.a, p.b, 1, 0)
        if d.agg != 125 or list(d.tuple) != [0, 2, 3]:
            return False
        for kind, k, want in (("ring", 4, 8), ("tree", 7, 8), ("path", 3, 2)):
            q = W.pattern(kind, k)
            if O.aut_count(k, q.a, q.b, lib=lib) != want:
                return False
        g = O.Instance.from_topology(W.torus3d(4), lib=lib)
        q = W.pattern("ring", 4)
        if g.decide(_idle(64), 4, q.a, q.b).classes != 240:
            return False
        rng = W.Rng(77, 1)
        for trial in range(40):
            n = int(rng.integers(3, 6, 1)[0])
            u, v, w, fill = _random_instance(rng, n)
            i2 = O.Instance(n, u, v, w, fill, lib=lib)
            busy = rng.uniform(n) < 0.2
            k = int(rng.integers(1, min(4, n), 1)[0])
            q = W.random_pattern(rng, k, 0.4)
            al, be = (int(x) for x in rng.integers(-2, 2, 2))
            d = i2.decide(busy, k, q.a, q.b, al, be)
            b = O.brute_force(n, u, v, w, fill, busy, k, q.a, q.b, al, be)
            if (d.status, d.score, d.tuple, d.classes) != (b.status, b.score, b.tuple, b.classes):
                return False
        return True
    except Exception:
        return False


def test_pins_pass_on_oracle():
    assert _pins_pass(O.load())


@pytest.mark.parametrize("name", sorted(_MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
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
    import ctypes  # noqa: F401  (loaded through O.load)
    lib = O.load(str(so))
    assert not _pins_pass(lib), f"planted mistake {name} not caught"
