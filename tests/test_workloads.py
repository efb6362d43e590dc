"""The seeded input generator produces the workloads it documents.

The generator feeds both the oracle and the CUDA path, so its structural
claims (sizes, regularity, link weights, request mixes, arrival processes)
are checked here on the CPU: a wrong topology would make every parity test
pass on the wrong input.
"""

import collections

import numpy as np
import pytest

from paper_2110_03214_gb300 import workloads as W


def _degrees(t):
    deg = np.zeros(t.n, np.int64)
    np.add.at(deg, t.u, 1)
    np.add.at(deg, t.v, 1)
    return deg


def _simple(t):
    assert np.all(t.u < t.v), "edges are stored with u < v (no self-loops)"
    keys = t.u.astype(np.int64) * t.n + t.v
    assert np.unique(keys).shape[0] == keys.shape[0], "duplicate edge"
    assert t.u.min() >= 0 and t.v.max() < t.n


def test_rng_is_counter_based_and_deterministic():
    a, b = W.Rng(5, 1), W.Rng(5, 1)
    x = np.concatenate([a.u64(3), a.u64(4)])
    assert np.array_equal(x, b.u64(7)), "draws depend only on (seed, stream, index)"
    assert not np.array_equal(W.Rng(5, 2).u64(7), x), "streams differ"
    ints = W.Rng(9, 0).integers(2, 5, 20000)
    assert ints.min() == 2 and ints.max() == 5, "integers(lo, hi) is inclusive"
    counts = np.bincount(ints - 2)
    assert np.all(np.abs(counts - 5000) < 400)
    u = W.Rng(9, 1).uniform(20000)
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01
    p = W.Rng(3, 3).permutation(50)
    assert sorted(p.tolist()) == list(range(50))


def test_hybrid_cube_mesh8():
    t = W.hybrid_cube_mesh8(W.Rng(1, 1))
    _simple(t)
    assert (t.n, t.m) == (8, 16)
    e = set(zip(t.u.tolist(), t.v.tolist()))
    for base in (0, 4):
        for i in range(base, base + 4):
            for j in range(i + 1, base + 4):
                assert (i, j) in e
    for i in range(4):
        assert (i, i + 4) in e
    assert set(t.w.tolist()) <= {25, 50}


@pytest.mark.parametrize("seed", [2, 17])
def test_random_regular32(seed):
    t = W.random_regular(W.Rng(seed, 1), 32, 6)
    _simple(t)
    assert (t.n, t.m) == (32, 96)
    assert np.all(_degrees(t) == 6)
    assert set(t.w.tolist()) == {25, 50}


def test_torus64():
    t = W.torus3d(4)
    _simple(t)
    assert (t.n, t.m) == (64, 192)
    assert np.all(_degrees(t) == 6)
    for a, b, w in zip(t.u.tolist(), t.v.tolist(), t.w.tolist()):
        xa, ya, za = a // 16, (a // 4) % 4, a % 4
        xb, yb, zb = b // 16, (b // 4) % 4, b % 4
        diff = [(xa - xb) % 4, (ya - yb) % 4, (za - zb) % 4]
        moved = [i for i, d in enumerate(diff) if d]
        assert len(moved) == 1 and diff[moved[0]] in (1, 3), (a, b)
        assert w == (50 if moved[0] == 0 else 25)


def test_dragonfly128():
    t = W.dragonfly(W.Rng(4, 1))
    _simple(t)
    assert t.n == 128
    g = lambda x: x // 8  # noqa: E731
    local = [(a, b, w) for a, b, w in zip(t.u.tolist(), t.v.tolist(), t.w.tolist()) if g(a) == g(b)]
    glob = [(a, b, w) for a, b, w in zip(t.u.tolist(), t.v.tolist(), t.w.tolist()) if g(a) != g(b)]
    assert len(local) == 16 * 28 and all(w == 50 for _, _, w in local)
    assert len(glob) == 120 and all(w == 25 for _, _, w in glob)
    pairs = collections.Counter((g(a), g(b)) for a, b, _ in glob)
    assert len(pairs) == 120 and max(pairs.values()) == 1, "one global link per group pair"
    ports = collections.Counter()
    for a, b, _ in glob:
        ports[a] += 1
        ports[b] += 1
    assert all(1 <= ports[v] <= 2 for v in range(128)), "each vertex takes 1-2 global links"


def test_boards256():
    t = W.boards256(W.Rng(5, 1))
    _simple(t)
    assert (t.n, t.m) == (256, 640)
    up = [(a, b, w) for a, b, w in zip(t.u.tolist(), t.v.tolist(), t.w.tolist()) if a // 8 != b // 8]
    assert len(up) == 128 and all(w == 10 for _, _, w in up)
    for a, b, _ in up:
        assert a % 8 == b % 8 and a % 8 < 4, "uplink j joins uplink j"
        assert (b // 8 - a // 8) % 32 in (1, 31), "boards form a ring"
    inner = [(a, b, w) for a, b, w in zip(t.u.tolist(), t.v.tolist(), t.w.tolist()) if a // 8 == b // 8]
    assert len(inner) == 32 * 16 and set(w for _, _, w in inner) <= {25, 50}


def test_dgx_fixture_links_of_the_worked_example():
    # Sec. 2.1-2.2 (1-indexed): 1-5 double NVLink, 1-2 single, 1-6 PCIe only.
    t = W.dgx_fixture()
    wt = {(a, b): w for a, b, w in zip(t.u.tolist(), t.v.tolist(), t.w.tolist())}
    assert wt[(0, 4)] == 50 and wt[(0, 1)] == 25 and (0, 5) not in wt
    assert t.fill_weight == 12
    assert sum(1 for e in ((0, 2), (0, 3), (2, 3)) if wt.get(e) == 25) == 1


def _busy_counts(wl):
    return np.asarray([int(sum(bin(int(x)).count("1") for x in row)) for row in wl.requests.busy])


def test_request_mixes():
    cm = W.workload("cube_mesh8")
    assert len(cm.requests) == 1000
    assert [p.name for p in cm.requests.patterns] == ["ring-4", "clique-3", "path-2"]
    c = _busy_counts(cm)
    assert c.min() == 0 and c.max() == 3
    assert np.all(np.bincount(cm.requests.pattern_index, minlength=3) > 250)

    rg = W.workload("regular32", num_requests=4000)
    assert [p.name for p in rg.requests.patterns] == ["ring-8", "tree-7", "clique-4"]
    c = _busy_counts(rg)
    assert c.min() == 0 and c.max() <= 16 and abs(c.mean() - 7.75) < 0.5  # floor(U[0,0.5]*32)
    frac = np.bincount(rg.requests.pattern_index) / 4000
    assert np.all(np.abs(frac - 1 / 3) < 0.04)
    assert np.all(rg.requests.alpha == 1) and np.all(rg.requests.beta == 1)

    to = W.workload("torus64", num_requests=6000)
    ks = collections.defaultdict(set)
    for i in to.requests.pattern_index.tolist():
        p = to.requests.patterns[i]
        ks[p.kind].add(p.k)
    assert ks["ring"] == set(range(2, 17)) and ks["tree"] == set(range(2, 17)) and ks["clique"] == {2, 3, 4}
    c = _busy_counts(to)
    assert c.max() <= int(0.6 * 64)

    # the same (name, seed) regenerates identical inputs
    again = W.workload("torus64", num_requests=6000)
    assert np.array_equal(again.requests.busy, to.requests.busy)
    assert np.array_equal(again.requests.pattern_index, to.requests.pattern_index)


def test_busy_masks_are_uniform_subsets():
    wl = W.workload("regular32", num_requests=3000)
    hits = np.zeros(32)
    for row in wl.requests.busy:
        hits += W.busy_to_bool(row, 32)
    assert np.all(np.abs(hits / hits.mean() - 1) < 0.12), "every vertex equally likely busy"
    assert np.all(wl.requests.busy[:, 1:] == 0), "no bits beyond n"


def test_served_trace_offers_the_stated_occupancy():
    tr = W.served_trace(20000, 1e4)
    assert np.all(np.diff(tr.at_ns) >= 0)
    span = (tr.at_ns[-1] - tr.at_ns[0]) * 1e-9
    assert abs(20000 / span - 1e4) / 1e4 < 0.03, "Poisson rate"
    ks = np.asarray([tr.patterns[i].k for i in tr.pattern_index], np.float64)
    offered = (ks * tr.lifetime_ns * 1e-9).sum() / span / tr.topology.n
    assert abs(offered - 0.6) < 0.05, "offered occupancy (Little's law)"


def test_sim_jobs_follow_the_section5_mix():
    jobs = W.sim_jobs(3000)
    sizes = np.asarray([jobs.patterns[i].k for i in jobs.pattern_index])
    assert sizes.min() == 1 and sizes.max() == 5
    assert jobs.duration.min() >= 100 and jobs.duration.max() <= 1000
    assert np.all(jobs.arrive == 0)
    assert all(jobs.patterns[i].kind == "ring" for i in jobs.pattern_index)
    by_net = dict(W.SIM_NETWORKS)
    assert all(bool(s) == by_net[n] for s, n in zip(jobs.sensitive.tolist(), jobs.network))
    assert len(set(jobs.network)) == len(W.SIM_NETWORKS)
