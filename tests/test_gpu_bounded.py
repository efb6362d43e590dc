"""GPU parity of the bounded mode (branch and bound, MAPA_MODE_BOUNDED).

The bounded mode must return the exhaustive decision exactly -- status,
score, AggBW, PreservedBW and tuple, ties included -- with count 0.  Checked
against the GPU's own exhaustive mode on the benchmark workloads, and
against the oracle's bounded search (pinned to the exhaustive oracle on the
CPU) on idle large graphs where exhaustive enumeration is large, through
every driver: independent batches (device-driven and chunked), mixed
batches, sequential commits and the single-request call.
"""

import dataclasses

import numpy as np
import pytest

from oracle import oracle as O
from paper_2110_03214_gb300 import build as B
from paper_2110_03214_gb300 import workloads as W

pytestmark = pytest.mark.gpu

OK, NO_FIT = 0, 1


@pytest.fixture(scope="module")
def M():
    B.build()
    from paper_2110_03214_gb300 import mapa

    return mapa


@pytest.fixture(scope="module")
def ctx(M):
    c = M.Context(0)
    yield c
    c.close()


def _key(r, k):
    return (int(r["status"]), int(r["score"]), int(r["agg"]), int(r["pres"]),
            tuple(int(x) for x in r["verts"][:k]) if int(r["status"]) == OK else ())


def _dec_key(d, k):
    if d.status == O.STATUS_NO_MATCH:
        return (NO_FIT, 0, 0, 0, ())
    assert d.status == O.STATUS_OK, d
    return (OK, d.score, d.agg, d.pres, tuple(d.tuple))


def _both_modes(M, ctx, wl, flags=0):
    tid = ctx.topology_load(wl.topology)
    pids = [ctx.pattern_load(p) for p in wl.requests.patterns]
    ex = ctx.allocate_batch(tid, ctx.requests(wl.requests, pids), flags)
    bd = ctx.allocate_batch(tid, ctx.requests(wl.requests, pids, mode=M.MAPA_MODE_BOUNDED), flags)
    return ex, bd


@pytest.mark.parametrize("name,num", [("cube_mesh8", 1000), ("regular32", 3000), ("torus64", 1500)])
def test_bounded_equals_exhaustive_on_workloads(M, ctx, name, num):
    wl = W.workload(name, num_requests=num)
    if name == "torus64":
        ks = np.asarray([wl.requests.patterns[i].k for i in wl.requests.pattern_index])
        wl = dataclasses.replace(wl, requests=wl.requests.subset(np.nonzero(ks <= 9)[0]))
    ex, bd = _both_modes(M, ctx, wl)
    for i in range(len(wl.requests)):
        k = wl.requests.patterns[wl.requests.pattern_index[i]].k
        assert _key(bd[i], k) == _key(ex[i], k), (name, i, bd[i], ex[i])
        assert int(bd[i]["count"]) == 0
    assert int((ex["status"] == OK).sum()) > 0


# (graph, pattern, whether the exhaustive oracle also judges policy (1, 1):
# only where it finishes in well under a minute on one host core)
@pytest.mark.parametrize("name,kind,k,full", [
    ("dragonfly128", "ring", 8, False), ("dragonfly128", "tree", 7, False), ("dragonfly128", "clique", 4, True),
    ("dragonfly128", "path", 8, False), ("boards256", "ring", 8, True), ("boards256", "tree", 7, False),
    ("boards256", "path", 8, False), ("torus64", "tree", 7, True), ("torus64", "path", 8, True),
])
def test_bounded_idle_large_graphs_match_oracle(M, ctx, name, kind, k, full):
    """Idle large graphs, three policies.  The bounded decision is judged
    by the GPU's own exhaustive mode (no cut-offs, so it shares no bound with
    either bounded search) and by the oracle's bounded search; where marked,
    the exhaustive oracle also judges the (1, 1) decision and its count."""
    topo = W.workload(name, num_requests=1).topology
    p = W.pattern(kind, k)
    tid = ctx.topology_load(topo)
    pid = ctx.pattern_load(p)
    inst = O.Instance.from_topology(topo)
    idle = np.zeros(topo.n, bool)
    for al, be in ((1, 1), (1, 0), (2, 1)):
        zero = np.zeros((1, 8), np.uint32)
        res = ctx.allocate_batch(tid, M.make_requests([pid], al, be, zero, mode=M.MAPA_MODE_BOUNDED))
        ex = ctx.allocate_batch(tid, M.make_requests([pid], al, be, zero))
        assert _key(res[0], k) == _key(ex[0], k), (name, kind, k, al, be, res[0], ex[0])
        assert int(res[0]["count"]) == 0 and int(ex[0]["count"]) > 0
        d = inst.decide_bounded(idle, k, p.a, p.b, al, be, max_nodes=5_000_000)
        assert _key(res[0], k) == _dec_key(d, k), (name, kind, k, al, be, res[0], d)
        if full and (al, be) == (1, 1):
            f = inst.decide(idle, k, p.a, p.b, al, be)
            assert _key(ex[0], k) == _dec_key(f, k) and int(ex[0]["count"]) == f.classes


def test_bounded_dragonfly_served_masks_match_oracle(M, ctx):
    # Busy masks at the served trace's occupancy, patterns up to 8 vertices.
    wl = W.workload("dragonfly128", num_requests=300, seed=11)
    ks = np.asarray([wl.requests.patterns[i].k for i in wl.requests.pattern_index])
    keep = np.nonzero(ks <= 8)[0][:120]
    reqs = wl.requests.subset(keep)
    tid = ctx.topology_load(wl.topology)
    pids = [ctx.pattern_load(p) for p in reqs.patterns]
    res = ctx.allocate_batch(tid, ctx.requests(reqs, pids, mode=M.MAPA_MODE_BOUNDED))
    inst = O.Instance.from_topology(wl.topology)
    for i in range(len(reqs)):
        p = reqs.patterns[reqs.pattern_index[i]]
        busy = W.busy_to_bool(reqs.busy[i], wl.topology.n)
        d = inst.decide_bounded(busy, p.k, p.a, p.b, int(reqs.alpha[i]), int(reqs.beta[i]), max_nodes=2_000_000)
        if d.status == O.STATUS_BUDGET:
            continue
        assert _key(res[i], p.k) == _dec_key(d, p.k), (i, res[i], d)


def test_bounded_mixed_batch(M, ctx):
    # Bounded and exhaustive requests of the same patterns in one batch: each
    # keeps its own semantics (count only for the exhaustive ones).
    wl = W.workload("regular32", num_requests=800, seed=9)
    tid = ctx.topology_load(wl.topology)
    pids = [ctx.pattern_load(p) for p in wl.requests.patterns]
    ex = ctx.allocate_batch(tid, ctx.requests(wl.requests, pids))
    mixed = ctx.requests(wl.requests, pids)
    mixed["mode"][1::2] = M.MAPA_MODE_BOUNDED
    got = ctx.allocate_batch(tid, mixed)
    for i in range(len(wl.requests)):
        k = wl.requests.patterns[wl.requests.pattern_index[i]].k
        assert _key(got[i], k) == _key(ex[i], k)
        assert int(got[i]["count"]) == (0 if i % 2 else int(ex[i]["count"]))


def test_bounded_chunked_path(M):
    # A frontier cap small enough that groups spill to the host-driven
    # chunked path, where the count and write passes both apply the cut-offs.
    wl = W.workload("regular32", num_requests=600, seed=4)
    with M.Context(0, frontier_mem_cap=64 << 20) as small:
        ex, bd = _both_modes(M, small, wl)
        st = small.stats()
    for i in range(len(wl.requests)):
        k = wl.requests.patterns[wl.requests.pattern_index[i]].k
        assert _key(bd[i], k) == _key(ex[i], k)
    assert st["kernel_launches"] > 0


def test_bounded_negative_weights_fall_back_to_full_enumeration(M, ctx):
    wl = W.workload("cube_mesh8", num_requests=300, seed=6)
    reqs = wl.requests
    reqs = W.Requests(reqs.patterns, reqs.pattern_index, np.full(len(reqs), -1, np.int32),
                      np.full(len(reqs), 2, np.int32), reqs.busy)
    wl2 = dataclasses.replace(wl, requests=reqs)
    ex, bd = _both_modes(M, ctx, wl2)
    for i in range(len(reqs)):
        k = reqs.patterns[reqs.pattern_index[i]].k
        assert _key(bd[i], k) == _key(ex[i], k)


def test_bounded_no_fit_and_budget(M, ctx):
    topo = W.torus3d(4)
    tid = ctx.topology_load(topo)
    c3 = ctx.pattern_load(W.pattern("clique", 3))  # no triangles in the torus
    req = M.make_requests([c3], 1, 1, np.zeros((1, 8), np.uint32), mode=M.MAPA_MODE_BOUNDED)
    assert int(ctx.allocate_batch(tid, req)[0]["status"]) == NO_FIT
    # with a negative weight nothing is cut, so a tiny budget is exceeded
    r8 = ctx.pattern_load(W.pattern("ring", 8))
    req = M.make_requests([r8], -1, 1, np.zeros((1, 8), np.uint32), max_embeddings=10, mode=M.MAPA_MODE_BOUNDED)
    assert int(ctx.allocate_batch(tid, req)[0]["status"]) == M.MAPA_E_BUDGET


def test_bounded_sequential_commits(M):
    # Sequential batches commit each decision; bounded and exhaustive runs
    # must leave the same decisions and the same occupancy.
    wl = W.workload("dragonfly128", num_requests=40, seed=2)
    ks = np.asarray([wl.requests.patterns[i].k for i in wl.requests.pattern_index])
    reqs = wl.requests.subset(np.nonzero(ks <= 8)[0])
    reqs = W.Requests(reqs.patterns, reqs.pattern_index, reqs.alpha, reqs.beta, np.zeros_like(reqs.busy))
    out = {}
    for mode in (M.MAPA_MODE_EXHAUSTIVE, M.MAPA_MODE_BOUNDED):
        with M.Context(0) as c:
            tid = c.topology_load(wl.topology)
            pids = [c.pattern_load(p) for p in reqs.patterns]
            res = c.allocate_batch(tid, c.requests(reqs, pids, mode=mode), M.MAPA_BATCH_SEQUENTIAL)
            out[mode] = ([_key(res[i], reqs.patterns[reqs.pattern_index[i]].k) for i in range(len(reqs))],
                         tuple(int(x) for x in c.occupancy(tid)))
    assert out[M.MAPA_MODE_BOUNDED] == out[M.MAPA_MODE_EXHAUSTIVE]


def test_bounded_single_request_call(M, ctx):
    topo = W.workload("dragonfly128", num_requests=1).topology
    with M.Context(0) as c:
        tid = c.topology_load(topo)
        pid = c.pattern_load(W.pattern("ring", 8))
        r = c.allocate(tid, pid, 1, 1, mode=M.MAPA_MODE_BOUNDED)
        p = W.pattern("ring", 8)
        d = O.Instance.from_topology(topo).decide_bounded(np.zeros(topo.n, bool), 8, p.a, p.b, 1, 1)
        assert _key(r, 8) == _dec_key(d, 8)
        assert int(r["job_id"]) >= 1 and int(r["count"]) == 0


def test_bounded_served_decisions_equal_exhaustive_on_their_snapshot(M):
    # The served loop with bounded-mode requests (parallel pass and chain):
    # every decision equals the exhaustive decision for that request alone
    # against the occupancy snapshot the server decided it on.
    tr = W.served_trace(400, rate=2e4, kmax_rt=7, seed=8)
    with M.Context(0) as c:
        tid = c.topology_load(tr.topology)
        pids = np.asarray([c.pattern_load(p) for p in tr.patterns], np.int32)
        ev = M.make_events(pids[tr.pattern_index], tr.at_ns, tr.lifetime_ns)
        ev["mode"] = M.MAPA_MODE_BOUNDED
        srv = M.mapa_serve_open(c.h, tid, 128, 0)
        try:
            M.mapa_serve_submit(srv, ev)
            M.mapa_serve_drain(srv, timeout_ms=120_000)
            out = M.mapa_serve_poll(srv, max_events=len(ev) + 16)
        finally:
            M.mapa_serve_close(srv)
        assert len(out) == len(ev)
        out = out[np.argsort(out["request_id"])]
        tid2 = c.topology_load(tr.topology)
        ref = c.allocate_batch(tid2, M.make_requests(ev["pattern_id"], 1, 1, out["snapshot"]))
    for i in range(len(ev)):
        k = tr.patterns[tr.pattern_index[i]].k
        assert _key(out["result"][i], k) == _key(ref[i], k), (i, out["result"][i], ref[i])
        assert int(out["result"][i]["count"]) == 0
