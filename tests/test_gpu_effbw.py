"""GPU parity of bandwidth-sensitive requests (Algorithm 1, first branch).

A request with MAPA_POLICY_BW_SENSITIVE gets the match with the largest
Predicted Effective Bandwidth (Eq. 2), ties to the lexicographically smallest
tuple; result.score = round(1000 * EffBW).  Compared bit-exactly (status,
AggBW, PreservedBW, count, tuple) with the oracle's oracle_decide_effbw,
through every driver.  The reported milli-GB/s value may differ by one:
with three-decimal coefficients Eq. 2 can land exactly on a half-milli value,
which two independent double evaluations round to either side.  The choice
itself cannot differ: the host-side test shows both rank every link-count
triple in the same order.
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


def _want(dec, k):
    if dec.status == O.STATUS_NO_MATCH:
        return (NO_FIT, 0, 0, 0, 0, ())
    assert dec.status == O.STATUS_OK, dec
    return (OK, dec.score, dec.agg, dec.pres, dec.classes, tuple(dec.tuple))


def _got(r, k):
    st = int(r["status"])
    if st != OK:
        return (st, 0, 0, 0, int(r["count"]), ())
    return (st, int(r["score"]), int(r["agg"]), int(r["pres"]), int(r["count"]),
            tuple(int(x) for x in r["verts"][:k]))


def _sensitive(M, ctx, topo, reqs, flags=0):
    tid = ctx.topology_load(topo)
    pids = [ctx.pattern_load(p) for p in reqs.patterns]
    q = ctx.requests(reqs, pids)
    q["flags"] = M.MAPA_POLICY_BW_SENSITIVE
    return ctx.allocate_batch(tid, q, flags)


def _same(got, want):
    # exact except the reported milli-GB/s value (index 1), within one
    return got[:1] + got[2:] == want[:1] + want[2:] and abs(got[1] - want[1]) <= 1


def _check_against_oracle(topo, reqs, res, idx):
    inst = O.Instance.from_topology(topo)
    for i in idx:
        p = reqs.patterns[reqs.pattern_index[i]]
        busy = W.busy_to_bool(reqs.busy[i], topo.n)
        dec, _ = inst.decide_effbw(busy, p.k, p.a, p.b)
        assert _same(_got(res[i], p.k), _want(dec, p.k)), (i, res[i], dec)


def test_worked_example_ideal_allocation(M, ctx):
    topo = W.dgx_fixture()
    tid = ctx.topology_load(topo)
    pid = ctx.pattern_load(W.pattern("clique", 3))
    req = M.make_requests([pid], 1, 1, np.zeros((1, 8), np.uint32), flags=M.MAPA_POLICY_BW_SENSITIVE)
    r = ctx.allocate_batch(tid, req)[0]
    p = W.pattern("clique", 3)
    dec, xyz = O.Instance.from_topology(topo).decide_effbw(np.zeros(8, bool), 3, p.a, p.b)
    assert xyz == (2, 1, 0)
    assert _same(_got(r, 3), _want(dec, 3))
    assert int(r["score"]) == 57857 and int(r["agg"]) == 125


def test_dgx_fixture_random_busy_with_pcie(M, ctx):
    # fill 12 makes every unlinked pair a PCIe link, so z counts too
    topo = W.dgx_fixture()
    rng = W.Rng(77, 2)
    pats = [W.pattern("ring", 4), W.pattern("clique", 3), W.pattern("tree", 5), W.pattern("path", 3),
            W.pattern("ring", 2), W.pattern("clique", 5)]
    n = 240
    idx = rng.integers(0, len(pats) - 1, n).astype(np.int32)
    busy = np.zeros((n, 8), np.uint32)
    for i in range(n):
        for v in range(8):
            if rng.uniform(1)[0] < 0.3:
                busy[i, 0] |= np.uint32(1 << v)
    reqs = W.Requests(pats, idx, np.ones(n, np.int32), np.ones(n, np.int32), busy)
    res = _sensitive(M, ctx, topo, reqs)
    _check_against_oracle(topo, reqs, res, range(n))


def test_cube_mesh_every_request(M, ctx):
    wl = W.workload("cube_mesh8")
    res = _sensitive(M, ctx, wl.topology, wl.requests)
    _check_against_oracle(wl.topology, wl.requests, res, range(len(wl.requests)))


def test_regular32_sample(M, ctx):
    wl = W.workload("regular32", num_requests=3000, seed=13)
    res = _sensitive(M, ctx, wl.topology, wl.requests)
    rng = W.Rng(13, 9)
    sample = sorted(set(rng.integers(0, len(wl.requests) - 1, 48).tolist()))
    _check_against_oracle(wl.topology, wl.requests, res, sample)


def test_mixed_batch_keeps_each_branch(M, ctx):
    wl = W.workload("regular32", num_requests=600, seed=14)
    tid = ctx.topology_load(wl.topology)
    pids = [ctx.pattern_load(p) for p in wl.requests.patterns]
    plain = ctx.allocate_batch(tid, ctx.requests(wl.requests, pids))
    q = ctx.requests(wl.requests, pids)
    q["flags"][::3] = M.MAPA_POLICY_BW_SENSITIVE
    mixed = ctx.allocate_batch(tid, q)
    sens = ctx.allocate_batch(tid, _flagged(M, ctx.requests(wl.requests, pids)))
    for i in range(len(wl.requests)):
        want = sens[i] if i % 3 == 0 else plain[i]
        assert np.array_equal(mixed[i], want), i


def _flagged(M, q):
    q["flags"] = M.MAPA_POLICY_BW_SENSITIVE
    return q


def test_chunked_path(M):
    wl = W.workload("regular32", num_requests=500, seed=15)
    with M.Context(0, frontier_mem_cap=64 << 20) as small:
        res = _sensitive(M, small, wl.topology, wl.requests)
    with M.Context(0) as big:
        ref = _sensitive(M, big, wl.topology, wl.requests)
    assert np.array_equal(res, ref)
    _check_against_oracle(wl.topology, wl.requests, res, range(0, len(wl.requests), 25))


def test_bounded_mode_makes_no_cut_for_sensitive(M, ctx):
    wl = W.workload("cube_mesh8", num_requests=300, seed=16)
    tid = ctx.topology_load(wl.topology)
    pids = [ctx.pattern_load(p) for p in wl.requests.patterns]
    ex = ctx.allocate_batch(tid, _flagged(M, ctx.requests(wl.requests, pids)))
    q = _flagged(M, ctx.requests(wl.requests, pids))
    q["mode"] = M.MAPA_MODE_BOUNDED
    bd = ctx.allocate_batch(tid, q)
    for i in range(len(wl.requests)):
        k = wl.requests.patterns[wl.requests.pattern_index[i]].k
        assert _got(bd[i], k)[:4] + _got(bd[i], k)[5:] == _got(ex[i], k)[:4] + _got(ex[i], k)[5:]
        assert int(bd[i]["count"]) == 0


def test_too_many_pattern_edges(M, ctx):
    topo = W.dgx_fixture()
    tid = ctx.topology_load(topo)
    pid = ctx.pattern_load(W.pattern("clique", 12))  # 66 edges
    req = M.make_requests([pid], 1, 1, np.zeros((1, 8), np.uint32), flags=M.MAPA_POLICY_BW_SENSITIVE)
    assert int(ctx.allocate_batch(tid, req)[0]["status"]) == M.MAPA_E_RANGE


def test_sequential_commits(M):
    wl = W.workload("cube_mesh8", num_requests=30, seed=17)
    reqs = dataclasses.replace(wl, requests=W.Requests(wl.requests.patterns, wl.requests.pattern_index,
                                                       wl.requests.alpha, wl.requests.beta,
                                                       np.zeros_like(wl.requests.busy))).requests
    with M.Context(0) as c:
        tid = c.topology_load(wl.topology)
        pids = [c.pattern_load(p) for p in reqs.patterns]
        res = c.allocate_batch(tid, _flagged(M, c.requests(reqs, pids)), M.MAPA_BATCH_SEQUENTIAL)
    # replay on the oracle: each decision against the vertices the earlier ones took
    inst = O.Instance.from_topology(wl.topology)
    taken = np.zeros(wl.topology.n, bool)
    for i in range(len(reqs)):
        p = reqs.patterns[reqs.pattern_index[i]]
        dec, _ = inst.decide_effbw(taken, p.k, p.a, p.b)
        assert _same(_got(res[i], p.k), _want(dec, p.k)), i
        if dec.status == O.STATUS_OK:
            taken[list(dec.tuple)] = True


def test_served_loop(M):
    tr = W.served_trace(300, rate=2e4, kmax_rt=6, seed=9)
    with M.Context(0) as c:
        tid = c.topology_load(tr.topology)
        pids = np.asarray([c.pattern_load(p) for p in tr.patterns], np.int32)
        ev = M.make_events(pids[tr.pattern_index], tr.at_ns, tr.lifetime_ns)
        ev["flags"] = M.MAPA_POLICY_BW_SENSITIVE
        srv = M.mapa_serve_open(c.h, tid, 128, 0)
        try:
            M.mapa_serve_submit(srv, ev)
            M.mapa_serve_drain(srv, timeout_ms=120_000)
            out = M.mapa_serve_poll(srv, max_events=len(ev) + 16)
        finally:
            M.mapa_serve_close(srv)
        out = out[np.argsort(out["request_id"])]
        tid2 = c.topology_load(tr.topology)
        alone = M.make_requests(ev["pattern_id"], 1, 1, out["snapshot"], flags=M.MAPA_POLICY_BW_SENSITIVE)
        ref = c.allocate_batch(tid2, alone)
    got = out["result"].copy()
    got["job_id"] = 0
    assert np.array_equal(got, ref)
    inst = O.Instance.from_topology(tr.topology)
    for i in range(0, len(ev), 23):
        p = tr.patterns[tr.pattern_index[i]]
        dec, _ = inst.decide_effbw(W.busy_to_bool(out["snapshot"][i], tr.topology.n), p.k, p.a, p.b)
        assert _same(_got(out["result"][i], p.k), _want(dec, p.k)), i
