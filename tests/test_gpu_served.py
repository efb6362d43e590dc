"""The served loop (continuous batching) on the GPU.

* every decision equals the one the batched path makes for that request
  alone against the occupancy snapshot the server decided it on, and a
  seeded sample equals the oracle's;
* arrival-order commit: of identical requests decided in one round the first
  commits, the others are decided again in order against the live occupancy;
* departures free vertices for later arrivals; an unknown job is rejected;
* one request per round (the plain form) reproduces sequential allocation;
* FIFO waiting: a request that does not fit waits until a lifetime ends;
* lifetimes are kept on the device: a job whose lifetime ends during a
  round's chain is freed before the chain's next decision.
"""

import numpy as np
import pytest

from helpers import assert_same
from oracle import oracle as O
from paper_2110_03214_gb300 import build as B
from paper_2110_03214_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    B.build()
    from paper_2110_03214_gb300 import mapa

    return mapa


def _serve(M, ctx, tid, events, max_batch, flags=0):
    srv = M.mapa_serve_open(ctx.h, tid, max_batch, flags)
    try:
        M.mapa_serve_submit(srv, events)
        M.mapa_serve_drain(srv, timeout_ms=120_000)
        out = M.mapa_serve_poll(srv, max_events=len(events) + 16)
        counters = M.mapa_serve_counters(srv)
    finally:
        M.mapa_serve_close(srv)
    return out, counters


def test_served_decisions_equal_alone_on_their_snapshot(M):
    tr = W.served_trace(600, rate=2e4, kmax_rt=7)
    with M.Context(0) as ctx:
        tid = ctx.topology_load(tr.topology)
        pids = np.asarray([ctx.pattern_load(p) for p in tr.patterns], np.int32)
        ev = M.make_events(pids[tr.pattern_index], tr.at_ns, tr.lifetime_ns)
        out, counters = _serve(M, ctx, tid, ev, max_batch=128)
        assert len(out) == len(ev)
        assert counters["decisions"] == len(ev)
        out = out[np.argsort(out["request_id"])]
        # replay every decision alone on its snapshot through the batched path
        alone = M.make_requests(ev["pattern_id"], 1, 1, out["snapshot"])
        tid2 = ctx.topology_load(tr.topology)
        ref = ctx.allocate_batch(tid2, alone)
        got = out["result"].copy()
        got["job_id"] = 0
        assert np.array_equal(got, ref)
        assert (out["result"]["job_id"][out["result"]["status"] == 0] > 0).all()
    inst = O.Instance.from_topology(tr.topology)
    for i in range(0, len(ev), 37):
        p = tr.patterns[tr.pattern_index[i]]
        busy = W.busy_to_bool(out["snapshot"][i], tr.topology.n)
        assert_same(out["result"][i], inst.decide(busy, p.k, p.a, p.b, 1, 1), p.k, where=f"served {i}")


def test_arrival_order_commit_and_conflict_redo(M):
    topo = W.hybrid_cube_mesh8(W.Rng(1, 1))
    with M.Context(0) as ctx:
        tid = ctx.topology_load(topo)
        k4 = ctx.pattern_load(W.pattern("clique", 4))
        # 48 requests arriving together: the parallel pass runs
        ev = M.make_events([k4] * 48, [0] * 48)
        out, counters = _serve(M, ctx, tid, ev, max_batch=64, flags=M.MAPA_SERVE_REJECT)
    out = out[np.argsort(out["request_id"])]
    st = out["result"]["status"]
    assert list(st) == [0, 0] + [1] * 46  # two K4 exist; the others find none
    # all 48 chose the same K4 against the shared snapshot; the first
    # commits, the rest are decided again in arrival order in the same round
    assert list(out["rounds"]) == [1] + [2] * 47
    assert counters["conflicts"] == 47 and counters["rounds"] == 1
    first, second = (set(out["result"]["verts"][i][:4].tolist()) for i in (0, 1))
    assert first.isdisjoint(second) and first | second == set(range(8))
    assert [bin(int(x[0])).count("1") for x in out["snapshot"]] == [0, 4] + [8] * 46


def test_departure_frees_vertices(M):
    topo = W.hybrid_cube_mesh8(W.Rng(1, 1))
    with M.Context(0) as ctx:
        tid = ctx.topology_load(topo)
        k4 = ctx.pattern_load(W.pattern("clique", 4))
        srv = M.mapa_serve_open(ctx.h, tid, 4)
        try:
            M.mapa_serve_submit(srv, M.make_events([k4, k4], [0, 0]))
            M.mapa_serve_drain(srv, 60_000)
            first = M.mapa_serve_poll(srv)
            jobs = sorted(int(j) for j in first["result"]["job_id"])
            dep = np.zeros(2, M.EVENT_DTYPE)
            dep["kind"] = M.MAPA_EVENT_DEPART
            dep["job_id"] = [jobs[0], 10**9]
            dep["request_id"] = [100, 101]
            M.mapa_serve_submit(srv, dep)
            M.mapa_serve_submit(srv, M.make_events([k4], [0], request_ids=[102]))
            M.mapa_serve_drain(srv, 60_000)
            later = M.mapa_serve_poll(srv)
        finally:
            M.mapa_serve_close(srv)
    later = later[np.argsort(later["request_id"])]
    assert list(later["kind"]) == [1, 1, 0]
    assert list(later["result"]["status"]) == [0, -7, 0]
    freed = set(first["result"]["verts"][list(first["result"]["job_id"]).index(jobs[0])][:4].tolist())
    assert set(later["result"]["verts"][2][:4].tolist()) == freed


def test_one_request_per_round_is_sequential_allocation(M):
    wl = W.workload("regular32", num_requests=30)
    with M.Context(0) as ctx:
        tid = ctx.topology_load(wl.topology)
        pids = np.asarray([ctx.pattern_load(p) for p in wl.requests.patterns], np.int32)
        ids = pids[wl.requests.pattern_index]
        out, counters = _serve(M, ctx, tid, M.make_events(ids, np.zeros(len(ids), np.int64)), max_batch=1,
                               flags=M.MAPA_SERVE_REJECT)
        out = out[np.argsort(out["request_id"])]
        tid2 = ctx.topology_load(wl.topology)
        seq = ctx.allocate_batch(tid2, M.make_requests(ids, 1, 1, np.zeros((len(ids), 8), np.uint32)),
                                 M.MAPA_BATCH_SEQUENTIAL)
    assert counters["conflicts"] == 0 and counters["rounds"] == len(ids)
    assert np.array_equal(out["result"], seq)


def test_fifo_request_waits_for_a_departure(M):
    topo = W.hybrid_cube_mesh8(W.Rng(1, 1))
    with M.Context(0) as ctx:
        tid = ctx.topology_load(topo)
        k4 = ctx.pattern_load(W.pattern("clique", 4))
        life = 20_000_000  # 20 ms
        ev = M.make_events([k4, k4, k4], [0, 0, 0], lifetime_ns=[life, life, 0])
        out, counters = _serve(M, ctx, tid, ev, max_batch=8)
    out = out[np.argsort(out["request_id"])]
    assert list(out["result"]["status"]) == [0, 0, 0]
    third = set(out["result"]["verts"][2][:4].tolist())
    assert third in ({0, 1, 2, 3}, {4, 5, 6, 7})
    # it waited for the first lifetime to end, then took a freed K4
    assert out["done_ns"][2] - out["done_ns"][0] >= life
    assert out["rounds"][2] >= 2


def test_lifetimes_end_on_the_device_between_chain_steps(M):
    """Three clique-4 requests in one round (straight to the chain, which
    decides them one after another) on the 8-vertex cube mesh, whose two K4
    differ in weight, each with a 1 ns lifetime: each job ends on the device
    before the next decision, so all three take the same best K4 against an
    empty machine, and nothing is held afterwards."""
    topo = W.hybrid_cube_mesh8(W.Rng(1, 1))
    with M.Context(0) as ctx:
        tid = ctx.topology_load(topo)
        k4 = ctx.pattern_load(W.pattern("clique", 4))
        ev = M.make_events([k4] * 3, [0] * 3, lifetime_ns=[1] * 3)
        out, counters = _serve(M, ctx, tid, ev, max_batch=8, flags=M.MAPA_SERVE_REJECT)
        left = ctx.occupancy(tid)
        # the same requests held until released: the second takes the other K4
        ev = M.make_events([k4] * 3, [0] * 3)
        held, _ = _serve(M, ctx, tid, ev, max_batch=8, flags=M.MAPA_SERVE_REJECT)
    out = out[np.argsort(out["request_id"])]
    held = held[np.argsort(held["request_id"])]
    assert counters["rounds"] == 1
    assert list(out["result"]["status"]) == [0, 0, 0]
    tuples = {tuple(int(x) for x in out["result"]["verts"][i][:4]) for i in range(3)}
    assert len(tuples) == 1
    assert not out["snapshot"].any() and not np.asarray(left).any()
    assert list(held["result"]["status"]) == [0, 0, 1]
    assert tuple(int(x) for x in held["result"]["verts"][0][:4]) in tuples


def test_admission_keeps_to_the_frontier_memory_budget(M):
    """Under a work budget a round admits requests only while their largest
    frontiers fit the context's frontier memory: with B = 2^12 partials on
    the 32-vertex graph (degree 6: at most 7 B entries of 20 bytes for
    ring-8, 560 KiB) and a 4 MiB frontier cap (16 MiB for the four
    concurrent groups), at most 29 of 200 waiting requests enter a round;
    every decision still equals the one taken alone on its snapshot."""
    wl = W.workload("regular32", num_requests=200)
    ring8 = [i for i, p in enumerate(wl.requests.patterns) if p.name == "ring-8"][0]
    with M.Context(0, frontier_mem_cap=4 << 20) as ctx:
        ctx.set_work_budget(1 << 12)
        tid = ctx.topology_load(wl.topology)
        pids = np.asarray([ctx.pattern_load(p) for p in wl.requests.patterns], np.int32)
        ev = M.make_events(np.full(200, pids[ring8]), np.zeros(200, np.int64))
        out, counters = _serve(M, ctx, tid, ev, max_batch=4096, flags=M.MAPA_SERVE_REJECT)
        out = out[np.argsort(out["request_id"])]
        alone = M.make_requests(ev["pattern_id"], 1, 1, out["snapshot"])
        tid2 = ctx.topology_load(wl.topology)
        ref = ctx.allocate_batch(tid2, alone)
    assert len(out) == 200
    assert counters["rounds"] >= 7
    got = out["result"].copy()
    got["job_id"] = 0
    assert np.array_equal(got, ref)


def test_fifo_head_is_answered_when_its_round_released_everything(M):
    """FIFO waiting with a job that ends inside its own round: the first
    request commits a K4 with a 1 ns lifetime (freed on the device before the
    next decision), the second asks for a K8, which the 8-vertex cube mesh
    does not hold, and waits at the head of the queue.  Nothing is left to
    release, so it is answered MAPA_NO_FIT at once (no wait for a departure
    that cannot come), and the request behind it is decided next."""
    topo = W.hybrid_cube_mesh8(W.Rng(1, 1))
    with M.Context(0) as ctx:
        tid = ctx.topology_load(topo)
        k4 = ctx.pattern_load(W.pattern("clique", 4))
        k8 = ctx.pattern_load(W.pattern("clique", 8))
        ev = M.make_events([k4, k8, k4], [0, 0, 0], lifetime_ns=[1, 0, 0])
        out, counters = _serve(M, ctx, tid, ev, max_batch=8)
    out = out[np.argsort(out["request_id"])]
    assert list(out["result"]["status"]) == [0, 1, 0]
    assert counters["decisions"] == 3
