"""GPU parity on the 256-vertex boards topology with its large patterns.

The workload: 32 boards of 8 accelerators (hybrid cube-mesh inside a board,
uplinks 0..3 of board b linked to those of board b + 1) and the patterns
ring-32, tree-31 and clique-8.  On a mostly idle machine the exact decision
for ring-32 or tree-31 is beyond any enumeration (the search visits about
10^10 partial matches on a single fully free 4-board region), so the parity
cases use free sets where the oracle finishes:

* ring-32 on "ladders": uplink j of every board (a 32-cycle through the
  uplinks) plus uplink j' of a run of 16-18 consecutive boards, which adds
  32-cycles that cross between the two rims;
* tree-31 on the vertex sets of placements of the 31-vertex binary tree
  (tests/golden/config5_tree_images.json) plus a few free neighbours, which
  adds other placements;
* clique-8, which never fits (a board holds no 5-clique).

Every case is decided by the exhaustive oracle (search-node cap; capped
cases are skipped and the compared count is asserted) and by the GPU in
exhaustive and bounded mode, in one mixed batch.  The tuples have 31-32
entries, so the frontier's tuple columns 5-8 (pattern vertices 16-31) are
written and read.  The work budget is checked on requests that cannot be
finished: they end with MAPA_E_BUDGET, the same way on every run, while the
other requests of the batch keep their exact results.
"""

import json
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from oracle import oracle as O
from paper_2110_03214_gb300 import build as B
from paper_2110_03214_gb300 import workloads as W

pytestmark = pytest.mark.gpu

OK, NO_FIT, E_BUDGET = 0, 1, -5
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def M():
    B.build()
    from paper_2110_03214_gb300 import mapa

    return mapa


@pytest.fixture(scope="module")
def env(M):
    wl = W.workload("boards256", num_requests=1)
    topo = wl.topology
    ctx = M.Context(0)
    tid = ctx.topology_load(topo)
    pats = {name: W.pattern(*name) for name in (("ring", 32), ("tree", 31), ("clique", 8))}
    pids = {name: ctx.pattern_load(p) for name, p in pats.items()}
    yield ctx, topo, tid, pats, pids
    ctx.close()


def _adjacency(topo):
    adj = {v: set() for v in range(topo.n)}
    for a, b in zip(topo.u, topo.v):
        adj[int(a)].add(int(b))
        adj[int(b)].add(int(a))
    return adj


def _ladder(j, j2, first, length):
    rim = {8 * b + j for b in range(32)}
    return rim | {8 * ((first + b) % 32) + j2 for b in range(length)}


def _cases(topo):
    """(pattern name, free set, alpha, beta) of every parity case."""
    cases = []
    for j, j2, first, length, al, be in ((0, 1, 0, 16, 1, 1), (1, 2, 5, 16, 1, 1), (2, 3, 11, 17, 1, 1),
                                         (3, 0, 20, 16, 1, 0), (0, 2, 27, 16, 2, 1), (1, 3, 8, 18, 0, 1)):
        cases.append((("ring", 32), _ladder(j, j2, first, length), al, be))
    rng = W.Rng(5, 31)
    for j in range(4):
        rim = {8 * b + j for b in range(32)}
        extra = {int(x) for x in rng.integers(0, topo.n - 1, 10)}
        cases.append((("ring", 32), rim | extra, 1, 1))
    adj = _adjacency(topo)
    with open(os.path.join(HERE, "golden", "config5_tree_images.json")) as f:
        images = json.load(f)["images"]
    rng = W.Rng(7, 7)
    for im in images:
        base = set(im["free"])
        around = sorted({y for x in base for y in adj[x]} - base)
        for extra, (al, be) in zip((0, 2, 4), ((1, 1), (1, 0), (1, 1))):
            pick = {int(around[i]) for i in rng.permutation(len(around))[:extra]}
            cases.append((("tree", 31), base | pick, al, be))
    for frac in (0.0, 0.5):
        keep = W.Rng(9, int(frac * 10)).uniform(topo.n) >= frac
        cases.append((("clique", 8), set(np.nonzero(keep)[0].tolist()), 1, 1))
    return cases


def _busy(topo, free):
    busy = np.ones(topo.n, bool)
    busy[sorted(free)] = False
    return busy


def _mask(busy):
    m = np.zeros(8, np.uint64)
    for v in np.nonzero(busy)[0]:
        m[v >> 5] |= np.uint64(1) << np.uint64(v & 31)
    return m.astype(np.uint32)


def _requests(M, topo, pids, cases, mode):
    names = [c[0] for c in cases]
    masks = np.stack([_mask(_busy(topo, c[1])) for c in cases])
    return M.make_requests(np.asarray([pids[n] for n in names], np.int32), np.asarray([c[2] for c in cases]),
                           np.asarray([c[3] for c in cases]), masks, mode=mode)


def _oracle(topo, pats, cases, max_nodes=200_000_000):
    inst = O.Instance.from_topology(topo)

    def one(c):
        p = pats[c[0]]
        return inst.decide(_busy(topo, c[1]), p.k, p.a, p.b, c[2], c[3], max_nodes=max_nodes)

    with ThreadPoolExecutor(os.cpu_count() or 8) as ex:
        return list(ex.map(one, cases))


def _key(r, k):
    st = int(r["status"])
    return (st, int(r["score"]), int(r["agg"]), int(r["pres"]), tuple(int(x) for x in r["verts"][:k]) if st == OK else ())


def test_large_patterns_match_oracle(M, env):
    ctx, topo, tid, pats, pids = env
    cases = _cases(topo)
    ex = ctx.allocate_batch(tid, _requests(M, topo, pids, cases, M.MAPA_MODE_EXHAUSTIVE))
    bd = ctx.allocate_batch(tid, _requests(M, topo, pids, cases, M.MAPA_MODE_BOUNDED))
    decs = _oracle(topo, pats, cases)
    compared = {("ring", 32): 0, ("tree", 31): 0, ("clique", 8): 0}
    classes = {("ring", 32): 0, ("tree", 31): 0}
    for i, (c, d) in enumerate(zip(cases, decs)):
        k = pats[c[0]].k
        assert _key(bd[i], k) == _key(ex[i], k), (i, c[0], bd[i], ex[i])
        assert int(bd[i]["count"]) == 0
        if d.status == O.STATUS_BUDGET:
            continue
        if d.status == O.STATUS_OK:
            want = (OK, d.score, d.agg, d.pres, tuple(d.tuple))
            assert _key(ex[i], k) == want, (i, c[0], ex[i], d)
            assert int(ex[i]["count"]) == d.classes, (i, c[0], int(ex[i]["count"]), d.classes)
            classes[c[0]] += d.classes
        else:
            assert d.status == O.STATUS_NO_MATCH and int(ex[i]["status"]) == NO_FIT, (i, c[0], ex[i], d)
        compared[c[0]] += 1
    assert compared[("ring", 32)] >= 9 and compared[("tree", 31)] >= 11 and compared[("clique", 8)] == 2, compared
    # several placements to choose from, not only forced ones
    assert classes[("ring", 32)] > compared[("ring", 32)] and classes[("tree", 31)] > compared[("tree", 31)]


def test_work_budget_on_unfinishable_requests(M, env):
    """Idle-machine ring-32 and tree-31 requests cannot be finished: under a
    work budget they end with MAPA_E_BUDGET (count 0, nothing chosen), the
    same way on every run and in either mode, and the finishable requests of
    the same batch keep their exact decisions."""
    ctx, topo, tid, pats, pids = env
    cases = _cases(topo)[:4] + _cases(topo)[10:13]
    idle = [(("ring", 32), set(range(topo.n)), 1, 1), (("tree", 31), set(range(topo.n)), 1, 1),
            (("ring", 32), set(range(64)), 1, 1)]
    want = ctx.allocate_batch(tid, _requests(M, topo, pids, cases, M.MAPA_MODE_EXHAUSTIVE))
    ctx.set_work_budget(1 << 23)
    try:
        for mode in (M.MAPA_MODE_EXHAUSTIVE, M.MAPA_MODE_BOUNDED):
            reqs = _requests(M, topo, pids, idle + cases, mode)
            first = ctx.allocate_batch(tid, reqs)
            again = ctx.allocate_batch(tid, reqs)
            assert np.array_equal(first, again)
            for i in range(len(idle)):
                assert int(first[i]["status"]) == E_BUDGET and int(first[i]["count"]) == 0, first[i]
                assert not first[i]["verts"].any()
            for i, c in enumerate(cases):
                k = pats[c[0]].k
                got = first[len(idle) + i]
                assert _key(got, k) == _key(want[i], k)
                if mode == M.MAPA_MODE_EXHAUSTIVE:
                    assert int(got["count"]) == int(want[i]["count"])
        # a single call under the budget behaves the same
        st = ctx.allocate_batch(tid, _requests(M, topo, pids, idle[:1], M.MAPA_MODE_BOUNDED))
        assert int(st[0]["status"]) == E_BUDGET
    finally:
        ctx.set_work_budget(0)


def test_frontier_chunks_with_large_patterns(M):
    """A 512 MiB frontier cap (room for little more than one 1024-parent tile
    of children per level at k = 32) forces the chunked, depth-first path on the
    ring-32 ladders; the decisions are those of the default cap."""
    wl = W.workload("boards256", num_requests=1)
    topo = wl.topology
    pats = {("ring", 32): W.pattern("ring", 32), ("tree", 31): W.pattern("tree", 31)}
    cases = [c for c in _cases(topo) if c[0] in pats][:8]
    out = []
    for cap in (0, 512 << 20):
        with M.Context(0, frontier_mem_cap=cap) as ctx:
            tid = ctx.topology_load(topo)
            pids = {n: ctx.pattern_load(p) for n, p in pats.items()}
            out.append(ctx.allocate_batch(tid, _requests(M, topo, pids, cases, M.MAPA_MODE_EXHAUSTIVE)))
    assert np.array_equal(out[0], out[1])
    assert (out[0]["status"] == OK).sum() >= 6


def test_anytime_past_budget(M, env):
    """MAPA_POLICY_ANYTIME in bounded mode: a request past the work budget
    returns a real match (status MAPA_INEXACT) whose score, AggBW and
    PreservedBW the oracle recomputes from its tuple, the same on every run;
    a request that finishes within the budget keeps its exact result; and a
    sequential batch commits the inexact decisions to the occupancy."""
    ctx, topo, tid, pats, pids = env
    cases = _cases(topo)[:3] + _cases(topo)[10:13] + _cases(topo)[-1:]
    heavy = [(("ring", 32), set(range(topo.n)), 1, 1), (("tree", 31), set(range(topo.n)), 1, 1),
             (("ring", 32), set(range(64)), 1, 1), (("tree", 31), set(range(80, 136)), 1, 0),
             (("ring", 32), set(range(40, 88)), 2, 1)]
    exact = ctx.allocate_batch(tid, _requests(M, topo, pids, cases, M.MAPA_MODE_BOUNDED))
    inst = O.Instance.from_topology(topo)
    ctx.set_work_budget(1 << 23)
    try:
        reqs = _requests(M, topo, pids, heavy + cases, M.MAPA_MODE_BOUNDED)
        reqs["flags"] |= M.MAPA_POLICY_ANYTIME
        first = ctx.allocate_batch(tid, reqs)
        assert np.array_equal(first, ctx.allocate_batch(tid, reqs))
        # the fallback depends on the request alone: the same on its own
        for i in (0, 2):
            assert np.array_equal(ctx.allocate_batch(tid, reqs[i:i + 1])[0], first[i])
        # the guided dive finds a match on the idle machine; on narrower free
        # sets it may not (then MAPA_E_BUDGET)
        assert int(first[0]["status"]) == M.MAPA_INEXACT and int(first[1]["status"]) == M.MAPA_INEXACT
        for i, c in enumerate(heavy):
            r, p = first[i], pats[c[0]]
            assert int(r["status"]) in (M.MAPA_INEXACT, M.MAPA_E_BUDGET) and int(r["count"]) == 0, r
            if int(r["status"]) != M.MAPA_INEXACT:
                assert not r["verts"].any()
                continue
            st, agg, pres, score = inst.score_tuple(_busy(topo, c[1]), p.k, p.a, p.b, c[2], c[3], r["verts"][: p.k])
            assert (st, agg, pres, score) == (0, int(r["agg"]), int(r["pres"]), int(r["score"])), (i, r)
        for i, c in enumerate(cases):
            k = pats[c[0]].k
            assert _key(first[len(heavy) + i], k) == _key(exact[i], k)
        # the inexact decisions commit like exact ones
        seq = _requests(M, topo, pids, heavy[:1] * 3, M.MAPA_MODE_BOUNDED)
        seq["flags"] |= M.MAPA_POLICY_ANYTIME
        seq["busy"][:] = 0
        done = ctx.allocate_batch(tid, seq, M.MAPA_BATCH_SEQUENTIAL)
        occ = ctx.occupancy(tid)
        held = set()
        for r in done:
            if int(r["status"]) in (M.MAPA_OK, M.MAPA_INEXACT):
                assert int(r["job_id"]) > 0
                vs = set(int(x) for x in r["verts"][:32])
                assert not (vs & held)
                held |= vs
        assert len(held) >= 64
        for v in held:
            assert (int(occ[v >> 5]) >> (v & 31)) & 1
        for r in done:
            if int(r["job_id"]) > 0:
                ctx.release(tid, int(r["job_id"]))
        assert not ctx.occupancy(tid).any()
    finally:
        ctx.set_work_budget(0)


def test_budget_with_chunked_frontier(M):
    """The work budget on the chunked path: with a 1 GiB frontier cap the
    served-snapshot requests' levels are produced in many chunks, and a
    request can pass its budget between the count pass of a level and a
    later chunk's write pass; the results equal those with a 16 GiB cap."""
    wl = W.workload("boards256", num_requests=300)
    out = []
    for cap in (16 << 30, 1 << 30):
        with M.Context(0, frontier_mem_cap=cap) as ctx:
            tid = ctx.topology_load(wl.topology)
            pids = [ctx.pattern_load(p) for p in wl.requests.patterns]
            reqs = ctx.requests(wl.requests, pids)
            reqs["flags"] |= M.MAPA_POLICY_ANYTIME
            ctx.set_work_budget(1 << 20)
            out.append(ctx.allocate_batch(tid, reqs))
            st = ctx.stats()
            assert st["expand_launches"] > 0
    assert np.array_equal(out[0], out[1])
    statuses = set(int(x) for x in out[0]["status"])
    assert {M.MAPA_INEXACT, M.MAPA_NO_FIT} <= statuses


@pytest.mark.parametrize("mode", [0, 1])
def test_anytime_with_shared_group_arrays(M, mode):
    """With per-kernel timing on, the pattern groups of a batch run one after
    another in one slot, sharing its per-request arrays, as they do whenever
    a batch has more groups than slots; an overflowed group redone on the
    chunked path must not see another group's state.  The anytime results
    under the work budget equal those of the concurrent run."""
    wl = W.workload("boards256", num_requests=300)
    with M.Context(0) as ctx:
        tid = ctx.topology_load(wl.topology)
        pids = [ctx.pattern_load(p) for p in wl.requests.patterns]
        reqs = ctx.requests(wl.requests, pids, mode=mode)
        reqs["flags"] |= M.MAPA_POLICY_ANYTIME
        ctx.set_work_budget(1 << 20)
        want = ctx.allocate_batch(tid, reqs)
        ctx.set_timing(True)
        got = ctx.allocate_batch(tid, reqs)
        ctx.set_timing(False)
    assert np.array_equal(got, want)
    assert int((want["status"] == M.MAPA_INEXACT).sum()) > 0


def test_budget_size_does_not_change_the_boards_decisions(M):
    """On the boards stream no ring-32 or tree-31 enumeration finishes within
    a work budget of 2^16 or of 2^20 partial matches, and every clique-8
    no-fit is proven far below either: the two budgets give the same result
    for every request (the benchmark's boards line runs at 2^16)."""
    wl = W.workload("boards256", num_requests=300)
    with M.Context(0) as ctx:
        tid = ctx.topology_load(wl.topology)
        pids = [ctx.pattern_load(p) for p in wl.requests.patterns]
        reqs = ctx.requests(wl.requests, pids)
        reqs["flags"] |= M.MAPA_POLICY_ANYTIME
        got = []
        for b in (1 << 16, 1 << 20):
            ctx.set_work_budget(b)
            got.append(ctx.allocate_batch(tid, reqs))
        ctx.set_work_budget(0)
    assert np.array_equal(got[0], got[1])
    st = got[0]["status"]
    assert int((st == M.MAPA_INEXACT).sum()) > 50 and int((st == M.MAPA_NO_FIT).sum()) >= 90


@pytest.mark.parametrize("name,mode", [("boards256", 0), ("boards256", 1), ("dragonfly128", 0)])
def test_block_dive_equals_the_one_warp_dive(M, monkeypatch, name, mode):
    """The guided dive of an anytime request runs on a block, its choices of
    phi(0) searched eight at a time; its outcome (fallback match, no-fit
    proof, bounded-mode seed) equals that of the one-warp dive for every
    request (MAPA_DIVE_BLOCK=0 selects the one-warp form)."""
    wl = W.workload(name, num_requests=300)
    out = []
    for flag in ("0", "1"):
        monkeypatch.setenv("MAPA_DIVE_BLOCK", flag)
        with M.Context(0) as ctx:
            tid = ctx.topology_load(wl.topology)
            pids = [ctx.pattern_load(p) for p in wl.requests.patterns]
            reqs = ctx.requests(wl.requests, pids, mode=mode)
            reqs["flags"] |= M.MAPA_POLICY_ANYTIME
            ctx.set_work_budget(1 << 16)
            out.append(ctx.allocate_batch(tid, reqs))
    assert np.array_equal(out[0], out[1])
    if name == "boards256":
        assert int((out[1]["status"] == M.MAPA_INEXACT).sum()) > 50


@pytest.mark.parametrize("env", [{"MAPA_DIVE_EAGER": "0"}, {"MAPA_HOST_HINT": "0"}])
def test_eager_dive_and_host_hint_keep_the_results(M, monkeypatch, env):
    """Two scheduling choices of the chunked path that must not change any
    result: the anytime dives started beside the enumeration (side stream)
    instead of after it, and a group sent straight to the chunked path after
    its device-driven run overflowed.  Three batches under a 1 GiB frontier
    cap (the first overflows, the others follow the hint) equal the same
    batches with the choice switched off."""
    wl = W.workload("boards256", num_requests=300)
    out = []
    for on in (False, True):
        for k, v in env.items():
            if on:
                monkeypatch.delenv(k, raising=False)
            else:
                monkeypatch.setenv(k, v)
        with M.Context(0, frontier_mem_cap=1 << 30) as ctx:
            tid = ctx.topology_load(wl.topology)
            pids = [ctx.pattern_load(p) for p in wl.requests.patterns]
            reqs = ctx.requests(wl.requests, pids)
            reqs["flags"] |= M.MAPA_POLICY_ANYTIME
            ctx.set_work_budget(1 << 16)
            out.append([ctx.allocate_batch(tid, reqs) for _ in range(3)])
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)
    assert all(np.array_equal(out[1][0], x) for x in out[1][1:])
