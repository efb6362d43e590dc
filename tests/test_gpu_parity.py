"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Bit-exact on status, score, AggBW, PreservedBW, count (matches modulo
automorphisms) and the chosen tuple.  Small cases are checked request by
request, including the full 10^4-request workload on the 32-vertex graph in
the launch configuration the benchmark times.
"""

import dataclasses
import os

import numpy as np
import pytest

from helpers import assert_same, check_result_properties, oracle_decisions
from oracle import oracle as O
from paper_2110_03214_gb300 import build as B
from paper_2110_03214_gb300 import workloads as W

pytestmark = pytest.mark.gpu


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


def _load(ctx, wl):
    tid = ctx.topology_load(wl.topology)
    pids = [ctx.pattern_load(p) for p in wl.requests.patterns]
    return tid, pids


def _run_and_compare(M, ctx, topo, reqs, idx=None, flags=0, max_maps=0):
    tid = ctx.topology_load(topo)
    pids = [ctx.pattern_load(p) for p in reqs.patterns]
    res = ctx.allocate_batch(tid, ctx.requests(reqs, pids), flags)
    inst = O.Instance.from_topology(topo)
    idx = list(range(len(reqs))) if idx is None else list(idx)
    decs = oracle_decisions(inst, topo.n, reqs, idx, max_maps=max_maps, threads=os.cpu_count() or 8)
    compared = 0
    for i, d in zip(idx, decs):
        if d.status == O.STATUS_BUDGET:
            continue
        assert_same(res[i], d, reqs.patterns[reqs.pattern_index[i]].k, where=f"request {i}")
        compared += 1
    return res, compared


def test_config1_every_request(M, ctx):
    wl = W.workload("cube_mesh8")
    _, compared = _run_and_compare(M, ctx, wl.topology, wl.requests)
    assert compared == 1000


def test_config2_every_request(M, ctx):
    """All 10^4 requests in one batch (the benchmark's workload and launch
    configuration), every decision compared with the oracle: status, score,
    AggBW, PreservedBW, count and tuple."""
    wl = W.workload("regular32")
    res, compared = _run_and_compare(M, ctx, wl.topology, wl.requests)
    assert compared == 10_000
    assert int(res["count"].sum()) > 10**7


def _config3_sample(reqs, n):
    """Seeded, input-only selection of torus requests for oracle parity: for
    every pattern of the batch (ring-k, tree-k for k in 2..16, clique-k for k
    in 2..4), the requests whose busy count is nearest to a few targets,
    lower for smaller patterns, among those with at least k free vertices
    (ties: the earlier request)."""
    busy = np.asarray([sum(bin(int(x)).count("1") for x in row) for row in reqs.busy])
    free = n - busy
    sample = []
    for pi, p in enumerate(reqs.patterns):
        targets = (38, 30, 20, 10, 4) if p.k <= 8 else ((38, 32, 26, 20) if p.k <= 12 else (38, 34, 31, 29))
        idx = np.nonzero(reqs.pattern_index == pi)[0]
        idx = idx[free[idx] >= p.k]
        chosen = []
        for tb in targets:
            for i in idx[np.argsort(np.abs(busy[idx] - tb), kind="stable")]:
                if int(i) not in chosen:
                    chosen.append(int(i))
                    break
        sample += chosen
    return sorted(sample)


def test_config3_every_pattern_size(M, ctx):
    """The torus workload's first 10^4 requests (ring/tree k in 2..16,
    clique k in 2..4, occupancy U[0, 0.6]) decided as one batch; a sample
    covering every pattern of the batch compared with the oracle (none
    skipped), every result re-scored from its tuple."""
    wl = W.workload("torus64", num_requests=10_000)
    reqs = wl.requests
    sample = _config3_sample(reqs, wl.topology.n)
    res, compared = _run_and_compare(M, ctx, wl.topology, reqs, idx=sample, max_maps=0)
    assert compared == len(sample)
    names = {reqs.patterns[reqs.pattern_index[i]].name for i in sample if int(res[i]["status"]) == 0}
    assert {f"tree-{k}" for k in range(2, 17)} <= names and {f"ring-{k}" for k in range(4, 17, 2)} <= names
    check_result_properties(O.Instance.from_topology(wl.topology), wl.topology.n, reqs, res)
    assert int(res["count"].sum()) > 10**11


def _random_busy_requests(rng, topo_n, patterns, count, lo_frac, hi_frac, alpha=1, beta=1):
    index = rng.integers(0, len(patterns) - 1, count).astype(np.int32)
    frac = lo_frac + (hi_frac - lo_frac) * rng.uniform(count)
    nbusy = np.floor(frac * topo_n).astype(np.int64)
    busy = W._busy_masks(rng, topo_n, nbusy)
    a = np.full(count, alpha, np.int32)
    b = np.full(count, beta, np.int32)
    return W.Requests(patterns, index, a, b, busy)


def test_dragonfly_128(M, ctx):
    topo = W.dragonfly(W.Rng(4, 1))
    pats = [W.pattern("ring", 4), W.pattern("ring", 6), W.pattern("tree", 5), W.pattern("tree", 7),
            W.pattern("clique", 3), W.pattern("clique", 4), W.pattern("path", 3)]
    reqs = _random_busy_requests(W.Rng(4, 7), topo.n, pats, 120, 0.55, 0.9)
    _, compared = _run_and_compare(M, ctx, topo, reqs, max_maps=3_000_000)
    assert compared >= 100


def test_boards_256(M, ctx):
    topo = W.boards256(W.Rng(5, 1))
    pats = [W.pattern("ring", 4), W.pattern("ring", 8), W.pattern("tree", 7), W.pattern("clique", 8),
            W.pattern("clique", 4), W.pattern("path", 5)]
    reqs = _random_busy_requests(W.Rng(5, 7), topo.n, pats, 80, 0.6, 0.9)
    _, compared = _run_and_compare(M, ctx, topo, reqs, max_maps=2_000_000)
    assert compared >= 60


@pytest.mark.parametrize("n", [5, 31, 32, 33, 63, 64, 65, 100, 128, 129, 200, 256])
def test_random_graphs_every_word_count(M, ctx, n):
    """Random weights (up to 8 classes), custom patterns (some disconnected), random policies."""
    rng = W.Rng(1000 + n, 1)
    deg = min(n - 1, 6)
    pairs = set()
    for v in range(n):
        for u in rng.integers(0, n - 1, deg).tolist():
            if u != v:
                pairs.add((min(u, v), max(u, v)))
    pairs = sorted(pairs)
    u = np.asarray([p[0] for p in pairs], np.int32)
    v = np.asarray([p[1] for p in pairs], np.int32)
    w = np.asarray([10, 12, 20, 25, 33, 40, 50, 64], np.int32)[rng.integers(0, 7, len(pairs))]
    topo = W.Topology(f"random-{n}", n, u, v, w)
    pats = [W.random_pattern(rng, int(k), 0.4, connected=bool(i % 3)) for i, k in enumerate(rng.integers(1, 6, 6))]
    pats += [W.pattern("ring", 5), W.pattern("tree", 6), W.pattern("path", 2), W.pattern("ring", 1)]
    reqs = _random_busy_requests(rng, n, pats, 60, 0.0 if n <= 40 else 0.5, 0.9)
    reqs.alpha[:] = rng.integers(-2, 3, len(reqs))
    reqs.beta[:] = rng.integers(-2, 3, len(reqs))
    _, compared = _run_and_compare(M, ctx, topo, reqs, max_maps=2_000_000)
    assert compared >= 30


def test_dgx_worked_example_through_gpu(M, ctx):
    topo = W.dgx_fixture()
    tid = ctx.topology_load(topo)
    pid = ctx.pattern_load(W.pattern("clique", 3))
    busy = np.zeros((1, 8), np.uint32)
    busy[0, 0] = 0xFF & ~((1 << 0) | (1 << 1) | (1 << 4))
    r = M.make_requests([pid], 1, 0, busy)
    res = ctx.allocate_batch(tid, r)[0]
    assert res["status"] == 0 and res["agg"] == 87
    r = M.make_requests([pid], 1, 0, np.zeros((1, 8), np.uint32))
    res = ctx.allocate_batch(tid, r)[0]
    assert res["status"] == 0 and res["agg"] == 125 and list(res["verts"][:3]) == [0, 2, 3]


def test_small_frontier_cap_forces_chunks(M):
    """A 64 MiB frontier forces depth-first chunking; results must not change."""
    wl = W.workload("regular32", num_requests=3000)
    with M.Context(0, frontier_mem_cap=64 << 20) as small:
        tid, pids = _load(small, wl)
        res_small = small.allocate_batch(tid, small.requests(wl.requests, pids))
        # three pattern groups; more fused-tail launches than groups means chunks were taken
        assert small.stats()["tail_launches"] > 3
    with M.Context(0) as big:
        tid, pids = _load(big, wl)
        res_big = big.allocate_batch(tid, big.requests(wl.requests, pids))
    assert np.array_equal(res_small, res_big)
    inst = O.Instance.from_topology(wl.topology)
    sample = list(range(0, 3000, 97))
    for i, d in zip(sample, oracle_decisions(inst, 32, wl.requests, sample)):
        assert_same(res_small[i], d, wl.requests.patterns[wl.requests.pattern_index[i]].k, where=f"req {i}")


def test_results_independent_of_batch_composition(M, ctx):
    wl = W.workload("regular32", num_requests=600)
    tid, pids = _load(ctx, wl)
    reqs = ctx.requests(wl.requests, pids)
    whole = ctx.allocate_batch(tid, reqs)
    rng = W.Rng(8, 8)
    perm = rng.permutation(len(reqs))
    shuffled = ctx.allocate_batch(tid, reqs[perm])
    assert np.array_equal(shuffled, whole[perm])
    for i in (0, 7, 301, 599):
        alone = ctx.allocate_batch(tid, reqs[i:i + 1])
        assert np.array_equal(alone[0], whole[i])


def test_edge_cases(M, ctx):
    topo = W.hybrid_cube_mesh8(W.Rng(1, 1))
    tid = ctx.topology_load(topo)
    ring4 = ctx.pattern_load(W.pattern("ring", 4))
    clique5 = ctx.pattern_load(W.pattern("clique", 5))
    one = ctx.pattern_load(W.pattern("ring", 1))
    allbusy = np.zeros((1, 8), np.uint32)
    allbusy[0, 0] = 0xFF
    some = np.zeros((1, 8), np.uint32)
    some[0, 0] = 0b11110000 | 0b1  # 3 free vertices < k = 4
    reqs = np.concatenate([
        M.make_requests([ring4], 1, 1, allbusy),
        M.make_requests([ring4], 1, 1, some),
        M.make_requests([clique5], 1, 1, np.zeros((1, 8), np.uint32)),
        M.make_requests([one], 0, 1, np.zeros((1, 8), np.uint32)),
        M.make_requests([1 << 30], 1, 1, np.zeros((1, 8), np.uint32)),
        M.make_requests([ring4], 1 << 24, 1, np.zeros((1, 8), np.uint32)),  # (2^24+1) * W(G) > 2^31
        M.make_requests([ring4], 1, 1, np.zeros((1, 8), np.uint32), max_embeddings=3),
    ])
    res = ctx.allocate_batch(tid, reqs)
    assert list(res["status"]) == [1, 1, 1, 0, -1, -2, -5]
    assert res["count"][3] == 8
    inst = O.Instance.from_topology(topo)
    d = inst.decide(np.zeros(8, bool), 1, [], [], 0, 1)
    assert_same(res[3], d, 1)
    assert len(ctx.allocate_batch(tid, reqs[:0])) == 0


def test_sequential_commits_and_release(M, ctx):
    """mapa_allocate commits against device occupancy (Sec. 3.6); replayed on the oracle."""
    wl = W.workload("cube_mesh8")
    tid, pids = _load(ctx, wl)
    inst = O.Instance.from_topology(wl.topology)
    busy = np.zeros(8, bool)
    jobs = []
    for step, pidx in enumerate([0, 1, 2, 2, 0]):
        p = wl.requests.patterns[pidx]
        res = ctx.allocate(tid, pids[pidx])
        d = inst.decide(busy, p.k, p.a, p.b, 1, 1)
        assert_same(res, d, p.k, where=f"step {step}")
        if d.status == O.STATUS_OK:
            assert res["job_id"] >= 1
            jobs.append((int(res["job_id"]), list(d.tuple)))
            busy[list(d.tuple)] = True
        occ = ctx.occupancy(tid)
        assert [(int(occ[0]) >> v) & 1 for v in range(8)] == busy.astype(int).tolist()
    job, verts = jobs[0]
    ctx.release(tid, job)
    busy[verts] = False
    occ = ctx.occupancy(tid)
    assert [(int(occ[0]) >> v) & 1 for v in range(8)] == busy.astype(int).tolist()
    with pytest.raises(M.MapaError) as ei:
        ctx.release(tid, job)
    assert ei.value.code == M.MAPA_E_STATE
    with pytest.raises(M.MapaError):
        ctx.release(tid, 10**9)


def test_sequential_batch_matches_replay(M, ctx):
    wl = W.workload("regular32", num_requests=40)
    tid, pids = _load(ctx, wl)
    reqs = ctx.requests(wl.requests, pids)
    reqs["busy"][:] = 0
    res = ctx.allocate_batch(tid, reqs, M.MAPA_BATCH_SEQUENTIAL)
    inst = O.Instance.from_topology(wl.topology)
    busy = np.zeros(32, bool)
    for i in range(len(reqs)):
        p = wl.requests.patterns[wl.requests.pattern_index[i]]
        d = inst.decide(busy, p.k, p.a, p.b, 1, 1)
        assert_same(res[i], d, p.k, where=f"seq {i}")
        if d.status == O.STATUS_OK:
            busy[list(d.tuple)] = True
        if busy.sum() > 24:
            break


def test_device_pointer_batch(M, ctx):
    torch = pytest.importorskip("torch")
    wl = W.workload("regular32", num_requests=500)
    tid, pids = _load(ctx, wl)
    reqs = ctx.requests(wl.requests, pids)
    host = ctx.allocate_batch(tid, reqs)
    dreq = torch.from_numpy(reqs.view(np.uint8)).cuda()
    dout = torch.zeros(len(reqs) * M.RESULT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    ctx.allocate_batch_device(tid, len(reqs), dreq.data_ptr(), dout.data_ptr())
    got = dout.cpu().numpy().view(M.RESULT_DTYPE)
    assert np.array_equal(got, host)


def test_autotune_keeps_results(M):
    """The autotuner only changes the fused tail depth, never a result."""
    wl = W.workload("torus64", num_requests=600)
    ks = np.asarray([wl.requests.patterns[i].k for i in wl.requests.pattern_index])
    reqs_w = wl.requests.subset(np.nonzero(ks <= 9)[0][:300])
    with M.Context(0) as c:
        tid = c.topology_load(wl.topology)
        pids = [c.pattern_load(p) for p in reqs_w.patterns]
        reqs = c.requests(reqs_w, pids)
        before = c.allocate_batch(tid, reqs)
        chosen = M.mapa_autotune(c.h, tid, reqs, len(pids))
        after = c.allocate_batch(tid, reqs)
    present = set(int(x) for x in reqs["pattern_id"])
    for p in range(len(pids)):
        if p in present:
            assert 1 <= chosen[p] <= min(3, reqs_w.patterns[p].k)
        else:
            assert chosen[p] == 0
    assert np.array_equal(before, after)


def test_graph_replay_matches_direct_launches(M, monkeypatch):
    """A batch shape seen twice is captured as a CUDA graph and replayed;
    replays give the results of direct launches."""
    wl = W.workload("regular32", num_requests=2000)
    monkeypatch.setenv("MAPA_GRAPHS", "0")
    with M.Context(0) as direct:
        tid, pids = _load(direct, wl)
        want = direct.allocate_batch(tid, direct.requests(wl.requests, pids))
    monkeypatch.setenv("MAPA_GRAPHS", "1")
    with M.Context(0) as graphed:
        tid, pids = _load(graphed, wl)
        reqs = graphed.requests(wl.requests, pids)
        for _ in range(4):  # run, capture, replay, replay
            got = graphed.allocate_batch(tid, reqs)
            assert np.array_equal(got, want)
        st = graphed.stats()
    assert st["requests"] == 4 * 2000 and st["kernel_launches"] > 0


@pytest.mark.parametrize("name,num", [("regular32", 3000), ("torus64", 800)])
def test_every_tail_depth_gives_the_same_results(M, monkeypatch, name, num):
    # depth 1, 2, 3 run different fused-tail forms (and 32- and 64-vertex
    # masks the short one); every result must be the same, and equal to the
    # oracle on a sample
    wl = W.workload(name, num_requests=num)
    if name == "torus64":
        ks = np.asarray([wl.requests.patterns[i].k for i in wl.requests.pattern_index])
        wl = dataclasses.replace(wl, requests=wl.requests.subset(np.nonzero(ks <= 9)[0]))
    out = {}
    for depth in (1, 2, 3):
        monkeypatch.setenv("MAPA_TAIL_DEPTH", str(depth))
        with M.Context(0) as c:
            tid = c.topology_load(wl.topology)
            pids = [c.pattern_load(p) for p in wl.requests.patterns]
            out[depth] = c.allocate_batch(tid, c.requests(wl.requests, pids))
    assert np.array_equal(out[1], out[2]) and np.array_equal(out[2], out[3])
    inst = O.Instance.from_topology(wl.topology)
    idx = list(range(0, len(wl.requests), max(1, len(wl.requests) // 40)))
    for i, d in zip(idx, oracle_decisions(inst, wl.topology.n, wl.requests, idx)):
        assert_same(out[3][i], d, wl.requests.patterns[wl.requests.pattern_index[i]].k, where=f"request {i}")


@pytest.mark.parametrize("name,num,mode", [("regular32", 600, 0), ("regular32", 600, 1), ("torus64", 800, 0),
                                           ("cube_mesh8", 300, 0)])
def test_root_split_shares_merge_to_unsplit(M, ctx, name, num, mode):
    """One request split into shares by the range of phi(0) (root_lo,
    root_hi), all shares decided in one batch and reduced with
    mapa_result_merge: status, score, AggBW, PreservedBW, count and tuple
    equal the unsplit decision (each match class is enumerated in exactly
    one share)."""
    wl = W.workload(name, num_requests=num)
    n = wl.topology.n
    tid, pids = _load(ctx, wl)
    reqs = ctx.requests(wl.requests, pids, mode=mode)
    whole = ctx.allocate_batch(tid, reqs)
    cuts = [0, n // 5, n // 2, (3 * n) // 4, n]
    shares = np.repeat(reqs, 4)
    for j in range(4):
        shares["root_lo"][j::4] = cuts[j]
        shares["root_hi"][j::4] = cuts[j + 1]
    parts = ctx.allocate_batch(tid, shares)
    for i in range(len(reqs)):
        got = M.mapa_result_merge(parts[4 * i:4 * i + 4])
        k = int(whole[i]["k"])
        want = whole[i]
        assert (int(got["status"]), int(got["score"]), int(got["agg"]), int(got["pres"]), int(got["count"])) == \
            (int(want["status"]), int(want["score"]), int(want["agg"]), int(want["pres"]), int(want["count"])), i
        assert np.array_equal(got["verts"][:k], want["verts"][:k]), i
    assert int((whole["status"] == 0).sum()) > 0


def test_root_split_when_the_tail_starts_at_vertex_zero(M, monkeypatch):
    """Patterns whose fused tail covers pattern vertex 0 (k = 1; k = 3 with a
    tail depth of 3): the share's range of phi(0) is applied inside the tail
    kernels (short tail, cooperative depth-3 tail, generic tail in bounded
    mode)."""
    monkeypatch.setenv("MAPA_TAIL_DEPTH", "3")
    topo = W.workload("regular32", num_requests=1).topology
    pats = [W.pattern("ring", 1), W.pattern("clique", 3), W.pattern("path", 3), W.pattern("tree", 3)]
    reqs_w = _random_busy_requests(W.Rng(77, 1), topo.n, pats, 200, 0.0, 0.5)
    with M.Context(0) as c:
        tid = c.topology_load(topo)
        pids = [c.pattern_load(p) for p in pats]
        for mode in (0, 1):
            reqs = c.requests(reqs_w, pids, mode=mode)
            whole = c.allocate_batch(tid, reqs)
            shares = np.repeat(reqs, 3)
            for j, (lo, hi) in enumerate(((0, 7), (7, 20), (20, 32))):
                shares["root_lo"][j::3] = lo
                shares["root_hi"][j::3] = hi
            parts = c.allocate_batch(tid, shares)
            for i in range(len(reqs)):
                got = M.mapa_result_merge(parts[3 * i:3 * i + 3])
                k = int(whole[i]["k"])
                assert (int(got["status"]), int(got["score"]), int(got["count"])) == \
                    (int(whole[i]["status"]), int(whole[i]["score"]), int(whole[i]["count"])), (mode, i)
                assert np.array_equal(got["verts"][:k], whole[i]["verts"][:k]), (mode, i)
