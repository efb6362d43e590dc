"""Multi-rank path of the benchmark on CPU (gloo, world size 2).

Independent requests shard over ranks with no exchange on the data path.
Two checks with real torch.distributed ranks on 127.0.0.1:

* one batch split into contiguous shares (shard_slice), each rank deciding
  its share -- through the oracle here, where no GPU exists -- and the
  decisions gathered on rank 0 equal the unsharded decisions of the whole
  batch, request for request;
* weak scaling (shard_workload: every rank its own batch of the workload's
  shape) with the job's figures combining the slowest rank's time and the
  matches of all ranks (combine_over_ranks).
"""

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

NREQ = 240


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _decide_all(wl, idx):
    """(status, score, agg, pres, classes, tuple) per request, from the oracle."""
    from oracle import oracle as O
    from paper_2110_03214_gb300 import workloads as W

    inst = O.Instance.from_topology(wl.topology)
    out = []
    for i in idx:
        p = wl.requests.patterns[wl.requests.pattern_index[i]]
        busy = W.busy_to_bool(wl.requests.busy[i], wl.topology.n)
        d = inst.decide(busy, p.k, p.a, p.b, int(wl.requests.alpha[i]), int(wl.requests.beta[i]))
        out.append((d.status, d.score, d.agg, d.pres, d.classes, tuple(d.tuple)))
    return out


def _rank(rank, world, port, q):
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    from paper_2110_03214_gb300 import workloads as W

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # strong split of one batch: decide the share, gather on rank 0
    wl = W.workload("regular32", num_requests=NREQ)
    lo, hi = bench.shard_slice(NREQ, rank, world)
    mine = _decide_all(wl, range(lo, hi))
    gathered = [None] * world if rank == 0 else None
    dist.gather_object((lo, hi, mine), gathered, dst=0)
    # weak scaling: own batch per rank, combined figures
    wk = bench.shard_workload(W, "regular32", 50, rank)
    res = bench.combine_over_ranks(dist, "cpu", 10.0 * (rank + 1), 0.5 + rank, 1000 + rank)
    q.put((rank, gathered, res, [p.name for p in wk.requests.patterns], wk.requests.busy.copy()))
    dist.barrier()
    dist.destroy_process_group()


def test_shard_slice_covers_every_request_once():
    import bench

    for count in (0, 1, 7, 240, 10_001):
        for world in (1, 2, 3, 8):
            spans = [bench.shard_slice(count, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == count
            assert all(spans[r][1] == spans[r + 1][0] for r in range(world - 1))
            assert max(h - l for l, h in spans) - min(h - l for l, h in spans) <= 1


def test_two_ranks_decide_their_shards():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(world):
        r, *rest = q.get(timeout=300)
        out[r] = rest
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # the union of the shards' decisions is the unsharded decision list
    from paper_2110_03214_gb300 import workloads as W

    gathered = sorted(out[0][0])
    assert [g[0] for g in gathered] == [0, NREQ // 2] and gathered[-1][1] == NREQ
    union = [d for _, _, part in gathered for d in part]
    whole = _decide_all(W.workload("regular32", num_requests=NREQ), range(NREQ))
    assert union == whole
    assert sum(1 for d in whole if d[0] == 0) > NREQ // 2
    # weak scaling: slowest rank's times, all ranks' matches
    for r in range(world):
        total_ms, e2e_s, emb = out[r][1]
        assert total_ms == 20.0 and e2e_s == 1.5 and emb == 2001.0
    assert out[0][2] == out[1][2]
    assert out[0][3].shape == out[1][3].shape and not np.array_equal(out[0][3], out[1][3])


def _rank_split(rank, world, port, q):
    """One large request split by phi(0): rank r decides its share of the
    vertex range through the oracle; rank 0 gathers one result per share
    (the exchange step) and reduces them with the library's merge."""
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    from oracle import oracle as O
    from paper_2110_03214_gb300 import mapa as M
    from paper_2110_03214_gb300 import workloads as W

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = W.workload("regular32", num_requests=12)
    inst = O.Instance.from_topology(wl.topology)
    lo, hi = bench.shard_slice(32, rank, world)
    mine = []
    for i in range(len(wl.requests)):
        p = wl.requests.patterns[wl.requests.pattern_index[i]]
        d = inst.decide_rooted(W.busy_to_bool(wl.requests.busy[i], 32), p.k, p.a, p.b, 1, 1, lo, hi)
        mine.append((d.status, d.score, d.agg, d.pres, d.maps, d.tuple, p.k))
    gathered = [None] * world if rank == 0 else None
    dist.gather_object(mine, gathered, dst=0)
    merged = None
    if rank == 0:
        merged = []
        for i in range(len(wl.requests)):
            parts = np.zeros(world, M.RESULT_DTYPE)
            for r in range(world):
                st, score, agg, pres, maps, tup, k = gathered[r][i]
                parts[r]["status"] = M.MAPA_OK if st == O.STATUS_OK else M.MAPA_NO_FIT
                parts[r]["score"], parts[r]["agg"], parts[r]["pres"] = score, agg, pres
                parts[r]["count"], parts[r]["k"] = maps, k
                parts[r]["verts"][: len(tup)] = tup
            m = M.mapa_result_merge(parts)
            merged.append((int(m["status"]), int(m["score"]), int(m["count"]), tuple(int(x) for x in m["verts"][: k])))
    q.put((rank, merged))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_split_one_request():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_split, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(world):
        r, merged = q.get(timeout=300)
        out[r] = merged
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    from oracle import oracle as O
    from paper_2110_03214_gb300 import workloads as W

    wl = W.workload("regular32", num_requests=12)
    inst = O.Instance.from_topology(wl.topology)
    for i, got in enumerate(out[0]):
        p = wl.requests.patterns[wl.requests.pattern_index[i]]
        d = inst.decide(W.busy_to_bool(wl.requests.busy[i], 32), p.k, p.a, p.b, 1, 1)
        assert got[2] == d.maps
        if d.status == O.STATUS_OK:
            assert got[0] == 0 and got[1] == d.score and got[3] == d.tuple
        else:
            assert got[0] == 1
