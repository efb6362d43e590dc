"""Multi-rank path of the benchmark on CPU (gloo, world size 2).

Independent requests shard over ranks with no exchange on the data path:
each rank decides its own batch of the workload's shape (weak scaling), and
the job's figures combine the slowest rank's time with the matches of all
ranks.  This checks the sharding and the combination with real
torch.distributed ranks on 127.0.0.1; the GPU part is the single-GPU path.
"""

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    from paper_2110_03214_gb300 import workloads as W

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = bench.shard_workload(W, "regular32", 50, rank)
    total_ms = 10.0 * (rank + 1)
    e2e_s = 0.5 + rank
    emb = 1000 + rank
    res = bench.combine_over_ranks(dist, "cpu", total_ms, e2e_s, emb)
    q.put((rank, res, [p.name for p in wl.requests.patterns], wl.requests.busy.copy(),
           wl.topology.u.copy(), wl.topology.v.copy()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_and_combine():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(world):
        r, *rest = q.get(timeout=120)
        out[r] = rest
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        total_ms, e2e_s, emb = out[r][0]
        assert total_ms == 20.0 and e2e_s == 1.5 and emb == 2001.0
    # same workload shape on every rank, different requests (and graphs)
    assert out[0][1] == out[1][1]
    assert out[0][2].shape == out[1][2].shape
    assert not np.array_equal(out[0][2], out[1][2])
