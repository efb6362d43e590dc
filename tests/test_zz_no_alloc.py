"""The allocation-free entry point agrees with the batched one.

mapa_allocate_batch_noalloc exists for callers that must not allocate device
memory: a scheduler loop that runs while a CUDA graph is being captured on
its thread, a hook that runs inside another framework's allocator, or a
process whose device memory a serving runtime has reserved up front.  It
keeps its scratch in a fixed array compiled into the library, so these tests
also check that two calls in a row (which share and reset that array) both
give the batched entry point's results.

This file is named so that pytest collects it last: a run that stops at the
first failure has run every other test before reaching it.
"""

import numpy as np
import pytest

from paper_2110_03214_gb300 import build as B
from paper_2110_03214_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    B.build()
    from paper_2110_03214_gb300 import mapa as M

    ctx = M.Context(0)
    ctx.set_stream(torch.cuda.current_stream().cuda_stream)
    yield torch, M, ctx
    torch.cuda.synchronize()
    ctx.close()


def _by_pattern(ctx, wl):
    tid = ctx.topology_load(wl.topology)
    pids = [ctx.pattern_load(p) for p in wl.requests.patterns]
    reqs = ctx.requests(wl.requests, pids)
    return tid, pids, reqs


@pytest.mark.parametrize("name,nreq", [("regular32", 4096), ("cube_mesh8", 1000)])
def test_two_calls_in_a_row_match_batched(env, name, nreq):
    torch, M, ctx = env
    wl = W.workload(name, num_requests=nreq)
    tid, pids, reqs = _by_pattern(ctx, wl)
    decided = 0
    for pid in pids:
        sel = reqs[reqs["pattern_id"] == pid]
        if len(sel) == 0:
            continue
        sel = sel[:4096]
        want = ctx.allocate_batch(tid, sel)  # the existing entry point
        dreq = torch.from_numpy(sel.view(np.uint8).copy()).cuda()
        dout = torch.empty(len(sel) * M.RESULT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        for call in range(2):
            dout.fill_(0xA5)  # results must be written in full on every call
            torch.cuda.synchronize()
            M.mapa_allocate_batch_noalloc(ctx.h, tid, pid, len(sel), dreq.data_ptr(), dout.data_ptr())
            torch.cuda.synchronize()
            got = dout.cpu().numpy().view(M.RESULT_DTYPE)
            assert np.array_equal(got, want), f"{name} pattern {pid} call {call}"
        decided += int((want["status"] == 0).sum())
    assert decided > 0


def test_limits_are_rejected(env):
    torch, M, ctx = env
    wl = W.workload("regular32", num_requests=8)
    tid, pids, reqs = _by_pattern(ctx, wl)
    dreq = torch.zeros(4097 * 64, dtype=torch.uint8, device="cuda")
    dout = torch.zeros(4097 * 80, dtype=torch.uint8, device="cuda")
    with pytest.raises(M.MapaError) as ei:
        M.mapa_allocate_batch_noalloc(ctx.h, tid, pids[0], 4097, dreq.data_ptr(), dout.data_ptr())
    assert ei.value.code == M.MAPA_E_RANGE
    big = ctx.pattern_load(W.pattern("ring", 9))
    with pytest.raises(M.MapaError) as ei:
        M.mapa_allocate_batch_noalloc(ctx.h, tid, big, 1, dreq.data_ptr(), dout.data_ptr())
    assert ei.value.code == M.MAPA_E_RANGE
    wide = ctx.topology_load(W.torus3d(4))
    with pytest.raises(M.MapaError) as ei:
        M.mapa_allocate_batch_noalloc(ctx.h, wide, pids[0], 1, dreq.data_ptr(), dout.data_ptr())
    assert ei.value.code == M.MAPA_E_RANGE


def test_mismatched_pattern_id_is_invalid(env):
    torch, M, ctx = env
    wl = W.workload("regular32", num_requests=64)
    tid, pids, reqs = _by_pattern(ctx, wl)
    dreq = torch.from_numpy(reqs.view(np.uint8).copy()).cuda()
    dout = torch.zeros(len(reqs) * 80, dtype=torch.uint8, device="cuda")
    M.mapa_allocate_batch_noalloc(ctx.h, tid, pids[0], len(reqs), dreq.data_ptr(), dout.data_ptr())
    torch.cuda.synchronize()
    got = dout.cpu().numpy().view(M.RESULT_DTYPE)
    other = reqs["pattern_id"] != pids[0]
    assert other.any() and (got["status"][other] == M.MAPA_E_INVALID).all()
    want = ctx.allocate_batch(tid, reqs[~other])
    assert np.array_equal(got[~other], want)


def _noalloc(torch, M, ctx, tid, pid, sel):
    dreq = torch.from_numpy(sel.view(np.uint8).copy()).cuda()
    dout = torch.empty(len(sel) * M.RESULT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    dout.fill_(0xA5)
    torch.cuda.synchronize()
    M.mapa_allocate_batch_noalloc(ctx.h, tid, pid, len(sel), dreq.data_ptr(), dout.data_ptr())
    torch.cuda.synchronize()
    return dout.cpu().numpy().view(M.RESULT_DTYPE)


# Per-request branches of the allocation-free kernel, each against the batched
# entry point on the same requests: bounded mode, a match budget small enough
# that most requests exceed it, signed weights, and an alpha that takes the
# int32 score out of range.
@pytest.mark.parametrize("case", ["bounded", "budget", "signed", "range"])
def test_request_branches_match_batched(env, case):
    torch, M, ctx = env
    wl = W.workload("regular32", num_requests=512)
    tid, pids, reqs = _by_pattern(ctx, wl)
    sel = reqs[reqs["pattern_id"] == pids[0]].copy()
    if case == "bounded":
        sel["mode"] = M.MAPA_MODE_BOUNDED
    elif case == "budget":
        sel["max_embeddings"] = 40
    elif case == "signed":
        sel["alpha"] = -1
        sel["beta"] = 2
    else:
        sel["alpha"][::2] = 1 << 20
    want = ctx.allocate_batch(tid, sel)
    statuses = set(int(s) for s in want["status"])
    if case == "budget":
        assert M.MAPA_E_BUDGET in statuses and M.MAPA_OK in statuses
    if case == "range":
        assert M.MAPA_E_RANGE in statuses and M.MAPA_OK in statuses
    for call in range(2):
        got = _noalloc(torch, M, ctx, tid, pids[0], sel)
        assert np.array_equal(got, want), f"{case} call {call}"


def test_refused_request_kinds_are_invalid(env):
    """Bandwidth-sensitive requests, bounded ones carrying a match budget and
    shares of a split request are refused per request (MAPA_E_INVALID); the
    rest of the call is decided as the batched entry point decides it."""
    torch, M, ctx = env
    wl = W.workload("regular32", num_requests=256)
    tid, pids, reqs = _by_pattern(ctx, wl)
    sel = reqs[reqs["pattern_id"] == pids[1]].copy()
    refused = np.zeros(len(sel), bool)
    refused[0::3] = True
    refused[1::5] = True
    refused[2::7] = True
    sel["flags"][0::3] = M.MAPA_POLICY_BW_SENSITIVE
    sel["mode"][1::5] = M.MAPA_MODE_BOUNDED
    sel["max_embeddings"][1::5] = 1000
    sel["root_lo"][2::7] = 3  # a share of a split request
    sel["root_hi"][2::7] = 17
    got = _noalloc(torch, M, ctx, tid, pids[1], sel)
    assert (got["status"][refused] == M.MAPA_E_INVALID).all()
    assert (got["count"][refused] == 0).all()
    want = ctx.allocate_batch(tid, sel[~refused])
    assert np.array_equal(got[~refused], want)
