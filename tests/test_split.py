"""Splitting one request by the value of phi(0) (CPU: no GPU needed).

A request's matches partition by the image of pattern vertex 0, so shares
over a partition of [0, n) can be decided apart (on different GPUs) and
reduced: the best share by score, then by the lexicographically smaller
tuple, with the counts summed.  Checked here:

* the library's host-only reduction (mapa_result_merge) on hand-made
  shares: ties, counts, errors, no-fits, inexact shares;
* the oracle's share decision (oracle_decide_rooted) against the plain
  oracle: the reduced shares give the unsplit decision and the shares' map
  counts add up to the unsplit one, on random graphs and the 32-vertex
  workload.
"""

import numpy as np
import pytest

from oracle import oracle as O
from paper_2110_03214_gb300 import build as B
from paper_2110_03214_gb300 import workloads as W


@pytest.fixture(scope="module")
def M():
    B.build()
    from paper_2110_03214_gb300 import mapa

    return mapa


def _res(M, status, score=0, verts=(), count=0, k=3):
    r = np.zeros(1, M.RESULT_DTYPE)[0]
    r["status"], r["score"], r["count"], r["k"] = status, score, count, k
    r["verts"][: len(verts)] = verts
    return r


def test_merge_rules(M):
    a = _res(M, M.MAPA_OK, 10, (4, 5, 6), 3)
    b = _res(M, M.MAPA_OK, 10, (2, 9, 1), 2)
    c = _res(M, M.MAPA_OK, 7, (0, 1, 2), 5)
    d = _res(M, M.MAPA_NO_FIT)
    got = M.mapa_result_merge(np.array([a, b, c, d]))
    assert int(got["status"]) == M.MAPA_OK and int(got["score"]) == 10
    assert tuple(got["verts"][:3]) == (2, 9, 1) and int(got["count"]) == 10
    # all no-fit
    got = M.mapa_result_merge(np.array([d, d]))
    assert int(got["status"]) == M.MAPA_NO_FIT and int(got["count"]) == 0
    # an error share makes the result that error
    e = _res(M, M.MAPA_E_BUDGET)
    got = M.mapa_result_merge(np.array([a, e, b]))
    assert int(got["status"]) == M.MAPA_E_BUDGET and not got["verts"].any()
    # an inexact share makes the result inexact; a higher inexact score wins
    f = _res(M, M.MAPA_INEXACT, 12, (7, 8, 3))
    got = M.mapa_result_merge(np.array([a, f]))
    assert int(got["status"]) == M.MAPA_INEXACT and int(got["score"]) == 12
    got = M.mapa_result_merge(np.array([f, _res(M, M.MAPA_OK, 20, (1, 2, 3))]))
    assert int(got["status"]) == M.MAPA_INEXACT and int(got["score"]) == 20
    # shares of different pattern sizes are refused
    with pytest.raises(M.MapaError):
        M.mapa_result_merge(np.array([a, _res(M, M.MAPA_OK, 1, (1, 2), k=2)]))


def _shares(n, cuts):
    edges = [0, *cuts, n]
    return [(edges[i], edges[i + 1]) for i in range(len(edges) - 1)]


def _merge_oracle_shares(M, inst, busy, p, al, be, shares):
    parts = []
    maps = 0
    for lo, hi in shares:
        d = inst.decide_rooted(busy, p.k, p.a, p.b, al, be, lo, hi)
        maps += d.maps
        st = M.MAPA_OK if d.status == O.STATUS_OK else M.MAPA_NO_FIT
        parts.append(_res(M, st, d.score, d.tuple, d.maps, p.k))
        if st == M.MAPA_OK:
            parts[-1]["agg"], parts[-1]["pres"] = d.agg, d.pres
    return M.mapa_result_merge(np.array(parts)), maps


def test_oracle_shares_reduce_to_the_unsplit_decision(M):
    rng = W.Rng(41, 1)
    checked = 0
    for trial in range(40):
        n = int(rng.integers(6, 12, 1)[0])
        pairs = sorted({(min(a, b), max(a, b)) for a, b in rng.integers(0, n - 1, 2 * 3 * n).reshape(-1, 2)
                        if a != b})
        u = np.asarray([q[0] for q in pairs], np.int32)
        v = np.asarray([q[1] for q in pairs], np.int32)
        w = np.asarray([25, 50, 12], np.int32)[rng.integers(0, 2, len(pairs))]
        inst = O.Instance(n, u, v, w)
        p = [W.pattern("ring", 4), W.pattern("path", 3), W.pattern("tree", 5), W.pattern("clique", 3)][trial % 4]
        busy = rng.uniform(n) < 0.2
        al, be = int(rng.integers(0, 2, 1)[0]), int(rng.integers(0, 2, 1)[0])
        whole = inst.decide(busy, p.k, p.a, p.b, al, be)
        cuts = sorted(set(int(x) for x in rng.integers(1, n - 1, 2)))
        got, maps = _merge_oracle_shares(M, inst, busy, p, al, be, _shares(n, cuts))
        assert maps == whole.maps
        if whole.status == O.STATUS_OK:
            assert int(got["status"]) == M.MAPA_OK
            assert (int(got["score"]), int(got["agg"]), int(got["pres"])) == (whole.score, whole.agg, whole.pres)
            assert tuple(int(x) for x in got["verts"][: p.k]) == whole.tuple
            checked += 1
        else:
            assert int(got["status"]) == M.MAPA_NO_FIT
    assert checked >= 20


def test_oracle_shares_on_the_32_vertex_workload(M):
    wl = W.workload("regular32", num_requests=40)
    inst = O.Instance.from_topology(wl.topology)
    for i in range(len(wl.requests)):
        p = wl.requests.patterns[wl.requests.pattern_index[i]]
        busy = W.busy_to_bool(wl.requests.busy[i], 32)
        whole = inst.decide(busy, p.k, p.a, p.b, 1, 1)
        got, maps = _merge_oracle_shares(M, inst, busy, p, 1, 1, _shares(32, [8, 13, 24]))
        assert maps == whole.maps
        if whole.status == O.STATUS_OK:
            assert tuple(int(x) for x in got["verts"][: p.k]) == whole.tuple
            assert int(got["score"]) == whole.score
