"""Shared helpers for the parity tests: run the oracle on requests and compare."""

from concurrent.futures import ThreadPoolExecutor

import numpy as np

from oracle import oracle as O
from paper_2110_03214_gb300 import workloads as W

OK, NO_FIT, E_BUDGET = 0, 1, -5


def oracle_decisions(inst, topo_n, reqs, idx, max_maps=0, threads=8):
    """Oracle decisions for requests `idx` of a workloads.Requests (threads release the GIL in ctypes)."""

    def one(i):
        p = reqs.patterns[reqs.pattern_index[i]]
        busy = W.busy_to_bool(reqs.busy[i], topo_n)
        return inst.decide(busy, p.k, p.a, p.b, int(reqs.alpha[i]), int(reqs.beta[i]), max_maps)

    with ThreadPoolExecutor(threads) as ex:
        return list(ex.map(one, idx))


def assert_same(res, dec, k, where=""):
    """Bit-exact comparison of one GPU result with one oracle decision."""
    if dec.status == O.STATUS_OK:
        got = (int(res["status"]), int(res["score"]), int(res["agg"]), int(res["pres"]), int(res["count"]),
               tuple(int(x) for x in res["verts"][:k]))
        want = (OK, dec.score, dec.agg, dec.pres, dec.classes, tuple(dec.tuple))
        assert got == want, f"{where}: gpu {got} != oracle {want}"
    elif dec.status == O.STATUS_NO_MATCH:
        assert int(res["status"]) == NO_FIT and int(res["count"]) == 0, f"{where}: gpu {res} != NO_FIT"
    else:
        raise AssertionError(f"{where}: oracle status {dec.status}")


def check_result_properties(inst, topo_n, reqs, results):
    """Size-independent checks: every OK result is a match whose score, AggBW
    and PreservedBW the oracle recomputes exactly from the tuple."""
    bad = []
    for i in range(len(reqs)):
        res = results[i]
        if int(res["status"]) != OK:
            assert int(res["status"]) == NO_FIT, (i, res)
            continue
        p = reqs.patterns[reqs.pattern_index[i]]
        busy = W.busy_to_bool(reqs.busy[i], topo_n)
        st, agg, pres, score = inst.score_tuple(busy, p.k, p.a, p.b, int(reqs.alpha[i]), int(reqs.beta[i]),
                                                res["verts"][: p.k])
        if (st, agg, pres, score) != (0, int(res["agg"]), int(res["pres"]), int(res["score"])):
            bad.append(i)
        if int(res["count"]) < 1:
            bad.append(i)
    assert not bad, f"results failing the tuple re-score: {bad[:10]}"
