"""Pins of the reference simulator (Sec. 6) over the oracle.

* a hand-worked Baseline schedule on the 8-GPU fixture;
* invariants of a FIFO cycle engine on seeded job files: starts follow the
  file order, every job runs for its duration, running allocations never
  share an accelerator, and nothing that fits is left unplaced;
* the logger's Predicted EffBW of the worked example's ideal allocation
  equals the paper's 57.85 GB/s;
* the paper's point about Preserve (Sec. 3.5.2, Sec. 5): placing an
  insensitive job by PreservedBW leaves a later sensitive job a better link
  mix than placing it by AggBW (Greedy).
"""

import numpy as np
import pytest

from oracle import sim as S
from paper_2110_03214_gb300 import workloads as W


def _jobs(ks, durations, sensitive, arrive=None):
    pats = [W.pattern("ring", k) for k in range(1, 9)]
    idx = np.asarray([k - 1 for k in ks], np.int32)
    arr = np.zeros(len(ks), np.int64) if arrive is None else np.asarray(arrive, np.int64)
    return W.SimJobs(pats, idx, arr, np.asarray(durations, np.int64), np.asarray(sensitive, np.int32),
                     ["x"] * len(ks))


def test_hand_worked_baseline_schedule():
    # 8 GPUs; at cycle 0 job 0 takes 0-3 and job 1 takes 4-7; job 2 waits until
    # job 1 ends at 5 and takes 4-5 (ends at 8); job 3 needs five GPUs, which
    # are free only once job 0 ends at 10, when 0-7 are all free again.
    jobs = _jobs([4, 4, 2, 5], [10, 5, 3, 4], [0, 0, 0, 0])
    recs = S.simulate(W.dgx_fixture(), jobs, S.BASELINE)
    assert [(r["start"], r["end"], r["verts"]) for r in recs] == [
        (0, 10, (0, 1, 2, 3)), (0, 5, (4, 5, 6, 7)), (5, 8, (4, 5)), (10, 14, (0, 1, 2, 3, 4))]


def test_job_larger_than_machine_is_logged_not_placed():
    jobs = _jobs([2, 8, 3], [5, 5, 5], [0, 0, 0])
    topo = W.dgx_fixture()
    recs = S.simulate(topo, dataclass_with_k(jobs, 1, 9), S.GREEDY)
    assert recs[1]["status"] == S.NOT_PLACED and recs[1]["start"] == 5
    assert recs[0]["status"] == recs[2]["status"] == S.PLACED


def dataclass_with_k(jobs, j, k):
    pats = list(jobs.patterns) + [W.pattern("ring", k)]
    idx = jobs.pattern_index.copy()
    idx[j] = len(pats) - 1
    return W.SimJobs(pats, idx, jobs.arrive, jobs.duration, jobs.sensitive, jobs.network)


@pytest.mark.parametrize("policy", [S.BASELINE, S.GREEDY, S.PRESERVE, S.EFFBW])
@pytest.mark.parametrize("topo", ["dgx", "torus2d16"])
def test_fifo_engine_invariants(policy, topo):
    t = W.dgx_fixture() if topo == "dgx" else W.torus2d16()
    jobs = W.sim_jobs(60, seed=3, arrival_gap=37)
    recs = S.simulate(t, jobs, policy)
    starts = [r["start"] for r in recs]
    assert starts == sorted(starts)
    for j, r in enumerate(recs):
        assert r["status"] == S.PLACED
        assert r["start"] >= jobs.arrive[j]
        assert r["end"] - r["start"] == jobs.duration[j]
        assert len(set(r["verts"])) == jobs.patterns[jobs.pattern_index[j]].k
    events = sorted({r["start"] for r in recs})
    for c in events:
        live = [r for r in recs if r["start"] <= c < r["end"]]
        used = [v for r in live for v in r["verts"]]
        assert len(used) == len(set(used)), c
    # FIFO and work conserving at the head: a job starts no later than the
    # first event at which it has arrived and enough GPUs are free (Baseline
    # needs only a count)
    if policy == S.BASELINE:
        for j, r in enumerate(recs):
            prev = recs[j - 1]["start"] if j else 0
            ok = [c for c in sorted({0, *(x["end"] for x in recs), *jobs.arrive.tolist()})
                  if c >= max(prev, jobs.arrive[j])
                  and t.n - sum(len(x["verts"]) for x in recs[:j] if x["start"] <= c < x["end"])
                  >= jobs.patterns[jobs.pattern_index[j]].k]
            assert r["start"] == ok[0], j


def test_logger_effbw_of_the_worked_example():
    jobs = W.SimJobs([W.pattern("clique", 3)], np.zeros(1, np.int32), np.zeros(1, np.int64),
                     np.ones(1, np.int64), np.ones(1, np.int32), ["VGG-16"])
    rec = S.simulate(W.dgx_fixture(), jobs, S.EFFBW)[0]
    assert rec["effbw_milli"] == 57857 and rec["agg"] == 125


def test_preserve_protects_a_later_sensitive_job():
    # an insensitive 2-GPU job, then a sensitive 3-GPU job, on the idle
    # 8-GPU fixture: Greedy spends a double NVLink pair on the first job
    pats = [W.pattern("ring", 2), W.pattern("clique", 3)]
    jobs = W.SimJobs(pats, np.asarray([0, 1], np.int32), np.zeros(2, np.int64), np.asarray([100, 100], np.int64),
                     np.asarray([0, 1], np.int32), ["GoogleNet", "VGG-16"])
    greedy = S.simulate(W.dgx_fixture(), jobs, S.GREEDY)
    preserve = S.simulate(W.dgx_fixture(), jobs, S.PRESERVE)
    assert greedy[0]["agg"] == 50
    assert preserve[1]["effbw_milli"] >= greedy[1]["effbw_milli"]
    assert preserve[1]["effbw_milli"] == 57857
