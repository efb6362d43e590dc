"""GPU parity of the simulator (mapa_simulate, Sec. 6) against the reference
simulator over the oracle (oracle/sim.py).

Same job file, same topology, same policy: every job gets the same start and
end cycle, the same accelerators and the same logged AggBW and PreservedBW;
the logged milli-GB/s EffBW may differ by one where Eq. 2 lands exactly on a
half milli-GB/s (two independent double evaluations round it either way).
"""

import numpy as np
import pytest

from oracle import sim as S
from paper_2110_03214_gb300 import build as B
from paper_2110_03214_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    B.build()
    from paper_2110_03214_gb300 import mapa

    return mapa


def _run(M, topo, jobs, policy):
    with M.Context(0) as c:
        tid = c.topology_load(topo)
        pids = np.asarray([c.pattern_load(p) for p in jobs.patterns], np.int32)
        table = M.make_sim_jobs(pids[jobs.pattern_index], jobs.arrive, jobs.duration, jobs.sensitive)
        return M.mapa_simulate(c.h, tid, policy, table)


@pytest.mark.parametrize("policy", [0, 1, 2, 3])
@pytest.mark.parametrize("topo,count,gap", [("dgx", 120, 0), ("torus2d16", 80, 25), ("cubemesh16", 80, 0)])
def test_simulator_matches_reference(M, policy, topo, count, gap):
    t = {"dgx": W.dgx_fixture, "torus2d16": W.torus2d16, "cubemesh16": W.cubemesh16}[topo]()
    jobs = W.sim_jobs(count, seed=21, arrival_gap=gap)
    got = _run(M, t, jobs, policy)
    want = S.simulate(t, jobs, policy)
    for j, w in enumerate(want):
        g = got[j]
        k = jobs.patterns[jobs.pattern_index[j]].k
        assert int(g["status"]) == (0 if w["status"] == S.PLACED else 1), j
        assert (int(g["start"]), int(g["end"])) == (w["start"], w["end"]), j
        if w["status"] == S.PLACED:
            assert tuple(int(x) for x in g["verts"][:k]) == w["verts"], j
            assert (int(g["agg"]), int(g["pres"])) == (w["agg"], w["pres"]), j
            assert abs(int(g["effbw_milli"]) - w["effbw_milli"]) <= 1, j


def test_simulator_rejects_bad_input(M):
    t = W.dgx_fixture()
    jobs = W.sim_jobs(5, seed=1)
    with M.Context(0) as c:
        tid = c.topology_load(t)
        pids = np.asarray([c.pattern_load(p) for p in jobs.patterns], np.int32)
        table = M.make_sim_jobs(pids[jobs.pattern_index], [5, 4, 6, 7, 8], jobs.duration, jobs.sensitive)
        with pytest.raises(M.MapaError):
            M.mapa_simulate(c.h, tid, 0, table)  # arrivals out of order
        table = M.make_sim_jobs(pids[jobs.pattern_index], 0, jobs.duration, jobs.sensitive)
        with pytest.raises(M.MapaError):
            M.mapa_simulate(c.h, tid, 9, table)  # unknown policy
