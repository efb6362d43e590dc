"""Reference simulator of Sec. 6 over the oracle -- TEST INFRASTRUCTURE ONLY.

Only tests/ may import this module.  It restates the simulation of Sec. 6
plainly: the job file is read in order into a FIFO queue; time advances from
one event (an arrival or the end of a job) to the next; at each event the
finished jobs give their accelerators back, then the queue head is placed
while it fits (a head that does not fit waits for the next job to end, and
one that does not fit on the idle machine is logged as not placed).  The
placement policies of Sec. 5 decide through the oracle:

* Baseline: the lowest free accelerator ids, in order;
* Greedy: the match with the largest AggBW;
* Preserve (Algorithm 1): the largest Predicted EffBW for a bandwidth-
  sensitive job, the largest PreservedBW otherwise;
* EffBW: the largest Predicted EffBW for every job.

Each placed job is logged with AggBW (Eq. 1), PreservedBW (Eq. 3) of the
accelerators left free, and round(1000 * Eq. 2) of its link mix.
"""

from __future__ import annotations

import math

import numpy as np

from oracle import oracle as O

BASELINE, GREEDY, PRESERVE, EFFBW = 0, 1, 2, 3
PLACED, NOT_PLACED = 0, 1

_TYPE = {50: 0, 25: 1, 20: 1, 12: 2}


def simulate(topo, jobs, policy: int):
    """Records (one dict per job, in file order) for a workloads.SimJobs."""
    inst = O.Instance.from_topology(topo)
    n = topo.n
    wm = inst.wmat.reshape(n, n)
    busy = np.zeros(n, bool)
    running = []  # (end, job)
    recs = [None] * len(jobs)
    head = 0
    t = int(jobs.arrive[0]) if len(jobs) else 0

    def place(j):
        p = jobs.patterns[jobs.pattern_index[j]]
        if policy == BASELINE:
            free = [v for v in range(n) if not busy[v]]
            return tuple(free[: p.k]) if len(free) >= p.k else None
        sensitive = policy == EFFBW or (policy == PRESERVE and jobs.sensitive[j])
        if sensitive:
            dec, _ = inst.decide_effbw(busy, p.k, p.a, p.b)
        elif policy == GREEDY:
            dec = inst.decide(busy, p.k, p.a, p.b, 1, 0)
        else:
            dec = inst.decide(busy, p.k, p.a, p.b, 0, 1)
        return tuple(dec.tuple) if dec.status == O.STATUS_OK else None

    def log(j, tup):
        p = jobs.patterns[jobs.pattern_index[j]]
        counts = [0, 0, 0]
        agg = 0
        for a, b in zip(p.a, p.b):
            w = int(wm[tup[a], tup[b]])
            agg += w
            if w in _TYPE:
                counts[_TYPE[w]] += 1
        free = [v for v in range(n) if not busy[v]]
        pres = sum(int(wm[a, b]) for i, a in enumerate(free) for b in free[i + 1:])
        return agg, pres, int(math.floor(1000.0 * O.effbw(*counts) + 0.5))

    while head < len(jobs) or running:
        for end, j in list(running):
            if end <= t:
                busy[list(recs[j]["verts"])] = False
        running = [(end, j) for end, j in running if end > t]
        while head < len(jobs) and jobs.arrive[head] <= t:
            j = head
            tup = place(j)
            if tup is not None:
                busy[list(tup)] = True
                agg, pres, eff = log(j, tup)
                end = t + int(jobs.duration[j])
                recs[j] = {"status": PLACED, "start": t, "end": end, "verts": tup, "agg": agg, "pres": pres,
                           "effbw_milli": eff}
                running.append((end, j))
                head += 1
            elif running:
                break
            else:
                recs[j] = {"status": NOT_PLACED, "start": t, "end": t, "verts": (), "agg": 0, "pres": 0,
                           "effbw_milli": 0}
                head += 1
        nexts = [end for end, _ in running]
        if head < len(jobs) and jobs.arrive[head] > t:
            nexts.append(int(jobs.arrive[head]))
        if not nexts:
            break
        t = min(nexts)
    return recs
