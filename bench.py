#!/usr/bin/env python
"""Benchmark of the MAPA allocation hot path on GB300.

One step = one mapa_allocate_batch call deciding every request of one batch:
enumerate the matches of each request's pattern on its free accelerators,
score them (alpha*AggBW + beta*PreservedBW, Eq. 1 and Eq. 3) and pick the
argmax (Algorithm 1).  Inputs are resident in HBM when the timed region
starts; the L2 is flushed between timed steps (a 256 MiB write).

Default workload: the 256-vertex boards machine (32 boards of 8, ring-32 /
tree-31 / clique-8), 3000 requests of its 10^6-request stream per step, each
with the occupancy a served run leaves, with the anytime fallback under a
work budget of 2^16 partial matches per request and a 16 GiB frontier cap
per pattern group (64 GiB for the four concurrent groups).  The line also carries the 10^4-request 32-vertex workload
(`config2`), decided exhaustively.

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle on
the host cores instead (the paper has no GPU implementation).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "embeddings scored/s & alloc decisions/s; p50/p99 decision latency vs plain"
UNIT = "embeddings/s"
SM_COUNT = 152
INT_LANES_PER_SM = 128  # 4 SM sub-partitions x 32 lanes issue one warp instruction per clock each


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="boards256", choices=("cube_mesh8", "regular32", "torus64", "dragonfly128", "boards256"))
    ap.add_argument("--requests", type=int, default=None,
                    help="requests per step (default: 3000 for boards256, the workload's size otherwise)")
    ap.add_argument("--work-budget", type=int, default=None,
                    help="partial matches a request may store (default: 2^16 for boards256, none otherwise)")
    ap.add_argument("--frontier-cap-gib", type=float, default=None,
                    help="frontier memory per pattern group (default: 16 for boards256, 4 otherwise)")
    ap.add_argument("--no-config2", action="store_true", help="skip the 32-vertex workload's extra figures")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="bounded oracle sample length")
    ap.add_argument("--plain-requests", type=int, default=300, help="requests timed through the plain per-request path")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--served-sweep", action="store_true", help="rate sweep of the served loop instead")
    ap.add_argument("--served-requests", type=int, default=3000, help="arrivals in the served comparison")
    ap.add_argument("--served-rate", type=float, default=1e4, help="Poisson rate of the served comparison")
    ap.add_argument("--served-kmax", type=int, default=8)
    ap.add_argument("--no-served-sweep", action="store_true", help="skip the rate sweep of the served loop (kmax 16)")
    ap.add_argument("--sim-jobs", type=int, default=0,
                    help="jobs of the simulator leg (Sec. 6 job file; 0 = skip)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default tail depths (profiling runs: timings under a profiler mislead the tuner)")
    return ap.parse_args()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1])]
        reasons = set()
        for r in rows:
            for name, col in (("hw_slowdown", 5), ("hw_thermal_slowdown", 6), ("sw_thermal_slowdown", 7),
                              ("sw_power_cap", 8)):
                if r[col].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": num(rows[0][2]),
                "samples": len(rows), "reasons": sorted(reasons)}


class NvmlSampler:
    """Polls SM clock and clock-event reasons through NVML every ~1 ms (read only)."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown"}

    def __init__(self, index: int):
        import ctypes
        import threading

        self.ok = False
        self.samples = []
        self.max_mhz = None
        self._stop = threading.Event()
        self._thread = None
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return
            h = ctypes.c_void_p()
            if lib.nvmlDeviceGetHandleByIndex_v2(index, ctypes.byref(h)) != 0:
                return
            self._lib, self._h, self._ct = lib, h, ctypes
            mx = ctypes.c_uint()
            if lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:
                self.max_mhz = float(mx.value)
            self._reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or getattr(
                lib, "nvmlDeviceGetCurrentClocksThrottleReasons", None)
            self.ok = True
        except OSError:
            pass

    def _run(self):
        ct = self._ct
        clk = ct.c_uint()
        rs = ct.c_ulonglong()
        while not self._stop.is_set():
            r = 0
            if self._reasons_fn is not None and self._reasons_fn(self._h, ct.byref(rs)) == 0:
                r = rs.value
            if self._lib.nvmlDeviceGetClockInfo(self._h, 1, ct.byref(clk)) == 0:
                self.samples.append((float(clk.value), r))
            time.sleep(0.001)

    def start(self):
        import threading

        if self.ok:
            self._thread = threading.Thread(target=self._run, daemon=True)
            self._thread.start()

    def stop(self):
        if not self._thread:
            return None
        self._stop.set()
        self._thread.join()
        if not self.samples:
            return None
        reasons = set()
        for _, r in self.samples:
            for bit, name in self.REASONS.items():
                if r & bit:
                    reasons.add(name)
        return {"sm_mhz": statistics.median(c for c, _ in self.samples), "sm_max_mhz": self.max_mhz,
                "samples": len(self.samples), "source": "nvml", "reasons": sorted(reasons)}


def _kernel_source_hash() -> str:
    """Hash of the sources that define the level and fused-tail kernels and
    their launches (a traffic record taken on other sources is not used)."""
    h = hashlib.sha256()
    for name in ("mapa_kernels.cuh", "mapa_runner.cuh"):
        with open(os.path.join(ROOT, "paper_2110_03214_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _expand_traffic_per_launch(workload: str, algorithmic_bytes: float):
    """DRAM bytes per launch of the level expansion: the committed ncu ratio
    of DRAM bytes to algorithmic frontier bytes over every expansion launch
    of a smaller batch of the same workload, times the algorithmic bytes of an
    average launch; None when the kernel source changed since the capture."""
    path = os.path.join(ROOT, "profiles", "k_expand_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except OSError:
        return None
    if rec.get("source_sha256_16") != _kernel_source_hash() or rec.get("workload") != workload:
        return None
    return rec["dram_bytes_per_algorithmic_byte"] * algorithmic_bytes


def _traffic_per_launch(workload: str, parents_per_launch: float):
    """DRAM bytes per launch of the fused-tail kernel: the committed ncu
    per-parent figure times the parents of an average launch, or None when
    the kernel source changed since the capture."""
    path = os.path.join(ROOT, "profiles", "k_last_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except OSError:
        return None
    if rec.get("source_sha256_16") != _kernel_source_hash() or rec.get("workload") != workload:
        return None
    return rec["dram_bytes_per_parent"] * parents_per_launch


def workload_settings(name: str, a) -> dict:
    """Requests per step, decision mode, policy flags, work budget and
    frontier cap of a workload's bench line."""
    big = name == "boards256"
    req = a.requests if a.requests else (3000 if big else None)
    return {
        "requests": req,
        # exhaustive: on this stream the bounded mode's degree term (a scan of
        # the free set per partial) costs 7x more than it prunes (2.85 s
        # against 0.40 s per 3000-request step, the same outcomes)
        "mode": 0,
        "flags": 2 if big else 0,  # MAPA_POLICY_ANYTIME
        # 2^16, the served sweep's budget: on this stream every request's
        # result is the same for any budget from 2^12 to 2^20 (no ring-32 or
        # tree-31 enumeration finishes within any of them), so a larger one
        # only adds enumeration that no decision uses
        "work_budget": a.work_budget if a.work_budget is not None else ((1 << 16) if big else 0),
        "frontier_cap": int((a.frontier_cap_gib if a.frontier_cap_gib else (16 if big else 4)) * (1 << 30)),
    }


def _oracle_sample(wl, budget_s: float, threads: int, start: int = 0, max_nodes: int = 0):
    """Runs the oracle over consecutive requests until budget_s elapses.
    Returns (matches scored once per distinct subgraph, requests, decisions,
    seconds): a request stopped at max_nodes search nodes still counts the
    matches it scored (maps / |Aut(P)|) but is not a decision."""
    from concurrent.futures import ThreadPoolExecutor

    from oracle import oracle as O
    from paper_2110_03214_gb300 import workloads as W

    inst = O.Instance.from_topology(wl.topology)
    reqs = wl.requests
    auts = [O.aut_count(p.k, p.a, p.b) for p in reqs.patterns]

    def one(i):
        p = reqs.patterns[reqs.pattern_index[i]]
        busy = W.busy_to_bool(reqs.busy[i], wl.topology.n)
        d = inst.decide(busy, p.k, p.a, p.b, int(reqs.alpha[i]), int(reqs.beta[i]), max_nodes=max_nodes)
        if d.status == O.STATUS_OK:
            return float(d.classes), 1
        if d.status == O.STATUS_NO_MATCH:
            return 0.0, 1
        return (float(d.maps) / auts[reqs.pattern_index[i]] if d.status == O.STATUS_BUDGET else 0.0), 0

    done, emb, decided = 0, 0.0, 0
    t0 = time.perf_counter()
    with ThreadPoolExecutor(threads) as ex:
        i = start
        while time.perf_counter() - t0 < budget_s and i < len(reqs):
            chunk = list(range(i, min(i + threads, len(reqs))))
            for e, dcd in ex.map(one, chunk):
                emb += e
                decided += dcd
            done += len(chunk)
            i += len(chunk)
    dt = time.perf_counter() - t0
    return emb, done, decided, dt


def _oracle_node_cap(settings) -> int:
    """Search-node cap of the oracle's timed sample: 2^22 nodes per request
    under a GPU work budget (one to two seconds of one host core on the
    256-vertex graph), 2^26 otherwise (a request with a large search space,
    such as ring-16 on an idle torus, would run for hours), so the sample
    stays within its time limit.  A capped request still counts the matches
    it scored; the figure is matches scored (or decisions) per second."""
    return 1 << 22 if settings["work_budget"] else 1 << 26


def shard_workload(W, name: str, num_requests, rank: int):
    """Rank r decides its own batch of the workload's shape (independent
    requests shard with no exchange; weak scaling): same topology recipe and
    request mix, seed offset by the rank."""
    return W.workload(name, num_requests=num_requests, seed=W.WORKLOADS.index(name) + 1 + 1000 * rank)


def shard_slice(count: int, rank: int, world: int) -> tuple[int, int]:
    """Rank r's contiguous share [lo, hi) of `count` independent requests
    (strong-scaling split of one batch: shares differ by at most one)."""
    lo = count * rank // world
    hi = count * (rank + 1) // world
    return lo, hi


def combine_over_ranks(dist, device, total_ms: float, e2e_s: float, emb_step: int):
    """Whole-job figures from per-rank ones: the slowest rank's times (max)
    and the matches of all ranks (sum)."""
    import torch

    t = torch.tensor([total_ms, e2e_s], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    e = torch.tensor([float(emb_step)], dtype=torch.float64, device=device)
    dist.all_reduce(e, op=dist.ReduceOp.SUM)
    return float(t[0].item()), float(t[1].item()), float(e[0].item())


def served_measure(M, W, rate: float, count: int, max_batch: int, kmax: int = 8, seed: int = 4, mode: int = 0,
                   flags: int = 0, budget: int = 0):
    """Drives the served loop with a Poisson trace on the 128-vertex dragonfly;
    returns decisions/s over the run and p50/p99 arrival-to-decision latency."""
    import numpy as np

    tr = W.served_trace(count, rate=rate, kmax_rt=kmax, seed=seed)
    with M.Context(0) as ctx:
        ctx.set_work_budget(budget)
        tid = ctx.topology_load(tr.topology)
        pids = np.asarray([ctx.pattern_load(p) for p in tr.patterns], np.int32)
        ev = M.make_events(pids[tr.pattern_index], tr.at_ns, tr.lifetime_ns, mode=mode, flags=flags)
        srv = M.mapa_serve_open(ctx.h, tid, max_batch)
        try:
            M.mapa_serve_submit(srv, ev)
            M.mapa_serve_drain(srv, timeout_ms=300_000)
            out = M.mapa_serve_poll(srv, max_events=count + 16)
            counters = M.mapa_serve_counters(srv)
        finally:
            M.mapa_serve_close(srv)
    lat = (out["done_ns"] - out["arrive_ns"]) / 1e6
    span = (out["done_ns"].max() - out["arrive_ns"].min()) / 1e9
    st = out["result"]["status"]
    return {
        "rate_per_s": rate, "requests": int(count), "max_batch": int(max_batch), "kmax": kmax,
        "decisions_per_s": float(len(out) / span), "p50_ms": float(np.percentile(lat, 50)),
        "p99_ms": float(np.percentile(lat, 99)), "rounds": counters["rounds"], "conflicts_redone": counters["conflicts"],
        "placed": int(((st == 0) | (st == 2)).sum()), "inexact": int((st == 2).sum()), "budget": int((st == -5).sum()),
        "matches_scored": int(out["result"]["count"].sum()),
        "trace_s": float((tr.at_ns[-1] - tr.at_ns[0]) / 1e9), "workload": tr.description,
        "mode": "bounded" if mode else "exhaustive", "anytime": bool(flags & 2), "work_budget_partials": budget,
    }


def served_sweep(M, W, kmax: int = 16, rates=(1e3, 1e4, 1e5, 1e6), budget: int = 1 << 16):
    """Config 4's sweep: Poisson arrivals at each rate on the dragonfly, pattern
    sizes 2..kmax, decided by the served loop in batched rounds (max_batch
    4096) and one request per round (max_batch 1, the plain per-request
    form), with the anytime fallback under a work budget of 2^16 partial
    matches (so an oversized request cannot stall the queue)."""
    out = []
    for rate in rates:
        count = int(min(3000, max(2000, rate * 1.0)))
        row = {"rate_per_s": rate}
        for mb, key in ((4096, "batched"), (1, "plain")):
            row[key] = served_measure(M, W, rate, count, mb, kmax=kmax, mode=0, flags=2, budget=budget)
        out.append(row)
    return out


def simulator_measure(M, W, jobs_count: int, seed: int = 6):
    """The simulator of Sec. 6 (mapa_simulate) on the 8-GPU fixture and the two
    16-GPU stand-ins: per policy, the quartiles of the logged Predicted EffBW
    of bandwidth-sensitive and -insensitive jobs, the makespan in cycles, and
    the decisions per second of the run (every non-Baseline decision on the
    GPU)."""
    import numpy as np

    names = {M.MAPA_SIM_BASELINE: "baseline", M.MAPA_SIM_GREEDY: "greedy", M.MAPA_SIM_PRESERVE: "preserve",
             M.MAPA_SIM_EFFBW: "effbw"}
    jobs = W.sim_jobs(jobs_count, seed=seed)
    out = {"jobs": jobs_count, "job_file": "uniform mix of Sec. 5 workloads, 1-5 GPUs, ring pattern, "
                                           "durations U[100,1000] cycles, all in the file at cycle 0"}
    for topo in (W.dgx_fixture(), W.torus2d16(), W.cubemesh16()):
        per = {}
        with M.Context(0) as c:
            tid = c.topology_load(topo)
            pids = np.asarray([c.pattern_load(p) for p in jobs.patterns], np.int32)
            table = M.make_sim_jobs(pids[jobs.pattern_index], jobs.arrive, jobs.duration, jobs.sensitive)
            for pol, name in names.items():
                t0 = time.perf_counter()
                rec = M.mapa_simulate(c.h, tid, pol, table)
                dt = time.perf_counter() - t0
                ok = rec["status"] == M.MAPA_OK
                q = {}
                for label, sel in (("sensitive", jobs.sensitive == 1), ("insensitive", jobs.sensitive == 0)):
                    e = rec["effbw_milli"][ok & sel] / 1000.0
                    q[label] = [round(float(np.percentile(e, p)), 3) for p in (25, 50, 75)] if len(e) else None
                per[name] = {"effbw_quartiles_gbps": q, "makespan_cycles": int(rec["end"].max()),
                             "decisions_per_s": round(jobs_count / dt, 1)}
        out[topo.name] = per
    return out


def run_served_sweep(a):
    """Served loop only: the rate sweep (batched rounds vs one request per
    round), one JSON line per rate."""
    import __graft_entry__

    __graft_entry__.build()
    from paper_2110_03214_gb300 import mapa as M
    from paper_2110_03214_gb300 import workloads as W

    for row in served_sweep(M, W, kmax=16):
        print(json.dumps(row), flush=True)


def run_reference(a):
    """The CPU oracle on the host cores (the reference arm)."""
    from paper_2110_03214_gb300 import workloads as W
    from oracle import oracle as O

    O.build()
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cfg = workload_settings(a.workload, a)
    wl = W.workload(a.workload, num_requests=cfg["requests"])
    threads = os.cpu_count() or 1
    cap = _oracle_node_cap(cfg)
    per_step = max(0.5, min(20.0, 120.0 / max(1, a.steps + a.warmup)))
    for _ in range(a.warmup):
        _oracle_sample(wl, per_step / 4, threads, max_nodes=cap)
    emb_total, req_total, dec_total, t_total = 0.0, 0, 0, 0.0
    start = 0
    for _ in range(a.steps):
        emb, done, decided, dt = _oracle_sample(wl, per_step, threads, start, max_nodes=cap)
        start = (start + done) % len(wl.requests)
        emb_total += emb
        req_total += done
        dec_total += decided
        t_total += dt
    unit = line_unit(a.workload)
    value = (dec_total if unit == "decisions/s" else emb_total) / t_total
    sample = (f"{req_total} requests of {wl.name} ({len(wl.requests)} in the batch), {per_step:.1f} s per step"
              + (f", at most {cap} search nodes per request" if cap else ""))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": unit, "n_gpus": a.gpus, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": 1000 * t_total / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "decisions_per_s": dec_total / t_total, "embeddings_per_s": emb_total / t_total,
        "config": {"workload": f"{wl.name}: {wl.description}", "requests_per_step": req_total // a.steps,
                   "l2": "host run"},
        "cpu_baseline": {"value": value, "unit": unit, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def measure_batch(M, W, torch, a, name, rank, world, dist, local, plain_requests):
    """Times one workload's batch: the timed device-buffer steps, a per-kernel
    timing pass for the roofline, the end-to-end host-buffer steps and the
    plain one-request-per-call path.  Returns the figures as a dict."""
    import numpy as np

    cfg = workload_settings(name, a)
    wl = shard_workload(W, name, cfg["requests"], rank)
    nreq = len(wl.requests)
    stream = torch.cuda.current_stream()
    ctx = M.Context(local, frontier_mem_cap=cfg["frontier_cap"])
    ctx.set_stream(stream.cuda_stream)
    ctx.set_work_budget(cfg["work_budget"])
    tid = ctx.topology_load(wl.topology)
    pids = [ctx.pattern_load(p) for p in wl.requests.patterns]
    reqs = ctx.requests(wl.requests, pids, mode=cfg["mode"])
    reqs["flags"] |= cfg["flags"]
    d_req = torch.from_numpy(reqs.view(np.uint8).copy()).cuda()
    d_out = torch.zeros(nreq * M.RESULT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def step():
        ctx.allocate_batch_device(tid, nreq, d_req.data_ptr(), d_out.data_ptr())

    # tail depths chosen by the autotuner on the workload (untimed)
    if a.no_autotune:
        tail_depths = "default"
    else:
        tuned = M.mapa_autotune(ctx.h, tid, reqs, len(pids))
        tail_depths = {wl.requests.patterns[i].name: int(tuned[p]) for i, p in enumerate(pids)}
        tail_depths["level_limits"] = {wl.requests.patterns[i].name: M.mapa_autotune_level_limit(ctx.h, tid, p)
                                       for i, p in enumerate(pids)}

    for _ in range(a.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    ref = d_out.cpu().numpy().view(M.RESULT_DTYPE).copy()

    ctx.stats_reset()
    clocks = ClockSampler(local)
    nvml = NvmlSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    nvml.start()
    times = []
    for _ in range(a.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = nvml.stop()
    smi = clocks.stop()
    if clk is None:
        clk = smi
    elif smi:
        clk["nvidia_smi_samples"] = smi["samples"]
    st = ctx.stats()
    got = d_out.cpu().numpy().view(M.RESULT_DTYPE)
    if not np.array_equal(got, ref):
        raise RuntimeError("results changed between steps")
    # roofline pass: the same step with every fused-tail and level-expansion
    # launch bracketed by CUDA events on the stream it runs on (per-kernel
    # timing runs the pattern groups one after another and bypasses graphs,
    # so it runs outside the timed region)
    ctx.stats_reset()
    ctx.set_timing(True)
    roof_steps = 3
    t_roof = []
    for _ in range(roof_steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        t_roof.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    st_roof = ctx.stats()
    ctx.set_timing(False)
    emb_step = int(st["embeddings"] // max(1, a.steps))
    total_ms = float(sum(times))

    # end to end through the public API with pinned host buffers
    h_req = torch.from_numpy(reqs.view(np.uint8).copy()).pin_memory()
    h_out = torch.zeros(nreq * M.RESULT_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
    e2e_times = []
    for i in range(a.warmup + a.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        M.lib.mapa_allocate_batch(ctx.h, tid, nreq, h_req.data_ptr(), h_out.data_ptr(), 0)
        t1 = time.perf_counter()
        if i >= a.warmup:
            e2e_times.append(t1 - t0)
    if not np.array_equal(h_out.numpy().view(M.RESULT_DTYPE), ref):
        raise RuntimeError("host-buffer path disagrees with the device path")
    e2e_s = sum(e2e_times)
    if world > 1:
        total_ms, e2e_s, emb_all = combine_over_ranks(dist, "cuda", total_ms, e2e_s, emb_step)
    else:
        emb_all = float(emb_step)

    # plain per-request path (mapa_allocate_batch with one request per call) for latency
    plain_lat = []
    for i in range(min(plain_requests, nreq)):
        t0 = time.perf_counter()
        ctx.allocate_batch(tid, reqs[i:i + 1])
        plain_lat.append(time.perf_counter() - t0)
    ctx.close()
    statuses = {int(k): int(v) for k, v in zip(*np.unique(ref["status"], return_counts=True))}
    decided = sum(v for k, v in statuses.items() if k >= 0)
    unit = line_unit(name)
    out = {
        "wl": wl, "nreq": nreq, "cfg": cfg, "ref": ref, "times": times, "total_ms": total_ms, "clocks": clk,
        "stats": st, "stats_roof": st_roof, "roof_steps": roof_steps, "roof_ms": t_roof, "tail_depths": tail_depths,
        "emb_step": emb_step, "emb_all": emb_all, "e2e_s": e2e_s,
        "embeddings_per_s": emb_all * a.steps / (total_ms / 1000.0),
        "decisions_per_s": decided * world * a.steps / (total_ms / 1000.0),
        "requests_per_s": nreq * world * a.steps / (total_ms / 1000.0),
        "statuses": {M_STATUS.get(k, str(k)): v for k, v in statuses.items()},
        "e2e": {"embeddings_per_s": emb_all * a.steps / e2e_s,
                "decisions_per_s": decided * world * a.steps / e2e_s,
                "h2d_bytes_per_step": nreq * M.REQUEST_DTYPE.itemsize,
                "d2h_bytes_per_step": nreq * M.RESULT_DTYPE.itemsize},
        "plain": {"decisions_per_s": len(plain_lat) / sum(plain_lat) if plain_lat else None,
                  "p50_ms": 1000 * float(np.percentile(plain_lat, 50)) if plain_lat else None,
                  "p99_ms": 1000 * float(np.percentile(plain_lat, 99)) if plain_lat else None,
                  "requests": len(plain_lat)},
    }
    key = "decisions_per_s" if unit == "decisions/s" else "embeddings_per_s"
    out["value"] = out[key]
    out["unit"] = unit
    out["e2e"]["value"] = out["e2e"][key]
    out["e2e"]["unit"] = unit
    return out


def line_unit(name: str) -> str:
    """Unit of a workload's headline value: matches scored per second, or
    decisions per second on the boards stream, where no request finishes an
    enumeration within its work budget (its decisions are exact no-fits,
    budget-capped inexact matches or budget ends) and the scored-match rate
    says nothing."""
    return "decisions/s" if name == "boards256" else UNIT


M_STATUS = {0: "ok", 1: "no_fit", 2: "inexact", -5: "budget", -2: "range", -1: "invalid"}


def roofline(r, peaks, peak_src, int_peak):
    """Roofline entry of the kernel that takes the larger share of the
    timing pass: the level expansion (frontier bytes against the measured
    copy bandwidth) or the fused tail (algorithmic integer operations
    against the measured integer issue rate)."""
    st = r["stats_roof"]
    n = r["roof_steps"]
    step_ms = statistics.median(r["roof_ms"])
    tail_ms, exp_ms = st["tail_ms"] / n, st["expand_ms"] / n
    if exp_ms >= tail_ms and st["expand_launches"]:
        launch_ms = st["expand_ms"] / st["expand_launches"]
        bytes_per_launch = st["expand_bytes"] / st["expand_launches"]
        achieved = bytes_per_launch / (launch_ms / 1000.0) / 1e9
        peak = float(peaks["hbm_gbs"])
        return {"bound": "hbm", "kernel": "level expansion (k_expand, or k_count + k_write when chunked)",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": _expand_traffic_per_launch(r["wl"].name, bytes_per_launch),
                "peak_source": f"{peak_src} hbm_gbs (copy bandwidth)",
                "algorithmic_bytes_per_launch": bytes_per_launch, "launch_ms": launch_ms,
                "launches_per_step": st["expand_launches"] / n, "share_of_step": exp_ms / step_ms,
                "tail_share_of_step": tail_ms / step_ms,
                "rest_of_step": "anytime dives (one warp per request, beside the chunked enumeration), budget "
                                "counts, set-up and finish",
                "measured": "separate 3-step pass, CUDA events around each launch on its stream, groups serial"}
    launch_ms = st["tail_ms"] / max(1, st["tail_launches"])
    ops_per_launch = st["tail_int_ops"] / max(1, st["tail_launches"])
    achieved = ops_per_launch / (launch_ms / 1000.0) / 1e9 if launch_ms > 0 else 0.0
    peak = int_peak["mix_gops"]
    traffic = _traffic_per_launch(f"{r['wl'].name}/{r['nreq']}", st["tail_parents"] / max(1, st["tail_launches"]))
    return {"bound": "alu", "kernel": "k_last_short (fused last two levels: score, count, argmax)",
            "achieved": achieved, "peak": peak, "unit": "Gop/s", "frac": achieved / peak if peak else None,
            "traffic": traffic, "peak_source": int_peak["source"], "launch_ms": launch_ms,
            "ops_per_launch": ops_per_launch, "launches_per_step": st["tail_launches"] / n,
            "share_of_step": tail_ms / step_ms, "expand_share_of_step": exp_ms / step_ms,
            "ops_units": "per parent (|back|+3)W, per tail node 2CW+|back|+4 plus its (|back|+3)W, per leaf 2CW+|back|+5",
            "measured": "separate 3-step pass, CUDA events around each launch on its stream, groups serial"}


def measure_int_peak(M, local, peaks):
    """Integer issue rate of this GPU measured by the library's probe kernel
    (no such figure in MEASURED_PEAKS.json); the lane-count figure beside it."""
    with M.Context(local) as c:
        plain = M.mapa_measure_int_peak(c.h, 0) / 1e9
        mix = M.mapa_measure_int_peak(c.h, 1) / 1e9
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    lanes = SM_COUNT * INT_LANES_PER_SM * sm_mhz * 1e6 / 1e9
    return {"logic_add_gops": plain, "mix_gops": mix, "lanes_x_clock_gops": lanes,
            "source": "measured: lop3/popc/add chains, one popc per three ops (mapa_measure_int_peak kind 1)"}


def run_ours(a):
    import numpy as np
    import torch
    import torch.distributed as dist

    import __graft_entry__

    __graft_entry__.build()
    from paper_2110_03214_gb300 import mapa as M
    from paper_2110_03214_gb300 import workloads as W

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    # Each rank decides its own batch of the same shape (independent requests shard with no exchange).
    r = measure_batch(M, W, torch, a, a.workload, rank, world, dist, local, a.plain_requests)
    peaks, peak_src = _peaks()
    int_peak = measure_int_peak(M, local, peaks)
    roof = roofline(r, peaks, peak_src, int_peak)
    wl, nreq, cfg = r["wl"], r["nreq"], r["cfg"]
    total_ms = r["total_ms"]
    if rank == 0:
        line = {
            "metric": METRIC, "value": r["value"], "unit": r["unit"], "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": total_ms / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic (seeded SplitMix64 generator)",
            "decisions_per_s": r["decisions_per_s"], "embeddings_per_s": r["embeddings_per_s"],
            "requests_per_s": r["requests_per_s"],
            "outcomes_per_step": r["statuses"],
            "latency_ms": {"batched_p50": statistics.median(r["times"]), "batched_p99": max(r["times"]),
                           "plain_p50": r["plain"]["p50_ms"], "plain_p99": r["plain"]["p99_ms"]},
            "plain": r["plain"],
            "config": {"workload": f"{wl.name}: {wl.description}", "requests_per_step": nreq,
                       "embeddings_per_step": r["emb_step"], "tail_depths": r["tail_depths"],
                       "mode": "bounded" if cfg["mode"] else "exhaustive",
                       "anytime": bool(cfg["flags"] & 2), "work_budget_partials": cfg["work_budget"],
                       "frontier_cap_bytes_per_group": cfg["frontier_cap"],
                       "parallelism": f"{world} independent shards" if world > 1 else "single GPU",
                       "l2": "flushed between timed steps (256 MiB write)"},
            "roofline": roof,
            "int_peak": int_peak,
            "gpu_launches": r["stats"]["kernel_launches"],
            "stats": r["stats"],
            "e2e": r["e2e"],
            "clocks": r["clocks"],
        }
        if world == 1 and a.workload != "regular32" and not a.no_config2:
            c2 = measure_batch(M, W, torch, a, "regular32", 0, 1, dist, local, a.plain_requests)
            line["config2"] = {
                "workload": f"{c2['wl'].name}: {c2['wl'].description}", "requests_per_step": c2["nreq"],
                "value": c2["value"], "unit": c2["unit"], "ms_per_step": c2["total_ms"] / a.steps,
                "decisions_per_s": c2["decisions_per_s"], "e2e": c2["e2e"], "plain": c2["plain"],
                "roofline": roofline(c2, peaks, peak_src, int_peak), "clocks": c2["clocks"],
                "gpu_launches": c2["stats"]["kernel_launches"], "embeddings_per_step": c2["emb_step"],
            }
        if world == 1 and a.served_requests > 0:
            sb = served_measure(M, W, a.served_rate, a.served_requests, 4096, kmax=a.served_kmax)
            sp = served_measure(M, W, a.served_rate, a.served_requests, 1, kmax=a.served_kmax)
            line["served"] = {"batched": sb, "plain": sp}
            line["latency_ms"].update({"served_batched_p50": sb["p50_ms"], "served_batched_p99": sb["p99_ms"],
                                       "served_plain_p50": sp["p50_ms"], "served_plain_p99": sp["p99_ms"]})
        if world == 1 and not a.no_served_sweep:
            line["served_sweep"] = served_sweep(M, W)
        if world == 1 and a.sim_jobs > 0:
            line["simulator"] = simulator_measure(M, W, a.sim_jobs)
        if world == 1 and not a.no_cpu_baseline:
            threads = os.cpu_count() or 1
            cap = _oracle_node_cap(cfg)
            emb, done, decided, dt = _oracle_sample(wl, a.cpu_seconds, threads, max_nodes=cap)
            line["cpu_baseline"] = {"value": (decided if r["unit"] == "decisions/s" else emb) / dt, "unit": r["unit"],
                                    "cores": threads, "kind": "oracle", "embeddings_per_s": emb / dt,
                                    "decisions_per_s": decided / dt,
                                    "sample": f"first {done} of {nreq} requests of {wl.name}, {dt:.1f} s"
                                              + (f", at most {cap} search nodes per request" if cap else "")}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    a = _args()
    if a.served_sweep:
        run_served_sweep(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
