"""Seeded synthetic workloads for the allocation hot path.

This module makes inputs only: topology graphs, pattern graphs and request
streams.  It holds none of the allocation arithmetic (no matching, scoring or
argmax), so the CPU oracle and the CUDA path can both be fed from it.

Randomness comes from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used in its counter form:
draw i of a stream is mix(seed + (i + 1) * 0x9E3779B97F4A7C15).  Because every
draw is a pure function of (seed, counter), the generator vectorises in numpy
and any slice of a stream can be reproduced without replaying the rest.

The hardware graphs follow the paper's abstraction (Sec. 3.2): vertices are
accelerators, an undirected edge carries the integer bandwidth of the best link
between two accelerators (Table 1 gives 20/25/50/12 GB/s link classes).  The
application graphs are the NCCL-style ring and tree shapes of Sec. 3.1 (Fig. 5)
plus clique (all-to-all) and path.
"""

from __future__ import annotations

import dataclasses

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

MAX_N = 256
MAX_K = 32
BUSY_WORDS = 8  # busy masks always carry 256 bits, bit v in word v // 32


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class Rng:
    """Counter-based SplitMix64 stream: (seed, stream) selects the sequence."""

    def __init__(self, seed: int, stream: int = 0):
        base = (int(seed) * 0x100000001B3 + int(stream) * 0x5851F42D4C957F2D) & (2**64 - 1)
        self._base = np.uint64(base)
        self._ctr = 0

    def u64(self, count: int) -> np.ndarray:
        idx = np.arange(self._ctr + 1, self._ctr + 1 + count, dtype=np.uint64)
        self._ctr += count
        with np.errstate(over="ignore"):
            return _mix(self._base + idx * _GOLDEN)

    def integers(self, lo: int, hi: int, count: int) -> np.ndarray:
        """Uniform integers in [lo, hi] (inclusive); modulo bias is below 2^-55."""
        span = np.uint64(hi - lo + 1)
        return (self.u64(count) % span).astype(np.int64) + lo

    def uniform(self, count: int) -> np.ndarray:
        """Uniform doubles in [0, 1) from the top 53 bits."""
        return (self.u64(count) >> np.uint64(11)).astype(np.float64) * (1.0 / 2**53)

    def permutation(self, n: int) -> np.ndarray:
        return np.argsort(self.u64(n), kind="stable")


# --------------------------------------------------------------------------
# Graph containers


@dataclasses.dataclass
class Topology:
    """Undirected weighted hardware graph; edge i is (u[i], v[i]) with weight w[i]."""

    name: str
    n: int
    u: np.ndarray
    v: np.ndarray
    w: np.ndarray
    fill_weight: int = 0  # >0: every non-adjacent pair gets this weight (Sec. 3.2)

    @property
    def m(self) -> int:
        return int(self.u.shape[0])


@dataclasses.dataclass
class Pattern:
    """Application graph with k vertices; edges (a[i], b[i])."""

    kind: str
    k: int
    a: np.ndarray
    b: np.ndarray

    @property
    def m(self) -> int:
        return int(self.a.shape[0])

    @property
    def name(self) -> str:
        return f"{self.kind}-{self.k}"


def _edges(pairs) -> tuple[np.ndarray, np.ndarray]:
    if not pairs:
        return np.zeros(0, np.int32), np.zeros(0, np.int32)
    arr = np.asarray(pairs, dtype=np.int32)
    return arr[:, 0].copy(), arr[:, 1].copy()


def pattern(kind: str, k: int) -> Pattern:
    """Built-in shapes.  k always counts vertices.

    ring-k: cycle 0-1-..-(k-1)-0 for k >= 3; ring-2 is one edge; ring-1 one vertex.
    tree-k: binary tree in heap order, parent(i) = (i - 1) // 2.
    clique-k: all pairs.  path-k: chain 0-1-..-(k-1).
    """
    if not (1 <= k <= MAX_K):
        raise ValueError(f"pattern size {k} outside 1..{MAX_K}")
    if kind == "ring":
        if k == 1:
            pairs = []
        elif k == 2:
            pairs = [(0, 1)]
        else:
            pairs = [(i, i + 1) for i in range(k - 1)] + [(0, k - 1)]
    elif kind == "tree":
        pairs = [((i - 1) // 2, i) for i in range(1, k)]
    elif kind == "clique":
        pairs = [(i, j) for i in range(k) for j in range(i + 1, k)]
    elif kind == "path":
        pairs = [(i, i + 1) for i in range(k - 1)]
    else:
        raise ValueError(f"unknown pattern kind {kind!r}")
    a, b = _edges(pairs)
    return Pattern(kind, k, a, b)


def random_pattern(rng: Rng, k: int, p_edge: float = 0.5, connected: bool = True) -> Pattern:
    """Random pattern with k vertices (edge (i, j) kept with probability p_edge).

    With connected=True each vertex i >= 1 also links to a random earlier vertex,
    so the pattern is connected in vertex-id order.
    """
    pairs = set()
    if connected:
        for i in range(1, k):
            j = int(rng.integers(0, i - 1, 1)[0])
            pairs.add((j, i))
    draws = rng.uniform(k * k)
    for i in range(k):
        for j in range(i + 1, k):
            if draws[i * k + j] < p_edge:
                pairs.add((i, j))
    a, b = _edges(sorted(pairs))
    return Pattern("custom", k, a, b)


# --------------------------------------------------------------------------
# Topologies


def hybrid_cube_mesh8(rng: Rng, weights=(25, 50)) -> Topology:
    """Two 4-cliques {0..3}, {4..7} plus the links i <-> i+4 (16 edges)."""
    pairs = [(i, j) for base in (0, 4) for i in range(base, base + 4) for j in range(i + 1, base + 4)]
    pairs += [(i, i + 4) for i in range(4)]
    u, v = _edges(pairs)
    w = np.asarray(weights, np.int32)[rng.integers(0, len(weights) - 1, len(pairs))]
    return Topology("hybrid-cube-mesh-8", 8, u, v, w.astype(np.int32))


def random_regular(rng: Rng, n: int = 32, degree: int = 6, weights=(25, 50), max_tries: int = 1_000_000) -> Topology:
    """Configuration model: pair the n*degree stubs at random, resample until simple."""
    stubs = np.repeat(np.arange(n, dtype=np.int64), degree)
    for _ in range(max_tries):
        perm = stubs[rng.permutation(stubs.shape[0])]
        a, b = perm[0::2], perm[1::2]
        if np.any(a == b):
            continue
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        key = lo * n + hi
        if np.unique(key).shape[0] != key.shape[0]:
            continue
        order = np.argsort(key)
        u, v = lo[order].astype(np.int32), hi[order].astype(np.int32)
        w = np.asarray(weights, np.int32)[rng.integers(0, len(weights) - 1, u.shape[0])]
        return Topology(f"random-{degree}-regular-{n}", n, u, v, w.astype(np.int32))
    raise RuntimeError("configuration model did not produce a simple graph")


def torus3d(dim: int = 4, w_x: int = 50, w_yz: int = 25) -> Topology:
    """dim^3 torus, vertex id = dim^2*x + dim*y + z; x-links weigh w_x, y/z-links w_yz."""
    n = dim ** 3
    pairs, ws = set(), {}
    for x in range(dim):
        for y in range(dim):
            for z in range(dim):
                s = dim * dim * x + dim * y + z
                for axis, (dx, dy, dz) in enumerate(((1, 0, 0), (0, 1, 0), (0, 0, 1))):
                    t = dim * dim * ((x + dx) % dim) + dim * ((y + dy) % dim) + (z + dz) % dim
                    e = (min(s, t), max(s, t))
                    if e[0] != e[1] and e not in pairs:
                        pairs.add(e)
                        ws[e] = w_x if axis == 0 else w_yz
    order = sorted(pairs)
    u, v = _edges(order)
    w = np.asarray([ws[e] for e in order], np.int32)
    return Topology(f"torus-{dim}x{dim}x{dim}", n, u, v, w)


def dragonfly(rng: Rng, groups: int = 16, group_size: int = 8, w_local: int = 50, w_global: int = 25) -> Topology:
    """groups x K_group_size (local links) plus one global link per pair of groups.

    Each group spreads its (groups - 1) global links over its vertices as evenly
    as possible (a seeded shuffle of the port list decides which vertex takes
    which partner group).
    """
    n = groups * group_size
    pairs, ws = [], []
    for g in range(groups):
        base = g * group_size
        for i in range(group_size):
            for j in range(i + 1, group_size):
                pairs.append((base + i, base + j))
                ws.append(w_local)
    ports = []
    for g in range(groups):
        need = groups - 1
        plist = np.asarray([i % group_size for i in range(need)], np.int64)
        ports.append(plist[rng.permutation(need)])
    slot = [0] * groups
    for g in range(groups):
        for h in range(g + 1, groups):
            pg = ports[g][slot[g]]
            ph = ports[h][slot[h]]
            slot[g] += 1
            slot[h] += 1
            pairs.append((g * group_size + int(pg), h * group_size + int(ph)))
            ws.append(w_global)
    order = np.lexsort((np.asarray([p[1] for p in pairs]), np.asarray([p[0] for p in pairs])))
    u = np.asarray([pairs[i][0] for i in order], np.int32)
    v = np.asarray([pairs[i][1] for i in order], np.int32)
    w = np.asarray([ws[i] for i in order], np.int32)
    return Topology(f"dragonfly-{groups}x{group_size}", n, u, v, w)


def boards256(rng: Rng, boards: int = 32, w_board=(25, 50), w_uplink: int = 10) -> Topology:
    """boards x hybrid cube-mesh of 8; local vertices 0..3 are uplinks.

    Uplink j of board b connects to uplink j of board (b + 1) mod boards.
    """
    pairs, ws = [], []
    for bidx in range(boards):
        t = hybrid_cube_mesh8(rng, w_board)
        base = 8 * bidx
        for a, b, w in zip(t.u, t.v, t.w):
            pairs.append((base + int(a), base + int(b)))
            ws.append(int(w))
    for bidx in range(boards):
        nb = (bidx + 1) % boards
        for j in range(4):
            a, b = 8 * bidx + j, 8 * nb + j
            pairs.append((min(a, b), max(a, b)))
            ws.append(w_uplink)
    order = sorted(range(len(pairs)), key=lambda i: pairs[i])
    u = np.asarray([pairs[i][0] for i in order], np.int32)
    v = np.asarray([pairs[i][1] for i in order], np.int32)
    w = np.asarray([ws[i] for i in order], np.int32)
    return Topology(f"boards-{boards}x8", 8 * boards, u, v, w)


def dgx_fixture() -> Topology:
    """8-GPU fixture built from the link facts stated in Sec. 2.1-2.2.

    1-indexed GPUs: 1-5 double NVLink (50), 1-2 single NVLink (25), 1-6 PCIe
    only; exactly one single link among 1-3, 1-4, 3-4; PCIe (12) fills every
    pair without NVLink.  Stored 0-indexed, with fill_weight = 12.  This is a
    fixture consistent with those statements, not the machine's full wiring.
    """
    one = {
        (1, 2): 25, (1, 3): 25, (1, 4): 50, (2, 3): 50, (2, 4): 25, (3, 4): 50,
        (5, 6): 25, (5, 7): 50, (5, 8): 25, (6, 7): 25, (6, 8): 50, (7, 8): 25,
        (1, 5): 50, (2, 6): 50, (3, 7): 25, (4, 8): 25,
    }
    order = sorted(one)
    u = np.asarray([a - 1 for a, _ in order], np.int32)
    v = np.asarray([b - 1 for _, b in order], np.int32)
    w = np.asarray([one[e] for e in order], np.int32)
    return Topology("dgx-fixture-8", 8, u, v, w, fill_weight=12)


def torus2d16(w_x: int = 50, w_y: int = 25, fill: int = 12) -> Topology:
    """16 accelerators on a 4x4 torus (id 4x + y): double NVLinks (w_x) along
    x, single NVLinks (w_y) along y, PCIe (fill) between every other pair.
    A stand-in for the Torus-2d of Sec. 6 with its three link types (the
    paper's wiring figure is not available)."""
    pairs = {}
    for x in range(4):
        for y in range(4):
            s = 4 * x + y
            for t, wt in ((4 * ((x + 1) % 4) + y, w_x), (4 * x + (y + 1) % 4, w_y)):
                pairs[(min(s, t), max(s, t))] = wt
    order = sorted(pairs)
    u, v = _edges(order)
    return Topology("torus2d-16", 16, u, v, np.asarray([pairs[e] for e in order], np.int32), fill_weight=fill)


def cubemesh16(link: int = 25, fill: int = 12) -> Topology:
    """Two 8-accelerator boards with the NVLink layout of dgx_fixture (ids
    0-7 and 8-15) joined by one single NVLink (link) between corresponding
    accelerators, PCIe (fill) elsewhere.  A stand-in for the Cube-mesh of
    Sec. 6 (wiring figure not available)."""
    board = dgx_fixture()
    u = np.concatenate([board.u, board.u + 8, np.arange(8, dtype=np.int32)]).astype(np.int32)
    v = np.concatenate([board.v, board.v + 8, np.arange(8, 16, dtype=np.int32)]).astype(np.int32)
    w = np.concatenate([board.w, board.w, np.full(8, link, np.int32)]).astype(np.int32)
    return Topology("cubemesh-16", 16, u, v, w, fill_weight=fill)


# --------------------------------------------------------------------------
# Requests


@dataclasses.dataclass
class Requests:
    """A batch of allocation requests against one topology.

    pattern_index[i] indexes `patterns`; busy[i] is a 256-bit mask (8 x u32).
    """

    patterns: list
    pattern_index: np.ndarray  # int32 [R]
    alpha: np.ndarray  # int32 [R]
    beta: np.ndarray  # int32 [R]
    busy: np.ndarray  # uint32 [R, 8]

    def __len__(self) -> int:
        return int(self.pattern_index.shape[0])

    def subset(self, idx) -> "Requests":
        idx = np.asarray(idx)
        return Requests(self.patterns, self.pattern_index[idx], self.alpha[idx], self.beta[idx], self.busy[idx])


def busy_to_bool(busy_row: np.ndarray, n: int) -> np.ndarray:
    """256-bit mask -> bool[n]."""
    bits = np.zeros(n, dtype=bool)
    for v in range(n):
        bits[v] = (int(busy_row[v >> 5]) >> (v & 31)) & 1
    return bits


def _busy_masks(rng: Rng, n: int, counts: np.ndarray) -> np.ndarray:
    """Uniform random subsets of {0..n-1} of the given sizes, as 256-bit masks."""
    r = counts.shape[0]
    keys = rng.u64(r * n).reshape(r, n)
    order = np.argsort(keys, axis=1, kind="stable")
    rank = np.empty_like(order)
    np.put_along_axis(rank, order, np.arange(n)[None, :].repeat(r, 0), axis=1)
    chosen = rank < counts[:, None]
    busy = np.zeros((r, BUSY_WORDS), np.uint64)
    for v in range(n):
        busy[:, v >> 5] |= chosen[:, v].astype(np.uint64) << np.uint64(v & 31)
    return busy.astype(np.uint32)


def boards_snapshots(rng: Rng, count: int, boards: int = 32, max_jobs: int = 7, strays: int = 8) -> np.ndarray:
    """Busy masks of the boards machine as a served run of 31-32-accelerator
    jobs leaves it: J ~ U{0..max_jobs} jobs, each holding a run of 4
    consecutive boards (32 accelerators; a tree-31 job, drawn with
    probability 1/2, leaves one of them free) at a uniform board offset (runs
    that overlap merge), plus U{0..strays} stray busy accelerators.  Returns
    [count, 8] uint32 masks."""
    n = 8 * boards
    jobs = rng.integers(0, max_jobs, count)
    first = rng.integers(0, boards - 1, count * max_jobs).reshape(count, max_jobs)
    tree = rng.uniform(count * max_jobs).reshape(count, max_jobs) < 0.5
    drop = rng.integers(0, 31, count * max_jobs).reshape(count, max_jobs)
    nstray = rng.integers(0, strays, count)
    stray = rng.integers(0, n - 1, count * max(strays, 1)).reshape(count, max(strays, 1))
    verts = (8 * first[:, :, None] + np.arange(32)[None, None, :]) % n  # [count, jobs, 32]
    keep = np.arange(max_jobs)[None, :, None] < jobs[:, None, None]
    keep = keep & ~(tree[:, :, None] & (np.arange(32)[None, None, :] == drop[:, :, None]))
    busy = np.zeros((count, n), bool)
    rows = np.broadcast_to(np.arange(count)[:, None, None], verts.shape)
    busy[rows[keep], verts[keep]] = True
    srows = np.broadcast_to(np.arange(count)[:, None], stray.shape)
    sk = np.arange(stray.shape[1])[None, :] < nstray[:, None]
    busy[srows[sk], stray[sk]] = True
    out = np.zeros((count, BUSY_WORDS), np.uint64)
    for v in range(n):
        out[:, v >> 5] |= busy[:, v].astype(np.uint64) << np.uint64(v & 31)
    return out.astype(np.uint32)


def _mix_patterns(rng: Rng, count: int, kmax_rt: int, clique_max: int):
    """Pattern mix shared by the batched and served workloads."""
    kinds = rng.integers(0, 2, count)
    k_rt = rng.integers(2, kmax_rt, count)
    k_cl = rng.integers(2, clique_max, count)
    pats, index, idx_of = [], np.zeros(count, np.int32), {}
    for i in range(count):
        kind = ("ring", "tree", "clique")[kinds[i]]
        k = int(k_cl[i] if kind == "clique" else k_rt[i])
        key = (kind, k)
        if key not in idx_of:
            idx_of[key] = len(pats)
            pats.append(pattern(kind, k))
        index[i] = idx_of[key]
    return pats, index


@dataclasses.dataclass
class Workload:
    name: str
    topology: Topology
    requests: Requests
    description: str


WORKLOADS = ("cube_mesh8", "regular32", "torus64", "dragonfly128", "boards256")


def workload(name: str, num_requests: int | None = None, seed: int | None = None) -> Workload:
    """The five workload shapes, each seeded by its own default seed.

    cube_mesh8:   8-vertex hybrid cube-mesh, 1000 independent requests, ring-4 /
                  clique-3 / path-2, 0-3 busy vertices.
    regular32:    32-vertex random 6-regular graph, 10^4 independent requests,
                  ring-8 / tree-7 / clique-4, occupancy U[0, 0.5].
    torus64:      4x4x4 torus, 10^5 requests, ring/tree k in 2..16, clique k
                  in 2..4, occupancy U[0, 0.6].
    dragonfly128: 16 groups x K8 plus one global link per group pair, request
                  mix of torus64, occupancy kept on the device (served).
    boards256:    32 boards x hybrid cube-mesh with a 4-uplink ring of boards,
                  ring-32 / tree-31 / clique-8, 10^6 requests, each with the
                  occupancy a served run leaves (boards_snapshots).
    """
    if name not in WORKLOADS:
        raise ValueError(f"unknown workload {name!r}; one of {WORKLOADS}")
    default_seed = WORKLOADS.index(name) + 1
    seed = default_seed if seed is None else seed
    trng = Rng(seed, 1)
    rrng = Rng(seed, 2)
    if name == "cube_mesh8":
        topo = hybrid_cube_mesh8(trng)
        r = 1000 if num_requests is None else num_requests
        pats = [pattern("ring", 4), pattern("clique", 3), pattern("path", 2)]
        index = rrng.integers(0, 2, r).astype(np.int32)
        busy = _busy_masks(rrng, topo.n, rrng.integers(0, 3, r))
        desc = "8-vertex hybrid cube-mesh, ring-4/clique-3/path-2, 0-3 busy vertices"
    elif name == "regular32":
        topo = random_regular(trng, 32, 6)
        r = 10_000 if num_requests is None else num_requests
        pats = [pattern("ring", 8), pattern("tree", 7), pattern("clique", 4)]
        index = rrng.integers(0, 2, r).astype(np.int32)
        u = rrng.uniform(r) * 0.5
        busy = _busy_masks(rrng, topo.n, np.floor(u * topo.n).astype(np.int64))
        desc = "32-vertex random 6-regular graph, ring-8/tree-7/clique-4, occupancy U[0,0.5]"
    elif name == "torus64":
        topo = torus3d(4)
        r = 100_000 if num_requests is None else num_requests
        pats, index = _mix_patterns(rrng, r, 16, 4)
        u = rrng.uniform(r) * 0.6
        busy = _busy_masks(rrng, topo.n, np.floor(u * topo.n).astype(np.int64))
        desc = "4x4x4 torus, ring/tree k in 2..16, clique k in 2..4, occupancy U[0,0.6]"
    elif name == "dragonfly128":
        topo = dragonfly(trng)
        r = 10_000 if num_requests is None else num_requests
        pats, index = _mix_patterns(rrng, r, 16, 4)
        busy = np.zeros((r, BUSY_WORDS), np.uint32)  # served: occupancy lives on the device
        desc = "128-vertex dragonfly (16 x K8 + one global link per group pair), served"
    else:
        topo = boards256(trng)
        r = 1_000_000 if num_requests is None else num_requests
        pats = [pattern("ring", 32), pattern("tree", 31), pattern("clique", 8)]
        index = rrng.integers(0, 2, r).astype(np.int32)
        busy = boards_snapshots(Rng(seed, 3), r)
        desc = ("256-vertex boards (32 x hybrid cube-mesh, 4-uplink ring of boards), ring-32/tree-31/clique-8, "
                "served-occupancy snapshots (0-7 jobs of 4 consecutive boards, 0-8 stray busy)")
    ones = np.ones(r, np.int32)
    reqs = Requests(pats, index, ones.copy(), ones.copy(), busy)
    return Workload(name, topo, reqs, desc)


def arrivals(rng: Rng, count: int, rate: float, mean_k: float, n: int, occupancy: float = 0.6):
    """Poisson arrivals at `rate` per second and exponential lifetimes.

    Mean lifetime tau = occupancy * n / (rate * mean_k), so the offered
    occupancy is about `occupancy` at every rate.  Returns (t_arrive, lifetime)
    in seconds.
    """
    gaps = -np.log1p(-rng.uniform(count)) / rate
    tau = occupancy * n / (rate * mean_k)
    life = -np.log1p(-rng.uniform(count)) * tau
    return np.cumsum(gaps), life


@dataclasses.dataclass
class ServedTrace:
    """A served workload: one topology and timed arrivals with lifetimes."""

    topology: Topology
    patterns: list
    pattern_index: np.ndarray  # int32 [R]
    at_ns: np.ndarray  # int64 [R], non-decreasing
    lifetime_ns: np.ndarray  # int64 [R]
    rate: float
    description: str


def served_trace(count: int, rate: float, kmax_rt: int = 8, clique_max: int = 4, occupancy: float = 0.6,
                 seed: int = 4) -> ServedTrace:
    """Poisson arrivals at `rate`/s on the 128-vertex dragonfly.

    Pattern mix as in torus64 (ring/tree k uniform in 2..kmax_rt, clique k in
    2..clique_max); exponential lifetimes with mean occupancy * n / (rate * E[k])
    so the offered occupancy is about `occupancy` at every rate.
    """
    trng = Rng(seed, 1)
    rrng = Rng(seed, 3)
    topo = dragonfly(trng)
    pats, index = _mix_patterns(rrng, count, kmax_rt, clique_max)
    ks = np.asarray([pats[i].k for i in index], np.float64)
    t, life = arrivals(rrng, count, rate, float(ks.mean()), topo.n, occupancy)
    desc = (f"128-vertex dragonfly, ring/tree k in 2..{kmax_rt}, clique k in 2..{clique_max}, "
            f"Poisson {rate:g}/s, offered occupancy {occupancy:g}")
    return ServedTrace(topo, pats, index, (t * 1e9).astype(np.int64), (life * 1e9).astype(np.int64), rate, desc)


# --------------------------------------------------------------------------
# Simulator job files (Sec. 5 and Sec. 6)

#: Workloads of the evaluation and their bandwidth sensitivity as Sec. 2.3
#: and Sec. 5 classify them.
SIM_NETWORKS = (("AlexNet", True), ("VGG-16", True), ("ResNet-50", True), ("Inception-v3", True),
                ("GoogleNet", False), ("CaffeNet", False), ("Cusimann", False), ("GMM", False), ("Jacobi", False))


@dataclasses.dataclass
class SimJobs:
    """A job file: job i runs network[i] on the pattern patterns[pattern_index[i]]."""

    patterns: list
    pattern_index: np.ndarray  # int32 [J]
    arrive: np.ndarray  # int64 [J], non-decreasing cycles
    duration: np.ndarray  # int64 [J] cycles
    sensitive: np.ndarray  # int32 [J]
    network: list

    def __len__(self) -> int:
        return int(self.pattern_index.shape[0])


def sim_jobs(count: int = 300, seed: int = 6, max_gpus: int = 5, duration=(100, 1000), arrival_gap: int = 0) -> SimJobs:
    """Job file in the manner of Sec. 5: a uniform mix of the workloads in
    SIM_NETWORKS, GPUs per job uniform in 1..max_gpus, each job's pattern the
    ring over its GPUs (the NCCL ring of Sec. 3.1; 1 GPU = one vertex, 2 =
    one edge), durations uniform in `duration` cycles.  With arrival_gap = 0
    every job is in the file at cycle 0 (the dispatcher reads it whole);
    otherwise job i arrives at i * arrival_gap.  Durations and the network mix
    are synthetic stand-ins for the measured execution times of the paper's
    runs, which are not available."""
    rng = Rng(seed, 11)
    pats = [pattern("ring", k) for k in range(1, max_gpus + 1)]
    gpus = rng.integers(1, max_gpus, count)
    net = rng.integers(0, len(SIM_NETWORKS) - 1, count)
    dur = rng.integers(int(duration[0]), int(duration[1]), count).astype(np.int64)
    arrive = np.arange(count, dtype=np.int64) * int(arrival_gap)
    sens = np.asarray([1 if SIM_NETWORKS[i][1] else 0 for i in net], np.int32)
    return SimJobs(pats, (gpus - 1).astype(np.int32), arrive, dur, sens, [SIM_NETWORKS[i][0] for i in net])
