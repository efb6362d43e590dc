"""Writes config5_tree_images.json: free sets for the tree-31 parity cases on
the 256-vertex boards topology.

Each entry is the vertex set of one placement of the 31-vertex binary tree
(heap order, parent(i) = (i - 1) // 2) in the boards topology of
workloads.workload("boards256"), found by a seeded randomized greedy
construction that prefers vertices with few links to the vertices already
placed, so the set induces few links beyond the tree's 30.  The sets are
inputs of the parity tests (busy = every other vertex), not expected
values: the tests get their expected decisions from the oracle.  This script
uses only the input generator and its own search; it calls neither the
oracle nor the CUDA library.

Run from the repository root:  python tests/golden/make_config5_fixtures.py
"""

import json
import os
import random
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from paper_2110_03214_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "config5_tree_images.json")


def main():
    topo = W.workload("boards256", num_requests=1).topology
    adj = {v: set() for v in range(topo.n)}
    for a, b in zip(topo.u, topo.v):
        adj[int(a)].add(int(b))
        adj[int(b)].add(int(a))

    def induced(vs):
        return sum(1 for a in vs for b in adj[a] if b in vs and a < b)

    images = []
    for seed, first_board in ((11, 0), (12, 9), (13, 17), (14, 24)):
        rnd = random.Random(seed)
        window = {(8 * first_board + j) % topo.n for j in range(64)}
        best = None
        for _ in range(30000):
            phi = [rnd.choice(sorted(window))]
            used = set(phi)
            for i in range(1, 31):
                par = phi[(i - 1) // 2]
                cand = sorted(x for x in adj[par] if x in window and x not in used)
                if not cand:
                    break
                pen = [sum(1 for y in adj[x] if y in used and y != par) + rnd.random() * 0.5 for x in cand]
                x = cand[pen.index(min(pen))]
                phi.append(x)
                used.add(x)
            if len(phi) == 31:
                e = induced(used)
                if best is None or e < best[0]:
                    best = (e, sorted(used))
        images.append({"seed": seed, "first_board": first_board, "induced_links": best[0], "free": best[1]})
    with open(OUT, "w") as f:
        json.dump({"topology": "boards256 (workloads.workload default seed)", "pattern": "tree-31",
                   "images": images}, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
