"""Write tests/golden/expected_counts.txt: oracle results (Algorithm 1, run by
the CPU oracle only) for the full-size seeded workloads, so the GPU tests can
compare at full size without re-running the oracle.

With --digests, write tests/golden/expected_digests.txt instead: SHA-256
digests of the oracle's per-vertex counts (over unified ids) and per-edge
counts (over the graph's distinct (u, v) pairs in ascending u * |V| + v
order) of the full-size Chung-Lu 1M x 200k x 20M graph, so that the GPU
arrays can be compared element by element at full size (see digest()).

Usage: python tests/golden/make_expected.py [workload ...] [--threads N] [--digests]
Existing lines for other workloads are kept.
"""
import argparse
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "expected_counts.txt")
OUT_DIGESTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "expected_digests.txt")
DIGEST_HEADER = """# SHA-256 of oracle per-vertex / per-edge butterfly counts (tip and wing
# counts, CPU oracle only) for full-size seeded workloads. Written by
# tests/golden/make_expected.py --digests. Columns: workload kind sha256, where
# kind is vertices (balanced then unbalanced, uint64 little-endian, unified ids)
# or edges (the same over the distinct (u, v) pairs in ascending u*|V| + v).
"""
HEADER = """# Oracle (Algorithm 1, CPU) results for the seeded full-size workloads.
# Written by tests/golden/make_expected.py, which calls only oracle/ (and the
# shared input generator synth/). Columns: workload balanced unbalanced wedges.
"""


def read():
    rows = {}
    if os.path.exists(OUT):
        for line in open(OUT):
            line = line.split("#", 1)[0].split()
            if len(line) == 4:
                rows[line[0]] = tuple(int(x) for x in line[1:])
    return rows


def digest(balanced, unbalanced) -> str:
    """SHA-256 of two count arrays as little-endian uint64, one after the other."""
    import hashlib

    import numpy as np
    h = hashlib.sha256()
    for a in (balanced, unbalanced):
        h.update(np.ascontiguousarray(a, dtype="<u8").tobytes())
    return h.hexdigest()


def edge_queries(g):
    """The graph's distinct (u, v) pairs in ascending u * |V| + v order."""
    import numpy as np
    pairs = np.unique(g.u.astype(np.int64) * g.n_v + g.v)
    return (pairs // g.n_v).astype(np.int32), (pairs % g.n_v).astype(np.int32)


def read_digests():
    rows = {}
    if os.path.exists(OUT_DIGESTS):
        for line in open(OUT_DIGESTS):
            f = line.split("#", 1)[0].split()
            if len(f) == 3:
                rows[(f[0], f[1])] = f[2]
    return rows


def write_digests(names):
    rows = read_digests()
    for name in names:
        g = synth.workload(name)
        t = time.time()
        rows[(name, "vertices")] = digest(*oracle.count_per_vertex(g.u, g.v, g.s, g.n_u, g.n_v))
        print(name, "vertices", f"{time.time() - t:.1f}s", flush=True)
        t = time.time()
        qu, qv = edge_queries(g)
        rows[(name, "edges")] = digest(*oracle.count_per_edge(g.u, g.v, g.s, g.n_u, g.n_v, qu, qv))
        print(name, "edges", f"{time.time() - t:.1f}s", flush=True)
        with open(OUT_DIGESTS, "w") as f:
            f.write(DIGEST_HEADER)
            for (w, kind) in sorted(rows):
                f.write(f"{w} {kind} {rows[(w, kind)]}\n")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workloads", nargs="*", default=["uniform-2k-3k-20k", "chunglu-1m-200k-20m"])
    ap.add_argument("--threads", type=int, default=synth.default_threads())
    ap.add_argument("--digests", action="store_true")
    a = ap.parse_args()
    if a.digests:
        write_digests(a.workloads if a.workloads != ["uniform-2k-3k-20k", "chunglu-1m-200k-20m"]
                      else ["chunglu-1m-200k-20m"])
        return
    rows = read()
    for name in a.workloads:
        t = time.time()
        g = synth.workload(name)
        rows[name] = oracle.count(g.u, g.v, g.s, g.n_u, g.n_v, threads=a.threads)
        print(name, rows[name], f"{time.time() - t:.1f}s", flush=True)
        with open(OUT, "w") as f:
            f.write(HEADER)
            for k in sorted(rows):
                f.write(f"{k} {rows[k][0]} {rows[k][1]} {rows[k][2]}\n")


if __name__ == "__main__":
    main()
