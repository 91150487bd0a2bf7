"""Write tests/golden/expected_counts.txt: oracle results (Algorithm 1, run by
the CPU oracle only) for the full-size seeded workloads, so the GPU tests can
compare at full size without re-running the oracle.

Usage: python tests/golden/make_expected.py [workload ...] [--threads N]
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workloads", nargs="*", default=["uniform-2k-3k-20k", "chunglu-1m-200k-20m"])
    ap.add_argument("--threads", type=int, default=synth.default_threads())
    a = ap.parse_args()
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
