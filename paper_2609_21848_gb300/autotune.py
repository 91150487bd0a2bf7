"""Autotuner for the counting tiers (``dbbc_set_tuning``).

A coordinate search over the tier thresholds, the hash-table load factor, the
hub work-item size and the lane-group density thresholds. Each candidate is
measured on the caller's own graphs: the graphs are built with that tuning
(tiers and hub items are decided at build time) and counted several times,
timed with CUDA events; the fastest median wins. Tuning never changes a count,
only the speed, so any candidate is safe.

Results are saved as JSON keyed by the GPU's name in ``tuning/`` next to this
file, one record per workload tuned on; :func:`apply_saved` (called when the
library is loaded, unless ``DBBC_NO_TUNING`` is set) applies the current GPU's
default record, or the record of a named workload.

    python -m paper_2609_21848_gb300.autotune --workload chunglu-1m-200k-20m
"""
from __future__ import annotations

import argparse
import json
import os
import re
import time

HERE = os.path.dirname(os.path.abspath(__file__))
TUNING_DIR = os.path.join(HERE, "tuning")

DEFAULT = {"light_max_work": 512, "medium_max_work": 4096, "hub_item_work": 1 << 20,
           "group_density": [40.0, 16.0, 6.0, 2.0], "hash_mult_log": 1, "list_density": 8.0, "list_group_log": 2,
           "finalize_window_wedges": 65536, "list_wide_density": 1e30}

SPACE = [
    ("light_max_work", [64, 128, 256, 512]),
    ("medium_max_work", [64, 128, 256, 512, 1024, 2048, 4096]),  # = light_max_work: no medium tier
    ("hash_mult_log", [1, 2]),
    ("hub_item_work", [1 << 19, 1 << 20, 1 << 21, 1 << 22]),
    ("group_density", [[40.0, 16.0, 6.0, 2.0], [64.0, 24.0, 8.0, 3.0], [24.0, 10.0, 4.0, 1.5],
                       [96.0, 32.0, 12.0, 4.0], [128.0, 48.0, 12.0, 4.0], [128.0, 48.0, 16.0, 6.0],
                       [192.0, 64.0, 16.0, 6.0], [256.0, 96.0, 24.0, 8.0]]),
    ("list_density", [0.0, 4.0, 8.0, 16.0, 32.0, 64.0, 128.0]),
    ("list_group_log", [2, 3, 4, 5]),
    ("finalize_window_wedges", [0, 16384, 65536, 262144, 2**64 - 1]),
    ("list_wide_density", [16.0, 32.0, 48.0, 1e30]),
]


def gpu_key(name: str | None = None) -> str:
    if name is None:
        import torch
        name = torch.cuda.get_device_name()
    return re.sub(r"[^A-Za-z0-9]+", "_", name).strip("_")


def saved_path(name: str | None = None) -> str:
    return os.path.join(TUNING_DIR, gpu_key(name) + ".json")


def apply_saved(workload: str | None = None) -> dict | None:
    """Apply the saved tuning of the current GPU (its default record, or the
    one tuned on `workload`), if any; returns it."""
    try:
        import torch
        if not torch.cuda.is_available():
            return None
        path = saved_path()
    except Exception:
        return None
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f)
    entry = rec["workloads"].get(workload or rec["default"])
    if entry is None:
        return None
    from . import dbbc_set_tuning
    dbbc_set_tuning(entry["tuning"])
    return entry["tuning"]


def measure(graphs, tuning: dict, repeats: int = 5, stream=None) -> float:
    """Median milliseconds of one count of all `graphs` (device COO tuples
    (u, v, s, n_u, n_v)) built with `tuning`; several graphs are counted as one
    batch plan."""
    import torch

    from . import (dbbc_batch_count_async, dbbc_batch_create, dbbc_count_async, dbbc_graph_from_coo,
                   dbbc_set_tuning)
    dbbc_set_tuning(tuning)
    handles = [dbbc_graph_from_coo(u, v, s, nu, nv, stream=stream) for (u, v, s, nu, nv) in graphs]
    plan = dbbc_batch_create(handles, stream) if len(handles) > 1 else None
    out = torch.zeros((len(handles), 2), dtype=torch.int64, device="cuda")
    times = []
    try:
        for k in range(repeats + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            if plan is not None:
                dbbc_batch_count_async(plan, out, stream)
            else:
                dbbc_count_async(handles[0], out[0], stream)
            e1.record()
            torch.cuda.synchronize()
            if k:
                times.append(e0.elapsed_time(e1))
    finally:
        if plan is not None:
            plan.free()
        for h in handles:
            h.free()
    times.sort()
    return times[len(times) // 2]


def tune(graphs, repeats: int = 5, log=print, start: dict | None = None) -> tuple[dict, float, float]:
    """Coordinate search from `start` (the defaults when None); returns (best
    tuning, its ms, the start's ms)."""
    best = dict(start or DEFAULT)
    best_ms = base_ms = measure(graphs, best, repeats)
    log(f"default: {base_ms:.3f} ms")
    for key, candidates in SPACE:
        for c in candidates:
            if c == best[key]:
                continue
            cand = dict(best)
            cand[key] = c
            if cand["medium_max_work"] < cand["light_max_work"]:
                continue
            ms = measure(graphs, cand, repeats)
            log(f"{key}={c}: {ms:.3f} ms")
            if ms < best_ms:
                best, best_ms = cand, ms
    from . import dbbc_set_tuning
    dbbc_set_tuning(best)
    return best, best_ms, base_ms


def save(tuning: dict, workload: str, ms: float, default_ms: float, path: str | None = None,
         make_default: bool = False) -> str:
    """Add (or replace) the record of `workload` in the GPU's tuning file."""
    import torch
    path = path or saved_path()
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    rec = {"gpu": torch.cuda.get_device_name(), "default": workload, "workloads": {}}
    if os.path.exists(path):
        with open(path) as f:
            rec = json.load(f)
    rec["workloads"][workload] = {"tuning": tuning, "count_ms": ms, "default_ms": default_ms,
                                  "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())}
    if make_default or rec.get("default") not in rec["workloads"]:
        rec["default"] = workload
    with open(path, "w") as f:
        json.dump(rec, f, indent=1)
    return path


def main():
    import sys

    import torch
    sys.path.insert(0, os.path.dirname(HERE))
    import synth

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="chunglu-1m-200k-20m")
    ap.add_argument("--graphs", type=int, default=512, help="graphs of the batch workload to tune on")
    ap.add_argument("--repeats", type=int, default=5)
    ap.add_argument("--out", default=None)
    ap.add_argument("--make-default", action="store_true", help="make this workload's tuning the GPU's default")
    ap.add_argument("--from-saved", action="store_true",
                    help="start the search from this workload's saved record instead of the defaults")
    a = ap.parse_args()
    os.environ["DBBC_NO_TUNING"] = "1"
    dev = torch.device("cuda")
    if a.workload == "batch-4096":
        gs = [synth.batch_graph(i) for i in range(a.graphs)]
    else:
        gs = [synth.workload(a.workload)]
    graphs = [tuple(torch.from_numpy(x).to(dev) for x in (g.u, g.v, g.s)) + (g.n_u, g.n_v) for g in gs]
    start = None
    if a.from_saved:
        path = a.out or saved_path()
        if os.path.exists(path):
            with open(path) as f:
                entry = json.load(f)["workloads"].get(a.workload)
            start = dict(DEFAULT, **entry["tuning"]) if entry else None
    best, ms, base = tune(graphs, a.repeats, start=start)
    path = save(best, a.workload, ms, base, a.out, a.make_default)
    print(json.dumps({"tuning": best, "count_ms": ms, "default_ms": base, "saved": path}))


if __name__ == "__main__":
    main()
