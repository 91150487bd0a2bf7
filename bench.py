#!/usr/bin/env python
"""Benchmark of balanced / unbalanced butterfly counting on GB300.

One step = one pass of the whole path over one synthetic graph already
resident in HBM: build (validate, keep-latest dedup, degrees, Def. 3 ranks,
sign-packed CSR, accepted-wedge work and tiers) + count (light / medium / hub
wedge aggregation, Lemma 1 finalisation, reduction) + free. The metric is
accepted wedges of Algorithm 1 per second (G wedges/s), whole job. The
default workload is the largest single graph (polarized, 20M x 2M vertices,
300M edges); its line also carries the batched form (4,096 resident graphs
counted by one replayed plan, against one count per graph) and the served form
(a Poisson stream of 100,000 requests at 2,000/s) as "batch" and "serve"
records, in graphs/s.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl dbbc|reference]

With N > 1 (launched by torchrun) every rank counts its own replica of the
graph (one GPU per rank, no collective on the data path; "replicas only").
``--impl reference`` times the CPU oracle (Algorithm 1 as written, all host
cores) on pivot samples of the same graph instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "G wedges/s and graphs/s, batched vs per-graph launches, bit-exact counts"
# the largest single graph: the headline line, which also carries the batched
# (4,096 graphs) and served (Poisson stream) records
DEFAULT_WORKLOAD = "polarized-20m-2m-300m"
UNIT = "G wedges/s"
L2_BYTES = 129 * 2**20

# Algorithmic bytes of the method (the roofline's numerator), per unit of
# work of Algorithm 1's Phase 5 with shared-memory counters:
#   per accepted wedge                     : 4 B CSR entry of the endpoint
#   per (pivot, lower neighbour) step      : 4 B pivot-row entry + 16 B row offsets + 8 B end probe
# (the global-counter terms of a touched-list design are zero: the hub
# sweep's counters live in shared memory).
B_WEDGE, B_LOWER = 4, 28
# Bytes the hub sweep's design adds on top (reported beside the roofline, not
# in it): per (item, neighbour) slot initialisation 8 B written, per
# (neighbour, window) cursor step 8 B slot read + 8 B written + 4 B first entry
# past the window, per list-mode visit the same 20 B + 8 B list append.
B_CUR_INIT, B_CUR_STEP, B_LIST_VISIT = 8, 20, 28


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["dbbc", "reference"], default="dbbc")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(synth.WORKLOADS) + ["batch-4096", "serve", "sign-sweep", "tips"])
    ap.add_argument("--n-graphs", type=int, default=4096, help="graphs in the batch-4096 workload")
    ap.add_argument("--requests", type=int, default=synth.SERVE["n_requests"],
                    help="requests of the served workload (and of the default line's serve record)")
    ap.add_argument("--large-pool", type=int, default=16,
                    help="distinct large graphs (5M-20M edges) the served stream's large requests are drawn from")
    ap.add_argument("--no-extras", action="store_true",
                    help="leave the batch and serve records out of the default single-graph line")
    ap.add_argument("--e2e-steps", type=int, default=None, help="steps of the host-buffer end-to-end timing")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--reference-seconds", type=float, default=120.0,
                    help="wall time of the reference arm's warm-up and timed steps together")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="scale a single-graph workload's vertices and edges (small cases for profiling; the "
                         "line then carries the scale and no stored-count check)")
    ap.add_argument("--partition", action="store_true",
                    help="with N > 1 GPUs: every rank counts its LPT share of the pivots of one graph (strong "
                         "scaling) instead of counting its own replica (weak scaling)")
    return ap.parse_args()


def cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def expected_counts(name):
    path = os.path.join(ROOT, "tests", "golden", "expected_counts.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        f = line.split("#", 1)[0].split()
        if len(f) == 4 and f[0] == name:
            return tuple(int(x) for x in f[1:])
    return None


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


KERNEL_SOURCES = ("count.cu", "sweep_device.cuh", "count_device.cuh", "internal.h", "common.cuh")


def kernel_source_sha() -> str:
    """Hash of the sources the counting kernels are built from."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2609_21848_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


def known_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel sources (profiles/traffic.txt: kernel workload sha bytes)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    sha = kernel_source_sha()
    for line in open(path):
        f = line.split("#", 1)[0].split()
        if len(f) == 4 and f[0] == kernel and f[1] == workload and f[2] == sha:
            return float(f[3])
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def run_reference(a):
    """The reference arm: the CPU oracle (Algorithm 1) on the host cores, each
    step a strided pivot sample of the same graph."""
    import oracle
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    nc = cores()
    if a.workload in ("batch-4096", "serve"):
        # graphs of the batch (the served stream's small requests) counted one
        # after another by the oracle; each
        # step a bounded sample of consecutive graphs (about 2 minutes overall)
        per_step = a.reference_seconds / max(1, a.steps + a.warmup)
        graphs = [synth.batch_graph(i) for i in range(min(a.n_graphs, 512))]
        k = 0
        done, t_total = 0, 0.0
        for step in range(a.warmup + a.steps):
            t0 = time.perf_counter()
            n_step = 0
            while time.perf_counter() - t0 < per_step:
                g = graphs[k % len(graphs)]
                oracle.count(g.u, g.v, g.s, g.n_u, g.n_v, threads=nc)
                k += 1
                n_step += 1
            if step >= a.warmup:
                done += n_step
                t_total += time.perf_counter() - t0
        value = done / t_total
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "graphs/s", "n_gpus": a.gpus,
                "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * t_total / a.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
                "data": "synthetic", "config": {"workload": a.workload, "parallelism": "host threads"},
                "cpu_baseline": {"value": value, "unit": "graphs/s", "cores": nc, "kind": "oracle",
                                 "sample": f"{done} batch graphs counted one after another, {nc} threads"},
                "e2e": {"value": value, "unit": "graphs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    # the sign sweep and the per-vertex/per-edge workload run on the Chung-Lu
    # topology; the oracle counts its totals there
    topology = {"sign-sweep": "chunglu-1m-200k-20m", "tips": "chunglu-1m-200k-20m"}.get(a.workload, a.workload)
    g = synth.workload(topology)
    t0 = time.perf_counter()
    bg = oracle.BuiltGraph(g.u, g.v, g.s, g.n_u, g.n_v)
    build_s = time.perf_counter() - t0
    # calibrate the stride so all warm-up + timed steps take --reference-seconds
    per_step = a.reference_seconds / max(1, a.steps + a.warmup)
    probe = max(1, bg.n // 4096)
    t0 = time.perf_counter()
    bg.count_sample(0, probe, nc)
    dt = max(time.perf_counter() - t0, 1e-3)
    step = max(1, int(probe * dt / per_step))
    for k in range(a.warmup):
        bg.count_sample(k % step, step, nc)
    wedges = 0
    t0 = time.perf_counter()
    for k in range(a.steps):
        wedges += bg.count_sample((a.warmup + k) % step, step, nc)[2]
    t = time.perf_counter() - t0
    value = wedges / t / 1e9
    sample = (f"Algorithm 1 on every {step}-th pivot (unified id order) of {topology}, {nc} threads, "
              f"graph built once untimed ({build_s:.1f} s)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * t / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": a.workload, "parallelism": "host threads"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nc, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(g, target_s: float) -> dict:
    import oracle
    nc = cores()
    t0 = time.perf_counter()
    bg = oracle.BuiltGraph(g.u, g.v, g.s, g.n_u, g.n_v)
    build_s = time.perf_counter() - t0
    # A strided probe sets the stride of the main sample; the rate is taken
    # over both, since one large hub can dominate either (the oracle
    # parallelises over pivots, so such a hub keeps one core busy alone).
    probe = max(1, bg.n // 4096)
    t0 = time.perf_counter()
    w0 = bg.count_sample(0, probe, nc)[2]
    dt = max(time.perf_counter() - t0, 1e-3)
    w, t, step = 0, 0.0, probe
    if dt < target_s:
        step = max(1, int(probe * dt / (target_s - dt)))
        t0 = time.perf_counter()
        w = bg.count_sample(1 % step, step, nc)[2]
        t = time.perf_counter() - t0
    bg.close()
    return {"value": (w0 + w) / (dt + t) / 1e9, "unit": UNIT, "cores": nc, "kind": "oracle",
            "sample": f"Algorithm 1 on every {probe}-th pivot and then every {step}-th pivot of the same graph "
                      f"({w0 + w} accepted wedges, {dt + t:.1f} s, {nc} threads; oracle graph build {build_s:.1f} s "
                      f"untimed)"}


def batch_record(a, torch, dbbc, world, rank, local, dist, barrier, graphs=None, with_cpu=True) -> dict:
    """The batched form: thousands of uneven resident graphs counted by one
    replayed CUDA graph (three kernels for all graphs), against the plain path
    of one synchronous count (one launch sequence) per graph. Metric: graphs/s.
    Returns the line (printed by run_batch, or attached to the default line)."""
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    t0 = time.perf_counter()
    if graphs is None:
        graphs = synth.batch(a.n_graphs)
    gen_s = time.perf_counter() - t0
    sizes = [g.m for g in graphs]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    U, V, S = (torch.from_numpy(np.concatenate([getattr(g, k) for g in graphs])).to(dev) for k in ("u", "v", "s"))
    torch.cuda.synchronize(dev)
    eb0, eb1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    eb0.record(stream)
    handles = [dbbc.dbbc_graph_from_coo(U[offs[i]:offs[i + 1]], V[offs[i]:offs[i + 1]], S[offs[i]:offs[i + 1]],
                                        g.n_u, g.n_v, stream=stream) for i, g in enumerate(graphs)]
    eb1.record(stream)
    torch.cuda.synchronize(dev)
    build_ms = eb0.elapsed_time(eb1)
    infos = [h.info for h in handles]
    wedges = sum(i["wedges"] for i in infos)
    # plain: one synchronous count per graph
    for h in handles[:64]:
        dbbc.dbbc_count(h, stream)
    barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    plain = [dbbc.dbbc_count(h, stream) for h in handles]
    torch.cuda.synchronize(dev)
    plain_s = time.perf_counter() - t0
    # batched: one plan, replayed
    plan = dbbc.dbbc_batch_create(handles, stream)
    d_out = torch.zeros((len(handles), 2), dtype=torch.int64, device=dev)
    for _ in range(a.warmup):
        dbbc.dbbc_batch_count_async(plan, d_out, stream)
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(local)
    barrier()
    torch.cuda.synchronize(dev)
    sampler.start()
    time.sleep(0.3)
    launches0 = dbbc.dbbc_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        dbbc.dbbc_batch_count_async(plan, d_out, stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    launches = dbbc.dbbc_kernel_launches() - launches0
    clocks = sampler.stop()
    barrier()
    t_ms = torch.tensor([e0.elapsed_time(e1)], dtype=torch.float64, device=dev)
    if dist is not None:
        dist.all_reduce(t_ms, op=dist.ReduceOp.MAX)
    t_ms = float(t_ms.item())
    got = [tuple(map(int, r)) for r in d_out.cpu().numpy().astype(np.uint64)]
    bit_exact_vs_plain = got == plain
    value = world * len(handles) * a.steps / (t_ms / 1e3)
    plain_gps = len(handles) / plain_s
    # end to end: host COO (pinned) -> one union build of all graphs ->
    # per-component counts on the host
    hU, hV, hS = (torch.from_numpy(np.concatenate([getattr(g, k) for g in graphs])).pin_memory()
                  for k in ("u", "v", "s"))
    nus, nvs = [g.n_u for g in graphs], [g.n_v for g in graphs]
    torch.cuda.synchronize(dev)
    e2e_times = []
    for _ in range(2):  # the first run warms the allocator pools
        t0 = time.perf_counter()
        with dbbc.dbbc_graph_from_coo_multi(hU, hV, hS, offs, nus, nvs, stream=stream) as hu_:
            bal, unb = dbbc.dbbc_count_components(hu_, stream)
        e2e_times.append(time.perf_counter() - t0)
    e2e_s = e2e_times[-1]
    e2e_exact = list(zip(bal.tolist(), unb.tolist())) == plain
    # the union path from device-resident COO (build + count), for comparison
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    with dbbc.dbbc_graph_from_coo_multi(U, V, S, offs, nus, nvs, stream=stream) as hu_:
        ub, uu = dbbc.dbbc_count_components(hu_, stream)
    union_s = time.perf_counter() - t0
    union_exact = list(zip(ub.tolist(), uu.tolist())) == plain

    # algorithmic bytes of one batch count (all tiers)
    nbytes = sum(B_WEDGE * i["wedges"] + B_LOWER * (i["lower_light"] + i["lower_medium"] + i["lower_hub"])
                 for i in infos)
    peaks, peak_kind = measured_peaks()
    per_replay_s = t_ms / 1e3 / a.steps
    achieved = nbytes / per_replay_s / 1e9
    line = {"metric": METRIC, "value": value, "unit": "graphs/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": t_ms / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": "batch-4096", "n_graphs": len(handles), "edges_total": int(offs[-1]),
                       "tuning": dbbc.dbbc_get_tuning(),
                       "wedges_per_step": wedges,
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                       "l2": "inputs larger than L2 (all graphs' CSR %.0f MB > 129 MB)" % (
                           sum(8 * i["m"] + 24 * (i["n_u"] + i["n_v"]) for i in infos) / 1e6)},
            "plain_graphs_per_s": plain_gps, "batched_over_plain": value / world / plain_gps,
            "batched_gwedges_per_s": wedges * a.steps / (t_ms / 1e3) / 1e9,
            "build_ms_all_graphs": build_ms, "generate_s": gen_s,
            "union_build_and_count_graphs_per_s": len(handles) / union_s, "union_bit_exact": union_exact,
            "bit_exact_vs_plain": bit_exact_vs_plain,
            "e2e": {"value": world * len(handles) / e2e_s, "unit": "graphs/s",
                    "h2d_bytes_per_step": 9 * int(offs[-1]), "d2h_bytes_per_step": 16 * len(handles),
                    "steps": 1, "bit_exact": e2e_exact},
            "roofline": {"bound": "hbm", "kernel": "batch count (light + medium + hub sweep, one CUDA graph)",
                         "achieved": achieved, "peak": float(peaks["hbm_gbs"]), "unit": "GB/s",
                         "frac": achieved / float(peaks["hbm_gbs"]), "traffic": None,
                         "peak_kind": f"of {peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                         "bytes_per_launch": nbytes, "ms_per_launch": 1e3 * per_replay_s},
            "gpu_launches": int(launches), "clocks": clocks}
    if with_cpu and rank == 0 and world == 1 and not a.no_cpu_baseline:
        import oracle
        nc = cores()
        t0 = time.perf_counter()
        done = 0
        k = 0
        while time.perf_counter() - t0 < a.cpu_seconds and k < len(graphs):
            g = graphs[k]
            oracle.count(g.u, g.v, g.s, g.n_u, g.n_v, threads=nc)
            done += 1
            k += 1
        t = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": done / t, "unit": "graphs/s", "cores": nc, "kind": "oracle",
                                "sample": f"the first {done} graphs of the batch, one after another, {nc} threads"}
    plan.free()
    for h in handles:
        h.free()
    return line


def run_batch(a, torch, dbbc, world, rank, local, dist, barrier):
    line = batch_record(a, torch, dbbc, world, rank, local, dist, barrier)
    if rank == 0:
        print(json.dumps(line), flush=True)


def serve_record(a, torch, dbbc, world, rank, local, dist, barrier, small=None) -> dict:
    """The served form: a Poisson stream at 2,000 requests/s, 99% graphs of the
    batch distribution and 1% large polarized graphs (5M-20M edges, drawn from
    a pool of --large-pool distinct graphs), served with continuous batching
    (paper_2609_21848_gb300.serve). Reports latency percentiles at that rate,
    the saturated throughput (every request arrives at once), and the plain
    path (one request at a time: build, count, free). Returns the line."""
    from paper_2609_21848_gb300.serve import DbbcBackend, Request, Server, poisson_arrivals
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    rate = synth.SERVE["rate"]
    n = a.requests
    t0 = time.perf_counter()
    if small is None:
        small = synth.batch(min(n, 4096))
    is_large = [synth.serve_is_large(i) for i in range(n)]
    n_large = sum(is_large)
    large = [synth.serve_large_graph(i) for i in range(min(a.large_pool, max(1, n_large)))] if n_large else []
    gen_s = time.perf_counter() - t0
    pinned = {}

    def pin(key, g):
        if key not in pinned:
            pinned[key] = tuple(torch.from_numpy(x).pin_memory() for x in (g.u, g.v, g.s)) + (g.n_u, g.n_v)
        return pinned[key]

    picks = []
    kl = 0
    for i in range(n):
        if is_large[i]:
            picks.append(("L", kl % len(large)))
            kl += 1
        else:
            picks.append(("S", i % len(small)))
    graph_of = {("S", j): small[j] for j in range(len(small))}
    graph_of.update({("L", j): large[j] for j in range(len(large))})
    # each distinct graph counted alone (reference answers for the served results)
    alone = {}
    for key in set(picks):
        g = graph_of[key]
        pu, pv, ps, nu, nv = pin(key, g)
        with dbbc.dbbc_graph_from_coo(pu, pv, ps, nu, nv, stream=stream) as h:
            alone[key] = dbbc.dbbc_count(h, stream)

    def requests(arrivals):
        out = []
        for i, key in enumerate(picks):
            pu, pv, ps, nu, nv = pin(key, graph_of[key])
            out.append(Request(i, pu, pv, ps, nu, nv, float(arrivals[i])))
        return out

    backend = DbbcBackend(local)
    torch.cuda.synchronize(dev)
    barrier()
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = dbbc.dbbc_kernel_launches()
    st = Server(backend).run(requests(poisson_arrivals(n, rate, seed=synth.SEED_BASE + 4)))
    torch.cuda.synchronize(dev)
    launches = dbbc.dbbc_kernel_launches() - launches0
    clocks = sampler.stop()
    nominal = st.summary()
    exact = all((r.balanced, r.unbalanced) == alone[picks[r.rid]] for r in st.results)
    # saturated: the whole stream at once
    st2 = Server(backend).run(requests(np.zeros(n)))
    torch.cuda.synchronize(dev)
    sat = st2.summary()
    exact = exact and all((r.balanced, r.unbalanced) == alone[picks[r.rid]] for r in st2.results)
    # plain: one request at a time
    n_plain = min(n, 1000)
    t0 = time.perf_counter()
    for i in range(n_plain):
        pu, pv, ps, nu, nv = pin(picks[i], graph_of[picks[i]])
        with dbbc.dbbc_graph_from_coo(pu, pv, ps, nu, nv, stream=stream) as h:
            dbbc.dbbc_count(h, stream)
    torch.cuda.synchronize(dev)
    plain_gps = n_plain / (time.perf_counter() - t0)
    value = world * sat["graphs_per_s"]
    edges = sum(graph_of[k].m for k in picks)
    line = {"metric": METRIC, "value": value, "unit": "graphs/s", "n_gpus": world, "steps": 1, "warmup": 0,
            "ms_per_step": 1e3 * sat["wall_s"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int64", "data": "synthetic",
            "config": {"workload": "serve", "requests": n, "rate_per_s": rate, "large_requests": n_large,
                       "tuning": dbbc.dbbc_get_tuning(),
                       "distinct_large_graphs": len(large), "edges_total": edges,
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                       "timing": "wall clock around the whole stream (host COO in pinned memory)"},
            "served_at_rate": {k: nominal[k] for k in ("graphs_per_s", "p50_ms", "p99_ms", "max_ms", "batches",
                                                     "wall_s")},
            "saturated": {k: sat[k] for k in ("graphs_per_s", "p50_ms", "p99_ms", "batches", "wall_s")},
            "plain_graphs_per_s": plain_gps, "served_over_plain": sat["graphs_per_s"] / plain_gps,
            "bit_exact_vs_alone": exact, "generate_s": gen_s,
            "e2e": {"value": value, "unit": "graphs/s", "h2d_bytes_per_step": 9 * edges,
                    "d2h_bytes_per_step": 16 * n, "steps": 1, "bit_exact": exact},
            "roofline": None, "gpu_launches": int(launches), "clocks": clocks}
    return line


def run_serve(a, torch, dbbc, world, rank, local, dist, barrier):
    line = serve_record(a, torch, dbbc, world, rank, local, dist, barrier)
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_sign_sweep(a, torch, dbbc, world, rank, local, dist, barrier):
    """The sign-ratio study (paper Section VI, "Sign Distribution"): the
    Chung-Lu 1M x 200k x 20M topology with P(+) from 0.1 to 0.9. The count
    time should not move (one packed counter per endpoint, no branch on the
    sign); the balanced / unbalanced split does, while their sum (the unsigned
    butterfly count) stays put."""
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    p = dict(synth.WORKLOADS["chunglu-1m-200k-20m"])
    p.pop("index")
    rows = []
    for pp in (0.1, 0.3, 0.5, 0.7, 0.9):
        p["p_plus"] = pp
        g = synth.generate(synth.SEED_BASE + 1, name=f"p+={pp}", **p)
        du, dv, ds = (torch.from_numpy(x).to(dev) for x in (g.u, g.v, g.s))
        times, counts = [], None
        for k in range(a.warmup + a.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            with dbbc.dbbc_graph_from_coo(du, dv, ds, g.n_u, g.n_v, stream=stream) as h:
                counts = dbbc.dbbc_count(h, stream)
                wedges = h.info["wedges"]
            e1.record(stream)
            torch.cuda.synchronize(dev)
            if k >= a.warmup:
                times.append(e0.elapsed_time(e1))
        times.sort()
        rows.append({"p_plus": pp, "ms_per_step": times[len(times) // 2], "balanced": counts[0],
                     "unbalanced": counts[1], "balanced_fraction": counts[0] / max(1, counts[0] + counts[1]),
                     "wedges": wedges})
    ms = [r["ms_per_step"] for r in rows]
    total = {r["balanced"] + r["unbalanced"] for r in rows}
    line = {"metric": METRIC, "value": world * rows[2]["wedges"] / (rows[2]["ms_per_step"] / 1e3) / 1e9,
            "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "ms_per_step": rows[2]["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": "sign-sweep", "topology": "chunglu-1m-200k-20m", "tuning": dbbc.dbbc_get_tuning()},
            "sweep": rows, "time_spread": (max(ms) - min(ms)) / min(ms),
            "unsigned_count_constant": len(total) == 1, "e2e": None, "roofline": None, "gpu_launches": None}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_tips(a, torch, dbbc, world, rank, local, dist, barrier):
    """Per-vertex ("tip") and per-edge ("wing") butterfly counts of the
    Chung-Lu 1M x 200k x 20M graph, built once: one step is one
    dbbc_count_vertices call (host output arrays) and one dbbc_count_edges
    call over every distinct edge (device queries and outputs). Both walk every
    accepted wedge twice (count, then credit)."""
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    g = synth.workload("chunglu-1m-200k-20m")
    pairs = np.unique(g.u.astype(np.int64) * g.n_v + g.v)
    qu = torch.from_numpy((pairs // g.n_v).astype(np.int32)).to(dev)
    qv = torch.from_numpy((pairs % g.n_v).astype(np.int32)).to(dev)
    du, dv, ds = (torch.from_numpy(x).to(dev) for x in (g.u, g.v, g.s))
    want = expected_counts("chunglu-1m-200k-20m")
    h = dbbc.dbbc_graph_from_coo(du, dv, ds, g.n_u, g.n_v, stream=stream)
    wedges = h.info["wedges"]
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    tv, te = [], []
    launches0 = 0
    sampler = ClockSampler(local)
    for k in range(a.warmup + a.steps):
        if k == a.warmup:
            barrier()
            torch.cuda.synchronize(dev)
            sampler.start()
            time.sleep(0.3)
            launches0 = dbbc.dbbc_kernel_launches()
        ev[0].record(stream)
        vb, vu = dbbc.dbbc_count_vertices(h, stream)
        ev[1].record(stream)
        eb, eu = dbbc.dbbc_count_edges(h, qu, qv, stream)
        ev[2].record(stream)
        torch.cuda.synchronize(dev)
        if k >= a.warmup:
            tv.append(ev[0].elapsed_time(ev[1]))
            te.append(ev[1].elapsed_time(ev[2]))
    launches = dbbc.dbbc_kernel_launches() - launches0
    clocks = sampler.stop()
    sums = (int(vb.sum(dtype=np.uint64)), int(vu.sum(dtype=np.uint64)), int(eb.sum().item()), int(eu.sum().item()))
    h.free()
    verified = None if want is None else sums == (4 * want[0], 4 * want[1], 4 * want[0], 4 * want[1])
    ms_v, ms_e = sum(tv) / len(tv), sum(te) / len(te)
    line = {"metric": METRIC, "value": world * wedges / (ms_v / 1e3) / 1e9, "unit": UNIT, "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms_v + ms_e, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": "tips", "graph": "chunglu-1m-200k-20m", "wedges": wedges,
                       "edge_queries": int(pairs.shape[0]), "tuning": dbbc.dbbc_get_tuning(),
                       "l2": "inputs larger than L2 (CSR %.0f MB > 129 MB)" % ((2 * g.m * 4 + (g.n_u + g.n_v) * 8) / 1e6)},
            "per_vertex": {"ms": ms_v, "gwedges_per_s": wedges / (ms_v / 1e3) / 1e9,
                           "output": "host arrays, 2 x 8 B per vertex"},
            "per_edge": {"ms": ms_e, "gwedges_per_s": wedges / (ms_e / 1e3) / 1e9,
                         "output": "device arrays, 2 x 8 B per queried edge"},
            "verified": verified, "e2e": None, "roofline": None, "gpu_launches": int(launches), "clocks": clocks}
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        import oracle
        gs = synth.workload("chunglu-1m-200k-20m", scale=0.05)
        w = oracle.count(gs.u, gs.v, gs.s, gs.n_u, gs.n_v, threads=1)[2]
        t0 = time.perf_counter()
        oracle.count_per_vertex(gs.u, gs.v, gs.s, gs.n_u, gs.n_v)
        t = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": w / t / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"oracle per-vertex counts of the 5% Chung-Lu graph ({w} wedges, {t:.1f} s, "
                                          "1 thread)"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
        return
    import torch
    import paper_2609_21848_gb300 as dbbc

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    # the autotuner's record for this workload on this GPU, if there is one
    from paper_2609_21848_gb300 import autotune
    dbbc.lib()
    tuned = autotune.apply_saved({"serve": "batch-4096", "sign-sweep": "chunglu-1m-200k-20m",
                                  "tips": "chunglu-1m-200k-20m"}.get(a.workload, a.workload))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    if a.workload in ("batch-4096", "serve", "sign-sweep", "tips"):
        fn = {"batch-4096": run_batch, "serve": run_serve, "sign-sweep": run_sign_sweep, "tips": run_tips}[a.workload]
        fn(a, torch, dbbc, world, rank, local, dist, barrier)
        if dist is not None:
            dist.destroy_process_group()
        return

    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    g = synth.workload(a.workload, scale=a.scale) if a.scale != 1.0 else synth.workload(a.workload)
    du, dv, ds = (torch.from_numpy(x).to(dev) for x in (g.u, g.v, g.s))
    torch.cuda.synchronize(dev)

    eb0, eb1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    partition = a.partition and world > 1

    def step(prof_acc=None):
        eb0.record(stream)
        h = dbbc.dbbc_graph_from_coo(du, dv, ds, g.n_u, g.n_v, stream=stream)
        eb1.record(stream)
        if partition:
            bal, unb = dbbc.dbbc_count_partition(h, rank, world, stream=stream)
            prof = {}
        else:
            bal, unb, prof = dbbc.dbbc_count_profiled(h, stream=stream)
        info = h.info
        h.free()
        if prof_acc is not None:
            for k, val in prof.items():
                prof_acc[k] = prof_acc.get(k, 0) + val
            prof_acc["ms_build"] = prof_acc.get("ms_build", 0.0) + eb0.elapsed_time(eb1)
        return bal, unb, info

    for _ in range(a.warmup):
        bal, unb, info = step()
    if partition:  # the parts' 16-byte results add up to the graph's counts
        t = torch.tensor([bal, unb], dtype=torch.int64, device=dev)
        dist.all_reduce(t)
        bal, unb = (int(x) for x in t.tolist())
    want = expected_counts(a.workload) if a.scale == 1.0 else None
    verified = None if want is None else ((bal, unb, info["wedges"]) == want)

    sampler = ClockSampler(local)
    prof = {}
    barrier()
    torch.cuda.synchronize(dev)
    sampler.start()
    time.sleep(0.3)
    launches0 = dbbc.dbbc_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        step(prof)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    launches = dbbc.dbbc_kernel_launches() - launches0
    clocks = sampler.stop()
    barrier()
    t_ms = torch.tensor([e0.elapsed_time(e1)], dtype=torch.float64, device=dev)
    if dist is not None:
        dist.all_reduce(t_ms, op=dist.ReduceOp.MAX)
    t_ms = float(t_ms.item())
    wedges = info["wedges"]
    value = (1 if partition else world) * wedges * a.steps / (t_ms / 1e3) / 1e9

    # end to end through the public API with host buffers (pinned), H2D + D2H inside
    e2e_steps = min(a.steps, 5) if a.e2e_steps is None else a.e2e_steps
    e2e = None
    if e2e_steps > 0:
        hu, hv, hs = (torch.from_numpy(x).pin_memory() for x in (g.u, g.v, g.s))
        barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            if partition:
                with dbbc.dbbc_graph_from_coo(hu, hv, hs, g.n_u, g.n_v, stream=stream) as he:
                    r = dbbc.dbbc_count_partition(he, rank, world, stream=stream)
            else:
                r = dbbc.count_coo(hu, hv, hs, g.n_u, g.n_v, stream=stream)
        torch.cuda.synchronize(dev)
        t_e2e = torch.tensor([time.perf_counter() - t0], dtype=torch.float64, device=dev)
        if dist is not None:
            dist.all_reduce(t_e2e, op=dist.ReduceOp.MAX)
        if partition:
            t = torch.tensor(list(r), dtype=torch.int64, device=dev)
            dist.all_reduce(t)
            r = tuple(int(x) for x in t.tolist())
        e2e = {"value": (1 if partition else world) * wedges * e2e_steps / float(t_e2e.item()) / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": 9 * g.m, "d2h_bytes_per_step": 16, "steps": e2e_steps,
               "bit_exact": r == (bal, unb)}

    # roofline of the dominant kernel (hub window sweep), from the live events
    peaks, peak_kind = measured_peaks()
    n_agg = max(1, int(prof.get("launches_hub_aggregate", 0)))
    agg_s = prof.get("ms_hub_aggregate", 0.0) / 1e3
    list_visits = prof.get("hub_list_visits", 0) / max(1, a.steps)
    bytes_hub_step = B_WEDGE * info["wedges_hub"] + B_LOWER * info["lower_hub"]
    overhead_hub_step = (B_CUR_INIT * info["hub_cursor_inits"] + B_CUR_STEP * info["hub_cursor_steps"]
                         + B_LIST_VISIT * list_visits)
    per_launch_bytes = bytes_hub_step * a.steps / n_agg
    per_launch_s = agg_s / n_agg
    achieved = per_launch_bytes / per_launch_s / 1e9 if per_launch_s > 0 else None
    peak = float(peaks["hbm_gbs"])
    roofline = {"bound": "hbm", "kernel": "hub_sweep_kernel", "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": (achieved / peak) if achieved else None,
                "traffic": known_traffic("hub_sweep_kernel", a.workload) if a.scale == 1.0 else None,
                "peak_kind": f"of {peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                "bytes_per_launch": per_launch_bytes,
                "bytes_model": "method terms: 4 B per accepted hub wedge + 28 B per hub lower-neighbour step",
                "design_overhead_bytes_per_launch": overhead_hub_step * a.steps / n_agg,
                "list_visits_per_launch": list_visits * a.steps / n_agg,
                "launches_per_step": n_agg / a.steps,
                "ms_per_launch": 1e3 * per_launch_s,
                "wedges_per_s_in_kernel": info["wedges_hub"] * a.steps / agg_s if agg_s > 0 else None}
    tiers_ms = {k: prof.get(k, 0.0) / a.steps for k in ("ms_build", "ms_light", "ms_medium", "ms_hub_aggregate",
                                                         "ms_total")}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": t_ms / a.steps, "higher_is_better": True,
            "scaling": "strong" if partition else "weak", "vs_baseline": None,
            "dtype": "int64", "data": "synthetic",
            "config": {"workload": a.workload, "scale": a.scale, "n_u": g.n_u, "n_v": g.n_v, "edges": g.m,
                       "tuning": dbbc.dbbc_get_tuning(),
                       "wedges_per_step": wedges,
                       "parallelism": (f"LPT pivot partition x{world}" if partition else f"replicas x{world}")
                       if world > 1 else "1 GPU",
                       "l2": "inputs larger than L2 (COO %.0f MB, CSR %.0f MB > 129 MB)" % (
                           g.m * 9 / 1e6, (2 * g.m * 4 + (g.n_u + g.n_v) * 8) / 1e6)},
            "verified": verified, "counts": {"balanced": bal, "unbalanced": unb},
            "count_ms_per_step": tiers_ms,
            "count_only_gwedges_per_s": wedges / (tiers_ms["ms_total"] / 1e3) / 1e9 if tiers_ms["ms_total"] else None,
            "e2e": e2e,
            "roofline": roofline, "gpu_launches": int(launches), "clocks": clocks}
    # the other half of the metric, on the same GPU after the timed region:
    # graphs/s of the batched (one replayed plan over 4,096 graphs) and served
    # (Poisson stream, continuous batching) forms against one launch per graph
    if a.workload == DEFAULT_WORKLOAD and a.scale == 1.0 and not a.no_extras:
        if world == 1:
            del du, dv, ds
            torch.cuda.synchronize(dev)
            autotune.apply_saved("batch-4096")
            small = synth.batch(a.n_graphs)
            b = batch_record(a, torch, dbbc, world, rank, local, dist, barrier, graphs=small, with_cpu=False)
            line["batch"] = {k: b[k] for k in ("value", "unit", "ms_per_step", "steps", "plain_graphs_per_s",
                                               "batched_over_plain", "bit_exact_vs_plain", "batched_gwedges_per_s",
                                               "union_build_and_count_graphs_per_s", "union_bit_exact", "e2e",
                                               "gpu_launches", "clocks")}
            line["batch"]["config"] = b["config"]
            s = serve_record(a, torch, dbbc, world, rank, local, dist, barrier, small=small)
            line["serve"] = {k: s[k] for k in ("value", "unit", "served_at_rate", "saturated", "plain_graphs_per_s",
                                               "served_over_plain", "bit_exact_vs_alone", "e2e", "gpu_launches",
                                               "clocks")}
            line["serve"]["config"] = s["config"]
            autotune.apply_saved(a.workload)
        else:
            line["batch"] = line["serve"] = {"skipped": "with N > 1 every rank counts a replica of the single "
                                                        "graph only; the batched and served forms run at N = 1"}
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(g, a.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
