"""Continuous-batching request loop for butterfly counting on one GPU.

Requests (a signed bipartite COO graph each) arrive over time. The loop:

* **admits** requests in arrival order while the device bytes they will need
  (``dbbc_estimate_bytes`` up front, the built handle's bytes afterwards) fit
  under a budget taken from the free HBM at start-up;
* **builds** admitted graphs on builder threads, each on its own CUDA stream,
  and keeps them resident until they are counted. A builder admits every small
  request that has arrived (while it fits) as one group and builds the group's
  disjoint union with one call (``dbbc_graph_from_coo_multi``); a large
  request is built alone;
* **counts** in lanes on their own streams: a batch lane counts one group at a
  time, per component (``dbbc_count_components``), and large lanes count big
  graphs one by one each, so a large request never holds up the small ones
  behind it;
* **completes** a request when its counts are on the host, frees its graph
  (returning its bytes to the budget), and records its latency from arrival.

Requests that arrive while others are on the GPU are admitted as memory frees
up, and their builds and counts overlap the work already running. The loop is
written against a small backend interface so that the scheduling can be tested
without a GPU (see ``tests/test_serve.py``); :class:`DbbcBackend` is the CUDA
one, calling the C ABI through this package's binding.
"""
from __future__ import annotations

import threading
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    u: object
    v: object
    s: object
    n_u: int
    n_v: int
    arrival: float = 0.0  # seconds from the start of the stream

    @property
    def m(self) -> int:
        return int(len(self.u))


@dataclass
class Result:
    rid: int
    balanced: int
    unbalanced: int
    arrival: float
    admitted: float
    built: float
    done: float
    large: bool

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclass
class ServeStats:
    results: list = field(default_factory=list)
    wall_s: float = 0.0
    batches: int = 0
    max_in_flight_bytes: int = 0

    def summary(self) -> dict:
        lat = np.array([r.latency for r in self.results]) if self.results else np.zeros(1)
        return {"requests": len(self.results), "wall_s": self.wall_s,
                "graphs_per_s": len(self.results) / self.wall_s if self.wall_s > 0 else 0.0,
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "max_ms": float(lat.max() * 1e3), "batches": self.batches,
                "max_in_flight_bytes": self.max_in_flight_bytes}


class DbbcBackend:
    """The CUDA backend: builds from host COO on a builder's stream and counts
    batches / large graphs on the lanes' streams."""

    def __init__(self, device: int = 0):
        import torch

        from . import dbbc_count, dbbc_count_components, dbbc_estimate_bytes, dbbc_graph_device_bytes, \
            dbbc_graph_from_coo, dbbc_graph_from_coo_multi
        self.torch = torch
        self.device = device
        torch.cuda.set_device(device)
        self._from_coo = dbbc_graph_from_coo
        self._count = dbbc_count
        self._from_coo_multi = dbbc_graph_from_coo_multi
        self._count_components = dbbc_count_components
        self._est = dbbc_estimate_bytes
        self._bytes = dbbc_graph_device_bytes
        self._streams = {}
        self._stages = {}
        self._lock = threading.Lock()

    def _stream(self, key):
        with self._lock:
            if key not in self._streams:
                self._streams[key] = self.torch.cuda.Stream(device=self.device)
            return self._streams[key]

    def free_memory(self) -> int:
        return int(self.torch.cuda.mem_get_info(self.device)[0])

    def estimate_bytes(self, req: Request) -> int:
        return self._est(req.m, req.n_u, req.n_v)

    def build(self, req: Request, lane: str):
        self.torch.cuda.set_device(self.device)
        return self._from_coo(req.u, req.v, req.s, req.n_u, req.n_v, stream=self._stream(lane))

    def device_bytes(self, handle) -> int:
        return self._bytes(handle)

    def build_many(self, reqs, lane: str):
        """One union handle for a group of requests (host COO gathered into a
        pinned staging buffer of this builder, then one build)."""
        torch = self.torch
        torch.cuda.set_device(self.device)
        parts = [[torch.as_tensor(getattr(r, k)) for r in reqs] for k in ("u", "v", "s")]
        total = sum(r.m for r in reqs)
        with self._lock:
            stage = self._stages.get(lane)
            if stage is None or stage[0].numel() < total:
                cap = max(total, 1 << 20)
                stage = (torch.empty(cap, dtype=torch.int32).pin_memory(),
                         torch.empty(cap, dtype=torch.int32).pin_memory(),
                         torch.empty(cap, dtype=torch.int8).pin_memory())
                self._stages[lane] = stage
        bu, bv, bs = (x[:total] for x in stage)
        if total:
            torch.cat(parts[0], out=bu)
            torch.cat(parts[1], out=bv)
            torch.cat(parts[2], out=bs)
        offs = np.zeros(len(reqs) + 1, np.int64)
        offs[1:] = np.cumsum([r.m for r in reqs])
        return self._from_coo_multi(bu, bv, bs, offs, [r.n_u for r in reqs], [r.n_v for r in reqs],
                                    stream=self._stream(lane))

    def count_components(self, handle, lane: str):
        self.torch.cuda.set_device(self.device)
        bal, unb = self._count_components(handle, stream=self._stream(lane))
        return list(zip(bal.tolist(), unb.tolist()))

    def count_one(self, handle, lane: str):
        self.torch.cuda.set_device(self.device)
        return self._count(handle, stream=self._stream(lane))

    def free(self, handle):
        handle.free()


class Server:
    """Continuous batching over a backend (see the module docstring)."""

    def __init__(self, backend, memory_budget: int | None = None, reserve_bytes: int = 2 << 30,
                 large_edges: int = 1_000_000, max_batch: int = 4096, max_group_edges: int = 1 << 26,
                 builders: int = 3, large_lanes: int = 2):
        self.backend = backend
        free = backend.free_memory()
        self.budget = int(memory_budget if memory_budget is not None else max(0, free - reserve_bytes))
        self.large_edges = large_edges
        self.max_batch = max_batch
        self.max_group_edges = max_group_edges
        self.n_builders = builders
        self.n_large_lanes = large_lanes
        self._cv = threading.Condition()
        self._arrived = deque()       # requests not yet admitted
        self._ready_small = deque()   # (group of requests, union handle, bytes, t_admit, t_built)
        self._ready_large = deque()   # ([request], handle, bytes, t_admit, t_built)
        self._in_flight = 0
        self._closed = False          # no more arrivals
        self._pending_builds = 0
        self._small_building = 0      # small groups being built
        self.stats = ServeStats()
        self._t0 = 0.0
        self._errors = []

    # ------------------------------------------------------------ arrivals
    def _now(self) -> float:
        return time.perf_counter() - self._t0

    def _feed(self, requests):
        for req in sorted(requests, key=lambda r: r.arrival):
            if self._errors:
                break
            delay = req.arrival - self._now()
            if delay > 0:
                time.sleep(delay)
            with self._cv:
                self._arrived.append(req)
                self._cv.notify_all()
        with self._cv:
            self._closed = True
            self._cv.notify_all()

    # ------------------------------------------------------------ admission + build
    def _admit(self):
        """Under the lock: pop the next admissible unit of work (a large request
        alone, or the run of small requests at the head of the arrivals that
        fits), or return None."""
        if not self._arrived:
            return None
        head = self._arrived[0]
        small = head.m < self.large_edges
        # continuous batching: while a small group is being built or waits for
        # the batch lane, later small requests keep accumulating into the next
        # group instead of forming many tiny ones
        if small and (self._small_building or self._ready_small):
            return None
        need = self.backend.estimate_bytes(head)
        # an empty device always admits (a request larger than the budget runs alone)
        if self._in_flight + need > self.budget and self._in_flight != 0:
            return None
        group = [self._arrived.popleft()]
        if small:
            self._small_building += 1
            edges = head.m
            while (self._arrived and self._arrived[0].m < self.large_edges and len(group) < self.max_batch
                   and edges + self._arrived[0].m <= self.max_group_edges):
                nxt = self.backend.estimate_bytes(self._arrived[0])
                if self._in_flight + need + nxt > self.budget:
                    break
                need += nxt
                edges += self._arrived[0].m
                group.append(self._arrived.popleft())
        self._in_flight += need
        self._pending_builds += 1
        self.stats.max_in_flight_bytes = max(self.stats.max_in_flight_bytes, self._in_flight)
        return group, need

    def _builder(self, idx: int):
        lane = f"build{idx}"
        while True:
            with self._cv:
                while True:
                    if self._errors:
                        return
                    unit = self._admit()
                    if unit is not None:
                        break
                    if self._closed and not self._arrived:
                        return
                    self._cv.wait()
            group, need = unit
            large = group[0].m >= self.large_edges
            t_admit = self._now()
            try:
                h = self.backend.build(group[0], lane) if large else self.backend.build_many(group, lane)
                nbytes = self.backend.device_bytes(h)
            except Exception as e:  # surfaced to the caller by run()
                with self._cv:
                    self._errors.append(e)
                    self._cv.notify_all()
                return
            t_built = self._now()
            with self._cv:
                self._in_flight += nbytes - need
                self._pending_builds -= 1
                if not large:
                    self._small_building -= 1
                (self._ready_large if large else self._ready_small).append((group, h, nbytes, t_admit, t_built))
                self._cv.notify_all()

    # ------------------------------------------------------------ counting lanes
    def _drained(self) -> bool:
        return self._closed and not self._arrived and self._pending_builds == 0

    def _lane(self, large: bool, idx: int = 0):
        lane = f"large{idx}" if large else "batch"
        ready = self._ready_large if large else self._ready_small
        while True:
            with self._cv:
                while not ready:
                    if self._errors or self._drained():
                        return
                    self._cv.wait()
                group, h, nbytes, t_admit, t_built = ready.popleft()
            try:
                if large:
                    counts = [self.backend.count_one(h, lane)]
                else:
                    counts = self.backend.count_components(h, lane)
                t_done = self._now()
                done = [Result(req.rid, int(bal), int(unb), req.arrival, t_admit, t_built, t_done, large)
                        for req, (bal, unb) in zip(group, counts)]
                self.backend.free(h)
            except Exception as e:  # surfaced to the caller by run()
                with self._cv:
                    self._errors.append(e)
                    self._cv.notify_all()
                return
            with self._cv:
                self.stats.results.extend(done)
                self._in_flight -= nbytes
                self.stats.batches += 1
                self._cv.notify_all()

    # ------------------------------------------------------------ driver
    def run(self, requests) -> ServeStats:
        """Serve `requests` (their .arrival fields are seconds from now) and
        return per-request results and timings."""
        self._t0 = time.perf_counter()
        threads = [threading.Thread(target=self._feed, args=(list(requests),), daemon=True)]
        threads += [threading.Thread(target=self._builder, args=(i,), daemon=True) for i in range(self.n_builders)]
        threads += [threading.Thread(target=self._lane, args=(False,), daemon=True)]
        threads += [threading.Thread(target=self._lane, args=(True, i), daemon=True)
                    for i in range(max(1, self.n_large_lanes))]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        self.stats.wall_s = self._now()
        if self._errors:
            raise self._errors[0]
        self.stats.results.sort(key=lambda r: r.rid)
        return self.stats


def poisson_arrivals(n: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times (seconds) of a Poisson stream of n requests at `rate`/s."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))
