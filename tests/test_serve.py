"""The continuous-batching loop (paper_2609_21848_gb300/serve.py) against a fake
backend on the CPU: every request completes with its own answer, admission
keeps the bytes in flight under the budget, large requests take the large
lane, and requests that arrive while a batch is counting are built meanwhile."""
import threading
import time

import numpy as np
import pytest

from paper_2609_21848_gb300.serve import Request, Server, poisson_arrivals


class FakeHandle:
    def __init__(self, req):
        self.req = req
        self.freed = False


class FakeGroup:
    def __init__(self, handles):
        self.handles = handles


class FakeBackend:
    """Answers are a function of the request id; timings are small sleeps."""

    def __init__(self, free=10_000_000, count_sleep=0.0, fail_build=None):
        self.free_bytes = free
        self.count_sleep = count_sleep
        self.fail_build = fail_build
        self.lock = threading.Lock()
        self.built = []
        self.freed = []
        self.batches = []
        self.in_flight = 0
        self.max_in_flight = 0

    def free_memory(self):
        return self.free_bytes

    def estimate_bytes(self, req):
        return 10 * req.m + 100

    def build(self, req, lane):
        if self.fail_build is not None and req.rid == self.fail_build:
            raise RuntimeError("build failed")
        time.sleep(0.0005)
        with self.lock:
            self.built.append((req.rid, time.perf_counter()))
            self.in_flight += 10 * req.m + 100
            self.max_in_flight = max(self.max_in_flight, self.in_flight)
        return FakeHandle(req)

    def build_many(self, reqs, lane):
        hs = [self.build(r, lane) for r in reqs]
        return FakeGroup(hs)

    def device_bytes(self, h):
        if isinstance(h, FakeGroup):
            return sum(self.device_bytes(x) for x in h.handles)
        return 10 * h.req.m + 100

    def answer(self, req):
        return req.rid * 7 + req.m, req.rid % 5

    def count_components(self, group, lane):
        assert lane == "batch" and isinstance(group, FakeGroup)
        time.sleep(self.count_sleep)
        with self.lock:
            self.batches.append(([h.req.rid for h in group.handles], time.perf_counter()))
        return [self.answer(h.req) for h in group.handles]

    def count_one(self, h, lane):
        assert lane.startswith("large")
        time.sleep(self.count_sleep)
        return self.answer(h.req)

    def free(self, h):
        if isinstance(h, FakeGroup):
            for x in h.handles:
                self.free(x)
            return
        assert not h.freed
        h.freed = True
        with self.lock:
            self.freed.append(h.req.rid)
            self.in_flight -= 10 * h.req.m + 100


def _requests(n, rate=5000.0, seed=1, big_every=0, big_m=5000):
    t = poisson_arrivals(n, rate, seed)
    reqs = []
    for i in range(n):
        m = big_m if big_every and i % big_every == 0 else 10 + (i * 37) % 200
        z = np.zeros(m, np.int32)
        reqs.append(Request(i, z, z, z.astype(np.int8), 10, 10, float(t[i])))
    return reqs


def test_every_request_gets_its_own_answer():
    be = FakeBackend()
    reqs = _requests(300)
    st = Server(be, memory_budget=1_000_000, large_edges=1000).run(reqs)
    assert [r.rid for r in st.results] == list(range(300))
    for r, q in zip(st.results, reqs):
        assert (r.balanced, r.unbalanced) == be.answer(q)
        assert r.done >= r.built >= r.admitted >= 0 and r.latency >= 0
    assert sorted(be.freed) == list(range(300))
    s = st.summary()
    assert s["requests"] == 300 and s["p99_ms"] >= s["p50_ms"] > 0


def test_admission_keeps_bytes_under_budget():
    be = FakeBackend()
    reqs = _requests(200, rate=1e6)  # all at once
    budget = 5000
    st = Server(be, memory_budget=budget, large_edges=10**9).run(reqs)
    assert len(st.results) == 200
    assert st.max_in_flight_bytes <= budget
    assert be.max_in_flight <= budget


def test_oversized_request_runs_alone():
    be = FakeBackend()
    reqs = _requests(20, rate=1e6, big_every=7, big_m=50_000)
    st = Server(be, memory_budget=3000, large_edges=10**9).run(reqs)
    assert len(st.results) == 20


def test_large_requests_take_the_large_lane():
    be = FakeBackend()
    reqs = _requests(100, big_every=10, big_m=3000)
    st = Server(be, memory_budget=10_000_000, large_edges=1000).run(reqs)
    large = {r.rid for r in st.results if r.large}
    assert large == {i for i in range(100) if i % 10 == 0}
    assert all(rid not in large for ids, _ in be.batches for rid in ids)


def test_arrivals_during_a_count_are_built_meanwhile_and_batched():
    be = FakeBackend(count_sleep=0.05)
    reqs = _requests(400, rate=4000.0)
    st = Server(be, memory_budget=10_000_000, large_edges=10**9).run(reqs)
    assert len(st.results) == 400
    # far fewer batches than requests: requests that arrived during a count
    # were admitted, built and then counted together
    assert len(be.batches) < 60
    # some request was built while an earlier batch was still counting
    built_at = dict(be.built)
    first_ids, first_done = be.batches[0]
    later = [rid for rid, t in built_at.items() if rid not in first_ids and t < first_done]
    assert later


def test_build_error_is_raised():
    be = FakeBackend(fail_build=5)
    with pytest.raises(RuntimeError, match="build failed"):
        Server(be, memory_budget=10_000_000).run(_requests(50))


def test_poisson_arrivals_rate():
    t = poisson_arrivals(20_000, 2000.0, seed=3)
    assert np.all(np.diff(t) > 0)
    assert abs(20_000 / t[-1] - 2000.0) < 60
