"""Failure paths of the C ABI, injected on the host (no GPU fault is made).

A test allocator, installed with dbbc_set_allocator, hands the library's
device allocations to torch's caching allocator and returns NULL from its
k-th call. Every allocation of a call is failed in turn, and each time:

* the call returns DBBC_ENOMEM;
* its output parameters are left untouched (the ABI's error convention);
* every allocation it made has been released again (nothing leaks);
* the next call on the same device succeeds and equals the oracle.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth
import paper_2609_21848_gb300 as dbbc

pytestmark = pytest.mark.gpu

SENTINEL = 0x5EED5EED5EED5EED


class FailingAllocator:
    """Device allocations through torch's caching allocator; the allocation
    with index `fail_at` (counted from installation) returns NULL."""

    def __init__(self):
        import torch
        self.torch = torch
        self.calls = 0
        self.fail_at = None
        self.live = {}
        self._refs = (dbbc._ALLOC_FN(self._alloc), dbbc._FREE_FN(self._free))

    def _alloc(self, size, stream, ctx):
        i = self.calls
        self.calls += 1
        if self.fail_at is not None and i == self.fail_at:
            return None
        p = self.torch.cuda.caching_allocator_alloc(int(size), self.torch.cuda.current_device(), int(stream or 0))
        self.live[int(p)] = int(size)
        return p

    def _free(self, ptr, stream, ctx):
        self.live.pop(int(ptr), None)
        self.torch.cuda.caching_allocator_delete(int(ptr))

    def __enter__(self):
        dbbc.lib().dbbc_set_allocator(ctypes.cast(self._refs[0], ctypes.c_void_p),
                                      ctypes.cast(self._refs[1], ctypes.c_void_p), None)
        return self

    def __exit__(self, *exc):
        self.torch.cuda.synchronize()
        dbbc.lib().dbbc_set_allocator(None, None, None)


def _graph():
    """A graph with light, medium and hub pivots, hub items in list mode."""
    g = synth.workload("chunglu-1m-200k-20m", scale=0.005)
    return g, oracle.count(g.u, g.v, g.s, g.n_u, g.n_v)


@pytest.fixture
def sparse_hubs():
    base = dbbc.dbbc_get_tuning()
    dbbc.dbbc_set_tuning({"list_density": 1e9, "light_max_work": 64, "medium_max_work": 512})
    yield
    dbbc.dbbc_set_tuning(base)


def _build_raw(g, stream):
    out = ctypes.c_void_p(SENTINEL)
    st = dbbc.lib().dbbc_graph_from_coo(g.u.ctypes.data, g.v.ctypes.data, g.s.ctypes.data, g.m, g.n_u, g.n_v, 0,
                                        stream, ctypes.byref(out))
    return st, out.value


def _sweep(alloc, call, check_untouched, reset=lambda: None):
    """Run `call` once to count its allocations, then fail each in turn
    (`reset` puts the output parameters back to their sentinels first)."""
    torch = alloc.torch
    before = dict(alloc.live)
    c0 = alloc.calls
    assert call() == dbbc.DBBC_OK
    n = alloc.calls - c0
    assert n > 0
    torch.cuda.synchronize()
    for k in range(n):
        reset()
        live0 = dict(alloc.live)
        alloc.fail_at = alloc.calls + k
        st = call()
        alloc.fail_at = None
        torch.cuda.synchronize()
        assert st == dbbc.DBBC_ENOMEM, (k, st)
        check_untouched()
        assert alloc.live == live0, f"allocation {k} of {n}: {len(alloc.live) - len(live0)} leaked"
    return n, before


def test_build_fails_cleanly_on_every_allocation(sparse_hubs):
    import torch
    g, want = _graph()
    stream = torch.cuda.current_stream().cuda_stream
    with FailingAllocator() as alloc:
        handles = []

        def call():
            st, h = _build_raw(g, stream)
            if st == dbbc.DBBC_OK:
                handles.append(h)
            else:
                assert h == SENTINEL  # *out untouched
            return st

        _sweep(alloc, call, lambda: None)
        for h in handles:
            dbbc.lib().dbbc_graph_free(h)
    with dbbc.dbbc_graph_from_coo(g.u, g.v, g.s, g.n_u, g.n_v) as h:
        assert dbbc.dbbc_count(h) + (h.info["wedges"],) == want


def test_count_fails_cleanly_on_every_allocation(sparse_hubs):
    import torch
    g, want = _graph()
    stream = torch.cuda.current_stream().cuda_stream
    with dbbc.dbbc_graph_from_coo(g.u, g.v, g.s, g.n_u, g.n_v) as h:
        assert h.info["n_hub"] > 0
        out = (ctypes.c_uint64 * 2)(SENTINEL, SENTINEL)
        base = ctypes.addressof(out)

        def call():
            return dbbc.lib().dbbc_count(h.handle, stream, base, base + 8)

        def untouched():
            assert list(out) == [SENTINEL, SENTINEL]

        def reset():
            out[0] = out[1] = SENTINEL

        with FailingAllocator() as alloc:
            n, _ = _sweep(alloc, call, untouched, reset)
        assert n >= 3  # status word, output pair, hub cursors / lists at least
        assert dbbc.dbbc_count(h) == want[:2]  # the same handle counts correctly afterwards


def test_count_vertices_fails_cleanly_on_every_allocation(sparse_hubs):
    import torch
    g, _ = _graph()
    stream = torch.cuda.current_stream().cuda_stream
    want_b, want_u = oracle.count_per_vertex(g.u, g.v, g.s, g.n_u, g.n_v)
    with dbbc.dbbc_graph_from_coo(g.u, g.v, g.s, g.n_u, g.n_v) as h:
        n = g.n_u + g.n_v
        vb = np.full(n, SENTINEL, np.uint64)
        vu = np.full(n, SENTINEL, np.uint64)

        def call():
            return dbbc.lib().dbbc_count_vertices(h.handle, stream, vb.ctypes.data, vu.ctypes.data)

        def untouched():
            assert np.all(vb == SENTINEL) and np.all(vu == SENTINEL)

        with FailingAllocator() as alloc:
            # the sweep's first, successful call writes the arrays: reset them
            assert call() == dbbc.DBBC_OK
            vb[:] = SENTINEL
            vu[:] = SENTINEL
            c0 = alloc.calls
            assert call() == dbbc.DBBC_OK
            n_alloc = alloc.calls - c0
            vb[:] = SENTINEL
            vu[:] = SENTINEL
            for k in range(n_alloc):
                live0 = dict(alloc.live)
                alloc.fail_at = alloc.calls + k
                st = call()
                alloc.fail_at = None
                torch.cuda.synchronize()
                assert st == dbbc.DBBC_ENOMEM, (k, st)
                untouched()
                assert alloc.live == live0
        gb, gu = dbbc.dbbc_count_vertices(h)
        assert np.array_equal(gb, want_b) and np.array_equal(gu, want_u)


def test_batch_plan_fails_cleanly_on_every_allocation(sparse_hubs):
    import torch
    graphs = [synth.batch_graph(i) for i in range(6)]
    want = [oracle.count(x.u, x.v, x.s, x.n_u, x.n_v)[:2] for x in graphs]
    stream = torch.cuda.current_stream().cuda_stream
    handles = [dbbc.dbbc_graph_from_coo(x.u, x.v, x.s, x.n_u, x.n_v) for x in graphs]
    try:
        arr = (ctypes.c_void_p * len(handles))(*[h.handle for h in handles])
        plans = []

        def call():
            out = ctypes.c_void_p(SENTINEL)
            st = dbbc.lib().dbbc_batch_create(arr, len(handles), stream, ctypes.byref(out))
            if st == dbbc.DBBC_OK:
                plans.append(out.value)
            else:
                assert out.value == SENTINEL
            return st

        with FailingAllocator() as alloc:
            _sweep(alloc, call, lambda: None)
            for p in plans:
                dbbc.lib().dbbc_batch_free(p)
        b, u = dbbc.dbbc_count_batch(handles)
        assert list(zip(b.tolist(), u.tolist())) == want
    finally:
        for h in handles:
            h.free()
