"""dbbc_count_noalloc, the entry point for callers that cannot allocate device
memory while counting (a fixed memory budget owned by another allocator, no
allocator calls while other work is captured into CUDA graphs). It takes its
scratch from a fixed array inside the library, so its results must equal
those of dbbc_count_async on the same graph and the oracle's, call after
call, even though every call reuses the same scratch; and it must not call
the library's allocator at all. This file is collected last so that a run
that stops at the first failure has run every other test before it."""
import ctypes

import numpy as np
import pytest

import oracle
import synth
import paper_2609_21848_gb300 as dbbc

pytestmark = pytest.mark.gpu

# the fixed scratch array (32 MiB) less its 256-byte header, in 8-byte cursors
NOALLOC_CURSORS = ((32 << 20) - 256) // 8


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return torch


class CountingAllocator:
    """Counts the library's device allocations (through torch's allocator)."""

    def __init__(self, torch):
        self.torch = torch
        self.calls = 0
        self._refs = (dbbc._ALLOC_FN(self._alloc), dbbc._FREE_FN(self._free))

    def _alloc(self, size, stream, ctx):
        self.calls += 1
        return self.torch.cuda.caching_allocator_alloc(int(size), self.torch.cuda.current_device(), int(stream or 0))

    def _free(self, ptr, stream, ctx):
        self.torch.cuda.caching_allocator_delete(int(ptr))

    def __enter__(self):
        dbbc.lib().dbbc_set_allocator(ctypes.cast(self._refs[0], ctypes.c_void_p),
                                      ctypes.cast(self._refs[1], ctypes.c_void_p), None)
        return self

    def __exit__(self, *exc):
        self.torch.cuda.synchronize()
        dbbc.lib().dbbc_set_allocator(None, None, None)


def _one_big_hub(n_leaf=50_000, n_other=200, seed=7):
    """U vertex 0 joined to n_leaf V vertices, each also joined to one of
    n_other other U vertices: the hub's lower neighbours (n_leaf of them) need
    more cursor scratch per CTA than the fixed array holds for every CTA, so
    the hub tier runs on fewer CTAs."""
    rng = np.random.default_rng(seed)
    v = np.arange(n_leaf)
    u = np.concatenate([np.zeros(n_leaf, np.int64), 1 + rng.integers(0, n_other, n_leaf)])
    s = np.where(rng.random(2 * n_leaf) < 0.5, 1, -1)
    return synth.Graph(u.astype(np.int32), np.concatenate([v, v]).astype(np.int32), s.astype(np.int8),
                       n_other + 1, n_leaf)


CASES = {
    "chunglu-5pct": lambda: synth.workload("chunglu-1m-200k-20m", scale=0.05),
    "uniform-2k-3k-20k": lambda: synth.workload("uniform-2k-3k-20k"),
    "one-big-hub": _one_big_hub,
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_noalloc_matches_count_async_and_the_oracle_on_two_calls(torch_cuda, case):
    torch = torch_cuda
    g = CASES[case]()
    want = oracle.count(g.u, g.v, g.s, g.n_u, g.n_v, threads=synth.default_threads())[:2]
    with dbbc.dbbc_graph_from_coo(g.u, g.v, g.s, g.n_u, g.n_v) as h:
        ref = torch.zeros(2, dtype=torch.int64, device="cuda")
        dbbc.dbbc_count_async(h, ref)
        torch.cuda.synchronize()
        assert tuple(int(x) for x in ref.cpu().numpy().astype(np.uint64)) == want
        info = h.info
        outs = [torch.full((2,), -1, dtype=torch.int64, device="cuda") for _ in range(2)]
        with CountingAllocator(torch) as alloc:
            for got in outs:  # two calls in a row, through the C ABI directly
                st = dbbc.lib().dbbc_count_noalloc(ctypes.c_void_p(h.handle),
                                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                                   ctypes.c_void_p(got.data_ptr()))
                assert st == dbbc.DBBC_OK
        assert alloc.calls == 0  # the library's allocator was never called
        for got in outs:
            assert torch.equal(got, ref), (got.tolist(), ref.tolist())
    if case != "uniform-2k-3k-20k":
        assert info["n_hub"] > 0  # the hub sweep (the scratch user) ran
    if case == "one-big-hub":
        # the array holds cursors for fewer CTAs than the full grid (152 SMs)
        assert NOALLOC_CURSORS // 50_000 < 152


def test_noalloc_rejects_bad_arguments(torch_cuda):
    assert dbbc.lib().dbbc_count_noalloc(None, None, None) == dbbc.DBBC_EINVAL
