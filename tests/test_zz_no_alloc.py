"""dbbc_count_noalloc, the entry point for callers that cannot allocate device
memory while counting (a fixed memory budget owned by another allocator, no
allocator calls while other work is captured into CUDA graphs). It takes its
scratch from a fixed array inside the library, so its results must equal
those of dbbc_count_async on the same graph, call after call, even though
every call reuses the same scratch. This file is collected last so that a run
that stops at the first failure has run every other test before it."""
import ctypes

import numpy as np
import pytest

import synth
import paper_2609_21848_gb300 as dbbc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return torch


@pytest.mark.parametrize("workload,scale", [("chunglu-1m-200k-20m", 0.05), ("uniform-2k-3k-20k", 1.0)])
def test_noalloc_matches_count_async_on_two_calls(torch_cuda, workload, scale):
    torch = torch_cuda
    g = synth.workload(workload, scale=scale)
    with dbbc.dbbc_graph_from_coo(g.u, g.v, g.s, g.n_u, g.n_v) as h:
        want = torch.zeros(2, dtype=torch.int64, device="cuda")
        dbbc.dbbc_count_async(h, want)
        torch.cuda.synchronize()
        for _ in range(2):
            got = torch.full((2,), -1, dtype=torch.int64, device="cuda")
            # through the C ABI directly
            st = dbbc.lib().dbbc_count_noalloc(ctypes.c_void_p(h.handle),
                                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                               ctypes.c_void_p(got.data_ptr()))
            assert st == dbbc.DBBC_OK
            torch.cuda.synchronize()
            assert torch.equal(got, want), (got.tolist(), want.tolist())
        if workload.startswith("chunglu"):
            assert h.info["n_hub"] > 0  # the hub sweep (the scratch user) ran


def test_noalloc_rejects_bad_arguments(torch_cuda):
    assert dbbc.lib().dbbc_count_noalloc(None, None, None) == dbbc.DBBC_EINVAL
