"""The served form on the GPU: a Poisson stream of uneven requests, with a few
large ones on the large lane, served with continuous batching; every result
must equal the count of the same graph alone (and the oracle's for a sample)."""
import os

import pytest

import oracle
import synth
import paper_2609_21848_gb300 as dbbc
from paper_2609_21848_gb300.serve import DbbcBackend, Request, Server, poisson_arrivals

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    dbbc.lib()
    return torch


def test_served_results_equal_alone_results(cuda):
    graphs = [synth.batch_graph(i) for i in range(300)]
    graphs += [synth.workload("chunglu-1m-200k-20m", scale=0.02), synth.workload("polarized-20m-2m-300m", scale=0.002)]
    alone = []
    for g in graphs:
        with dbbc.dbbc_graph_from_coo(g.u, g.v, g.s, g.n_u, g.n_v) as h:
            alone.append(dbbc.dbbc_count(h))
    t = poisson_arrivals(len(graphs), 2000.0, seed=11)
    order = list(range(len(graphs)))
    order.insert(40, order.pop(-1))   # the large ones arrive early, amid small ones
    order.insert(120, order.pop(-1))
    reqs = [Request(k, graphs[i].u, graphs[i].v, graphs[i].s, graphs[i].n_u, graphs[i].n_v, float(t[k]))
            for k, i in enumerate(order)]
    st = Server(DbbcBackend(0), large_edges=300_000).run(reqs)
    assert len(st.results) == len(reqs)
    for r in st.results:
        assert (r.balanced, r.unbalanced) == alone[order[r.rid]], r.rid
    assert sum(r.large for r in st.results) == 2
    assert st.batches < len(reqs)
    nc = max(1, len(os.sched_getaffinity(0)))
    for i in range(0, 300, 15):
        g = graphs[i]
        assert alone[i] == oracle.count(g.u, g.v, g.s, g.n_u, g.n_v, threads=nc)[:2]
