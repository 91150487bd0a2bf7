"""Pivot partitioning for several GPUs (Phase 3 greedy bin packing): the
library's LPT against the oracle's and the paper's Example 2, and a two-rank
gloo run on the CPU in which each rank sums the oracle's per-pivot counts of
its LPT share and one all-reduce recovers the graph's totals."""
import os

import numpy as np
import pytest

import oracle
import synth
import paper_2609_21848_gb300 as dbbc
from conftest import read_golden


@pytest.fixture(scope="module", autouse=True)
def _lib():
    dbbc.build()
    dbbc.lib()


def test_lpt_example2():
    g = read_golden("phase3_examples.txt")
    work = g["example2_work"][0]
    part, loads = dbbc.dbbc_lpt_partition(work, g["example2_bins"][0][0])
    assert sorted(loads.tolist(), reverse=True) == g["example2_greedy_loads"][0]
    assert max(loads) / min(loads) == pytest.approx(19 / 16)


@pytest.mark.parametrize("seed", range(5))
def test_lpt_matches_oracle(seed):
    rng = np.random.default_rng(seed)
    work = rng.integers(0, 10**6, size=int(rng.integers(1, 3000)), dtype=np.uint64)
    for parts in (1, 2, 3, 7, 16):
        a_part, a_loads = dbbc.dbbc_lpt_partition(work, parts)
        b_part, b_loads = oracle.lpt(work, parts)
        assert np.array_equal(a_part, b_part) and np.array_equal(a_loads, b_loads)
        assert int(a_loads.sum()) == int(work.sum())


def test_lpt_rejects_bad_arguments():
    with pytest.raises(dbbc.DbbcError):
        dbbc.dbbc_lpt_partition([1, 2, 3], 0)


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import torch
    g = synth.workload("chunglu-1m-200k-20m", scale=0.004)
    bal, unb, wed = oracle.count_per_pivot(g.u, g.v, g.s, g.n_u, g.n_v)
    piv = np.nonzero(wed)[0]
    part, loads = dbbc.dbbc_lpt_partition(wed[piv], world)
    mine = piv[part == rank]
    t = torch.tensor([int(bal[mine].sum()), int(unb[mine].sum()), int(wed[mine].sum())], dtype=torch.int64)
    dist.all_reduce(t)
    q.put((rank, t.tolist(), int(loads.max()), int(loads.min())))
    dist.destroy_process_group()


def test_two_rank_partition_sums_to_total():
    import multiprocessing as mp
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    g = synth.workload("chunglu-1m-200k-20m", scale=0.004)
    want = list(oracle.count(g.u, g.v, g.s, g.n_u, g.n_v))
    for rank, tot, hi, lo in out:
        assert tot == want
        assert hi <= 2 * lo + 10**6  # LPT keeps the two shares close
