"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle,
bit-exact, on worked examples, closed forms, edge cases, seeded synthetic
graphs that span every counting tier, and the full-size Chung-Lu workload."""
import math
import os

import numpy as np
import pytest

import oracle
import synth
import paper_2609_21848_gb300 as dbbc
from conftest import read_golden
from gpu_util import assert_parity, gpu_count, host_csr

pytestmark = pytest.mark.gpu

NCPU = max(1, len(os.sched_getaffinity(0)))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    dbbc.lib()


def _rand(rng, n_u, n_v, m, p_plus=0.5):
    pairs = rng.choice(n_u * n_v, size=min(m, n_u * n_v), replace=False)
    return (pairs // n_v).astype(np.int32), (pairs % n_v).astype(np.int32), \
        np.where(rng.random(pairs.shape[0]) < p_plus, 1, -1).astype(np.int8)


def _kab(a, b, sign=None):
    u, v = np.meshgrid(np.arange(a), np.arange(b), indexing="ij")
    u, v = u.ravel().astype(np.int32), v.ravel().astype(np.int32)
    s = np.ones(u.shape[0], np.int8) if sign is None else sign(u, v).astype(np.int8)
    return u, v, s


# ------------------------------------------------------------- paper examples
def test_worked_example():
    g = read_golden("worked_example_k22.txt")
    e = np.array(g["edge"])
    bal, unb, info = gpu_count(e[:, 0], e[:, 1], e[:, 2], g["n_u"][0][0], g["n_v"][0][0])
    assert (bal, unb) == (1, 0)
    assert info["wedges"] == g["expect"][3][1]


def test_all_sign_patterns_of_k22():
    u, v = np.array([0, 0, 1, 1]), np.array([0, 1, 0, 1])
    for bits in range(16):
        s = np.array([-1 if bits >> i & 1 else 1 for i in range(4)])
        k = bin(bits).count("1")
        assert gpu_count(u, v, s, 2, 2)[:2] == ((1, 0) if k % 2 == 0 else (0, 1))


@pytest.mark.parametrize("a,b", [(2, 3), (9, 7), (40, 60), (120, 90), (300, 200)])
def test_complete_bipartite(a, b):
    u, v, s = _kab(a, b)
    bal, unb, info = gpu_count(u, v, s, a, b)
    assert (bal, unb) == (math.comb(a, 2) * math.comb(b, 2), 0)
    assert info["wedges"] == (b * math.comb(a, 2) if b > a else a * math.comb(b, 2))


def test_complete_bipartite_camp_signs_spans_tiers():
    rng = np.random.default_rng(5)
    a, b = 260, 180
    cu, cv = rng.choice([-1, 1], size=a), rng.choice([-1, 1], size=b)
    u, v, s = _kab(a, b, lambda x, y: cu[x] * cv[y])
    bal, unb, info = gpu_count(u, v, s, a, b)
    assert (bal, unb) == (math.comb(a, 2) * math.comb(b, 2), 0)
    assert info["n_light"] > 0 and info["n_medium"] > 0 and info["n_hub"] > 0


# ------------------------------------------------------------- edge cases
@pytest.mark.parametrize("edges,n_u,n_v", [
    ([], 0, 0), ([], 5, 3), ([(0, 0, 1)], 1, 1), ([(0, j, 1) for j in range(50)], 1, 50),
    ([(i, 0, -1) for i in range(70)], 70, 1), ([(0, 0, 1), (1, 0, -1), (1, 1, 1), (2, 1, -1)], 3, 2),
])
def test_degenerate(edges, n_u, n_v):
    e = np.array(edges, np.int64).reshape(-1, 3)
    bal, unb, info = gpu_count(e[:, 0], e[:, 1], e[:, 2], n_u, n_v)
    assert (bal, unb) == (0, 0)


@pytest.mark.parametrize("bad", ["u", "v", "sign0", "sign2", "neg_u"])
def test_invalid_input_is_einval(bad):
    u, v, s = np.array([0, 1, 1]), np.array([0, 0, 1]), np.array([1, -1, 1])
    if bad == "u":
        u[1] = 2
    elif bad == "v":
        v[0] = 7
    elif bad == "sign0":
        s[2] = 0
    elif bad == "sign2":
        s[0] = 2
    else:
        u[0] = -3
    with pytest.raises(dbbc.DbbcError) as ei:
        dbbc.dbbc_graph_from_coo(u, v, s, 2, 2)
    assert ei.value.status == dbbc.DBBC_EINVAL


def test_duplicates_keep_latest_and_reject_flag():
    rng = np.random.default_rng(9)
    u, v, s = _rand(rng, 50, 40, 900)
    pick = rng.choice(u.shape[0], 200, replace=False)
    u2, v2 = np.concatenate([u, u[pick]]), np.concatenate([v, v[pick]])
    s2 = np.concatenate([s, -s[pick]]).astype(np.int8)
    info = assert_parity(u2, v2, s2, 50, 40)
    assert info["m"] == 900 and info["m_input"] == 1100
    with pytest.raises(dbbc.DbbcError) as ei:
        dbbc.dbbc_graph_from_coo(u2, v2, s2, 50, 40, reject_duplicates=True)
    assert ei.value.status == dbbc.DBBC_EINVAL
    with dbbc.dbbc_graph_from_coo(u, v, s, 50, 40, reject_duplicates=True) as g:
        assert dbbc.dbbc_count(g) == oracle.count(u, v, s, 50, 40)[:2]


@pytest.mark.parametrize("seed", range(8))
def test_random_small_vs_brute_force(seed):
    rng = np.random.default_rng(1000 + seed)
    n_u, n_v = int(rng.integers(2, 30)), int(rng.integers(2, 30))
    u, v, s = _rand(rng, n_u, n_v, int(rng.integers(1, n_u * n_v + 1)), float(rng.random()))
    assert gpu_count(u, v, s, n_u, n_v)[:2] == oracle.brute_force(u, v, s, n_u, n_v)


# ------------------------------------------------------------- seeded workloads
@pytest.mark.parametrize("device_input", [False, True])
def test_uniform_2k_3k_20k(device_input):
    g = synth.workload("uniform-2k-3k-20k")
    assert_parity(g.u, g.v, g.s, g.n_u, g.n_v, device_input=device_input)


@pytest.mark.parametrize("scale", [0.002, 0.01, 0.05])
def test_chunglu_scaled(scale):
    g = synth.workload("chunglu-1m-200k-20m", scale=scale)
    info = assert_parity(g.u, g.v, g.s, g.n_u, g.n_v, threads=NCPU)
    assert info["n_pivots"] > 0


@pytest.mark.parametrize("scale", [0.0005, 0.002])
def test_polarized_scaled(scale):
    g = synth.workload("polarized-20m-2m-300m", scale=scale)
    assert_parity(g.u, g.v, g.s, g.n_u, g.n_v, threads=NCPU)


def test_dense_hub_graph_ragged_sizes():
    # a few dense hubs over a sparse background: hub tier with many chunks,
    # side sizes that are not multiples of any tile
    rng = np.random.default_rng(77)
    n_u, n_v = 3001, 1777
    hubs = rng.choice(n_u, 7, replace=False)
    u = [np.repeat(hubs, n_v)]
    v = [np.tile(np.arange(n_v), hubs.shape[0])]
    bu, bv, _ = _rand(rng, n_u, n_v, 30_000)
    u = np.concatenate(u + [bu]).astype(np.int32)
    v = np.concatenate(v + [bv]).astype(np.int32)
    s = np.where(rng.random(u.shape[0]) < 0.6, 1, -1).astype(np.int8)
    info = assert_parity(u, v, s, n_u, n_v, threads=NCPU)
    assert info["n_hub"] > 0


# ------------------------------------------------------------- CSR export
@pytest.mark.parametrize("which", ["uniform", "chunglu"])
def test_csr_export_matches_host_build(which):
    if which == "uniform":
        g = synth.workload("uniform-2k-3k-20k")
    else:
        g = synth.workload("chunglu-1m-200k-20m", scale=0.005)
    want = host_csr(g.u, g.v, g.s, g.n_u, g.n_v)
    _, _, wed = oracle.count_per_pivot(g.u, g.v, g.s, g.n_u, g.n_v, threads=NCPU)
    with dbbc.dbbc_graph_from_coo(g.u, g.v, g.s, g.n_u, g.n_v) as h:
        got = dbbc.dbbc_graph_export(h)
    assert np.array_equal(got["row_ptr"], want["row_ptr"])
    assert np.array_equal(got["col"], want["col"])
    assert np.array_equal(got["vertex"], want["vertex"])
    assert np.array_equal(got["lower"].astype(np.int64), want["lower"])
    assert np.array_equal(got["work"], wed[got["vertex"]])


# ------------------------------------------------------------- batch / async / allocator
def test_batch_and_async_match_single_counts():
    import torch
    graphs = [synth.batch_graph(i) for i in range(12)]
    want = [oracle.count(g.u, g.v, g.s, g.n_u, g.n_v)[:2] for g in graphs]
    handles = [dbbc.dbbc_graph_from_coo(g.u, g.v, g.s, g.n_u, g.n_v) for g in graphs]
    try:
        bal, unb = dbbc.dbbc_count_batch(handles)
        assert list(zip(bal.tolist(), unb.tolist())) == want
        d_out = torch.zeros((len(handles), 2), dtype=torch.int64, device="cuda")
        dbbc.dbbc_count_batch_async(handles, d_out)
        got = d_out.cpu().numpy().astype(np.uint64)
        assert [tuple(map(int, r)) for r in got] == want
        one = torch.zeros(2, dtype=torch.int64, device="cuda")
        dbbc.dbbc_count_async(handles[3], one)
        assert tuple(map(int, one.cpu().tolist())) == want[3]
    finally:
        for h in handles:
            h.free()


def test_batch_plan_capture_and_replay_mixed_graphs():
    """A batch plan over uneven graphs (empty, tiny, light-only and hub-heavy):
    the first count captures the CUDA graph, the second replays it; both must
    equal the oracle for every graph."""
    import torch
    graphs = [synth.batch_graph(i) for i in range(40)]
    graphs.append(synth.Graph(np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int8), 5, 7))
    graphs.append(synth.workload("chunglu-1m-200k-20m", scale=0.01))
    graphs.append(synth.workload("uniform-2k-3k-20k"))
    u, v, s = _kab(150, 90)
    graphs.append(synth.Graph(u, v, s, 150, 90))
    want = [oracle.count(g.u, g.v, g.s, g.n_u, g.n_v, threads=NCPU)[:2] for g in graphs]
    handles = [dbbc.dbbc_graph_from_coo(g.u, g.v, g.s, g.n_u, g.n_v) for g in graphs]
    try:
        with dbbc.dbbc_batch_create(handles) as b:
            for _ in range(2):
                bal, unb = dbbc.dbbc_batch_count(b)
                assert list(zip(bal.tolist(), unb.tolist())) == want
            d_out = torch.full((len(handles), 2), -1, dtype=torch.int64, device="cuda")
            dbbc.dbbc_batch_count_async(b, d_out)
            got = [tuple(map(int, r)) for r in d_out.cpu().numpy().astype(np.uint64)]
            assert got == want
    finally:
        for h in handles:
            h.free()


@pytest.mark.parametrize("medium_max_work", [4096, 256])
def test_batch_plan_wide_and_narrow_hub_items(medium_max_work):
    """A plan whose hub items go to both CTA shapes: the hubs of a 1M-edge
    Chung-Lu graph (items of more than 2^20 estimated wedges and windows wider
    than a narrow CTA's) on the full-window CTAs, the small graphs' items on the
    narrow ones, counted side by side; every graph equals the oracle."""
    base = dbbc.dbbc_get_tuning()
    graphs = [synth.workload("chunglu-1m-200k-20m", scale=0.05)] + [synth.batch_graph(i) for i in range(24)]
    want = [oracle.count(g.u, g.v, g.s, g.n_u, g.n_v, threads=NCPU)[:2] for g in graphs]
    try:
        dbbc.dbbc_set_tuning({"light_max_work": 128, "medium_max_work": medium_max_work, "hub_item_work": 1 << 22})
        handles = [dbbc.dbbc_graph_from_coo(g.u, g.v, g.s, g.n_u, g.n_v) for g in graphs]
        try:
            assert max(h.info["wedges_hub"] for h in handles[:1]) > 1 << 22  # the large graph has large hub items
            with dbbc.dbbc_batch_create(handles) as b:
                for _ in range(2):  # capture, then replay
                    bal, unb = dbbc.dbbc_batch_count(b)
                    assert list(zip(bal.tolist(), unb.tolist())) == want
        finally:
            for h in handles:
                h.free()
    finally:
        dbbc.dbbc_set_tuning(base)


def _union_inputs(graphs):
    u = np.concatenate([g.u for g in graphs]).astype(np.int32)
    v = np.concatenate([g.v for g in graphs]).astype(np.int32)
    s = np.concatenate([g.s for g in graphs]).astype(np.int8)
    off = np.concatenate([[0], np.cumsum([g.m for g in graphs])]).astype(np.int64)
    return u, v, s, off, [g.n_u for g in graphs], [g.n_v for g in graphs]


@pytest.mark.parametrize("device_input,finalize", [(False, None), (True, None), (False, 0), (False, 2**64 - 1)])
def test_union_build_counts_each_component_exactly(device_input, finalize):
    """dbbc_graph_from_coo_multi: per-component counts equal each graph counted
    alone (oracle), the plain count of the union is their sum, and duplicates
    stay within their own component. Components start at arbitrary (odd) ranks,
    so 8-bit counter windows start at odd ranks too; `finalize` forces every hub
    window through one Lemma 1 mode (scan on clear, or per wedge)."""
    import torch
    base = dbbc.dbbc_get_tuning()
    if finalize is not None:
        dbbc.dbbc_set_tuning({"finalize_window_wedges": finalize, "light_max_work": 16, "medium_max_work": 64})
    try:
        _union_case(device_input, torch)
    finally:
        dbbc.dbbc_set_tuning(base)


def _union_case(device_input, torch):
    rng = np.random.default_rng(21)
    graphs = [synth.batch_graph(i) for i in range(30)]
    graphs.insert(3, synth.Graph(np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int8), 4, 9))
    graphs.insert(10, synth.workload("chunglu-1m-200k-20m", scale=0.01))
    gd = synth.batch_graph(77)  # a graph with conflicting duplicates
    pick = rng.choice(gd.m, 50, replace=False)
    graphs.append(synth.Graph(np.concatenate([gd.u, gd.u[pick]]), np.concatenate([gd.v, gd.v[pick]]),
                              np.concatenate([gd.s, -gd.s[pick]]).astype(np.int8), gd.n_u, gd.n_v))
    u, v, s, off, nu, nv = _union_inputs(graphs)
    want = [oracle.count(g.u, g.v, g.s, g.n_u, g.n_v, threads=NCPU)[:2] for g in graphs]
    if device_input:
        u, v, s = (torch.from_numpy(x).cuda() for x in (u, v, s))
    with dbbc.dbbc_graph_from_coo_multi(u, v, s, off, nu, nv) as h:
        assert h.info["n_components"] == len(graphs)
        bal, unb = dbbc.dbbc_count_components(h)
        assert list(zip(bal.tolist(), unb.tolist())) == want
        assert dbbc.dbbc_count(h) == (sum(w[0] for w in want), sum(w[1] for w in want))
        assert h.info["wedges"] == sum(oracle.count(g.u, g.v, g.s, g.n_u, g.n_v, threads=NCPU)[2] for g in graphs)


def test_union_build_validates_each_component():
    graphs = [synth.batch_graph(i) for i in range(4)]
    u, v, s, off, nu, nv = _union_inputs(graphs)
    u[off[2]] = nu[2]  # out of range for graph 2 (in range for the union)
    with pytest.raises(dbbc.DbbcError) as ei:
        dbbc.dbbc_graph_from_coo_multi(u, v, s, off, nu, nv)
    assert ei.value.status == dbbc.DBBC_EINVAL


@pytest.mark.parametrize("tuning", [
    dict(light_max_work=1, medium_max_work=1, hub_item_work=1024, group_density=[40.0, 16.0, 6.0, 2.0],
         hash_mult_log=1),   # every pivot in the hub sweep, many small items
    dict(light_max_work=512, medium_max_work=4096, hub_item_work=1 << 22, group_density=[0.0, 0.0, 0.0, 0.0],
         hash_mult_log=3),   # 32-lane groups everywhere, sparse hash tables
    dict(light_max_work=16, medium_max_work=64, hub_item_work=4096, group_density=[1e9, 1e9, 1e9, 1e9],
         hash_mult_log=2),   # one lane per segment
    dict(light_max_work=1, medium_max_work=1, hub_item_work=1024, group_density=[40.0, 16.0, 6.0, 2.0],
         hash_mult_log=1, list_density=1e9, list_group_log=0),   # every pivot a list-mode hub, one lane
    dict(light_max_work=64, medium_max_work=512, hub_item_work=1 << 20, group_density=[40.0, 16.0, 6.0, 2.0],
         hash_mult_log=2, list_density=1e9, list_group_log=5),   # list mode with whole-warp groups
    dict(light_max_work=512, medium_max_work=4096, hub_item_work=1 << 22, group_density=[40.0, 16.0, 6.0, 2.0],
         hash_mult_log=2, list_density=0.0, list_group_log=2),   # no list mode
    dict(light_max_work=1, medium_max_work=1, hub_item_work=1024, group_density=[40.0, 16.0, 6.0, 2.0],
         hash_mult_log=1, list_density=8.0, list_group_log=3,
         finalize_window_wedges=0),   # every hub window finalised by a scan of its counters
    dict(light_max_work=1, medium_max_work=1, hub_item_work=1024, group_density=[0.0, 0.0, 0.0, 0.0],
         hash_mult_log=1, list_density=0.0, finalize_window_wedges=0),   # scan-finalised, 32-lane groups
    dict(light_max_work=1, medium_max_work=1, hub_item_work=1024, group_density=[1e9, 1e9, 1e9, 1e9],
         hash_mult_log=1, list_density=1e9, list_group_log=0,
         finalize_window_wedges=2**64 - 1),   # every wedge's Lemma 1 term from its atomic, one lane
    dict(light_max_work=1, medium_max_work=1, hub_item_work=1024, group_density=[40.0, 16.0, 6.0, 2.0],
         hash_mult_log=1, list_density=1e9, list_group_log=2,
         list_wide_density=0.0),   # every pivot a list-mode hub, 8-lane groups
])
def test_counts_do_not_depend_on_tuning(tuning):
    base = dbbc.dbbc_get_tuning()
    g = synth.workload("chunglu-1m-200k-20m", scale=0.01)
    want = oracle.count(g.u, g.v, g.s, g.n_u, g.n_v, threads=NCPU)
    graphs = [synth.batch_graph(i) for i in range(8)]
    want_b = [oracle.count(x.u, x.v, x.s, x.n_u, x.n_v)[:2] for x in graphs]
    try:
        dbbc.dbbc_set_tuning(tuning)
        bal, unb, info = gpu_count(g.u, g.v, g.s, g.n_u, g.n_v)
        assert (bal, unb, info["wedges"]) == want
        handles = [dbbc.dbbc_graph_from_coo(x.u, x.v, x.s, x.n_u, x.n_v) for x in graphs]
        try:
            b, u = dbbc.dbbc_count_batch(handles)
            assert list(zip(b.tolist(), u.tolist())) == want_b
        finally:
            for h in handles:
                h.free()
    finally:
        dbbc.dbbc_set_tuning(base)


def test_sign_ratio_changes_the_split_not_the_total():
    """Section VI sign-ratio study on a scaled Chung-Lu topology: the same
    edges with P(+) from 0.1 to 0.9 give the same accepted wedges and the same
    balanced + unbalanced total (the unsigned count), while the split moves;
    every point matches the oracle."""
    p = dict(synth.WORKLOADS["chunglu-1m-200k-20m"])
    p.pop("index")
    for k in ("n_u", "n_v", "m"):
        p[k] = p[k] // 200
    p["cap_u"] = p["cap_v"] = 100
    totals, fracs, wedges = set(), [], set()
    for pp in (0.1, 0.5, 0.9):
        p["p_plus"] = pp
        g = synth.generate(synth.SEED_BASE + 1, **p)
        bal, unb, info = gpu_count(g.u, g.v, g.s, g.n_u, g.n_v)
        assert (bal, unb, info["wedges"]) == oracle.count(g.u, g.v, g.s, g.n_u, g.n_v, threads=NCPU)
        totals.add(bal + unb)
        wedges.add(info["wedges"])
        fracs.append(bal / (bal + unb))
    assert len(totals) == 1 and len(wedges) == 1
    assert fracs[1] < fracs[0] and fracs[1] < fracs[2]  # P(+) = 1/2 balances least


def _lpt_parts_from_export(h, parts):
    """The pivots of each LPT part, recomputed from the exported CSR: pivots
    are the rows with at least two lower neighbours and accepted wedges, in
    descending work (ties by row); Phase 3's greedy packing of their work
    (dbbc_lpt_partition, itself checked against the oracle's LPT on the CPU)
    assigns each to a part. Returns the unified ids of each part's pivots."""
    ex = dbbc.dbbc_graph_export(h)
    rows = np.nonzero((ex["lower"] >= 2) & (ex["work"] > 0))[0]
    rows = rows[np.lexsort((rows, -ex["work"][rows].astype(np.float64)))]
    assert np.all(np.diff(ex["work"][rows].astype(np.int64)) <= 0)
    part, _ = dbbc.dbbc_lpt_partition(ex["work"][rows], parts)
    return [ex["vertex"][rows[part == p]] for p in range(parts)]


@pytest.mark.parametrize("parts", [1, 2, 3, 8])
def test_partition_parts_match_the_oracle(parts):
    """dbbc_count_partition (Phase 3 greedy packing, Section IV-A, Example 2):
    each part's counts equal the oracle's per-pivot counts summed over that
    part's pivots, on a graph with hubs (several work items each), medium and
    light pivots; the parts add up to the oracle's totals (Theorem 1)."""
    g = synth.workload("chunglu-1m-200k-20m", scale=0.02)
    bal, unb, wed = oracle.count_per_pivot(g.u, g.v, g.s, g.n_u, g.n_v, threads=NCPU)
    want_total = oracle.count(g.u, g.v, g.s, g.n_u, g.n_v, threads=NCPU)[:2]
    base = dbbc.dbbc_get_tuning()
    dbbc.dbbc_set_tuning({"hub_item_work": 1 << 14})  # several sweep items per hub
    try:
        with dbbc.dbbc_graph_from_coo(g.u, g.v, g.s, g.n_u, g.n_v) as h:
            info = h.info
            assert info["n_hub"] > 0 and info["n_medium"] > 0 and info["n_light"] > 0
            got = [dbbc.dbbc_count_partition(h, p, parts) for p in range(parts)]
            ids = _lpt_parts_from_export(h, parts)
    finally:
        dbbc.dbbc_set_tuning(base)
    for p in range(parts):
        assert got[p] == (int(bal[ids[p]].sum()), int(unb[ids[p]].sum())), p
    assert (sum(x[0] for x in got), sum(x[1] for x in got)) == want_total
    if parts > 1:
        assert all(x != (0, 0) for x in got)


def test_torch_allocator_hook():
    g = synth.workload("chunglu-1m-200k-20m", scale=0.003)
    want = oracle.count(g.u, g.v, g.s, g.n_u, g.n_v, threads=NCPU)[:2]
    dbbc.dbbc_set_allocator(True)
    try:
        assert gpu_count(g.u, g.v, g.s, g.n_u, g.n_v)[:2] == want
    finally:
        dbbc.dbbc_set_allocator(False)
    assert gpu_count(g.u, g.v, g.s, g.n_u, g.n_v)[:2] == want


def test_repeated_counts_are_identical():
    g = synth.workload("chunglu-1m-200k-20m", scale=0.01)
    with dbbc.dbbc_graph_from_coo(g.u, g.v, g.s, g.n_u, g.n_v) as h:
        first = dbbc.dbbc_count(h)
        for _ in range(3):
            assert dbbc.dbbc_count(h) == first


# ------------------------------------------------------------- full size
def test_chunglu_1m_200k_20m_full_size():
    g = synth.workload("chunglu-1m-200k-20m")
    assert_parity(g.u, g.v, g.s, g.n_u, g.n_v, threads=NCPU)


def _expected(name):
    from conftest import GOLDEN
    for line in open(os.path.join(GOLDEN, "expected_counts.txt")):
        f = line.split("#", 1)[0].split()
        if len(f) == 4 and f[0] == name:
            return tuple(int(x) for x in f[1:])
    return None


def test_chunglu_full_size_matches_stored_oracle_counts():
    g = synth.workload("chunglu-1m-200k-20m")
    bal, unb, info = gpu_count(g.u, g.v, g.s, g.n_u, g.n_v)
    assert (bal, unb, info["wedges"]) == _expected("chunglu-1m-200k-20m")


def test_invariants_at_full_size_polarized():
    """The 300M-edge polarized graph: the counts equal the oracle's (stored by
    tests/golden/make_expected.py); balanced + unbalanced equals the unsigned
    count; switching (negating every edge at a random vertex set) changes
    neither count."""
    if os.environ.get("DBBC_SKIP_HUGE"):
        pytest.skip("DBBC_SKIP_HUGE set")
    import torch
    g = synth.workload("polarized-20m-2m-300m")
    dev = torch.device("cuda")
    u, v, s = (torch.from_numpy(x).to(dev) for x in (g.u, g.v, g.s))
    with dbbc.dbbc_graph_from_coo(u, v, s, g.n_u, g.n_v) as h:
        bal, unb = dbbc.dbbc_count(h)
        wedges = h.info["wedges"]
    assert (bal, unb, wedges) == _expected("polarized-20m-2m-300m")
    with dbbc.dbbc_graph_from_coo(u, v, torch.ones_like(s), g.n_u, g.n_v) as h:
        assert dbbc.dbbc_count(h) == (bal + unb, 0)
    rng = np.random.default_rng(3)
    fu = torch.from_numpy(np.where(rng.random(g.n_u) < 0.5, -1, 1).astype(np.int8)).to(dev)
    fv = torch.from_numpy(np.where(rng.random(g.n_v) < 0.5, -1, 1).astype(np.int8)).to(dev)
    s2 = s * fu[u.long()] * fv[v.long()]
    with dbbc.dbbc_graph_from_coo(u, v, s2, g.n_u, g.n_v) as h:
        assert dbbc.dbbc_count(h) == (bal, unb)
        assert h.info["wedges"] == wedges
    assert bal > unb > 0
