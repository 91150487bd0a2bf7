"""GPU parity of the per-vertex counts (dbbc_count_vertices) against the
oracle's per-vertex Algorithm 1 and brute-force enumeration, element by
element: tiny graphs, closed forms, every counting tier (light and medium hash
tables, narrow and wide hub windows), tuning settings that move pivots between
tiers, union handles, and the sum invariant at full size."""
import math
import os

import numpy as np
import pytest

import oracle
import synth
import paper_2609_21848_gb300 as dbbc
from conftest import read_golden

pytestmark = pytest.mark.gpu

NCPU = max(1, len(os.sched_getaffinity(0)))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    dbbc.lib()


def gpu_vertices(u, v, s, n_u, n_v):
    with dbbc.dbbc_graph_from_coo(u, v, s, n_u, n_v) as g:
        vb, vu = dbbc.dbbc_count_vertices(g)
        tot = dbbc.dbbc_count(g)
        info = g.info
    return vb, vu, tot, info


def assert_vertex_parity(u, v, s, n_u, n_v, brute=False):
    want_b, want_u = (oracle.brute_force_per_vertex if brute else oracle.count_per_vertex)(u, v, s, n_u, n_v)
    vb, vu, tot, info = gpu_vertices(u, v, s, n_u, n_v)
    assert vb.shape == (n_u + n_v,) and vu.shape == (n_u + n_v,)
    bad = np.flatnonzero((vb != want_b) | (vu != want_u))
    assert bad.size == 0, f"{bad.size} vertices differ, first {bad[:5]}: GPU {vb[bad[:5]]}/{vu[bad[:5]]} " \
                          f"oracle {want_b[bad[:5]]}/{want_u[bad[:5]]}"
    # every butterfly has four vertices
    assert int(vb.sum(dtype=np.uint64)) == 4 * tot[0] and int(vu.sum(dtype=np.uint64)) == 4 * tot[1]
    return info


def _rand(rng, n_u, n_v, m, p_plus=0.5):
    pairs = rng.choice(n_u * n_v, size=min(m, n_u * n_v), replace=False)
    return (pairs // n_v).astype(np.int32), (pairs % n_v).astype(np.int32), \
        np.where(rng.random(pairs.shape[0]) < p_plus, 1, -1).astype(np.int8)


def _kab(a, b, sign=None):
    u, v = np.meshgrid(np.arange(a), np.arange(b), indexing="ij")
    u, v = u.ravel().astype(np.int32), v.ravel().astype(np.int32)
    s = np.ones(u.shape[0], np.int8) if sign is None else sign(u, v).astype(np.int8)
    return u, v, s


def test_worked_example_every_vertex_in_the_one_butterfly():
    g = read_golden("worked_example_k22.txt")
    e = np.array(g["edge"])
    n_u, n_v = g["n_u"][0][0], g["n_v"][0][0]
    vb, vu, tot, _ = gpu_vertices(e[:, 0], e[:, 1], e[:, 2], n_u, n_v)
    assert tot == (1, 0)
    want_b, want_u = oracle.brute_force_per_vertex(e[:, 0], e[:, 1], e[:, 2], n_u, n_v)
    assert vb.tolist() == want_b.tolist() and vu.tolist() == want_u.tolist()


def test_all_sign_patterns_of_k22():
    u, v = np.array([0, 0, 1, 1]), np.array([0, 1, 0, 1])
    for bits in range(16):
        s = np.array([-1 if bits >> i & 1 else 1 for i in range(4)])
        vb, vu, _, _ = gpu_vertices(u, v, s, 2, 2)
        even = bin(bits).count("1") % 2 == 0
        assert vb.tolist() == [int(even)] * 4 and vu.tolist() == [int(not even)] * 4


@pytest.mark.parametrize("seed", range(8))
def test_random_small_vs_brute_force(seed):
    rng = np.random.default_rng(300 + seed)
    n_u, n_v = int(rng.integers(2, 40)), int(rng.integers(2, 40))
    u, v, s = _rand(rng, n_u, n_v, int(rng.integers(1, n_u * n_v + 1)), p_plus=rng.random())
    assert_vertex_parity(u, v, s, n_u, n_v, brute=True)


@pytest.mark.parametrize("a,b", [(2, 3), (9, 7), (120, 90), (300, 200)])
def test_complete_bipartite_closed_form(a, b):
    # in K(a,b) every U vertex lies in (a-1) C(b,2) butterflies, every V vertex
    # in (b-1) C(a,2); with campaign signs (s = c_u c_v) all are balanced
    rng = np.random.default_rng(a * 1000 + b)
    cu, cv = rng.choice([-1, 1], size=a), rng.choice([-1, 1], size=b)
    u, v, s = _kab(a, b, lambda x, y: cu[x] * cv[y])
    vb, vu, _, info = gpu_vertices(u, v, s, a, b)
    assert vb[:a].tolist() == [(a - 1) * math.comb(b, 2)] * a
    assert vb[a:].tolist() == [(b - 1) * math.comb(a, 2)] * b
    assert not vu.any()


def test_random_signs_spanning_tiers_vs_oracle():
    rng = np.random.default_rng(5)
    a, b = 260, 180
    u, v, s = _kab(a, b, lambda x, y: rng.choice([-1, 1], size=x.shape))
    info = assert_vertex_parity(u, v, s, a, b)
    assert info["n_light"] > 0 and info["n_medium"] > 0 and info["n_hub"] > 0


@pytest.mark.parametrize("edges,n_u,n_v", [
    ([], 0, 0), ([], 5, 3), ([(0, 0, 1)], 1, 1), ([(0, j, 1) for j in range(50)], 1, 50),
    ([(i, 0, -1) for i in range(40)], 40, 1), ([(0, 0, 1), (1, 1, -1)], 4, 4),
])
def test_degenerate(edges, n_u, n_v):
    e = np.array(edges, np.int64).reshape(-1, 3)
    vb, vu, tot, _ = gpu_vertices(e[:, 0].astype(np.int32), e[:, 1].astype(np.int32), e[:, 2].astype(np.int8),
                                  n_u, n_v)
    assert vb.shape == (n_u + n_v,) and not vb.any() and not vu.any() and tot == (0, 0)


@pytest.mark.parametrize("scale", [0.002, 0.01])
def test_chunglu_scaled(scale):
    g = synth.workload("chunglu-1m-200k-20m", scale=scale)
    info = assert_vertex_parity(g.u, g.v, g.s, g.n_u, g.n_v)
    assert info["n_pivots"] > 0


def test_polarized_scaled():
    g = synth.workload("polarized-20m-2m-300m", scale=0.0005)
    assert_vertex_parity(g.u, g.v, g.s, g.n_u, g.n_v)


def test_uniform_2k_3k_20k():
    g = synth.workload("uniform-2k-3k-20k")
    assert_vertex_parity(g.u, g.v, g.s, g.n_u, g.n_v)


def test_dense_hubs_ragged_sizes():
    rng = np.random.default_rng(77)
    n_u, n_v = 3001, 1777
    hubs = rng.choice(n_u, 7, replace=False)
    bu, bv, _ = _rand(rng, n_u, n_v, 30_000)
    u = np.concatenate([np.repeat(hubs, n_v), bu]).astype(np.int32)
    v = np.concatenate([np.tile(np.arange(n_v), hubs.shape[0]), bv]).astype(np.int32)
    s = np.where(rng.random(u.shape[0]) < 0.6, 1, -1).astype(np.int8)
    info = assert_vertex_parity(u, v, s, n_u, n_v)
    assert info["n_hub"] > 0


def test_wide_hub_window():
    # one U hub over 70,000 V vertices of degree 2: more than 2^16 lower
    # neighbours, so its sweep uses 32-bit counter halves
    rng = np.random.default_rng(11)
    n_u, n_v = 101, 70_000
    other = rng.integers(1, n_u, size=n_v)
    u = np.concatenate([np.zeros(n_v, np.int64), other]).astype(np.int32)
    v = np.concatenate([np.arange(n_v), np.arange(n_v)]).astype(np.int32)
    s = np.where(rng.random(u.shape[0]) < 0.5, 1, -1).astype(np.int8)
    info = assert_vertex_parity(u, v, s, n_u, n_v)
    assert info["n_hub"] >= 1 and info["lower_hub"] >= 1 << 16


@pytest.mark.parametrize("tuning", [
    dict(light_max_work=1, medium_max_work=1, hub_item_work=1024, group_density=[40.0, 16.0, 6.0, 2.0],
         hash_mult_log=1),   # every pivot in the hub sweep, many small items
    dict(light_max_work=16, medium_max_work=64, hub_item_work=4096, group_density=[1e9, 1e9, 1e9, 1e9],
         hash_mult_log=3),
])
def test_counts_do_not_depend_on_tuning(tuning):
    base = dbbc.dbbc_get_tuning()
    g = synth.workload("chunglu-1m-200k-20m", scale=0.005)
    want_b, want_u = oracle.count_per_vertex(g.u, g.v, g.s, g.n_u, g.n_v)
    try:
        dbbc.dbbc_set_tuning(tuning)
        vb, vu, _, _ = gpu_vertices(g.u, g.v, g.s, g.n_u, g.n_v)
    finally:
        dbbc.dbbc_set_tuning(base)
    assert np.array_equal(vb, want_b) and np.array_equal(vu, want_u)


def test_union_handle_uses_union_ids():
    graphs = [synth.batch_graph(i) for i in range(6)] + [synth.workload("uniform-2k-3k-20k")]
    off = np.concatenate([[0], np.cumsum([x.u.shape[0] for x in graphs])])
    nu = [x.n_u for x in graphs]
    nv = [x.n_v for x in graphs]
    with dbbc.dbbc_graph_from_coo_multi(np.concatenate([x.u for x in graphs]), np.concatenate([x.v for x in graphs]),
                                        np.concatenate([x.s for x in graphs]), off, nu, nv) as g:
        vb, vu = dbbc.dbbc_count_vertices(g)
    NU = sum(nu)
    uo = np.concatenate([[0], np.cumsum(nu)])
    vo = np.concatenate([[0], np.cumsum(nv)])
    for i, x in enumerate(graphs):
        wb, wu = oracle.count_per_vertex(x.u, x.v, x.s, x.n_u, x.n_v)
        assert np.array_equal(vb[uo[i]:uo[i + 1]], wb[:x.n_u]) and np.array_equal(vu[uo[i]:uo[i + 1]], wu[:x.n_u])
        assert np.array_equal(vb[NU + vo[i]:NU + vo[i + 1]], wb[x.n_u:])
        assert np.array_equal(vu[NU + vo[i]:NU + vo[i + 1]], wu[x.n_u:])


def _digest(balanced, unbalanced):
    """SHA-256 of two count arrays as little-endian uint64, one after the other
    (the form tests/golden/make_expected.py stores for the oracle's arrays)."""
    import hashlib
    h = hashlib.sha256()
    for a in (balanced, unbalanced):
        h.update(np.ascontiguousarray(a, dtype="<u8").tobytes())
    return h.hexdigest()


def _stored_digest(workload, kind):
    return dict(read_golden("expected_digests.txt")[workload])[kind]


def test_chunglu_full_size_matches_the_oracle_element_by_element():
    """At 1M x 200k x 20M edges: every vertex's balanced and unbalanced counts
    equal the oracle's (compared through the SHA-256 of the whole arrays that
    the oracle's per-vertex walk stored), each array sums to four times the
    stored totals, and two calls give the same arrays."""
    g = synth.workload("chunglu-1m-200k-20m")
    exp = read_golden("expected_counts.txt")["chunglu-1m-200k-20m"][0]
    vb, vu, tot, _ = gpu_vertices(g.u, g.v, g.s, g.n_u, g.n_v)
    assert tot == (exp[0], exp[1])
    assert int(vb.sum(dtype=np.uint64)) == 4 * exp[0]
    assert int(vu.sum(dtype=np.uint64)) == 4 * exp[1]
    assert _digest(vb, vu) == _stored_digest("chunglu-1m-200k-20m", "vertices")
    vb2, vu2, _, _ = gpu_vertices(g.u, g.v, g.s, g.n_u, g.n_v)
    assert np.array_equal(vb, vb2) and np.array_equal(vu, vu2)


# ------------------------------------------------------------- per-edge counts
def gpu_edges(u, v, s, n_u, n_v, qu=None, qv=None, device=False):
    if qu is None:
        qu, qv = u, v
    with dbbc.dbbc_graph_from_coo(u, v, s, n_u, n_v) as g:
        if device:
            import torch
            eb, eu = dbbc.dbbc_count_edges(g, torch.as_tensor(np.asarray(qu, np.int32)).cuda(),
                                           torch.as_tensor(np.asarray(qv, np.int32)).cuda())
            eb, eu = eb.cpu().numpy(), eu.cpu().numpy()
        else:
            eb, eu = dbbc.dbbc_count_edges(g, qu, qv)
        tot = dbbc.dbbc_count(g)
    return eb, eu, tot


def assert_edge_parity(u, v, s, n_u, n_v, brute=False, device=False):
    fn = oracle.brute_force_per_edge if brute else oracle.count_per_edge
    # every distinct input pair once, in a shuffled order, plus some non-edges
    rng = np.random.default_rng(len(u))
    pairs = np.unique(np.asarray(u, np.int64) * n_v + np.asarray(v, np.int64))
    rng.shuffle(pairs)
    extra = rng.integers(0, n_u * n_v, size=min(64, n_u * n_v)) if n_u * n_v else np.zeros(0, np.int64)
    q = np.concatenate([pairs, extra])
    qu, qv = (q // n_v).astype(np.int32), (q % n_v).astype(np.int32)
    want_b, want_u = fn(u, v, s, n_u, n_v, qu, qv)
    eb, eu, tot = gpu_edges(u, v, s, n_u, n_v, qu, qv, device=device)
    bad = np.flatnonzero((eb != want_b) | (eu != want_u))
    assert bad.size == 0, f"{bad.size} edges differ, first {bad[:5]}: GPU {eb[bad[:5]]}/{eu[bad[:5]]} " \
                          f"oracle {want_b[bad[:5]]}/{want_u[bad[:5]]}"
    k = pairs.shape[0]
    assert int(eb[:k].sum(dtype=np.uint64)) == 4 * tot[0] and int(eu[:k].sum(dtype=np.uint64)) == 4 * tot[1]


@pytest.mark.parametrize("seed", range(6))
def test_edges_random_small_vs_brute_force(seed):
    rng = np.random.default_rng(400 + seed)
    n_u, n_v = int(rng.integers(2, 40)), int(rng.integers(2, 40))
    u, v, s = _rand(rng, n_u, n_v, int(rng.integers(1, n_u * n_v + 1)), p_plus=rng.random())
    assert_edge_parity(u, v, s, n_u, n_v, brute=True)


def test_edges_complete_bipartite_closed_form():
    a, b = 300, 200
    rng = np.random.default_rng(9)
    cu, cv = rng.choice([-1, 1], size=a), rng.choice([-1, 1], size=b)
    u, v, s = _kab(a, b, lambda x, y: cu[x] * cv[y])
    eb, eu, _ = gpu_edges(u, v, s, a, b)
    assert eb.tolist() == [(a - 1) * (b - 1)] * (a * b) and not eu.any()


def test_edges_repeated_pairs_and_non_edges():
    u, v, s = [0, 0, 0, 1, 1], [0, 0, 1, 0, 1], [-1, 1, 1, 1, 1]
    eb, eu, _ = gpu_edges(u, v, s, 3, 3, qu=[0, 0, 0, 1, 1, 2, 2, 0], qv=[0, 0, 1, 0, 1, 2, 0, 2])
    assert eb.tolist() == [1, 1, 1, 1, 1, 0, 0, 0] and not eu.any()


def test_edges_out_of_range_is_einval():
    with dbbc.dbbc_graph_from_coo([0, 1], [0, 1], [1, 1], 2, 2) as g:
        for qu, qv in (([2], [0]), ([0], [2]), ([-1], [0])):
            with pytest.raises(dbbc.DbbcError):
                dbbc.dbbc_count_edges(g, qu, qv)
        eb, eu = dbbc.dbbc_count_edges(g, [], [])
        assert eb.shape == (0,)


@pytest.mark.parametrize("device", [False, True])
def test_edges_uniform_2k_3k_20k(device):
    g = synth.workload("uniform-2k-3k-20k")
    assert_edge_parity(g.u, g.v, g.s, g.n_u, g.n_v, device=device)


def test_edges_spanning_tiers():
    rng = np.random.default_rng(5)
    a, b = 260, 180
    u, v, s = _kab(a, b, lambda x, y: rng.choice([-1, 1], size=x.shape))
    assert_edge_parity(u, v, s, a, b)


@pytest.mark.parametrize("scale", [0.002, 0.01])
def test_edges_chunglu_scaled(scale):
    g = synth.workload("chunglu-1m-200k-20m", scale=scale)
    assert_edge_parity(g.u, g.v, g.s, g.n_u, g.n_v)


def test_edges_polarized_scaled():
    g = synth.workload("polarized-20m-2m-300m", scale=0.0005)
    assert_edge_parity(g.u, g.v, g.s, g.n_u, g.n_v)


def test_edges_dense_and_wide_hubs():
    rng = np.random.default_rng(77)
    n_u, n_v = 3001, 1777
    hubs = rng.choice(n_u, 7, replace=False)
    bu, bv, _ = _rand(rng, n_u, n_v, 30_000)
    u = np.concatenate([np.repeat(hubs, n_v), bu]).astype(np.int32)
    v = np.concatenate([np.tile(np.arange(n_v), hubs.shape[0]), bv]).astype(np.int32)
    s = np.where(rng.random(u.shape[0]) < 0.6, 1, -1).astype(np.int8)
    assert_edge_parity(u, v, s, n_u, n_v)
    n_u, n_v = 101, 70_000
    other = rng.integers(1, n_u, size=n_v)
    u = np.concatenate([np.zeros(n_v, np.int64), other]).astype(np.int32)
    v = np.concatenate([np.arange(n_v), np.arange(n_v)]).astype(np.int32)
    s = np.where(rng.random(u.shape[0]) < 0.5, 1, -1).astype(np.int8)
    assert_edge_parity(u, v, s, n_u, n_v)


def test_edges_do_not_depend_on_tuning():
    base = dbbc.dbbc_get_tuning()
    g = synth.workload("chunglu-1m-200k-20m", scale=0.005)
    want_b, want_u = oracle.count_per_edge(g.u, g.v, g.s, g.n_u, g.n_v)
    try:
        dbbc.dbbc_set_tuning(dict(light_max_work=1, medium_max_work=1, hub_item_work=1024,
                                  group_density=[40.0, 16.0, 6.0, 2.0], hash_mult_log=1))
        eb, eu, _ = gpu_edges(g.u, g.v, g.s, g.n_u, g.n_v)
    finally:
        dbbc.dbbc_set_tuning(base)
    assert np.array_equal(eb, want_b) and np.array_equal(eu, want_u)


def test_edges_chunglu_full_size_match_the_oracle():
    g = synth.workload("chunglu-1m-200k-20m")
    exp = read_golden("expected_counts.txt")["chunglu-1m-200k-20m"][0]
    pairs = np.unique(g.u.astype(np.int64) * g.n_v + g.v)
    eb, eu, tot = gpu_edges(g.u, g.v, g.s, g.n_u, g.n_v, (pairs // g.n_v).astype(np.int32),
                            (pairs % g.n_v).astype(np.int32))
    assert tot == (exp[0], exp[1])
    assert int(eb.sum(dtype=np.uint64)) == 4 * exp[0] and int(eu.sum(dtype=np.uint64)) == 4 * exp[1]
    # every edge against the oracle's per-edge walk (stored as a digest)
    assert _digest(eb, eu) == _stored_digest("chunglu-1m-200k-20m", "edges")
