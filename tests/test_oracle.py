"""Pins for the CPU oracle: worked example, closed forms, invariants and
independent cross-checks (brute force of Def. 1-2, pair counting, Gram identity).
No GPU is needed."""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth
from conftest import read_golden


def _rand_graph(rng, n_u, n_v, m, p_plus=0.5):
    pairs = rng.choice(n_u * n_v, size=min(m, n_u * n_v), replace=False)
    u = (pairs // n_v).astype(np.int32)
    v = (pairs % n_v).astype(np.int32)
    s = np.where(rng.random(u.shape[0]) < p_plus, 1, -1).astype(np.int8)
    return u, v, s


def _kab(a, b, sign=None):
    u, v = np.meshgrid(np.arange(a), np.arange(b), indexing="ij")
    u = u.ravel().astype(np.int32)
    v = v.ravel().astype(np.int32)
    s = np.ones(u.shape[0], np.int8) if sign is None else sign(u, v).astype(np.int8)
    return u, v, s


# --------------------------------------------------------------- worked example
def test_worked_example_fig8():
    g = read_golden("worked_example_k22.txt")
    n_u, n_v = g["n_u"][0][0], g["n_v"][0][0]
    e = np.array(g["edge"])
    u, v, s = e[:, 0], e[:, 1], e[:, 2]
    bal, unb, wed = oracle.count(u, v, s, n_u, n_v)
    assert (bal, unb) == (g["expect"][0][1], g["expect"][1][1])
    assert oracle.brute_force(u, v, s, n_u, n_v) == (bal, unb)
    b, ub, w = oracle.count_per_pivot(u, v, s, n_u, n_v)
    pivot = n_u + g["expect"][2][1]  # unified id of right vertex 8
    assert b[pivot] == 1 and b.sum() == 1 and ub.sum() == 0
    assert w[pivot] == g["expect"][3][1]  # B1[5] = 2 at pivot 8


# --------------------------------------------------------------- Def. 2 / Fig. 3
def test_all_16_sign_patterns_of_k22():
    u = np.array([0, 0, 1, 1])
    v = np.array([0, 1, 0, 1])
    n_bal = 0
    for signs in itertools.product([1, -1], repeat=4):
        s = np.array(signs)
        k = sum(x < 0 for x in signs)
        want = (1, 0) if k % 2 == 0 else (0, 1)
        assert oracle.count(u, v, s, 2, 2)[:2] == want, signs
        assert oracle.brute_force(u, v, s, 2, 2) == want
        n_bal += want[0]
    assert n_bal == 8  # Fig. 3: k in {0,2,4} balanced, k in {1,3} unbalanced


@pytest.mark.parametrize("k_neg,balanced", [(0, True), (1, False), (2, True), (3, False), (4, True)])
def test_fig3_classes(k_neg, balanced):
    u = np.array([0, 0, 1, 1])
    v = np.array([0, 1, 0, 1])
    s = np.array([-1] * k_neg + [1] * (4 - k_neg))
    assert oracle.count(u, v, s, 2, 2)[:2] == ((1, 0) if balanced else (0, 1))


# --------------------------------------------------------------- closed forms
@pytest.mark.parametrize("a,b", [(2, 2), (2, 5), (5, 2), (4, 4), (7, 3), (3, 9), (12, 11)])
def test_complete_bipartite_all_positive(a, b):
    u, v, s = _kab(a, b)
    bal, unb, wed = oracle.count(u, v, s, a, b)
    assert bal == math.comb(a, 2) * math.comb(b, 2) and unb == 0
    # Accepted wedges of Algorithm 1 on K(a,b): the higher-priority side
    # (larger degree, or V on equal degree since V ids are larger) pivots;
    # pivot number i of that side sees i lower endpoints through every middle.
    assert wed == (b * math.comb(a, 2) if b > a else a * math.comb(b, 2))


@pytest.mark.parametrize("seed", range(3))
def test_wedge_total_does_not_depend_on_signs(seed):
    rng = np.random.default_rng(50 + seed)
    a, b = 5, 7
    u, v, _ = _kab(a, b)
    s = rng.choice([-1, 1], size=u.shape[0])
    assert oracle.count(u, v, s, a, b)[2] == b * math.comb(a, 2)
    u, v, s = _rand_graph(rng, 15, 15, 120)
    assert oracle.count(u, v, s, 15, 15)[2] == oracle.count(u, v, np.ones_like(s), 15, 15)[2]


@pytest.mark.parametrize("seed", range(4))
def test_switching_equivalent_signing_is_all_balanced(seed):
    rng = np.random.default_rng(seed)
    a, b = 6, 8
    cu = rng.choice([-1, 1], size=a)
    cv = rng.choice([-1, 1], size=b)
    u, v, s = _kab(a, b, lambda x, y: cu[x] * cv[y])
    assert oracle.count(u, v, s, a, b)[:2] == (math.comb(a, 2) * math.comb(b, 2), 0)


def test_all_negative_complete_bipartite_is_balanced():
    u, v, s = _kab(5, 6, lambda x, y: -np.ones_like(x))
    assert oracle.count(u, v, s, 5, 6)[:2] == (math.comb(5, 2) * math.comb(6, 2), 0)


@pytest.mark.parametrize("name,edges,n_u,n_v", [
    ("empty", [], 3, 3),
    ("no vertices", [], 0, 0),
    ("single edge", [(0, 0, 1)], 1, 1),
    ("star", [(0, j, (-1) ** j) for j in range(9)], 1, 9),
    ("path", [(0, 0, 1), (1, 0, -1), (1, 1, 1), (2, 1, -1)], 3, 2),
    ("cycle-free tree", [(0, 0, 1), (0, 1, 1), (1, 1, -1), (2, 1, 1), (2, 2, -1)], 3, 3),
])
def test_degenerate_graphs_have_no_butterflies(name, edges, n_u, n_v):
    e = np.array(edges, dtype=np.int64).reshape(-1, 3)
    assert oracle.count(e[:, 0], e[:, 1], e[:, 2], n_u, n_v)[:2] == (0, 0)


# --------------------------------------------------------------- invariants
@pytest.mark.parametrize("seed", range(6))
def test_matches_brute_force_on_random_tiny_graphs(seed):
    rng = np.random.default_rng(100 + seed)
    n_u, n_v = int(rng.integers(2, 14)), int(rng.integers(2, 14))
    m = int(rng.integers(1, n_u * n_v + 1))
    u, v, s = _rand_graph(rng, n_u, n_v, m, p_plus=float(rng.random()))
    assert oracle.count(u, v, s, n_u, n_v)[:2] == oracle.brute_force(u, v, s, n_u, n_v)


@pytest.mark.parametrize("seed", range(3))
def test_balanced_plus_unbalanced_is_unsigned_count(seed):
    rng = np.random.default_rng(200 + seed)
    u, v, s = _rand_graph(rng, 20, 25, 220)
    bal, unb, _ = oracle.count(u, v, s, 20, 25)
    ones = np.ones_like(s)
    assert oracle.count(u, v, ones, 20, 25)[:2] == (bal + unb, 0)


@pytest.mark.parametrize("seed", range(3))
def test_switching_invariance(seed):
    rng = np.random.default_rng(300 + seed)
    u, v, s = _rand_graph(rng, 30, 20, 250)
    base = oracle.count(u, v, s, 30, 20)
    flip_u = rng.random(30) < 0.5
    flip_v = rng.random(20) < 0.5
    s2 = (s * np.where(flip_u[u], -1, 1) * np.where(flip_v[v], -1, 1)).astype(np.int8)
    assert oracle.count(u, v, s2, 30, 20)[:2] == base[:2]
    assert oracle.count(u, v, -s, 30, 20)[:2] == base[:2]  # global negation


@pytest.mark.parametrize("seed", range(3))
def test_id_permutation_and_side_swap_invariance(seed):
    # Theorem 1: every butterfly is counted once at its highest-priority vertex,
    # whatever the total order, so relabelling changes nothing.
    rng = np.random.default_rng(400 + seed)
    u, v, s = _rand_graph(rng, 25, 35, 300)
    base = oracle.count(u, v, s, 25, 35)[:2]
    pu, pv = rng.permutation(25), rng.permutation(35)
    assert oracle.count(pu[u], pv[v], s, 25, 35)[:2] == base
    assert oracle.count(v, u, s, 35, 25)[:2] == base
    order = rng.permutation(u.shape[0])
    assert oracle.count(u[order], v[order], s[order], 25, 35)[:2] == base


def test_duplicates_keep_the_latest_sign():
    rng = np.random.default_rng(7)
    u, v, s = _rand_graph(rng, 12, 12, 90)
    pick = rng.choice(u.shape[0], size=30, replace=False)
    # append conflicting duplicates: the later (flipped) sign must win
    u2 = np.concatenate([u, u[pick]])
    v2 = np.concatenate([v, v[pick]])
    s2 = np.concatenate([s, -s[pick]]).astype(np.int8)
    s_final = s.copy()
    s_final[pick] = -s[pick]
    want = oracle.count(u, v, s_final, 12, 12)
    assert oracle.count(u2, v2, s2, 12, 12) == want
    assert oracle.brute_force(u2, v2, s2, 12, 12) == want[:2]
    assert oracle.pair_count(u2, v2, s2, 12, 12) == want[:2]
    # and a duplicate placed *before* the original loses
    u3 = np.concatenate([u[pick], u])
    v3 = np.concatenate([v[pick], v])
    s3 = np.concatenate([-s[pick], s]).astype(np.int8)
    assert oracle.count(u3, v3, s3, 12, 12) == oracle.count(u, v, s, 12, 12)


@pytest.mark.parametrize("bad", ["u_high", "u_neg", "v_high", "sign0", "sign2"])
def test_invalid_input_is_rejected(bad):
    u = np.array([0, 1, 1], np.int32)
    v = np.array([0, 0, 1], np.int32)
    s = np.array([1, -1, 1], np.int8)
    if bad == "u_high":
        u[1] = 2
    elif bad == "u_neg":
        u[0] = -1
    elif bad == "v_high":
        v[2] = 2
    elif bad == "sign0":
        s[0] = 0
    else:
        s[2] = 2
    with pytest.raises(ValueError):
        oracle.count(u, v, s, 2, 2)
    with pytest.raises(ValueError):
        oracle.brute_force(u, v, s, 2, 2)


# --------------------------------------------------------------- cross-checks
def test_uniform_2k_3k_20k_three_ways():
    g = synth.workload("uniform-2k-3k-20k")
    bal, unb, wed = oracle.count(g.u, g.v, g.s, g.n_u, g.n_v)
    assert (bal, unb) == oracle.pair_count(g.u, g.v, g.s, g.n_u, g.n_v)
    assert (bal, unb) == oracle.gram_count(g.u, g.v, g.s, g.n_u, g.n_v)
    assert oracle.count(g.u, g.v, g.s, g.n_u, g.n_v, threads=4) == (bal, unb, wed)
    # iid signs with P(+) = 1/2: balanced and unbalanced are equally likely per
    # butterfly, so the split is near one half (loose statistical check).
    assert abs(bal / (bal + unb) - 0.5) < 0.1


@pytest.mark.parametrize("seed", range(3))
def test_gram_identity_on_random_graphs(seed):
    rng = np.random.default_rng(500 + seed)
    u, v, s = _rand_graph(rng, 60, 80, 1500, p_plus=0.7)
    want = oracle.pair_count(u, v, s, 60, 80)
    assert oracle.gram_count(u, v, s, 60, 80) == want
    assert oracle.count(u, v, s, 60, 80)[:2] == want


def test_per_pivot_sums_to_totals():
    rng = np.random.default_rng(11)
    u, v, s = _rand_graph(rng, 40, 50, 700)
    bal, unb, wed = oracle.count(u, v, s, 40, 50)
    b, ub, w = oracle.count_per_pivot(u, v, s, 40, 50, threads=3)
    assert (int(b.sum()), int(ub.sum()), int(w.sum())) == (bal, unb, wed)


# --------------------------------------------------------------- Phase 3 examples
def test_eq1_example1():
    g = read_golden("phase3_examples.txt")
    degs = g["example1_degrees"][0]
    # pivot U0 joined to V0, V1, V2; V_j gets extra neighbours to reach its degree
    edges = []
    nxt = 1
    for j, d in enumerate(degs):
        edges.append((0, j))
        for _ in range(d - 1):
            edges.append((nxt, j))
            nxt += 1
    e = np.array(edges)
    W = oracle.workload_eq1(e[:, 0], e[:, 1], np.ones(len(edges), np.int8), nxt, len(degs))
    assert int(W[0]) == g["example1_workload"][0][0]


def test_lpt_example2():
    g = read_golden("phase3_examples.txt")
    work = g["example2_work"][0]
    P = g["example2_bins"][0][0]
    bins, loads = oracle.lpt(work, P)
    assert sorted(loads.tolist(), reverse=True) == g["example2_greedy_loads"][0]
    naive = [sum(work[i * 2:(i + 1) * 2]) for i in range(P)]
    assert naive == g["example2_naive_loads"][0]
    assert max(loads) / min(loads) == pytest.approx(19 / 16)


# --------------------------------------------------------------- per-vertex counts
@pytest.mark.parametrize("seed", range(6))
def test_per_vertex_matches_brute_force(seed):
    rng = np.random.default_rng(600 + seed)
    n_u, n_v = int(rng.integers(2, 12)), int(rng.integers(2, 12))
    u, v, s = _rand_graph(rng, n_u, n_v, int(rng.integers(1, n_u * n_v + 1)), float(rng.random()))
    b, ub = oracle.count_per_vertex(u, v, s, n_u, n_v)
    bb, bub = oracle.brute_force_per_vertex(u, v, s, n_u, n_v)
    assert np.array_equal(b, bb) and np.array_equal(ub, bub)


@pytest.mark.parametrize("a,b", [(2, 2), (3, 5), (6, 4)])
def test_per_vertex_complete_bipartite(a, b):
    u, v, s = _kab(a, b)
    bal, unb = oracle.count_per_vertex(u, v, s, a, b)
    # a U vertex shares a butterfly with each other U vertex over each pair of V
    assert bal[:a].tolist() == [(a - 1) * math.comb(b, 2)] * a
    assert bal[a:].tolist() == [(b - 1) * math.comb(a, 2)] * b
    assert unb.sum() == 0


def test_per_vertex_sums_to_four_times_the_totals():
    g = synth.workload("uniform-2k-3k-20k")
    bal, unb, _ = oracle.count(g.u, g.v, g.s, g.n_u, g.n_v)
    b, ub = oracle.count_per_vertex(g.u, g.v, g.s, g.n_u, g.n_v)
    assert int(b.sum()) == 4 * bal and int(ub.sum()) == 4 * unb


def test_per_vertex_worked_example():
    g = read_golden("worked_example_k22.txt")
    e = np.array(g["edge"])
    b, ub = oracle.count_per_vertex(e[:, 0], e[:, 1], e[:, 2], 8, 9)
    # the single balanced butterfly {2,7} x {5,8} contains exactly those four vertices
    assert sorted(np.nonzero(b)[0].tolist()) == [2, 7, 8 + 5, 8 + 8] and b.sum() == 4 and ub.sum() == 0


# --------------------------------------------------------------- per-edge counts
@pytest.mark.parametrize("seed", range(6))
def test_per_edge_matches_brute_force(seed):
    rng = np.random.default_rng(700 + seed)
    n_u, n_v = int(rng.integers(2, 12)), int(rng.integers(2, 12))
    u, v, s = _rand_graph(rng, n_u, n_v, int(rng.integers(1, n_u * n_v + 1)), float(rng.random()))
    # queries: every cell of the biadjacency, edges and non-edges alike
    qu, qv = np.meshgrid(np.arange(n_u), np.arange(n_v), indexing="ij")
    b, ub = oracle.count_per_edge(u, v, s, n_u, n_v, qu.ravel(), qv.ravel())
    bb, bub = oracle.brute_force_per_edge(u, v, s, n_u, n_v, qu.ravel(), qv.ravel())
    assert np.array_equal(b, bb) and np.array_equal(ub, bub)


@pytest.mark.parametrize("a,b", [(2, 2), (3, 5), (6, 4)])
def test_per_edge_complete_bipartite(a, b):
    # an edge (u, v) of K(a,b) closes a butterfly with every other u' and v'
    u, v, s = _kab(a, b)
    bal, unb = oracle.count_per_edge(u, v, s, a, b)
    assert bal.tolist() == [(a - 1) * (b - 1)] * (a * b) and unb.sum() == 0


def test_per_edge_sums_to_four_times_the_totals():
    g = synth.workload("uniform-2k-3k-20k")
    bal, unb, _ = oracle.count(g.u, g.v, g.s, g.n_u, g.n_v)
    # one query per distinct pair
    pairs = np.unique(g.u.astype(np.int64) * g.n_v + g.v)
    b, ub = oracle.count_per_edge(g.u, g.v, g.s, g.n_u, g.n_v, pairs // g.n_v, pairs % g.n_v)
    assert int(b.sum()) == 4 * bal and int(ub.sum()) == 4 * unb


def test_per_edge_worked_example_and_non_edges():
    g = read_golden("worked_example_k22.txt")
    e = np.array(g["edge"])
    b, ub = oracle.count_per_edge(e[:, 0], e[:, 1], e[:, 2], 8, 9)
    # the butterfly {2,7} x {5,8}: each of its four edges is in it, no other edge is
    in_bf = np.isin(e[:, 0], [2, 7]) & np.isin(e[:, 1], [5, 8])
    assert b.tolist() == in_bf.astype(int).tolist() and ub.sum() == 0
    b, ub = oracle.count_per_edge(e[:, 0], e[:, 1], e[:, 2], 8, 9, [0, 7], [0, 0])
    assert b.tolist() == [0, 0] and ub.tolist() == [0, 0]


def test_per_edge_repeated_pairs_answer_for_the_kept_edge():
    # K(2,2) whose edge (0,0) is first negative and then positive: the latest
    # sign wins, so the butterfly is balanced and both copies report it
    u, v, s = [0, 0, 0, 1, 1], [0, 0, 1, 0, 1], [-1, 1, 1, 1, 1]
    b, ub = oracle.count_per_edge(u, v, s, 2, 2)
    assert b.tolist() == [1] * 5 and ub.tolist() == [0] * 5
