"""The seeded input generator: reproducible, thread-count independent, distinct
in-range edges of the requested shape."""
import numpy as np
import pytest

import synth

M64 = (1 << 64) - 1


def _splitmix64_sequence(x, n):
    """SplitMix64 as published (Steele, Lea and Flood 2014), written out in Python."""
    out = []
    for _ in range(n):
        x = (x + 0x9E3779B97F4A7C15) & M64
        z = x
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
        out.append(z ^ (z >> 31))
    return out


def test_splitmix_matches_definition():
    for state in (0, 1234567, 0xDBBC0003):
        seq = _splitmix64_sequence(state, 6)
        assert [synth.splitmix_raw(state, k) for k in range(6)] == seq
    # published first outputs for state 1234567
    assert _splitmix64_sequence(1234567, 2) == [6457827717110365317, 3203168211198807973]


def test_uniform_workload_shape_and_determinism():
    g = synth.workload("uniform-2k-3k-20k")
    assert g.m == 20_000 and g.n_u == 2_000 and g.n_v == 3_000
    assert g.u.min() >= 0 and g.u.max() < 2_000 and g.v.min() >= 0 and g.v.max() < 3_000
    assert np.unique(g.u.astype(np.int64) * 3_000 + g.v).size == g.m
    assert set(np.unique(g.s).tolist()) == {-1, 1}
    assert abs((g.s == 1).mean() - 0.5) < 0.02
    g1 = synth.generate(synth.SEED_BASE, 2_000, 3_000, 20_000, threads=1)
    g4 = synth.generate(synth.SEED_BASE, 2_000, 3_000, 20_000, threads=4)
    for a, b in ((g.u, g1.u), (g.v, g1.v), (g.s, g1.s), (g1.u, g4.u), (g1.v, g4.v), (g1.s, g4.s)):
        assert np.array_equal(a, b)


def test_chung_lu_weights_sum_and_cap():
    d = synth.chung_lu_weights(100_000, 1.9, 2e6, 5_000.0)
    assert d.sum() == pytest.approx(2e6, rel=1e-9)
    assert d.max() <= 5_000.0 + 1e-6
    assert np.all(np.diff(d) <= 1e-9)


def test_chung_lu_small_is_power_law_like():
    g = synth.generate(synth.SEED_BASE + 1, 20_000, 4_000, 200_000, model="chung-lu", gamma_u=2.1, gamma_v=1.9,
                       cap_u=2_000, cap_v=2_000, signs="iid", p_plus=0.8)
    assert np.unique(g.u.astype(np.int64) * g.n_v + g.v).size == g.m
    dv = np.bincount(g.v, minlength=g.n_v)
    assert dv.max() > 20 * dv.mean()  # heavy tail
    assert abs((g.s == 1).mean() - 0.8) < 0.02


def test_camp_signs_agree_with_camps():
    g = synth.workload("polarized-20m-2m-300m", scale=0.0005)
    assert np.unique(g.u.astype(np.int64) * g.n_v + g.v).size == g.m
    assert abs((g.s == 1).mean() - 0.5) < 0.05


def test_batch_sizes_in_range():
    for i in range(64):
        nu, nv, m = synth.batch_sizes(i)
        assert 100 <= nu <= 20_000 and 100 <= nv <= 20_000
        assert 1 <= m <= max(500, 200_000) and m <= nu * nv // 2
    g = synth.batch_graph(5)
    assert np.unique(g.u.astype(np.int64) * g.n_v + g.v).size == g.m


def test_empty_graph():
    g = synth.generate(1, 10, 10, 0)
    assert g.m == 0


@pytest.mark.timeout(60)
def test_small_graph_with_large_sides_terminates():
    # m far below the side sizes: the first insertion window must not
    # overfill the first-occurrence set (it used to probe forever)
    g = synth.batch_graph(144)
    assert (g.n_u, g.n_v, g.m) == (16158, 394, 1001)
    assert np.unique(g.u.astype(np.int64) * g.n_v + g.v).size == g.m
    g = synth.generate(7, 20_000, 20_000, 10, model="chung-lu", gamma_u=2.2, gamma_v=2.2)
    assert g.m == 10


def test_whole_batch_generates():
    gs = synth.batch(256)
    assert len(gs) == 256 and all(g.m > 0 for g in gs)
