"""The autotuner's coordinate search, on the CPU: `measure` (which needs a GPU)
is replaced by a cost function of the tuning, so the test checks the search
itself: one pass over every coordinate in order, the start point it is given,
never a medium threshold below the light one, and the best point found."""
import pytest

from paper_2609_21848_gb300 import autotune


@pytest.fixture
def fake_measure(monkeypatch):
    seen = []

    def cost(graphs, tuning, repeats=5, stream=None):
        seen.append(dict(tuning))
        # a bowl with its minimum at light = medium = 128, list_density = 64
        c = 10.0
        c += abs(tuning["light_max_work"] - 128) / 64
        c += abs(tuning["medium_max_work"] - 128) / 64
        c += abs(tuning["list_density"] - 64.0) / 32
        return c

    monkeypatch.setattr(autotune, "measure", cost)
    set_calls = []
    import paper_2609_21848_gb300 as dbbc
    monkeypatch.setattr(dbbc, "dbbc_set_tuning", lambda t: set_calls.append(dict(t)))
    return seen, set_calls


def test_search_finds_the_bowl_minimum_from_the_defaults(fake_measure):
    seen, set_calls = fake_measure
    best, ms, base = autotune.tune(graphs=None, log=lambda *a: None)
    assert best["light_max_work"] == 128 and best["medium_max_work"] == 128 and best["list_density"] == 64.0
    assert ms < base
    assert seen[0] == autotune.DEFAULT  # the first point timed is the start
    assert all(t["medium_max_work"] >= t["light_max_work"] for t in seen)
    assert set_calls[-1] == best  # the winner is applied


def test_search_starts_from_a_given_record(fake_measure):
    seen, _ = fake_measure
    start = dict(autotune.DEFAULT, light_max_work=128, medium_max_work=256, list_density=128.0)
    best, ms, base = autotune.tune(graphs=None, log=lambda *a: None, start=start)
    assert seen[0] == start
    assert best["medium_max_work"] == 128 and best["list_density"] == 64.0
    # one pass: every candidate of every coordinate is timed at most once
    assert len(seen) <= 1 + sum(len(c) for _, c in autotune.SPACE)
