"""Host-side helpers of bench.py (no GPU): stored counts, the traffic record
keyed by the kernel sources' hash, measured peaks, and the argument defaults
the benchmark contract relies on."""
import importlib.util
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_expected_counts_are_read_from_the_golden_file():
    b = load_bench()
    assert b.expected_counts("uniform-2k-3k-20k") == (577, 515, 81835)
    assert b.expected_counts("no-such-workload") is None


def test_traffic_record_is_keyed_by_the_kernel_sources():
    b = load_bench()
    sha = b.kernel_source_sha()
    assert len(sha) == 12 and all(ch in "0123456789abcdef" for ch in sha)
    rows = [line.split() for line in open(os.path.join(ROOT, "profiles", "traffic.txt"))
            if line.strip() and not line.startswith("#")]
    assert rows and all(len(r) == 4 and int(r[3]) > 0 for r in rows)
    # a record whose hash is not the current sources' is not reported
    assert b.known_traffic("hub_sweep_kernel", "no-such-workload") is None


def test_measured_peaks_are_used():
    """The peak file written for this machine pool is used when present;
    without it the bench falls back to the earlier GB300 measurement and says so."""
    b = load_bench()
    peaks, kind = b.measured_peaks()
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        assert kind == "measured" and float(peaks["hbm_gbs"]) > 1000
    else:
        assert kind == "fallback" and peaks["hbm_gbs"] == 6800.0


def test_default_arguments_keep_the_contract(monkeypatch):
    b = load_bench()
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = b.parse()
    assert a.gpus == 1 and a.warmup >= 3 and a.steps >= 1 and a.impl == "dbbc"
    # the headline is the largest single graph, with the batched and served records attached
    assert a.workload == "polarized-20m-2m-300m" and a.scale == 1.0 and not a.no_extras
    assert a.requests == 100_000 and a.large_pool >= 16


def run_reference_arm(extra_env=None):
    import json
    import subprocess
    env = dict(os.environ, **(extra_env or {}))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "uniform-2k-3k-20k", "--steps", "2", "--warmup", "1", "--reference-seconds", "3"],
                       capture_output=True, text=True, env=env, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [line for line in r.stdout.splitlines() if line.startswith("{")]
    return [json.loads(line) for line in lines]


def test_reference_arm_prints_one_contract_line():
    """The reference arm times the oracle on the host cores and prints one
    JSON line with the keys the benchmark contract asks of it."""
    (line,) = run_reference_arm()
    assert line["impl"] == "reference" and line["unit"] == "G wedges/s" and line["value"] > 0
    assert line["steps"] == 2 and line["warmup"] == 1 and line["higher_is_better"] is True
    assert line["config"]["workload"] == "uniform-2k-3k-20k"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_runs_on_rank_zero_only():
    assert run_reference_arm({"RANK": "1", "WORLD_SIZE": "2"}) == []
