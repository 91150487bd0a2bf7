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
    b = load_bench()
    peaks, kind = b.measured_peaks()
    assert kind == "measured" and float(peaks["hbm_gbs"]) > 1000


def test_default_arguments_keep_the_contract(monkeypatch):
    b = load_bench()
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = b.parse()
    assert a.gpus == 1 and a.warmup >= 3 and a.steps >= 1 and a.impl == "dbbc"
    assert a.workload == "chunglu-1m-200k-20m" and a.scale == 1.0
