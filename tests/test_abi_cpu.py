"""The C-ABI library builds for sm_103a, loads on a machine without a GPU and
exports every entry point that include/dbbc.h declares. Only calls that touch
no CUDA state are made here (argument checks, strings, size estimates)."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2609_21848_gb300 as dbbc
from paper_2609_21848_gb300 import buildlib

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "dbbc.h")


@pytest.fixture(scope="module")
def lib():
    buildlib.build()
    return dbbc.lib()


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^DBBC_API [^(]*?\b(dbbc_\w+)\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for want in ("dbbc_graph_from_coo", "dbbc_count", "dbbc_count_batch", "dbbc_count_batch_async",
                 "dbbc_graph_device_bytes", "dbbc_estimate_bytes", "dbbc_graph_free", "dbbc_set_allocator",
                 "dbbc_status_string"):
        assert want in names
    assert set(names) == set(dbbc.EXPORTED)


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", dbbc.LIB_PATH], capture_output=True, text=True, check=True)
    exported = set(re.findall(r"\bT (dbbc_\w+)", out.stdout))
    for name in declared_symbols():
        assert name in exported, name
        assert hasattr(lib, name)


def test_status_strings_and_version(lib):
    assert dbbc.dbbc_status_string(dbbc.DBBC_OK) == "ok"
    for code in range(1, 7):
        assert dbbc.dbbc_status_string(code) not in ("", "ok", "unknown status")
    assert dbbc.dbbc_status_string(99) == "unknown status"
    assert re.fullmatch(r"\d+\.\d+\.\d+", dbbc.dbbc_version())


def test_argument_errors_need_no_gpu(lib):
    h = ctypes.c_void_p()
    L = dbbc.lib()
    assert L.dbbc_graph_from_coo(None, None, None, -1, 2, 2, 0, None, ctypes.byref(h)) == dbbc.DBBC_EINVAL
    assert L.dbbc_graph_from_coo(None, None, None, 5, 2, 2, 0, None, ctypes.byref(h)) == dbbc.DBBC_EINVAL
    assert L.dbbc_graph_from_coo(None, None, None, 0, -1, 2, 0, None, ctypes.byref(h)) == dbbc.DBBC_EINVAL
    assert L.dbbc_graph_from_coo(None, None, None, 0, 2, 2, 0x10, None, ctypes.byref(h)) == dbbc.DBBC_EINVAL
    assert L.dbbc_graph_from_coo(None, None, None, 0, 2, 2, 0, None, None) == dbbc.DBBC_EINVAL
    assert L.dbbc_graph_from_coo(None, None, None, 1 << 31, 2, 2, 0, None, ctypes.byref(h)) == dbbc.DBBC_EINVAL
    assert L.dbbc_count(None, None, None, None) == dbbc.DBBC_EINVAL
    assert L.dbbc_count_async(None, None, None) == dbbc.DBBC_EINVAL
    assert L.dbbc_count_vertices(None, None, None, None) == dbbc.DBBC_EINVAL
    assert L.dbbc_count_edges(None, None, None, None, 0, 0, None, None) == dbbc.DBBC_EINVAL
    assert L.dbbc_count_batch(None, -1, None, None, None) == dbbc.DBBC_EINVAL
    assert L.dbbc_graph_get_info(None, None) == dbbc.DBBC_EINVAL
    assert L.dbbc_graph_export(None, None, None, None, None, None, None) == dbbc.DBBC_EINVAL
    assert L.dbbc_graph_device_bytes(None) == 0
    L.dbbc_graph_free(None)


def test_estimate_bytes_grows_with_size(lib):
    a = dbbc.dbbc_estimate_bytes(1_000, 100, 100)
    b = dbbc.dbbc_estimate_bytes(1_000_000, 100_000, 100_000)
    assert 0 < a < b
    assert dbbc.dbbc_estimate_bytes(-1, 1, 1) == 0


def test_tuning_round_trip_and_validation(lib):
    base = dbbc.dbbc_get_tuning()
    try:
        t = dict(light_max_work=128, medium_max_work=2048, hub_item_work=1 << 19,
                 group_density=[64.0, 24.0, 8.0, 3.0], hash_mult_log=2, list_density=12.0, list_group_log=4,
                 finalize_window_wedges=1 << 17, list_wide_density=24.0)
        dbbc.dbbc_set_tuning(t)
        assert dbbc.dbbc_get_tuning() == t
        for bad in (dict(t, light_max_work=0), dict(t, light_max_work=1024), dict(t, medium_max_work=64),
                    dict(t, medium_max_work=8192), dict(t, hub_item_work=10), dict(t, hash_mult_log=0),
                    dict(t, hash_mult_log=4), dict(t, group_density=[1.0, 2.0, 3.0, 4.0]),
                    dict(t, list_density=-1.0), dict(t, list_group_log=1), dict(t, list_group_log=6),
                    dict(t, list_wide_density=-1.0)):
            with pytest.raises(dbbc.DbbcError):
                dbbc.dbbc_set_tuning(bad)
        assert dbbc.dbbc_get_tuning() == t  # rejected settings change nothing
        dbbc.dbbc_set_tuning({"hash_mult_log": 3})  # keys left out keep their values
        assert dbbc.dbbc_get_tuning() == dict(t, hash_mult_log=3)
        dbbc.dbbc_set_tuning(None)
        from paper_2609_21848_gb300 import autotune
        assert dbbc.dbbc_get_tuning() == autotune.DEFAULT
    finally:
        dbbc.dbbc_set_tuning(base)


def test_tuning_reads_are_whole_under_concurrent_sets(lib):
    """Threads that set and read the tuning at once (as the serving loop's
    builder threads may) only ever read one of the settings some thread set."""
    import threading
    base = dbbc.dbbc_get_tuning()
    a = dict(light_max_work=128, medium_max_work=1024, hub_item_work=1 << 19,
             group_density=[40.0, 16.0, 6.0, 2.0], hash_mult_log=1, list_density=4.0, list_group_log=2,
             finalize_window_wedges=0, list_wide_density=32.0)
    b = dict(light_max_work=512, medium_max_work=4096, hub_item_work=1 << 22,
             group_density=[128.0, 48.0, 12.0, 4.0], hash_mult_log=3, list_density=32.0, list_group_log=5,
             finalize_window_wedges=2**64 - 1, list_wide_density=1e30)
    seen, errors = [], []

    def writer(t):
        try:
            for _ in range(2000):
                dbbc.dbbc_set_tuning(t)  # every key given: nothing merged from the current values
        except Exception as e:  # pragma: no cover - reported below
            errors.append(e)

    def reader():
        for _ in range(2000):
            seen.append(dbbc.dbbc_get_tuning())

    try:
        threads = [threading.Thread(target=writer, args=(t,)) for t in (a, b)] + [threading.Thread(target=reader)]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
        assert not errors
        assert all(r in (a, b, base) for r in seen)
    finally:
        dbbc.dbbc_set_tuning(base)


def test_timeout_status_is_reserved():
    """DBBC_ETIMEOUT is reserved: no kernel of the library waits on a flag, a
    peer or a barrier that another launch sets, so no call returns it."""
    text = open(HEADER).read()
    assert "reserved" in text.split("DBBC_ETIMEOUT = 4,", 1)[1].split("\n", 1)[0]
    assert dbbc.dbbc_status_string(4) == "bounded device wait gave up"


def test_regular_build_is_not_checked(lib):
    """The regular library checks no index in its kernels, reports so, and
    its check-flag query needs no GPU (it returns 0 without synchronizing)."""
    if dbbc.dbbc_is_checked():
        pytest.skip("DBBC_LIBRARY names the checked build")
    assert lib.dbbc_is_checked() == 0
    assert dbbc.dbbc_checked_flags() == 0
    assert lib.dbbc_checked_flags(None) == dbbc.DBBC_EINVAL


def test_checked_build_flags_are_separate():
    """The checked build goes to its own folder with its own flag stamp, so it
    never replaces the regular library."""
    assert os.path.dirname(os.path.join(buildlib.CHECKED_DIR, "libdbbc.so")) != os.path.dirname(buildlib.LIB)
    assert buildlib.CHECKED_FLAGS == ["-DDBBC_CHECKED=1"]
    assert not buildlib.up_to_date(buildlib.LIB, buildlib.CHECKED_FLAGS)
