import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: larger CPU cases")


def read_golden(name):
    """Parse a golden fixture: '#' comments, then 'key value...' lines."""
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, *vals = line.split()
            out.setdefault(key, []).append([int(x) if x.lstrip("-").isdigit() else x for x in vals])
    return out


def pytest_runtest_teardown(item, nextitem):
    """Under the bounds-checked library (the library built with
    -DDBBC_CHECKED=1, loaded through DBBC_LIBRARY), every GPU test must also
    leave no bounds violation recorded by any kernel it ran."""
    if item.get_closest_marker("gpu") is None:
        return
    mod = sys.modules.get("paper_2609_21848_gb300")
    if mod is None or getattr(mod, "_lib", None) is None or not mod.dbbc_is_checked():
        return
    flags = mod.dbbc_checked_flags()
    assert flags == 0, f"{item.nodeid}: a kernel recorded bounds violations (flags {flags:#x})"
