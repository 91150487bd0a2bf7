"""Seeded synthetic signed bipartite graphs shared by the oracle tests and the GPU path.

This package draws inputs only; it contains none of the counting arithmetic.
The generator itself is C (``synth.c``, built into ``_build/libsynth.so``);
this module marshals arguments and names the workloads by what they are:

==========================  ===============================================================
workload                    graph
==========================  ===============================================================
``uniform-2k-3k-20k``       |U|=2,000, |V|=3,000, 20,000 distinct uniform edges, P(+)=0.5
``chunglu-1m-200k-20m``     Chung-Lu |U|=1M, |V|=200k, 20M edges, gamma 2.1 / 1.9,
                            expected degree cap 20k, iid P(+)=0.8
``polarized-20m-2m-300m``   Chung-Lu |U|=20M, |V|=2M, 300M edges, gamma 2.0 / 1.8,
                            degree cap 1M, two camps, P(agree with camps)=0.9
``batch-4096``              4,096 graphs, |U|,|V| log-uniform [100, 20k], m log-uniform
                            [500, 200k] capped at |U||V|/2, Chung-Lu gamma 2.2 (cap = other
                            side's size), P(+)=0.6
==========================  ===============================================================

The paper's own datasets (KONECT and other repositories) are not available;
these shapes stand in for them (rating-network-like iid signs, power-law
degrees, a camp model for polarized graphs).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "libsynth.so")
_lib = None

SEED_BASE = 0xDBBC0000


def build(force: bool = False) -> str:
    """Compile ``libsynth.so`` with the host C compiler (portable flags only)."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    src = os.path.join(_HERE, "synth.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", src, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        lib.synth_graph.restype = ctypes.c_int
        lib.synth_graph.argtypes = [
            ctypes.c_uint64, ctypes.c_int, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
            ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
            ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
        ]
        lib.synth_splitmix_raw.restype = ctypes.c_uint64
        lib.synth_splitmix_raw.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.synth_splitmix_at.restype = ctypes.c_uint64
        lib.synth_splitmix_at.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
        lib.synth_chung_lu_weights.restype = ctypes.c_int
        lib.synth_chung_lu_weights.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_void_p]
        lib.synth_batch_sizes.restype = None
        lib.synth_batch_sizes.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)]
        _lib = lib
    return _lib


def default_threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


@dataclass
class Graph:
    """COO signed bipartite graph: u in [0, n_u), v in [0, n_v), s in {+1, -1}."""
    u: np.ndarray
    v: np.ndarray
    s: np.ndarray
    n_u: int
    n_v: int
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.u.shape[0])


def splitmix_raw(state: int, k: int) -> int:
    return int(_load().synth_splitmix_raw(state, k))


def splitmix_at(seed: int, stream: int, k: int) -> int:
    return int(_load().synth_splitmix_at(seed, stream, k))


def chung_lu_weights(n: int, gamma: float, m: float, cap: float) -> np.ndarray:
    d = np.empty(n, dtype=np.float64)
    rc = _load().synth_chung_lu_weights(n, gamma, m, cap, d.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"synth_chung_lu_weights failed: {rc}")
    return d


def generate(seed: int, n_u: int, n_v: int, m: int, model: str = "uniform", gamma_u: float = 2.0,
             gamma_v: float = 2.0, cap_u: float | None = None, cap_v: float | None = None,
             signs: str = "iid", p_plus: float = 0.5, p_camp: float = 0.9, threads: int | None = None,
             name: str = "") -> Graph:
    """Draw one graph. ``cap_u`` caps the expected degree of U vertices (at most |V|)."""
    lib = _load()
    u = np.empty(m, dtype=np.int32)
    v = np.empty(m, dtype=np.int32)
    s = np.empty(m, dtype=np.int8)
    cu = float(min(cap_u if cap_u is not None else n_v, n_v))
    cv = float(min(cap_v if cap_v is not None else n_u, n_u))
    rc = lib.synth_graph(seed, 0 if model == "uniform" else 1, n_u, n_v, m, gamma_u, gamma_v, cu, cv,
                         0 if signs == "iid" else 1, p_plus, p_camp, threads or default_threads(),
                         u.ctypes.data, v.ctypes.data, s.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"synth_graph failed with code {rc}")
    return Graph(u, v, s, n_u, n_v, name)


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------
WORKLOADS = {
    "uniform-2k-3k-20k": dict(index=0, n_u=2_000, n_v=3_000, m=20_000, model="uniform", signs="iid", p_plus=0.5),
    "chunglu-1m-200k-20m": dict(index=1, n_u=1_000_000, n_v=200_000, m=20_000_000, model="chung-lu",
                                gamma_u=2.1, gamma_v=1.9, cap_u=20_000, cap_v=20_000, signs="iid", p_plus=0.8),
    "polarized-20m-2m-300m": dict(index=2, n_u=20_000_000, n_v=2_000_000, m=300_000_000, model="chung-lu",
                                  gamma_u=2.0, gamma_v=1.8, cap_u=1_000_000, cap_v=1_000_000, signs="camp",
                                  p_camp=0.9),
}
BATCH = dict(index=3, n_graphs=4096, lo_n=100, hi_n=20_000, lo_m=500, hi_m=200_000, gamma=2.2, p_plus=0.6)


def workload(name: str, threads: int | None = None, scale: float = 1.0) -> Graph:
    """One named single-graph workload. ``scale`` < 1 shrinks |U|, |V| and m together
    (same shape, used for quick tests); ``scale=1`` is the full size."""
    p = dict(WORKLOADS[name])
    idx = p.pop("index")
    if scale != 1.0:
        p["n_u"] = max(4, int(p["n_u"] * scale))
        p["n_v"] = max(4, int(p["n_v"] * scale))
        p["m"] = max(1, int(p["m"] * scale))
        for k in ("cap_u", "cap_v"):
            if k in p:
                p[k] = max(2.0, p[k] * scale)
    return generate(SEED_BASE + idx, threads=threads, name=name, **p)


def batch_sizes(g: int, seed: int = SEED_BASE + 3) -> tuple[int, int, int]:
    lib = _load()
    nu, nv, m = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    b = BATCH
    lib.synth_batch_sizes(seed, g, b["lo_n"], b["hi_n"], b["lo_m"], b["hi_m"], ctypes.byref(nu),
                          ctypes.byref(nv), ctypes.byref(m))
    return nu.value, nv.value, m.value


def batch_graph(g: int, seed: int = SEED_BASE + 3, threads: int = 1) -> Graph:
    """Graph ``g`` of the batched workload (4,096 uneven Chung-Lu graphs)."""
    nu, nv, m = batch_sizes(g, seed)
    b = BATCH
    return generate(seed * 65537 + g, nu, nv, m, model="chung-lu", gamma_u=b["gamma"], gamma_v=b["gamma"],
                    cap_u=nv, cap_v=nu, signs="iid", p_plus=b["p_plus"], threads=threads, name=f"batch[{g}]")


SERVE = dict(index=4, rate=2000.0, n_requests=100_000, large_fraction=0.01, large_lo=5_000_000,
             large_hi=20_000_000, avg_degree=13.6)


def serve_large_graph(i: int, seed: int = SEED_BASE + 4, threads: int | None = None) -> Graph:
    """Large request i of the served stream: a polarized Chung-Lu graph like the
    300M-edge one (gamma 2.0 / 1.8, camp signs), m log-uniform in [5M, 20M],
    |U| + |V| = m / 13.6 (that graph's average degree), |U| = |V| / 4."""
    key = splitmix_at(seed, 0x2000 + i, 0)
    lo, hi = np.log(SERVE["large_lo"]), np.log(SERVE["large_hi"])
    m = int(round(np.exp(lo + (hi - lo) * ((key >> 11) / 2.0**53))))
    n = int(m / SERVE["avg_degree"])
    n_u, n_v = n // 5, n - n // 5
    return generate(seed * 131 + i, n_u, n_v, m, model="chung-lu", gamma_u=2.0, gamma_v=1.8,
                    cap_u=min(1_000_000, n_v), cap_v=min(1_000_000, n_u), signs="camp", p_camp=0.9,
                    threads=threads, name=f"serve-large[{i}]")


def serve_is_large(i: int, seed: int = SEED_BASE + 4) -> bool:
    """Whether request i of the served stream is a large one (1% of requests)."""
    return (splitmix_at(seed, 0x3000, i) >> 11) / 2.0**53 < SERVE["large_fraction"]


def batch(n_graphs: int = 4096, seed: int = SEED_BASE + 3, threads: int | None = None) -> list[Graph]:
    from concurrent.futures import ThreadPoolExecutor
    nt = threads or default_threads()
    with ThreadPoolExecutor(max_workers=nt) as ex:
        return list(ex.map(lambda g: batch_graph(g, seed, 1), range(n_graphs)))
