"""CPU oracle for balanced / unbalanced butterfly counts. TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The product path (the CUDA library and
its binding) never does, and shares no code with it.

Functions and the passages they follow (paper: "Distributed Balanced Butterfly
Counting in Signed Bipartite Graphs"):

* :func:`count` / :func:`count_per_pivot` -- Algorithm 1, Phase 5 (Section IV-A)
  with the Def. 3 vertex priority, plus the unbalanced count from Lemma 1,
  case 3. Plain serial C++ (``dbbc_oracle.cpp``); ``threads > 1`` splits the
  pivots across host threads with private buckets, as Phase 5 does with TBB.
* :func:`brute_force` -- Def. 1 and Def. 2 enumerated over all
  {u1,u2} x {v1,v2} (C++, dense sign matrix, tiny graphs only).
* :func:`pair_count` -- the textbook wedge-pair count with no vertex priority:
  for every pair u1 < u2, p = common neighbours with equal signs, q = with
  unequal signs; balanced += C(p,2) + C(q,2), unbalanced += p*q (Lemma 1).
  Pure Python, shares no code with the C++.
* :func:`gram_count` -- the same totals by linear algebra: with S the signed
  biadjacency (+1/-1/0) and A = |S|, for i < j, (AA^T)_ij = p + q and
  (SS^T)_ij = p - q, so balanced + unbalanced = sum C((AA^T)_ij, 2) and
  balanced - unbalanced = sum ((SS^T)_ij^2 - (AA^T)_ij) / 2.
* :func:`count_per_vertex` -- butterflies containing each vertex (the "tip"
  input of the paper's applications), Algorithm 1 plus a second walk of each
  pivot's wedges for the middle vertices; :func:`brute_force_per_vertex`
  enumerates Def. 1-2 for the same numbers.
* :func:`count_per_edge` -- butterflies containing each queried edge (the
  "wing" input), Algorithm 1 with the same second walk crediting both edges of
  every wedge; :func:`brute_force_per_edge` enumerates Def. 1-2 for them.
* :func:`workload_eq1` -- Eq. (1) of Phase 3; :func:`lpt` -- the Phase 3 greedy
  bin packing of Example 2.

Duplicates keep the latest occurrence (Section V, dataset preprocessing); ids
outside [0, |U|) x [0, |V|) or signs other than +1 / -1 raise ``ValueError``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

OK, BAD_INPUT, OVERFLOW_64 = 0, 1, 5


def build(force: bool = False) -> str:
    """Compile the C++ oracle with the host compiler (no GPU, portable flags)."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    src = os.path.join(_HERE, "dbbc_oracle.cpp")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        extra = os.environ.get("DBBC_ORACLE_CFLAGS", "").split()
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", *extra, src, "-o", tmp])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        graph_args = [P, P, P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32]
        lib.oracle_count.argtypes = graph_args + [ctypes.c_int, P, P, P]
        lib.oracle_count_per_pivot.argtypes = graph_args + [ctypes.c_int, P, P, P]
        lib.oracle_brute_force.argtypes = graph_args + [P, P]
        lib.oracle_workload_eq1.argtypes = graph_args + [P]
        lib.oracle_lpt.argtypes = [P, ctypes.c_int64, ctypes.c_int32, P, P]
        lib.oracle_count_per_vertex.argtypes = graph_args + [P, P]
        lib.oracle_count_per_vertex.restype = ctypes.c_int
        lib.oracle_brute_force_per_vertex.argtypes = graph_args + [P, P]
        lib.oracle_brute_force_per_vertex.restype = ctypes.c_int
        lib.oracle_count_per_edge.argtypes = graph_args + [P, P, ctypes.c_int64, P, P]
        lib.oracle_count_per_edge.restype = ctypes.c_int
        lib.oracle_brute_force_per_edge.argtypes = graph_args + [P, P, ctypes.c_int64, P, P]
        lib.oracle_brute_force_per_edge.restype = ctypes.c_int
        lib.oracle_graph_new.argtypes = graph_args + [ctypes.POINTER(ctypes.c_int)]
        lib.oracle_graph_new.restype = P
        lib.oracle_graph_count_sample.argtypes = [P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, P, P, P]
        lib.oracle_graph_count_sample.restype = ctypes.c_int
        lib.oracle_graph_free.argtypes = [P]
        lib.oracle_graph_free.restype = None
        for f in (lib.oracle_count, lib.oracle_count_per_pivot, lib.oracle_brute_force, lib.oracle_workload_eq1,
                  lib.oracle_lpt):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _coo(u, v, s):
    u = np.ascontiguousarray(u, dtype=np.int32)
    v = np.ascontiguousarray(v, dtype=np.int32)
    s = np.ascontiguousarray(s, dtype=np.int8)
    if not (u.shape == v.shape == s.shape) or u.ndim != 1:
        raise ValueError("u, v, s must be 1-D arrays of equal length")
    return u, v, s


def _check(rc: int):
    if rc == BAD_INPUT:
        raise ValueError("invalid signed bipartite graph (id out of range or sign not +1/-1)")
    if rc == OVERFLOW_64:
        raise OverflowError("count does not fit in 64 bits")
    if rc != OK:
        raise RuntimeError(f"oracle error {rc}")


def count(u, v, s, n_u: int, n_v: int, threads: int = 1) -> tuple[int, int, int]:
    """(balanced, unbalanced, accepted wedges) by Algorithm 1."""
    u, v, s = _coo(u, v, s)
    out = (ctypes.c_uint64 * 3)()
    rc = _load().oracle_count(u.ctypes.data, v.ctypes.data, s.ctypes.data, u.shape[0], n_u, n_v, threads,
                              ctypes.addressof(out), ctypes.addressof(out) + 8, ctypes.addressof(out) + 16)
    _check(rc)
    return int(out[0]), int(out[1]), int(out[2])


def count_per_pivot(u, v, s, n_u: int, n_v: int, threads: int = 1):
    """Per-pivot (balanced, unbalanced, wedges) arrays over unified ids
    (u -> u, v -> n_u + v)."""
    u, v, s = _coo(u, v, s)
    n = n_u + n_v
    b = np.zeros(n, np.uint64)
    ub = np.zeros(n, np.uint64)
    w = np.zeros(n, np.uint64)
    rc = _load().oracle_count_per_pivot(u.ctypes.data, v.ctypes.data, s.ctypes.data, u.shape[0], n_u, n_v,
                                        threads, b.ctypes.data, ub.ctypes.data, w.ctypes.data)
    _check(rc)
    return b, ub, w


def count_per_vertex(u, v, s, n_u: int, n_v: int):
    """Balanced and unbalanced butterflies containing each vertex (arrays over
    unified ids u -> u, v -> n_u + v), following Algorithm 1 with a second
    walk of each pivot's wedges for the middle vertices."""
    u, v, s = _coo(u, v, s)
    b = np.zeros(n_u + n_v, np.uint64)
    ub = np.zeros(n_u + n_v, np.uint64)
    _check(_load().oracle_count_per_vertex(u.ctypes.data, v.ctypes.data, s.ctypes.data, u.shape[0], n_u, n_v,
                                           b.ctypes.data, ub.ctypes.data))
    return b, ub


def brute_force_per_vertex(u, v, s, n_u: int, n_v: int):
    """Per-vertex counts by enumerating Def. 1-2 directly (tiny graphs)."""
    u, v, s = _coo(u, v, s)
    b = np.zeros(n_u + n_v, np.uint64)
    ub = np.zeros(n_u + n_v, np.uint64)
    _check(_load().oracle_brute_force_per_vertex(u.ctypes.data, v.ctypes.data, s.ctypes.data, u.shape[0], n_u,
                                                 n_v, b.ctypes.data, ub.ctypes.data))
    return b, ub


def _per_edge(fn, u, v, s, n_u, n_v, qu, qv):
    u, v, s = _coo(u, v, s)
    if qu is None:
        qu, qv = u, v
    qu = np.ascontiguousarray(qu, dtype=np.int32)
    qv = np.ascontiguousarray(qv, dtype=np.int32)
    if qu.shape != qv.shape:
        raise ValueError("qu and qv differ in length")
    b = np.zeros(max(qu.shape[0], 1), np.uint64)
    ub = np.zeros(max(qu.shape[0], 1), np.uint64)
    _check(fn(u.ctypes.data, v.ctypes.data, s.ctypes.data, u.shape[0], n_u, n_v, qu.ctypes.data, qv.ctypes.data,
              qu.shape[0], b.ctypes.data, ub.ctypes.data))
    return b[:qu.shape[0]], ub[:qu.shape[0]]


def count_per_edge(u, v, s, n_u: int, n_v: int, qu=None, qv=None):
    """Balanced and unbalanced butterflies containing each queried pair
    (qu[i], qv[i]) (default: the input edges, a repeated pair answering for the
    edge it became); a pair that is not an edge gets zeros. Algorithm 1 with a
    second walk crediting both edges of every wedge."""
    return _per_edge(_load().oracle_count_per_edge, u, v, s, n_u, n_v, qu, qv)


def brute_force_per_edge(u, v, s, n_u: int, n_v: int, qu=None, qv=None):
    """Per-edge counts by enumerating Def. 1-2 directly (tiny graphs)."""
    return _per_edge(_load().oracle_brute_force_per_edge, u, v, s, n_u, n_v, qu, qv)


class BuiltGraph:
    """A graph built once by the oracle and counted on pivot samples (for
    timing Algorithm 1 alone). Pivots are unified ids first, first+step, ..."""

    def __init__(self, u, v, s, n_u: int, n_v: int):
        u, v, s = _coo(u, v, s)
        st = ctypes.c_int(0)
        self._h = _load().oracle_graph_new(u.ctypes.data, v.ctypes.data, s.ctypes.data, u.shape[0], n_u, n_v,
                                           ctypes.byref(st))
        _check(st.value)
        self.n = n_u + n_v

    def count_sample(self, first: int = 0, step: int = 1, threads: int = 1) -> tuple[int, int, int]:
        out = (ctypes.c_uint64 * 3)()
        base = ctypes.addressof(out)
        _check(_load().oracle_graph_count_sample(self._h, first, step, threads, base, base + 8, base + 16))
        return int(out[0]), int(out[1]), int(out[2])

    def close(self):
        if self._h:
            _load().oracle_graph_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def brute_force(u, v, s, n_u: int, n_v: int) -> tuple[int, int]:
    """(balanced, unbalanced) by enumerating Def. 1-2 directly (tiny graphs)."""
    u, v, s = _coo(u, v, s)
    out = (ctypes.c_uint64 * 2)()
    rc = _load().oracle_brute_force(u.ctypes.data, v.ctypes.data, s.ctypes.data, u.shape[0], n_u, n_v,
                                    ctypes.addressof(out), ctypes.addressof(out) + 8)
    _check(rc)
    return int(out[0]), int(out[1])


def workload_eq1(u, v, s, n_u: int, n_v: int) -> np.ndarray:
    """Eq. (1): W(x) = sum over neighbours y of d(y), per unified id."""
    u, v, s = _coo(u, v, s)
    W = np.zeros(n_u + n_v, np.uint64)
    _check(_load().oracle_workload_eq1(u.ctypes.data, v.ctypes.data, s.ctypes.data, u.shape[0], n_u, n_v,
                                       W.ctypes.data))
    return W


def lpt(work, n_bins: int) -> tuple[np.ndarray, np.ndarray]:
    """Phase 3 greedy bin packing: (bin of every item, load of every bin)."""
    work = np.ascontiguousarray(work, dtype=np.uint64)
    bins = np.zeros(work.shape[0], np.int32)
    loads = np.zeros(n_bins, np.uint64)
    _check(_load().oracle_lpt(work.ctypes.data, work.shape[0], n_bins, bins.ctypes.data, loads.ctypes.data))
    return bins, loads


# ---------------------------------------------------------------------------
# Independent cross-checks in Python (no shared code with the C++ above)
# ---------------------------------------------------------------------------
def _latest_signs(u, v, s, n_u, n_v) -> dict:
    latest = {}
    for a, b, c in zip(np.asarray(u).tolist(), np.asarray(v).tolist(), np.asarray(s).tolist()):
        if not (0 <= a < n_u and 0 <= b < n_v) or c not in (1, -1):
            raise ValueError("invalid signed bipartite graph")
        latest[(a, b)] = c
    return latest


def pair_count(u, v, s, n_u: int, n_v: int) -> tuple[int, int]:
    """Wedge-pair count over unordered pairs u1 < u2 (no vertex priority)."""
    latest = _latest_signs(u, v, s, n_u, n_v)
    by_v: dict[int, list] = {}
    for (a, b), c in latest.items():
        by_v.setdefault(b, []).append((a, c))
    same: dict = {}
    diff: dict = {}
    for nbrs in by_v.values():
        nbrs.sort()
        for i in range(len(nbrs)):
            a, ca = nbrs[i]
            for j in range(i + 1, len(nbrs)):
                b, cb = nbrs[j]
                if ca == cb:
                    same[(a, b)] = same.get((a, b), 0) + 1
                else:
                    diff[(a, b)] = diff.get((a, b), 0) + 1
    bal = unb = 0
    for key in set(same) | set(diff):
        p, q = same.get(key, 0), diff.get(key, 0)
        bal += p * (p - 1) // 2 + q * (q - 1) // 2
        unb += p * q
    return bal, unb


def gram_count(u, v, s, n_u: int, n_v: int) -> tuple[int, int]:
    """Totals from the Gram matrices of the signed and unsigned biadjacency."""
    latest = _latest_signs(u, v, s, n_u, n_v)
    S = np.zeros((n_u, n_v), dtype=np.float64)
    for (a, b), c in latest.items():
        S[a, b] = c
    A = np.abs(S)
    G = A @ A.T  # p + q per pair (exact: small integers in float64)
    H = S @ S.T  # p - q per pair
    iu = np.triu_indices(n_u, k=1)
    g = np.rint(G[iu]).astype(np.int64)
    h = np.rint(H[iu]).astype(np.int64)
    total = int((g * (g - 1) // 2).sum())
    diff = int(((h * h - g) // 2).sum())
    return (total + diff) // 2, (total - diff) // 2
