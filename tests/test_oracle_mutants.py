"""The oracle's pins must catch plausible mistakes. Each case copies the oracle
source, plants one mistake in the copy (on the CPU), builds it, and checks that
at least one pin fails against the planted copy. The real oracle is untouched."""
import ctypes
import math
import os
import subprocess

import numpy as np
import pytest

import oracle

SRC = os.path.join(os.path.dirname(oracle.__file__), "dbbc_oracle.cpp")

MUTANTS = {
    # (swapping the two classes outright is not a mistake: both totals are
    # symmetric in B1 and B2)
    "class from one edge's sign": ("if (uv.second == vw.second) B1[w]++; else B2[w]++;",
                                   "if (vw.second > 0) B1[w]++; else B2[w]++;"),
    "tie-break dropped": ("  return a < b;\n}", "  return false;\n}"),
    "middle not filtered": ("if (!lower_priority(g, v, u)) continue;", ""),
    "endpoint compared with middle": ("if (!lower_priority(g, w, u)) continue;",
                                      "if (!lower_priority(g, w, v)) continue;"),
    "unbalanced uses p*p": ("unb += static_cast<u128>(B1[w]) * B2[w];", "unb += static_cast<u128>(B1[w]) * B1[w];"),
    "choose2 off by one": ("x * (x - 1) / 2", "x * (x + 1) / 2"),
    "asymmetric term dropped": ("bal += choose2(B1[w]) + choose2(B2[w]);", "bal += choose2(B1[w]);"),
    "keep first duplicate": ("latest[key] = s[i];", "latest.emplace(key, s[i]);"),
    "buckets not reset": ("        B1[w] = 0;\n", ""),
    "sides share ids": ("int32_t b = n_u + static_cast<int32_t>", "int32_t b = static_cast<int32_t>"),
    "wedge term dropped": ("wed += static_cast<u128>(B1[w]) + B2[w];", "wed += static_cast<u128>(B1[w]);"),
}


def _build_mutant(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name!r} not found exactly once"
    path = tmp_path / "mutant.cpp"
    path.write_text(src.replace(old, new))
    so = tmp_path / "mutant.so"
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-pthread", str(path), "-o", str(so)])
    lib = ctypes.CDLL(str(so))
    P = ctypes.c_void_p
    lib.oracle_count.argtypes = [P, P, P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int, P, P, P]
    lib.oracle_count.restype = ctypes.c_int
    return lib


def _count(lib, u, v, s, n_u, n_v):
    u = np.ascontiguousarray(u, np.int32)
    v = np.ascontiguousarray(v, np.int32)
    s = np.ascontiguousarray(s, np.int8)
    out = (ctypes.c_uint64 * 3)()
    base = ctypes.addressof(out)
    rc = lib.oracle_count(u.ctypes.data, v.ctypes.data, s.ctypes.data, u.shape[0], n_u, n_v, 1, base, base + 8,
                          base + 16)
    return None if rc else tuple(int(x) for x in out)


def _pins_hold(lib) -> bool:
    # worked example (Section IV-C)
    if _count(lib, [2, 2, 7, 7], [5, 8, 5, 8], [-1] * 4, 8, 9)[:2] != (1, 0):
        return False
    # K(a,b) closed forms, balanced and wedges
    for a, b in [(2, 5), (5, 2), (4, 4), (3, 6)]:
        uu, vv = np.meshgrid(np.arange(a), np.arange(b), indexing="ij")
        r = _count(lib, uu.ravel(), vv.ravel(), np.ones(a * b), a, b)
        if r != (math.comb(a, 2) * math.comb(b, 2), 0, b * math.comb(a, 2) if b > a else a * math.comb(b, 2)):
            return False
        # the accepted-wedge total does not depend on the signs
        sg = np.where((uu.ravel() + 2 * vv.ravel()) % 3 == 0, -1, 1)
        if _count(lib, uu.ravel(), vv.ravel(), sg, a, b)[2] != r[2]:
            return False
    # brute force on random small graphs (brute force is the unplanted oracle's)
    rng = np.random.default_rng(1)
    for _ in range(8):
        n_u, n_v = int(rng.integers(3, 10)), int(rng.integers(3, 10))
        pairs = rng.choice(n_u * n_v, size=int(rng.integers(4, n_u * n_v + 1)), replace=False)
        u, v = pairs // n_v, pairs % n_v
        s = rng.choice([-1, 1], size=u.shape[0])
        if _count(lib, u, v, s, n_u, n_v)[:2] != oracle.brute_force(u, v, s, n_u, n_v):
            return False
        # keep-latest duplicates: an earlier copy with some signs flipped loses
        # (flipping all of them would be a global negation, which changes nothing)
        flip = np.where(rng.random(u.shape[0]) < 0.5, -1, 1)
        u2, v2 = np.concatenate([u, u]), np.concatenate([v, v])
        s2 = np.concatenate([s * flip, s])
        if _count(lib, u2, v2, s2, n_u, n_v)[:2] != oracle.brute_force(u, v, s, n_u, n_v):
            return False
    return True


VERTEX_MUTANTS = {
    "middle counts itself": ("bal[pv.first] += same - 1;", "bal[pv.first] += same;"),
    "middle unbalanced uses the same class": ("unb[pv.first] += other;", "unb[pv.first] += same;"),
    "endpoint not credited": ("      bal[w] += c;\n", ""),
    "pivot not credited": ("      unb[p] += d;\n", ""),
}


def _vertex_pins_hold(lib) -> bool:
    P = ctypes.c_void_p
    lib.oracle_count_per_vertex.argtypes = [P, P, P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, P, P]
    lib.oracle_count_per_vertex.restype = ctypes.c_int
    rng = np.random.default_rng(3)
    for _ in range(6):
        n_u, n_v = int(rng.integers(3, 9)), int(rng.integers(3, 9))
        pairs = rng.choice(n_u * n_v, size=int(rng.integers(6, n_u * n_v + 1)), replace=False)
        u = (pairs // n_v).astype(np.int32)
        v = (pairs % n_v).astype(np.int32)
        s = rng.choice([-1, 1], size=u.shape[0]).astype(np.int8)
        b = np.zeros(n_u + n_v, np.uint64)
        ub = np.zeros(n_u + n_v, np.uint64)
        if lib.oracle_count_per_vertex(u.ctypes.data, v.ctypes.data, s.ctypes.data, u.shape[0], n_u, n_v,
                                       b.ctypes.data, ub.ctypes.data):
            return False
        bb, bub = oracle.brute_force_per_vertex(u, v, s, n_u, n_v)
        if not (np.array_equal(b, bb) and np.array_equal(ub, bub)):
            return False
    return True


EDGE_MUTANTS = {
    "edge pairs with itself": ("const u128 same = (sym ? B1[vw.first] : B2[vw.first]) - 1;",
                               "const u128 same = (sym ? B1[vw.first] : B2[vw.first]);"),
    "far edge not credited": ("for (uint64_t e : {key(p, pv.first), key(pv.first, vw.first)})",
                              "for (uint64_t e : {key(p, pv.first)})"),
    "edge unbalanced from the same class": ("const u128 other = sym ? B2[vw.first] : B1[vw.first];",
                                            "const u128 other = sym ? B1[vw.first] : B2[vw.first];"),
    "edge key ignores the sides": ("    if (a >= n_u) std::swap(a, b);\n", ""),
}


def _edge_pins_hold(lib) -> bool:
    P = ctypes.c_void_p
    lib.oracle_count_per_edge.argtypes = [P, P, P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, P, P,
                                          ctypes.c_int64, P, P]
    lib.oracle_count_per_edge.restype = ctypes.c_int
    rng = np.random.default_rng(4)
    for _ in range(6):
        n_u, n_v = int(rng.integers(3, 9)), int(rng.integers(3, 9))
        pairs = rng.choice(n_u * n_v, size=int(rng.integers(6, n_u * n_v + 1)), replace=False)
        u = (pairs // n_v).astype(np.int32)
        v = (pairs % n_v).astype(np.int32)
        s = rng.choice([-1, 1], size=u.shape[0]).astype(np.int8)
        b = np.zeros(u.shape[0], np.uint64)
        ub = np.zeros(u.shape[0], np.uint64)
        if lib.oracle_count_per_edge(u.ctypes.data, v.ctypes.data, s.ctypes.data, u.shape[0], n_u, n_v,
                                     u.ctypes.data, v.ctypes.data, u.shape[0], b.ctypes.data, ub.ctypes.data):
            return False
        bb, bub = oracle.brute_force_per_edge(u, v, s, n_u, n_v)
        if not (np.array_equal(b, bb) and np.array_equal(ub, bub)):
            return False
    return True


def test_unplanted_copy_passes(tmp_path):
    lib = _build_mutant(tmp_path, "none", "// CPU oracle", "// CPU oracle")
    assert _pins_hold(lib)
    assert _vertex_pins_hold(lib)
    assert _edge_pins_hold(lib)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    lib = _build_mutant(tmp_path, name, old, new)
    assert not _pins_hold(lib), f"pins did not catch: {name}"


@pytest.mark.parametrize("name", sorted(VERTEX_MUTANTS))
def test_planted_per_vertex_mistake_is_caught(tmp_path, name):
    old, new = VERTEX_MUTANTS[name]
    lib = _build_mutant(tmp_path, name, old, new)
    assert not _vertex_pins_hold(lib), f"pins did not catch: {name}"


@pytest.mark.parametrize("name", sorted(EDGE_MUTANTS))
def test_planted_per_edge_mistake_is_caught(tmp_path, name):
    old, new = EDGE_MUTANTS[name]
    lib = _build_mutant(tmp_path, name, old, new)
    assert not _edge_pins_hold(lib), f"pins did not catch: {name}"
