"""Python binding of the dbbc C ABI (``include/dbbc.h``): balanced / unbalanced
butterfly counts of signed bipartite graphs on one GB300 GPU.

This module only marshals arguments (numpy arrays or torch tensors to
pointers, streams to ``cudaStream_t``) and calls ``_build/libdbbc.so``; every
step of the computation runs in the library's CUDA kernels. There is no CPU
fallback: if the library has not been built, :func:`lib` raises.

Functions carry the C names (``EXPORTED`` lists them all):

- graphs: :func:`dbbc_graph_from_coo`, :func:`dbbc_graph_from_coo_multi`,
  :func:`dbbc_graph_get_info`, :func:`dbbc_graph_device_bytes`,
  :func:`dbbc_estimate_bytes`, :func:`dbbc_graph_export`, :func:`dbbc_graph_free`;
- counts: :func:`dbbc_count`, :func:`dbbc_count_async`,
  :func:`dbbc_count_profiled`, :func:`dbbc_count_noalloc`,
  :func:`dbbc_count_components`, :func:`dbbc_count_vertices`,
  :func:`dbbc_count_edges`;
- many graphs: :func:`dbbc_count_batch`, :func:`dbbc_count_batch_async`,
  :func:`dbbc_batch_create`, :func:`dbbc_batch_count`,
  :func:`dbbc_batch_count_async`, :func:`dbbc_batch_free`;
- several GPUs: :func:`dbbc_lpt_partition`, :func:`dbbc_count_partition`;
- housekeeping: :func:`dbbc_set_tuning`, :func:`dbbc_get_tuning`,
  :func:`dbbc_set_allocator`, :func:`dbbc_kernel_launches`,
  :func:`dbbc_status_string`, :func:`dbbc_version`;
- the bounds-checked debug build (``buildlib.build_checked()``, loaded when
  ``DBBC_LIBRARY`` names it): :func:`dbbc_is_checked`, :func:`dbbc_checked_flags`.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("DBBC_LIBRARY") or os.path.join(_HERE, "_build", "libdbbc.so")

DBBC_OK, DBBC_EINVAL, DBBC_ENOMEM, DBBC_ECUDA, DBBC_ETIMEOUT, DBBC_EOVERFLOW, DBBC_EINTERNAL = range(7)
DBBC_INPUT_HOST, DBBC_INPUT_DEVICE, DBBC_DUP_KEEP_LAST, DBBC_DUP_REJECT = 0, 1, 0, 2

EXPORTED = (
    "dbbc_graph_from_coo", "dbbc_count", "dbbc_count_async", "dbbc_count_batch", "dbbc_count_batch_async",
    "dbbc_graph_get_info", "dbbc_graph_device_bytes", "dbbc_estimate_bytes", "dbbc_graph_free",
    "dbbc_graph_export", "dbbc_set_allocator", "dbbc_status_string", "dbbc_version", "dbbc_count_profiled",
    "dbbc_kernel_launches", "dbbc_count_noalloc", "dbbc_batch_create", "dbbc_batch_count_async",
    "dbbc_batch_count", "dbbc_batch_free", "dbbc_graph_from_coo_multi", "dbbc_count_components",
    "dbbc_set_tuning", "dbbc_get_tuning", "dbbc_lpt_partition", "dbbc_count_partition",
    "dbbc_count_vertices", "dbbc_count_edges", "dbbc_is_checked", "dbbc_checked_flags",
)


class DbbcError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {dbbc_status_string(status)} (status {status})")


class GraphInfo(ctypes.Structure):
    _fields_ = [("n_u", ctypes.c_int32), ("n_v", ctypes.c_int32), ("m_input", ctypes.c_int64),
                ("m", ctypes.c_int64), ("wedges", ctypes.c_uint64), ("n_pivots", ctypes.c_int64),
                ("n_light", ctypes.c_int64), ("n_medium", ctypes.c_int64), ("n_hub", ctypes.c_int64),
                ("wedges_light", ctypes.c_uint64), ("wedges_medium", ctypes.c_uint64),
                ("wedges_hub", ctypes.c_uint64), ("lower_light", ctypes.c_int64), ("lower_medium", ctypes.c_int64),
                ("lower_hub", ctypes.c_int64), ("hub_items", ctypes.c_int64), ("hub_cursor_inits", ctypes.c_int64),
                ("hub_cursor_steps", ctypes.c_int64), ("device_bytes", ctypes.c_size_t),
                ("n_components", ctypes.c_int32)]


class CountProfile(ctypes.Structure):
    _fields_ = [("ms_light", ctypes.c_float), ("ms_medium", ctypes.c_float), ("ms_hub_aggregate", ctypes.c_float),
                ("ms_hub_finalize", ctypes.c_float), ("ms_total", ctypes.c_float),
                ("launches_light", ctypes.c_int64), ("launches_medium", ctypes.c_int64),
                ("launches_hub_aggregate", ctypes.c_int64), ("launches_hub_finalize", ctypes.c_int64),
                ("hub_list_visits", ctypes.c_uint64)]


class Tuning(ctypes.Structure):
    _fields_ = [("light_max_work", ctypes.c_uint64), ("medium_max_work", ctypes.c_uint64),
                ("hub_item_work", ctypes.c_uint64), ("group_density", ctypes.c_double * 4),
                ("hash_mult_log", ctypes.c_int32), ("list_density", ctypes.c_double),
                ("list_group_log", ctypes.c_int32), ("finalize_window_wedges", ctypes.c_uint64),
                ("list_wide_density", ctypes.c_double)]


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
_lib = None
_allocator_refs = None


def build(force: bool = False) -> str:
    """Compile the library in-tree (needs nvcc; see ``buildlib.py``)."""
    from . import buildlib
    return buildlib.build(force=force)


def lib() -> ctypes.CDLL:
    """The loaded CUDA library. Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2609_21848_gb300.build() "
                               "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        P, I32, I64, U32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
        st = ctypes.c_int
        L.dbbc_graph_from_coo.argtypes = [P, P, P, I64, I32, I32, U32, P, ctypes.POINTER(P)]
        L.dbbc_graph_from_coo.restype = st
        L.dbbc_count.argtypes = [P, P, P, P]
        L.dbbc_count.restype = st
        L.dbbc_count_profiled.argtypes = [P, P, P, P, ctypes.POINTER(CountProfile)]
        L.dbbc_count_profiled.restype = st
        L.dbbc_kernel_launches.argtypes = []
        L.dbbc_kernel_launches.restype = ctypes.c_uint64
        L.dbbc_lpt_partition.argtypes = [P, I64, I32, P, P]
        L.dbbc_lpt_partition.restype = st
        L.dbbc_count_partition.argtypes = [P, P, I32, I32, P, P]
        L.dbbc_count_partition.restype = st
        L.dbbc_set_tuning.argtypes = [ctypes.POINTER(Tuning)]
        L.dbbc_set_tuning.restype = st
        L.dbbc_get_tuning.argtypes = [ctypes.POINTER(Tuning)]
        L.dbbc_get_tuning.restype = None
        L.dbbc_graph_from_coo_multi.argtypes = [P, P, P, P, P, P, I32, U32, P, ctypes.POINTER(P)]
        L.dbbc_graph_from_coo_multi.restype = st
        L.dbbc_count_components.argtypes = [P, P, P, P]
        L.dbbc_count_components.restype = st
        L.dbbc_count_vertices.argtypes = [P, P, P, P]
        L.dbbc_count_vertices.restype = st
        L.dbbc_count_edges.argtypes = [P, P, P, P, I64, U32, P, P]
        L.dbbc_count_edges.restype = st
        L.dbbc_batch_create.argtypes = [P, I32, P, ctypes.POINTER(P)]
        L.dbbc_batch_create.restype = st
        L.dbbc_batch_count_async.argtypes = [P, P, P]
        L.dbbc_batch_count_async.restype = st
        L.dbbc_batch_count.argtypes = [P, P, P, P]
        L.dbbc_batch_count.restype = st
        L.dbbc_batch_free.argtypes = [P]
        L.dbbc_batch_free.restype = None
        L.dbbc_count_noalloc.argtypes = [P, P, P]
        L.dbbc_count_noalloc.restype = st
        L.dbbc_count_async.argtypes = [P, P, P]
        L.dbbc_count_async.restype = st
        L.dbbc_count_batch.argtypes = [P, I32, P, P, P]
        L.dbbc_count_batch.restype = st
        L.dbbc_count_batch_async.argtypes = [P, I32, P, P]
        L.dbbc_count_batch_async.restype = st
        L.dbbc_graph_get_info.argtypes = [P, ctypes.POINTER(GraphInfo)]
        L.dbbc_graph_get_info.restype = st
        L.dbbc_graph_device_bytes.argtypes = [P]
        L.dbbc_graph_device_bytes.restype = ctypes.c_size_t
        L.dbbc_estimate_bytes.argtypes = [I64, I32, I32]
        L.dbbc_estimate_bytes.restype = ctypes.c_size_t
        L.dbbc_graph_free.argtypes = [P]
        L.dbbc_graph_free.restype = None
        L.dbbc_graph_export.argtypes = [P, P, P, P, P, P, P]
        L.dbbc_graph_export.restype = st
        L.dbbc_set_allocator.argtypes = [P, P, P]
        L.dbbc_set_allocator.restype = None
        L.dbbc_status_string.argtypes = [st]
        L.dbbc_status_string.restype = ctypes.c_char_p
        L.dbbc_version.argtypes = []
        L.dbbc_version.restype = ctypes.c_char_p
        L.dbbc_is_checked.argtypes = []
        L.dbbc_is_checked.restype = ctypes.c_int
        L.dbbc_checked_flags.argtypes = [P]
        L.dbbc_checked_flags.restype = st
        _lib = L
        if not os.environ.get("DBBC_NO_TUNING"):
            from . import autotune
            autotune.apply_saved()
    return _lib


def _check(status: int, where: str):
    if status != DBBC_OK:
        raise DbbcError(status, where)


def _stream_ptr(stream) -> int:
    """cudaStream_t of a torch stream, an int, or the current torch stream."""
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return int(torch.cuda.current_stream().cuda_stream)
        except ImportError:  # pragma: no cover
            pass
        return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _array_ptr(x, dtype):
    """(pointer, length, on_device, keepalive) for a numpy array or torch tensor."""
    try:
        import torch
        if isinstance(x, torch.Tensor):
            tdt = {np.int32: torch.int32, np.int8: torch.int8}[dtype]
            if x.dtype != tdt or not x.is_contiguous():
                x = x.to(tdt).contiguous()
            return x.data_ptr(), int(x.numel()), x.is_cuda, x
    except ImportError:  # pragma: no cover
        pass
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data, int(a.shape[0]), False, a


class Graph:
    """Owning wrapper of a ``dbbc_graph*`` handle."""

    def __init__(self, handle: int):
        self.handle = handle

    def free(self):
        if self.handle:
            lib().dbbc_graph_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.free()

    @property
    def info(self) -> dict:
        return dbbc_graph_get_info(self)


def dbbc_graph_from_coo(u, v, sign, n_u: int, n_v: int, *, reject_duplicates: bool = False, stream=None) -> Graph:
    """Build a graph from COO arrays (numpy / host tensors, or CUDA tensors)."""
    pu, mu, du, ku = _array_ptr(u, np.int32)
    pv, mv, dv, kv = _array_ptr(v, np.int32)
    ps, ms, ds, ks = _array_ptr(sign, np.int8)
    if not (mu == mv == ms):
        raise ValueError("u, v and sign must have the same length")
    if not (du == dv == ds):
        raise ValueError("u, v and sign must all be on the host or all on the device")
    flags = (DBBC_INPUT_DEVICE if du else DBBC_INPUT_HOST) | (DBBC_DUP_REJECT if reject_duplicates else 0)
    h = ctypes.c_void_p()
    _check(lib().dbbc_graph_from_coo(pu, pv, ps, mu, n_u, n_v, flags, _stream_ptr(stream), ctypes.byref(h)),
           "dbbc_graph_from_coo")
    del ku, kv, ks
    return Graph(h.value)


def dbbc_graph_from_coo_multi(u, v, sign, edge_offsets, n_u, n_v, *, reject_duplicates: bool = False,
                              stream=None) -> Graph:
    """Build the disjoint union of several graphs (edges of graph i at
    [edge_offsets[i], edge_offsets[i+1]), ids local to graph i) as one handle;
    see :func:`dbbc_count_components`."""
    pu, mu, du, ku = _array_ptr(u, np.int32)
    pv, mv, dv, kv = _array_ptr(v, np.int32)
    ps, ms, ds, ks = _array_ptr(sign, np.int8)
    off = np.ascontiguousarray(edge_offsets, dtype=np.int64)
    nu = np.ascontiguousarray(n_u, dtype=np.int32)
    nv = np.ascontiguousarray(n_v, dtype=np.int32)
    k = nu.shape[0]
    if not (mu == mv == ms) or nv.shape[0] != k or off.shape[0] != k + 1 or (k and off[-1] != mu):
        raise ValueError("inconsistent arrays")
    if not (du == dv == ds):
        raise ValueError("u, v and sign must all be on the host or all on the device")
    flags = (DBBC_INPUT_DEVICE if du else DBBC_INPUT_HOST) | (DBBC_DUP_REJECT if reject_duplicates else 0)
    h = ctypes.c_void_p()
    _check(lib().dbbc_graph_from_coo_multi(pu, pv, ps, off.ctypes.data, nu.ctypes.data, nv.ctypes.data, k, flags,
                                           _stream_ptr(stream), ctypes.byref(h)), "dbbc_graph_from_coo_multi")
    del ku, kv, ks
    return Graph(h.value)


def dbbc_count_components(g: Graph, stream=None) -> tuple[np.ndarray, np.ndarray]:
    """Per-component (balanced, unbalanced) of a union handle."""
    n = dbbc_graph_get_info(g)["n_components"]
    bal = np.zeros(max(n, 1), np.uint64)
    unb = np.zeros(max(n, 1), np.uint64)
    _check(lib().dbbc_count_components(g.handle, _stream_ptr(stream), bal.ctypes.data, unb.ctypes.data),
           "dbbc_count_components")
    return bal[:n], unb[:n]


def dbbc_count_vertices(g: Graph, stream=None) -> tuple[np.ndarray, np.ndarray]:
    """(balanced, unbalanced) butterflies containing each vertex, indexed by
    unified id (U vertex u at u, V vertex v at n_u + v); synchronous."""
    info = dbbc_graph_get_info(g)
    n = int(info["n_u"]) + int(info["n_v"])
    bal = np.zeros(max(n, 1), np.uint64)
    unb = np.zeros(max(n, 1), np.uint64)
    _check(lib().dbbc_count_vertices(g.handle, _stream_ptr(stream), bal.ctypes.data, unb.ctypes.data),
           "dbbc_count_vertices")
    return bal[:n], unb[:n]


def dbbc_count_edges(g: Graph, qu, qv, stream=None):
    """(balanced, unbalanced) butterflies containing each queried edge
    (qu[i], qv[i]); zeros for a pair that is not an edge. Host arrays in give
    numpy uint64 arrays out; CUDA tensors in give CUDA uint64 tensors out."""
    pu, ku_n, du, ku = _array_ptr(qu, np.int32)
    pv, kv_n, dv, kv = _array_ptr(qv, np.int32)
    if ku_n != kv_n:
        raise ValueError("qu and qv differ in length")
    if du != dv:
        raise ValueError("qu and qv must both be on the host or both on the device")
    k = ku_n
    if du:
        import torch
        dev = qu.device
        bal = torch.zeros(max(k, 1), dtype=torch.uint64, device=dev)
        unb = torch.zeros(max(k, 1), dtype=torch.uint64, device=dev)
        pb, pub = bal.data_ptr(), unb.data_ptr()
    else:
        bal = np.zeros(max(k, 1), np.uint64)
        unb = np.zeros(max(k, 1), np.uint64)
        pb, pub = bal.ctypes.data, unb.ctypes.data
    _check(lib().dbbc_count_edges(g.handle, _stream_ptr(stream), pu, pv, k,
                                  DBBC_INPUT_DEVICE if du else DBBC_INPUT_HOST, pb, pub), "dbbc_count_edges")
    del ku, kv
    return bal[:k], unb[:k]


def dbbc_count(g: Graph, stream=None) -> tuple[int, int]:
    """(balanced, unbalanced) of one graph; synchronous."""
    out = (ctypes.c_uint64 * 2)()
    base = ctypes.addressof(out)
    _check(lib().dbbc_count(g.handle, _stream_ptr(stream), base, base + 8), "dbbc_count")
    return int(out[0]), int(out[1])


def dbbc_count_profiled(g: Graph, stream=None) -> tuple[int, int, dict]:
    """(balanced, unbalanced, per-tier profile) of one graph; synchronous."""
    out = (ctypes.c_uint64 * 2)()
    base = ctypes.addressof(out)
    prof = CountProfile()
    _check(lib().dbbc_count_profiled(g.handle, _stream_ptr(stream), base, base + 8, ctypes.byref(prof)),
           "dbbc_count_profiled")
    return int(out[0]), int(out[1]), {name: getattr(prof, name) for name, _ in CountProfile._fields_}


def dbbc_kernel_launches() -> int:
    """Kernels the library has launched in this process."""
    return int(lib().dbbc_kernel_launches())


def dbbc_count_noalloc(g: Graph, d_out, stream=None) -> None:
    """Enqueue a count that allocates no device memory (scratch comes from a
    fixed array inside the library; see dbbc.h). ``d_out``: device tensor of
    at least 2 x 64-bit. Calls must not overlap on the GPU."""
    _check(lib().dbbc_count_noalloc(g.handle, _stream_ptr(stream), d_out.data_ptr()), "dbbc_count_noalloc")


def dbbc_count_async(g: Graph, d_out, stream=None) -> None:
    """Enqueue a count writing {balanced, unbalanced} into device tensor ``d_out``
    (at least 2 x 64-bit, e.g. ``torch.empty(2, dtype=torch.int64, device='cuda')``)."""
    _check(lib().dbbc_count_async(g.handle, _stream_ptr(stream), d_out.data_ptr()), "dbbc_count_async")


def _handles(graphs):
    arr = (ctypes.c_void_p * len(graphs))(*[g.handle for g in graphs])
    return arr


def dbbc_count_batch(graphs, stream=None) -> tuple[np.ndarray, np.ndarray]:
    n = len(graphs)
    bal = np.zeros(n, np.uint64)
    unb = np.zeros(n, np.uint64)
    if n == 0:
        return bal, unb
    _check(lib().dbbc_count_batch(_handles(graphs), n, _stream_ptr(stream), bal.ctypes.data, unb.ctypes.data),
           "dbbc_count_batch")
    return bal, unb


def dbbc_count_batch_async(graphs, d_out, stream=None) -> None:
    """Enqueue counts of all graphs into device tensor ``d_out`` of shape [n, 2] (64-bit)."""
    if len(graphs) == 0:
        return
    _check(lib().dbbc_count_batch_async(_handles(graphs), len(graphs), _stream_ptr(stream), d_out.data_ptr()),
           "dbbc_count_batch_async")


class Batch:
    """Owning wrapper of a ``dbbc_batch*`` plan; keeps its graphs alive."""

    def __init__(self, handle: int, graphs):
        self.handle = handle
        self.graphs = list(graphs)

    def free(self):
        if self.handle:
            lib().dbbc_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.free()

    def __len__(self):
        return len(self.graphs)


def dbbc_batch_create(graphs, stream=None) -> Batch:
    """Plan a batched count of resident graphs (replayed as one CUDA graph)."""
    h = ctypes.c_void_p()
    _check(lib().dbbc_batch_create(_handles(graphs), len(graphs), _stream_ptr(stream), ctypes.byref(h)),
           "dbbc_batch_create")
    return Batch(h.value, graphs)


def dbbc_batch_count_async(b: Batch, d_out=None, stream=None) -> None:
    """Replay the plan; ``d_out`` (device tensor [n, 2] of 64-bit, optional) receives the counts."""
    _check(lib().dbbc_batch_count_async(b.handle, _stream_ptr(stream), d_out.data_ptr() if d_out is not None else None),
           "dbbc_batch_count_async")


def dbbc_batch_count(b: Batch, stream=None) -> tuple[np.ndarray, np.ndarray]:
    n = len(b)
    bal = np.zeros(n, np.uint64)
    unb = np.zeros(n, np.uint64)
    _check(lib().dbbc_batch_count(b.handle, _stream_ptr(stream), bal.ctypes.data, unb.ctypes.data),
           "dbbc_batch_count")
    return bal, unb


def dbbc_batch_free(b: Batch) -> None:
    b.free()


def dbbc_graph_get_info(g: Graph) -> dict:
    info = GraphInfo()
    _check(lib().dbbc_graph_get_info(g.handle, ctypes.byref(info)), "dbbc_graph_get_info")
    return {name: getattr(info, name) for name, _ in GraphInfo._fields_}


def dbbc_graph_device_bytes(g: Graph) -> int:
    return int(lib().dbbc_graph_device_bytes(g.handle if g is not None else None))


def dbbc_estimate_bytes(m: int, n_u: int, n_v: int) -> int:
    return int(lib().dbbc_estimate_bytes(m, n_u, n_v))


def dbbc_graph_free(g: Graph) -> None:
    g.free()


def dbbc_graph_export(g: Graph, stream=None) -> dict:
    """Host copies of the device CSR (see ``dbbc_graph_export`` in dbbc.h)."""
    info = dbbc_graph_get_info(g)
    n = info["n_u"] + info["n_v"]
    out = dict(row_ptr=np.zeros(n + 1, np.int64), col=np.zeros(2 * info["m"], np.uint32),
               lower=np.zeros(n, np.uint32), vertex=np.zeros(n, np.int32), work=np.zeros(n, np.uint64))
    _check(lib().dbbc_graph_export(g.handle, _stream_ptr(stream), *(out[k].ctypes.data for k in
                                                                     ("row_ptr", "col", "lower", "vertex", "work"))),
           "dbbc_graph_export")
    return out


def dbbc_set_allocator(use_torch: bool = True) -> None:
    """Route the library's device allocations through torch's caching allocator
    (``use_torch=True``) or back to cudaMallocAsync (``False``)."""
    global _allocator_refs
    if not use_torch:
        lib().dbbc_set_allocator(None, None, None)
        _allocator_refs = None
        return
    import torch

    def _alloc(size, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(size), torch.cuda.current_device(), int(stream or 0))
        except Exception:
            return None

    def _free(ptr, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    refs = (_ALLOC_FN(_alloc), _FREE_FN(_free))
    lib().dbbc_set_allocator(ctypes.cast(refs[0], ctypes.c_void_p), ctypes.cast(refs[1], ctypes.c_void_p), None)
    _allocator_refs = refs


def dbbc_lpt_partition(work, n_parts: int) -> tuple[np.ndarray, np.ndarray]:
    """Greedy bin packing (Phase 3): (part of every item, load of every part)."""
    w = np.ascontiguousarray(work, dtype=np.uint64)
    part = np.zeros(w.shape[0], np.int32)
    loads = np.zeros(n_parts, np.uint64)
    _check(lib().dbbc_lpt_partition(w.ctypes.data, w.shape[0], n_parts, part.ctypes.data, loads.ctypes.data),
           "dbbc_lpt_partition")
    return part, loads


def dbbc_count_partition(g: Graph, part: int, n_parts: int, stream=None) -> tuple[int, int]:
    """(balanced, unbalanced) of the pivots LPT assigns to `part` of `n_parts`."""
    out = (ctypes.c_uint64 * 2)()
    base = ctypes.addressof(out)
    _check(lib().dbbc_count_partition(g.handle, _stream_ptr(stream), part, n_parts, base, base + 8),
           "dbbc_count_partition")
    return int(out[0]), int(out[1])


def dbbc_set_tuning(tuning: dict | None) -> None:
    """Set the tier tuning for graphs built afterwards (None: defaults). Keys:
    light_max_work, medium_max_work, hub_item_work, group_density (4 values),
    hash_mult_log, list_density, list_group_log, finalize_window_wedges,
    list_wide_density; keys left out keep their current values."""
    if tuning is None:
        _check(lib().dbbc_set_tuning(None), "dbbc_set_tuning")
        return
    tuning = {**dbbc_get_tuning(), **tuning}
    t = Tuning(int(tuning["light_max_work"]), int(tuning["medium_max_work"]), int(tuning["hub_item_work"]),
               (ctypes.c_double * 4)(*[float(x) for x in tuning["group_density"]]), int(tuning["hash_mult_log"]),
               float(tuning["list_density"]), int(tuning["list_group_log"]),
               min(int(tuning["finalize_window_wedges"]), 2**64 - 1), float(tuning["list_wide_density"]))
    _check(lib().dbbc_set_tuning(ctypes.byref(t)), "dbbc_set_tuning")


def dbbc_get_tuning() -> dict:
    t = Tuning()
    lib().dbbc_get_tuning(ctypes.byref(t))
    return {"light_max_work": t.light_max_work, "medium_max_work": t.medium_max_work,
            "hub_item_work": t.hub_item_work, "group_density": list(t.group_density),
            "hash_mult_log": t.hash_mult_log, "list_density": t.list_density, "list_group_log": t.list_group_log,
            "finalize_window_wedges": t.finalize_window_wedges, "list_wide_density": t.list_wide_density}


def dbbc_status_string(status: int) -> str:
    return lib().dbbc_status_string(status).decode()


def dbbc_version() -> str:
    return lib().dbbc_version().decode()


def dbbc_is_checked() -> bool:
    """True when the loaded library is the bounds-checked build (-DDBBC_CHECKED=1)."""
    return bool(lib().dbbc_is_checked())


def dbbc_checked_flags() -> int:
    """Bounds-check flags recorded since the last call (2: an index left its
    array), then cleared; always 0 in a regular build. Synchronizes the device."""
    f = ctypes.c_uint32(0)
    _check(lib().dbbc_checked_flags(ctypes.byref(f)), "dbbc_checked_flags")
    return f.value


def count_coo(u, v, sign, n_u: int, n_v: int, stream=None) -> tuple[int, int]:
    """Build, count and free in one call (the end-to-end path)."""
    with dbbc_graph_from_coo(u, v, sign, n_u, n_v, stream=stream) as g:
        return dbbc_count(g, stream)
