"""Helpers shared by the GPU tests: run a graph through the C ABI and the
oracle, and build a CSR on the host (independently of both) to check the
device export."""
import numpy as np

import oracle
import paper_2609_21848_gb300 as dbbc


def gpu_count(u, v, s, n_u, n_v, device_input=False, **kw):
    if device_input:
        import torch
        u = torch.as_tensor(np.asarray(u, np.int32)).cuda()
        v = torch.as_tensor(np.asarray(v, np.int32)).cuda()
        s = torch.as_tensor(np.asarray(s, np.int8)).cuda()
    with dbbc.dbbc_graph_from_coo(u, v, s, n_u, n_v, **kw) as g:
        bal, unb = dbbc.dbbc_count(g)
        info = g.info
    return bal, unb, info


def assert_parity(u, v, s, n_u, n_v, threads=1, device_input=False):
    want = oracle.count(u, v, s, n_u, n_v, threads=threads)
    bal, unb, info = gpu_count(u, v, s, n_u, n_v, device_input=device_input)
    assert (bal, unb) == want[:2], f"GPU {(bal, unb)} != oracle {want[:2]}"
    assert info["wedges"] == want[2], f"GPU wedges {info['wedges']} != oracle {want[2]}"
    return info


def host_csr(u, v, s, n_u, n_v):
    """Keep-latest dedup, Def. 3 ranks per side, rows sorted by neighbour rank,
    written with numpy sorts (no code shared with the oracle or the library)."""
    u = np.asarray(u, np.int64)
    v = np.asarray(v, np.int64)
    s = np.asarray(s, np.int64)
    key = u * max(n_v, 1) + v
    order = np.argsort(key, kind="stable")
    ks = key[order]
    last = np.ones(ks.shape[0], bool)
    if ks.shape[0]:
        last[:-1] = ks[1:] != ks[:-1]
    keep = order[last]
    u, v, s = u[keep], v[keep], s[keep]
    n = n_u + n_v
    deg = np.bincount(u, minlength=n_u).tolist() + np.bincount(v, minlength=n_v).tolist()
    deg = np.array(deg, np.int64)
    uid = np.arange(n)
    rank_u = np.empty(n_u, np.int64)
    rank_u[np.lexsort((uid[:n_u], deg[:n_u]))] = np.arange(n_u)
    rank_v = np.empty(n_v, np.int64)
    rank_v[np.lexsort((uid[n_u:], deg[n_u:]))] = np.arange(n_v)
    rows = np.concatenate([rank_u[u], n_u + rank_v[v]])
    cols = np.concatenate([rank_v[v], rank_u[u]])
    neg = np.concatenate([s < 0, s < 0]).astype(np.int64)
    o = np.lexsort((cols, rows))
    rows, cols, neg = rows[o], cols[o], neg[o]
    row_ptr = np.zeros(n + 1, np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    col = (cols << 1 | neg).astype(np.uint32)
    vertex = np.empty(n, np.int64)
    vertex[rank_u] = np.arange(n_u)
    vertex[n_u + rank_v] = n_u + np.arange(n_v)
    # lower-priority neighbours: Def. 3 over unified ids (u -> u, v -> n_u + v)
    me = vertex[rows]
    nb_vertex = vertex[np.where(rows < n_u, n_u + cols, cols)]
    lower_flag = (deg[nb_vertex] < deg[me]) | ((deg[nb_vertex] == deg[me]) & (nb_vertex < me))
    lower = np.bincount(rows, weights=lower_flag, minlength=n).astype(np.int64)
    return dict(row_ptr=row_ptr, col=col, vertex=vertex, lower=lower)
