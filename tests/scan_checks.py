"""Shared assertions for SCAN results (oracle pins and GPU parity).

A result is a dict with ``core`` uint8[n], ``cid`` int32[n], ``label`` uint8[n]
and ``pairs`` int32[k, 2] (vertex, cluster id) ascending.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

CORE, BORDER, HUB, OUTLIER = 0, 1, 2, 3


def assert_same(a: dict, b: dict, what: str = ""):
    """Bit-exact equality of two results, with the first differing index."""
    for key in ("core", "cid", "label"):
        x, y = np.asarray(a[key]), np.asarray(b[key])
        assert x.shape == y.shape, f"{what} {key}: shape {x.shape} vs {y.shape}"
        if not np.array_equal(x, y):
            i = int(np.flatnonzero(x != y)[0])
            raise AssertionError(f"{what} {key}[{i}]: {x[i]} vs {y[i]} ({int((x != y).sum())} differ)")
    pa, pb = np.asarray(a["pairs"]).reshape(-1, 2), np.asarray(b["pairs"]).reshape(-1, 2)
    assert pa.shape == pb.shape, f"{what} border pairs: {len(pa)} vs {len(pb)}"
    if not np.array_equal(pa, pb):
        i = int(np.flatnonzero((pa != pb).any(axis=1))[0])
        raise AssertionError(f"{what} border pair {i}: {pa[i]} vs {pb[i]}")


def similar_mask(graph, cn: np.ndarray, p: int, q: int) -> np.ndarray:
    """Per-slot eps-test from closed common counts, in Python integers."""
    deg = np.diff(graph.offsets).astype(np.int64)
    src = np.repeat(np.arange(graph.n, dtype=np.int64), deg)
    dst = graph.adj.astype(np.int64)
    du, dv = deg[src] + 1, deg[dst] + 1
    c = cn.astype(object)
    lhs = c * c * (q * q)
    rhs = (p * p) * du.astype(object) * dv.astype(object)
    return np.asarray(lhs >= rhs, dtype=bool)


def check_invariants(graph, res: dict, cn: np.ndarray, p: int, q: int, mu: int):
    """Properties every SCAN result must have, recomputed independently
    (connected components by scipy, memberships by set logic)."""
    n = graph.n
    deg = np.diff(graph.offsets).astype(np.int64)
    src = np.repeat(np.arange(n, dtype=np.int64), deg)
    dst = graph.adj.astype(np.int64)
    core, cid, label = (np.asarray(res[k]) for k in ("core", "cid", "label"))
    pairs = np.asarray(res["pairs"]).reshape(-1, 2)

    # sigma symmetric: the count of (u,v) equals the count of (v,u)
    key = src * n + dst
    rkey = dst * n + src
    order = np.argsort(key)
    pos = np.searchsorted(key[order], rkey)
    assert np.array_equal(cn[order[pos]], cn), "common counts not symmetric"
    assert (cn >= 2).all(), "adjacent pair must share both endpoints"

    S = similar_mask(graph, cn, p, q)
    eps_deg = 1 + np.bincount(src[S], minlength=n)  # sigma(u,u) = 1 counts u itself
    assert np.array_equal(core.astype(bool), eps_deg >= mu), "core flags disagree with |N_eps| >= mu"

    # clusters = connected components of the core eps-graph; id = smallest member
    cc = S & core[src].astype(bool) & core[dst].astype(bool)
    A = sp.coo_matrix((np.ones(int(cc.sum())), (src[cc], dst[cc])), shape=(n, n)).tocsr()
    _, comp = connected_components(A, directed=False)
    cores = np.flatnonzero(core)
    assert (cid[core == 0] == -1).all(), "non-core with a cluster id"
    if len(cores):
        assert (cid[cores] >= 0).all(), "core without a cluster"
        mins = {}
        for v in cores:
            mins.setdefault(comp[v], v)
        expect = np.array([mins[comp[v]] for v in cores])
        assert np.array_equal(cid[cores], expect), "cluster ids are not the components' smallest core"

    # border memberships: exactly the clusters of eps-similar core neighbours
    bs = S & core[src].astype(bool) & ~core[dst].astype(bool)
    want = sorted(set(zip(dst[bs].tolist(), cid[src[bs]].tolist())))
    got = [tuple(x) for x in pairs.tolist()]
    assert got == want, "border pairs differ from eps-similar core witnesses"

    # labels
    member = np.zeros(n, bool)
    member[pairs[:, 0]] = True
    memberships = {}
    for v, c in got:
        memberships.setdefault(v, set()).add(c)
    for v in cores:
        memberships[v] = {int(cid[v])}
    for u in range(n):
        if core[u]:
            assert label[u] == CORE
        elif member[u]:
            assert label[u] == BORDER
        else:
            seen = set()
            for w in graph.adj[graph.offsets[u]:graph.offsets[u + 1]]:
                seen |= memberships.get(int(w), set())
            assert label[u] == (HUB if len(seen) >= 2 else OUTLIER), f"vertex {u} hub/outlier"
