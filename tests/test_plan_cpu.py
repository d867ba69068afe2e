"""The paper's edge extended subgraph partition (Section 5, Algorithm 5's
CPU part), planned by the library on the host (no GPU), against a literal
set-based restatement of the same greedy rule written here.

Definition (Edge Extended Subgraph): the subgraph of an edge set S holds S and
every edge incident to an edge of S. Algorithm 5 takes the edges in order
into the current subgraph with their incident edges, and closes the subgraph
when Memof(G_s) + Memof(G'_s) + 15 |V(G)| would exceed the device memory,
Memof(G) = 25 |E(G)| + 4 |V(G)|.
"""
import numpy as np
import pytest

import graphgen as gg


@pytest.fixture(scope="module")
def ps():
    from paper_2311_12281_gb300 import _build
    _build.build()
    import paper_2311_12281_gb300 as mod
    return mod


def literal_plan(g, mem):
    off, adj = g.offsets, g.adj
    rows = [set(adj[off[x]:off[x + 1]].tolist()) for x in range(g.n)]
    es, vs, k, total = set(), set(), 0, 0
    for u in range(g.n):
        for v in adj[off[u]:off[u + 1]].tolist():  # CSR order
            if v <= u:
                continue
            inc = {(min(x, y), max(x, y)) for x in (u, v) for y in rows[x]}
            new = inc - es
            if not new:
                continue
            newv = {x for e in new for x in e} - vs
            if es and 25 * (len(es) + len(new)) + 4 * (len(vs) + len(newv)) + 15 * g.n > mem:
                total += 25 * len(es) + 4 * len(vs)
                k += 1
                es, vs = set(), set()
                new = inc
                newv = {x for e in inc for x in e}
            es |= new
            vs |= newv
    if es:
        total += 25 * len(es) + 4 * len(vs)
        k += 1
    return k, total


@pytest.mark.parametrize("which", ["rmat", "chung_lu", "star", "union"])
def test_plan_matches_the_literal_rule(ps, which):
    if which == "rmat":
        g = gg.rmat(9, 8, seed=4)
    elif which == "chung_lu":
        g = gg.chung_lu(800, 6.0, 2.1, seed=9)
    elif which == "star":
        g = gg.from_edges(200, [(0, i) for i in range(1, 200)] + [(i, i + 1) for i in range(1, 199, 2)])
    else:
        g, _ = gg.disjoint_union([gg.rmat(7, 8, seed=s) for s in range(3)] + [gg.from_edges(4, [])])
    whole = 25 * g.m + 4 * g.n + 15 * g.n
    for frac in (0.15, 0.3, 0.6, 2.0):
        mem = int(frac * whole)
        got = ps.scan_plan_edge_extended(g.n, g.offsets, g.adj, mem)
        assert got == literal_plan(g, mem), f"{which} at {frac} of the whole graph"
    # a budget that holds the whole graph: one subgraph of exactly the whole graph
    assert ps.scan_plan_edge_extended(g.n, g.offsets, g.adj, 10 * whole) == (1, 25 * g.m + 4 * int(
        (np.diff(g.offsets) > 0).sum()))


def test_plan_rejects_malformed_input(ps):
    with pytest.raises(ps.ScanError):
        ps.scan_plan_edge_extended(3, np.array([0, 2, 1, 2]), np.array([1, 2], np.int32), 1 << 20)
    with pytest.raises(ps.ScanError):
        ps.scan_plan_edge_extended(2, np.array([0, 1, 2]), np.array([1, 5], np.int32), 1 << 20)
