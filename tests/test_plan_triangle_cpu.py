"""The plan of triangle counting over vertex-block pairs out of core, made by
the library on the host (no GPU), against a literal restatement written here.

A triangle a < b < c in (deg, id) rank is found at b (Section 4.1's
orientation), with its three counts in out(a) and out(b), so the pair
(block of a, block of b) needs only those two blocks. Blocks are cut in rank
order from whole out-lists (12 B per row, 8 B per oriented edge) so that
three block slots fit 90 % of what the per-vertex state (19 B per vertex,
a bit per slot) leaves; each block is moved once as the resident block and
once per later pair that streams it (12 B per row and per oriented edge).
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
    deg = g.degrees().tolist()
    n, nnz = g.n, g.nnz
    if n == 0:
        return 0, 0, 0
    key = [(deg[v], v) for v in range(n)]
    rows = [g.adj[g.offsets[v]:g.offsets[v + 1]].tolist() for v in range(n)]
    outs = [[w for w in rows[v] if key[w] > key[v]] for v in range(n)]
    state = 19 * (n + 1) + nnz // 8 + 16
    cap = 0.9 * (mem - state) / 3.0
    blk = [0] * n
    edges, nrows = [], []
    used, e_cur, r_cur = 0.0, 0, 0
    for v in sorted(range(n), key=lambda x: key[x]):
        row = 12.0 + 8.0 * len(outs[v])
        assert row <= cap
        if used + row > cap and r_cur > 0:
            edges.append(e_cur)
            nrows.append(r_cur)
            used, e_cur, r_cur = 0.0, 0, 0
        blk[v] = len(edges)
        used += row
        e_cur += len(outs[v])
        r_cur += 1
    edges.append(e_cur)
    nrows.append(r_cur)
    work = {(blk[a], blk[b]) for a in range(n) for b in outs[a]}
    assert all(i <= j for (i, j) in work)  # rank-ordered blocks: a below b never lies in a later block
    moved = [12 * r + 12 * e for r, e in zip(nrows, edges)]
    total = sum(moved) + sum(moved[j] for (i, j) in work if j > i)
    assert sum(edges) == nnz // 2  # every undirected edge is one oriented edge
    return len(edges), len(work), total


def graphs():
    union, _ = gg.disjoint_union([gg.rmat(8, 8, seed=s) for s in range(3)] + [gg.from_edges(6, [])])
    return {
        "rmat11": gg.rmat(11, 16, seed=3),
        "chung_lu": gg.chung_lu(3000, 12.0, 2.1, seed=7),
        "star_path": gg.from_edges(600, [(0, i) for i in range(1, 600)] + [(i, i + 1) for i in range(1, 599, 2)]),
        "union_with_isolated": union,
    }


@pytest.mark.parametrize("name", list(graphs().keys()))
@pytest.mark.parametrize("slack", [2, 6, 40, 10 ** 6])
def test_plan_matches_literal_restatement(ps, name, slack):
    g = graphs()[name]
    state = 19 * (g.n + 1) + g.nnz // 8 + 16
    dmax = int(g.degrees().max(initial=0))
    mem = state + slack * (12 + 8 * dmax) * 4  # room for a few of the widest out-lists, up to all of them
    want = literal_plan(g, mem)
    got = ps.scan_plan_triangle_blocks(g.n, g.offsets, g.adj, mem)
    assert got == want, f"{name} mem={mem}: {got} vs {want}"


def test_one_block_moves_the_oriented_graph_once(ps):
    g = gg.rmat(10, 8, seed=1)
    nb, npairs, moved = ps.scan_plan_triangle_blocks(g.n, g.offsets, g.adj, 1 << 40)
    assert (nb, npairs) == (1, 1)
    assert moved == 12 * g.n + 12 * (g.nnz // 2)


def test_more_memory_never_means_more_blocks(ps):
    g = gg.chung_lu(4000, 16.0, 2.1, seed=9)
    state = 19 * (g.n + 1) + g.nnz // 8 + 16
    plans = [ps.scan_plan_triangle_blocks(g.n, g.offsets, g.adj, state + extra) for extra in
             (200_000, 400_000, 800_000, 1_600_000, 3_200_000)]
    counts = [p[0] for p in plans]
    assert counts == sorted(counts, reverse=True)
    assert all(p[2] >= 12 * g.n + 12 * (g.nnz // 2) for p in plans)


def test_empty_graph_and_errors(ps):
    assert ps.scan_plan_triangle_blocks(0, np.zeros(1, np.int64), np.zeros(0, np.int32), 1 << 20) == (0, 0, 0)
    g = gg.rmat(9, 8, seed=2)
    with pytest.raises(ps.ScanError) as ei:  # not even the per-vertex state fits
        ps.scan_plan_triangle_blocks(g.n, g.offsets, g.adj, 1000)
    assert ei.value.status == ps.SCAN_EBUDGET
    # a star of 10,000 leaves with room for one leaf's out-list (20 B) per slot: every leaf is a
    # block of its own, more than the 8,192 blocks a plan may have
    star = gg.from_edges(10001, [(0, i) for i in range(1, 10001)])
    state = 19 * 10002 + star.nnz // 8 + 16
    with pytest.raises(ps.ScanError) as ei:
        ps.scan_plan_triangle_blocks(star.n, star.offsets, star.adj, state + 3 * 30)
    assert ei.value.status == ps.SCAN_EBUDGET
    bad = gg.from_csr(np.array([0, 1, 2], np.int64), np.array([5, 0], np.int32))
    with pytest.raises(ps.ScanError) as ei:
        ps.scan_plan_triangle_blocks(bad.n, bad.offsets, bad.adj, 1 << 30)
    assert ei.value.status == ps.SCAN_EINVAL
