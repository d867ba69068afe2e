"""Out-of-core (partitioned) clustering vs the CPU oracle, bit-exact.

The CSR stays in host memory and is streamed in row blocks (Section 5's
setting). Lemma 5.1 says an edge's similarity needs only its endpoints'
rows, so the result must equal the resident one whatever the block plan:
the tests force many small blocks, blocks of a single row, and a plan sized
from a budget too small to hold the graph resident.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
from conftest import load_golden
from scan_checks import assert_same

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ps():
    from paper_2311_12281_gb300 import _build
    _build.build()
    import paper_2311_12281_gb300 as mod
    return mod


@pytest.fixture(scope="module")
def ctx(ps):
    c = ps.Context(0)
    yield c
    c.close()


def fig1():
    gd = load_golden("fig1.txt")
    e = list(map(int, gd["edges"][0].split()))
    return gg.from_edges(int(gd["n"][0]), list(zip(e[0::2], e[1::2])))


def graphs():
    star_path = gg.from_edges(3000, [(0, i) for i in range(1, 3000)] + [(i, i + 1) for i in range(1, 2999, 2)])
    union, _ = gg.disjoint_union([gg.rmat(9, 8, seed=s) for s in range(3)] + [gg.from_edges(5, [])])
    return {
        "fig1": fig1(),
        "hub_via_border": gg.from_edges(10, [(0, 1), (0, 2), (0, 4), (0, 6), (2, 7), (2, 9), (3, 9), (5, 9), (8, 9)]),
        "rmat12": gg.rmat(12, 16, seed=21),
        "chung_lu": gg.chung_lu(6007, 24.0, 2.1, seed=44),
        "star_path": star_path,
        "union_with_isolated": union,
    }


PARAMS = [(1, 5, 2), (1, 2, 3), (3, 5, 3), (7, 10, 5), (2, 5, 10)]


@pytest.mark.parametrize("name", list(graphs().keys()))
@pytest.mark.parametrize("nblocks", [1, 4, 23])
def test_partitioned_matches_oracle(ps, ctx, name, nblocks):
    g = graphs()[name]
    cn = oracle.common_counts(g)
    block_slots = max(1, -(-g.nnz // nblocks))
    dg = ctx.load_partitioned(g, block_slots)
    try:
        # rows are packed into a block up to block_slots slots (a longer row alone)
        widest = max(block_slots, int(g.degrees().max(initial=0)))
        assert dg.blocks >= max(1, -(-g.nnz // widest))
        for (p, q, mu) in PARAMS:
            # every query starts from a clean state: run them back to back
            want = oracle.scan_from_counts(g, cn, p, q, mu)
            assert_same(dg.query(p, q, mu), want, f"{name} blocks={dg.blocks} eps={p}/{q} mu={mu}")
    finally:
        dg.free()


def test_single_row_blocks_equal_resident(ps, ctx):
    g = gg.chung_lu(150, 8.0, 2.1, seed=5)
    dp = ctx.load_partitioned(g, 1)
    dr = ctx.load(g)
    try:
        # block_slots 1: every row of two or more slots is a block of its own
        assert dp.blocks >= int((g.degrees() > 1).sum())
        for (p, q, mu) in [(1, 2, 2), (3, 10, 4)]:
            want = dr.query(p, q, mu, ps.SCAN_Q_RECOMPUTE)
            assert_same(want, oracle.scan(g, p, q, mu))
            assert_same(dp.query(p, q, mu), want)
    finally:
        dp.free()
        dr.free()


def test_pinned_borrow_flag_loads_partitioned(ps, ctx):
    g = gg.rmat(11, 16, seed=3)
    dg = ctx.load(g, ps.SCAN_LOAD_PINNED_BORROW)
    try:
        assert dg.blocks >= 1
        for mode in (ps.SCAN_Q_AUTO, ps.SCAN_Q_RECOMPUTE, ps.SCAN_Q_PLAIN):
            assert_same(dg.query(1, 2, 3, mode), oracle.scan(g, 1, 2, 3))
    finally:
        dg.free()


def test_budget_too_small_for_resident_plans_blocks(ps):
    g = gg.chung_lu(20000, 16.0, 2.1, seed=3)
    c = ps.Context(0, budget_bytes=3 << 20)
    try:
        with pytest.raises(ps.ScanError) as ei:
            c.load(g)
        assert ei.value.status == ps.SCAN_EBUDGET
        dg = c.load_partitioned(g)  # block_slots 0: planned from what the budget leaves
        assert dg.blocks > 1
        assert c.device_bytes <= 3 << 20
        for (p, q, mu) in [(1, 2, 3), (3, 5, 5)]:
            assert_same(dg.query(p, q, mu), oracle.scan(g, p, q, mu))
        dg.free()
        assert c.device_bytes == 0
    finally:
        c.close()


def test_resident_only_calls_are_rejected(ps, ctx):
    g = gg.rmat(8, 8, seed=1)
    dg = ctx.load_partitioned(g, 100)
    try:
        for call in (lambda: dg.set_strategy(ps.SCAN_STRATEGY_OWNER), lambda: dg.counts(),
                     lambda: ps.scan_graph_autotune(dg.handle)):
            with pytest.raises(ps.ScanError) as ei:
                call()
            assert ei.value.status == ps.SCAN_EINVAL
        assert_same(dg.query(1, 2, 2), oracle.scan(g, 1, 2, 2))
    finally:
        dg.free()


def test_empty_and_edgeless_graphs(ps, ctx):
    for g in (gg.from_csr(np.zeros(1, np.int64), np.zeros(0, np.int32)), gg.from_edges(9, [])):
        dg = ctx.load_partitioned(g, 1)
        r = dg.query(1, 2, 2)
        assert_same(r, oracle.scan(g, 1, 2, 2))
        dg.free()


@pytest.mark.parametrize("case", ["self_loop", "unsorted", "out_of_range", "count_asymmetric"])
def test_malformed_csr_rejected_at_load(ps, ctx, case):
    off, adj = {
        "self_loop": ([0, 1, 2], [0, 0]),
        "unsorted": ([0, 2, 3, 4], [2, 1, 0, 0]),
        "out_of_range": ([0, 1, 2], [5, 0]),
        "count_asymmetric": ([0, 1, 2, 2], [1, 2]),
    }[case]
    g = gg.from_csr(np.array(off, np.int64), np.array(adj, np.int32))
    with pytest.raises(ps.ScanError) as ei:
        ctx.load_partitioned(g, 1)
    assert ei.value.status == ps.SCAN_EINVAL


def test_balanced_asymmetry_is_reported_by_the_query(ps, ctx):
    # (0,1) and (3,2) have no mirrors; the counts of entries above and below
    # their rows balance, so only the query's mirror lookup can see it
    g = gg.from_csr(np.array([0, 1, 1, 1, 2], np.int64), np.array([1, 2], np.int32))
    dg = ctx.load_partitioned(g, 1)
    try:
        with pytest.raises(ps.ScanError) as ei:
            dg.query(1, 2, 2)
        assert ei.value.status == ps.SCAN_EINVAL
    finally:
        dg.free()


def test_partitioned_graph_cannot_join_a_batch(ps, ctx):
    g = gg.rmat(8, 8, seed=2)
    dp = ctx.load_partitioned(g, 100)
    dr = ctx.load(g)
    try:
        with pytest.raises(ps.ScanError) as ei:
            ps.scan_query_batch([dr.handle, dp.handle], [(1, 2, 2), (1, 2, 2)])
        assert ei.value.status == ps.SCAN_EINVAL
    finally:
        dp.free()
        dr.free()


@pytest.mark.parametrize("name", ["rmat12", "chung_lu", "star_path", "union_with_isolated"])
def test_zero_copy_reads_match_copied_blocks_and_oracle(ps, ctx, name):
    # the streamed blocks read in place from the pinned host CSR (the host
    # link instead of copies): same answers, fewer bytes copied
    g = graphs()[name]
    slots = max(64, g.nnz // 9)
    dg = ctx.load_partitioned(g, block_slots=slots)
    try:
        assert dg.blocks > 1
        for (p, q, mu) in PARAMS[:3]:
            want = oracle.scan(g, p, q, mu)
            b0 = dg.transfer_bytes
            copied = dg.query(p, q, mu)
            copied_bytes = dg.transfer_bytes - b0
            dg.set_zero_copy(True)
            b1 = dg.transfer_bytes
            zc = dg.query(p, q, mu)
            zc_bytes = dg.transfer_bytes - b1
            dg.set_zero_copy(False)
            assert_same(copied, want, f"{name} copied eps={p}/{q} mu={mu}")
            assert_same(zc, want, f"{name} zero-copy eps={p}/{q} mu={mu}")
            assert zc_bytes < copied_bytes
    finally:
        dg.free()


def test_zero_copy_is_refused_for_a_resident_graph(ps, ctx):
    dg = ctx.load(gg.rmat(8, 8, seed=1))
    try:
        with pytest.raises(ps.ScanError) as ei:
            dg.set_zero_copy(True)
        assert ei.value.status == ps.SCAN_EINVAL
    finally:
        dg.free()
