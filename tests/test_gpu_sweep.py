"""Parameter sweeps (scan_query_sweep) against the oracle and single queries.

A sweep answers k (eps, mu) queries on one graph in order, each result's
copy to the host overlapping the next query (two device output sets used in
turn). Every answer must be bit-exact with the oracle at its (eps, mu) and
with the single-query call; the fallbacks (no room for the second set, a
partitioned graph, one query) must give the same answers; invalid
parameters anywhere in the list fail before any work; a bounded loop that
gives up in one query fails the whole sweep and leaves the context usable.
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
    union, _ = gg.disjoint_union([gg.rmat(9, 8, seed=s) for s in range(3)] + [gg.from_edges(7, [])])
    return {
        "fig1": fig1(),
        "rmat12": gg.rmat(12, 16, seed=5),
        "chung_lu": gg.chung_lu(5000, 20.0, 2.1, seed=8),
        "union_with_isolated": union,
        "edgeless": gg.from_edges(9, []),
        "empty": gg.from_csr(np.zeros(1, np.int64), np.zeros(0, np.int32)),
    }


# seven eps x three mu, with a repeat, so that both output sets are reused
SWEEP = [(p, q, mu) for (p, q) in [(1, 5), (3, 10), (2, 5), (1, 2), (3, 5), (7, 10), (9, 10)] for mu in (2, 3, 5)]
SWEEP.append((1, 2, 3))


@pytest.mark.parametrize("name", list(graphs().keys()))
@pytest.mark.parametrize("mode", ["RECOMPUTE", "AUTO", "BUILD_CACHE", "PLAIN"])
def test_sweep_matches_oracle_and_single_queries(ps, ctx, name, mode):
    g = graphs()[name]
    m = getattr(ps, "SCAN_Q_" + mode)
    cn = oracle.common_counts(g)
    dg = ctx.load(g)
    try:
        res = dg.sweep(SWEEP, m)
        assert len(res) == len(SWEEP)
        for (p, q, mu), r in zip(SWEEP, res):
            assert_same(r, oracle.scan_from_counts(g, cn, p, q, mu), f"{name} {mode} eps={p}/{q} mu={mu}")
        for j in (0, 7, len(SWEEP) - 1):
            p, q, mu = SWEEP[j]
            assert_same(dg.query(p, q, mu, m), res[j], f"{name} single query {j}")
    finally:
        dg.free()


def test_second_sweep_reuses_the_second_output_set(ps, ctx):
    g = gg.rmat(11, 16, seed=2)
    dg = ctx.load(g)
    try:
        before = ps.scan_graph_device_bytes(dg.handle)
        first = dg.sweep(SWEEP[:5], ps.SCAN_Q_RECOMPUTE)
        grown = ps.scan_graph_device_bytes(dg.handle)
        # the second set: core, cid, label for n + 1 vertices, room for nnz pairs, a count
        assert grown - before >= 6 * (g.n + 1) + 8 * g.nnz
        second = dg.sweep(SWEEP[:5], ps.SCAN_Q_RECOMPUTE)
        assert ps.scan_graph_device_bytes(dg.handle) == grown
        for a, b in zip(first, second):
            assert_same(a, b, "second sweep")
    finally:
        dg.free()


def test_results_outlive_later_sweeps_and_the_graph(ps, ctx):
    # each result owns its host arrays: later sweeps reuse the device sets, not them
    g = gg.chung_lu(3000, 12.0, 2.1, seed=3)
    dg = ctx.load(g)
    a = dg.sweep(SWEEP[:4], ps.SCAN_Q_RECOMPUTE)
    dg.sweep(SWEEP[4:9], ps.SCAN_Q_RECOMPUTE)
    dg.free()
    for (p, q, mu), r in zip(SWEEP[:4], a):
        assert_same(r, oracle.scan(g, p, q, mu), f"kept eps={p}/{q} mu={mu}")


def test_one_query_sweep(ps, ctx):
    g = gg.rmat(10, 8, seed=4)
    dg = ctx.load(g)
    try:
        (r,) = dg.sweep([(3, 5, 3)])
        assert_same(r, oracle.scan(g, 3, 5, 3))
    finally:
        dg.free()


def test_sweep_without_room_for_the_second_set_runs_one_query_at_a_time(ps):
    g = gg.chung_lu(20000, 16.0, 2.1, seed=3)
    with ps.Context(0) as probe:
        dg = probe.load(g)
        dg.query(1, 2, 3, ps.SCAN_Q_RECOMPUTE)
        need = probe.device_bytes
        dg.free()
    # room for the graph and its first query, not for another 8 nnz bytes of pairs
    c = ps.Context(0, budget_bytes=need + 4 * g.nnz)
    try:
        dg = c.load(g)
        dg.query(1, 2, 3, ps.SCAN_Q_RECOMPUTE)
        held = ps.scan_graph_device_bytes(dg.handle)
        res = dg.sweep(SWEEP[:6], ps.SCAN_Q_RECOMPUTE)
        assert ps.scan_graph_device_bytes(dg.handle) == held  # no second set
        for (p, q, mu), r in zip(SWEEP[:6], res):
            assert_same(r, oracle.scan(g, p, q, mu), f"budget eps={p}/{q} mu={mu}")
        dg.free()
        assert c.device_bytes == 0
    finally:
        c.close()


def test_partitioned_graph_sweeps_one_query_at_a_time(ps, ctx):
    g = gg.rmat(11, 16, seed=9)
    dg = ctx.load_partitioned(g, max(64, g.nnz // 7))
    try:
        assert dg.blocks > 1
        res = dg.sweep(SWEEP[:5])
        for (p, q, mu), r in zip(SWEEP[:5], res):
            assert_same(r, oracle.scan(g, p, q, mu), f"partitioned eps={p}/{q} mu={mu}")
    finally:
        dg.free()


@pytest.mark.parametrize("bad", [(0, 2, 3), (3, 2, 3), (1, 0, 3), (1, 2, 1)])
def test_invalid_parameters_anywhere_fail_before_any_work(ps, ctx, bad):
    g = gg.rmat(9, 8, seed=1)
    dg = ctx.load(g)
    try:
        launches = ctx.kernel_launches
        with pytest.raises(ps.ScanError) as ei:
            dg.sweep([(1, 2, 3), (3, 5, 2), bad, (1, 2, 2)])
        assert ei.value.status == ps.SCAN_EINVAL
        assert ctx.kernel_launches == launches
        with pytest.raises(ps.ScanError) as ei:
            dg.sweep([])
        assert ei.value.status == ps.SCAN_EINVAL
        assert_same(dg.sweep([(1, 2, 3), (3, 5, 2)])[1], oracle.scan(g, 3, 5, 2))
    finally:
        dg.free()


def test_a_loop_that_gives_up_fails_the_sweep_and_the_context_recovers(ps):
    # the square of a path: at mu = 2 one cluster spans every vertex, so a
    # union-find cap of one iteration gives up in every query
    n = 3000
    g = gg.from_edges(n + 5, [(i, i + 1) for i in range(n - 1)] + [(i, i + 2) for i in range(n - 2)])
    with ps.Context(0) as c:
        dg = c.load(g)
        ps.scan_ctx_set_loop_limit(c.handle, 1)
        with pytest.raises(ps.ScanError) as ei:
            dg.sweep([(1, 2, 2), (3, 5, 2), (1, 2, 3)], ps.SCAN_Q_RECOMPUTE)
        assert ei.value.status == ps.SCAN_ETIMEOUT, str(ei.value)
        ps.scan_ctx_set_loop_limit(c.handle, 0)
        res = dg.sweep([(1, 2, 2), (3, 5, 2), (1, 2, 3)], ps.SCAN_Q_RECOMPUTE)
        for (p, q, mu), r in zip([(1, 2, 2), (3, 5, 2), (1, 2, 3)], res):
            assert_same(r, oracle.scan(g, p, q, mu), f"after the cap eps={p}/{q} mu={mu}")
        dg.free()
