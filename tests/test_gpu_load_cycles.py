"""Graphs loaded, queried and freed over and over in one context.

These tests load, sweep and free graphs of different sizes in one context,
with other graphs alive in between, and check every answer against the
oracle and the context's byte count after each free; a budgeted context
must never report more than its budget.
"""
import pytest

import graphgen as gg
import oracle
from scan_checks import assert_same

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ps():
    from paper_2311_12281_gb300 import _build
    _build.build()
    import paper_2311_12281_gb300 as mod
    return mod


QUERIES = [(1, 2, 3), (3, 10, 2), (7, 10, 5)]


def check(dg, g, what):
    for (p, q, mu), r in zip(QUERIES, dg.sweep(QUERIES)):
        assert_same(r, oracle.scan(g, p, q, mu), f"{what} eps={p}/{q} mu={mu}")


def test_load_free_cycles_stay_exact(ps):
    shapes = [gg.rmat(12, 16, seed=1), gg.chung_lu(9000, 14.0, 2.1, seed=2), gg.rmat(11, 8, seed=3),
              gg.rmat(12, 16, seed=1), gg.chung_lu(20000, 10.0, 2.3, seed=4)]
    with ps.Context(0) as ctx:
        for i, g in enumerate(shapes):
            dg = ctx.load(g)
            check(dg, g, f"cycle {i}")
            dg.free()
            assert ctx.device_bytes == 0


def test_graphs_freed_and_loaded_while_other_graphs_live(ps):
    a, b, c = gg.rmat(12, 16, seed=5), gg.chung_lu(6000, 12.0, 2.1, seed=6), gg.rmat(12, 12, seed=7)
    with ps.Context(0) as ctx:
        da = ctx.load(a)
        db = ctx.load(b)
        check(da, a, "a")
        held_b = ps.scan_graph_device_bytes(db.handle)
        da.free()
        assert ctx.device_bytes == held_b
        dc = ctx.load(c)  # b still resident
        check(dc, c, "c")
        check(db, b, "b")
        dc.free()
        db.free()
        assert ctx.device_bytes == 0


def test_budgeted_context_reports_at_most_its_budget(ps):
    g = gg.chung_lu(20000, 16.0, 2.1, seed=3)
    with ps.Context(0) as probe:
        dg = probe.load(g)
        dg.query(1, 2, 3)
        need = probe.device_bytes
        dg.free()
    budget = need + (1 << 20)
    with ps.Context(0, budget_bytes=budget) as ctx:
        for i in range(3):
            dg = ctx.load(g)
            assert_same(dg.query(1, 2, 3), oracle.scan(g, 1, 2, 3), f"budgeted cycle {i}")
            assert ctx.device_bytes <= budget
            dg.free()
            assert ctx.device_bytes == 0
