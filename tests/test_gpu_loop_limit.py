"""The bounded union-find loops' error path, through the C ABI.

Every device loop of the library has an iteration cap; a query whose loops
run out returns SCAN_ETIMEOUT. scan_ctx_set_loop_limit lowers the
union-find cap (Algorithm 3's root walks and hook retries) so a test can
reach that path without any fault: with a cap of one iteration, any cluster
of two or more cores has a core whose root walk gives up. The next query,
with the compiled cap restored, must succeed on the same context and match
the oracle, resident and out of core.
"""
import numpy as np
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


def chain(n=3000):
    """The square of a path: every edge has sigma >= 1/2 and every vertex is a
    core at mu = 2, so one cluster spans all n vertices (a long union-find
    chain); a few isolated vertices at the end."""
    edges = [(i, i + 1) for i in range(n - 1)] + [(i, i + 2) for i in range(n - 2)]
    return gg.from_edges(n + 5, edges)


@pytest.mark.parametrize("mode", ["RECOMPUTE", "AUTO"])
def test_union_find_cap_gives_etimeout_then_the_context_recovers(ps, mode):
    g = chain()
    want = oracle.scan(g, 1, 2, 2)
    assert len(set(want["cid"][want["core"] == 1].tolist())) == 1
    m = getattr(ps, "SCAN_Q_" + mode)
    with ps.Context(0) as ctx:
        dg = ctx.load(g)
        if mode == "AUTO":
            dg.query(1, 2, 2, ps.SCAN_Q_BUILD_CACHE)
        assert_same(dg.query(1, 2, 2, m), want, "before the cap")  # also captures a replay
        assert_same(dg.query(1, 2, 2, m), want, "replayed")
        ps.scan_ctx_set_loop_limit(ctx.handle, 1)
        for _ in range(2):
            with pytest.raises(ps.ScanError) as ei:
                dg.query(1, 2, 2, m)
            assert ei.value.status == ps.SCAN_ETIMEOUT, str(ei.value)
        ps.scan_ctx_set_loop_limit(ctx.handle, 0)
        assert_same(dg.query(1, 2, 2, m), want, "after the cap is lifted")
        assert_same(dg.query(3, 5, 3, m), oracle.scan(g, 3, 5, 3), "another query after")


def test_union_find_cap_out_of_core(ps):
    g = chain(4000)
    want = oracle.scan(g, 1, 2, 2)
    with ps.Context(0) as ctx:
        dg = ctx.load_partitioned(g, block_slots=2000)
        assert dg.blocks > 4
        assert_same(dg.query(1, 2, 2), want, "partitioned, before the cap")
        ps.scan_ctx_set_loop_limit(ctx.handle, 1)
        with pytest.raises(ps.ScanError) as ei:
            dg.query(1, 2, 2)
        assert ei.value.status == ps.SCAN_ETIMEOUT, str(ei.value)
        ps.scan_ctx_set_loop_limit(ctx.handle, 0)
        assert_same(dg.query(1, 2, 2), want, "partitioned, after the cap is lifted")


def test_a_cap_above_the_chain_depth_changes_nothing(ps):
    # a generous cap (far above what this graph's loops need) gives the same answer
    g = gg.rmat(12, 8, seed=3)
    want = oracle.scan(g, 1, 2, 3)
    with ps.Context(0) as ctx:
        dg = ctx.load(g)
        ps.scan_ctx_set_loop_limit(ctx.handle, 1 << 16)
        assert_same(dg.query(1, 2, 3, ps.SCAN_Q_RECOMPUTE), want)
        ps.scan_ctx_set_loop_limit(ctx.handle, 0)
        assert_same(dg.query(1, 2, 3, ps.SCAN_Q_RECOMPUTE), want)
