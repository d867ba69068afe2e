"""The query server: continuous batching over resident graphs with cached
counts. Every result must equal the single query run alone and the oracle,
whatever the mix, the admission order or the evictions (tolerance 0)."""
import random
import threading

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


def pool():
    graphs = [gg.rmat(10 + (k % 3), 16, seed=4000 + k) for k in range(6)]
    graphs += [gg.chung_lu(3000 + 700 * k, 12.0 + 4 * k, 2.1, seed=4100 + k) for k in range(4)]
    graphs += [gg.from_edges(4, [(0, 1), (1, 2), (0, 2)]), gg.from_edges(3, [])]
    return graphs


def requests(count, ngraphs, seed):
    rng = random.Random(seed)
    return [(rng.randrange(ngraphs), rng.randint(4, 16), 20, rng.randint(2, 10)) for _ in range(count)]


class Expected:
    """Oracle answers, memoised per (graph, eps, mu)."""

    def __init__(self, graphs):
        self.graphs = graphs
        self.cn = {}
        self.memo = {}

    def __call__(self, gi, p, q, mu):
        key = (gi, p, q, mu)
        if key not in self.memo:
            if gi not in self.cn:
                self.cn[gi] = oracle.common_counts(self.graphs[gi])
            self.memo[key] = oracle.scan_from_counts(self.graphs[gi], self.cn[gi], p, q, mu)
        return self.memo[key]


@pytest.mark.parametrize("use_cache", [True, False])
def test_results_in_the_mix_equal_results_alone(ps, use_cache):
    graphs = pool()
    want = Expected(graphs)
    reqs = requests(240, len(graphs), seed=7)
    # alone: one query at a time on a plain context
    alone = {}
    with ps.Context(0) as c:
        for gi in sorted({r[0] for r in reqs}):
            dg = c.load(graphs[gi])
            for r in {r for r in reqs if r[0] == gi}:
                alone[r] = dg.query(r[1], r[2], r[3], ps.SCAN_Q_RECOMPUTE)
    # mixed: submitted from 3 threads into 8 slots
    ctx = ps.scan_ctx_create(0)
    srv = ps.scan_server_create(ctx, max_inflight=8, use_cache=use_cache)
    try:
        ids = [ps.scan_server_add_graph(srv, g) for g in graphs]
        tickets = [None] * len(reqs)

        def submitter(part):
            for i in part:
                gi, p, q, mu = reqs[i]
                tickets[i] = ps.scan_server_submit(srv, ids[gi], p, q, mu)

        threads = [threading.Thread(target=submitter, args=(range(k, len(reqs), 3),)) for k in range(3)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        for i, r in enumerate(reqs):
            got, lat = ps.scan_server_wait(srv, tickets[i])
            assert lat >= 0
            assert_same(got, alone[r], f"request {i} {r} vs alone")
            assert_same(got, want(*r), f"request {i} {r} vs oracle")
        st = ps.scan_server_stats(srv)
        assert st["completed"] == len(reqs) and st["rejected"] == 0
        assert st["max_inflight"] > 1, "no two requests were ever in flight together"
        if use_cache:
            assert 0 < st["cache_builds"] <= len(graphs)
        else:
            assert st["cache_builds"] == 0
        assert st["p99_ms"] >= st["p50_ms"] > 0
    finally:
        ps.scan_server_destroy(srv)
        ps.scan_ctx_destroy(ctx)


def test_admission_evicts_caches_then_graphs_under_a_small_budget(ps):
    graphs = [gg.chung_lu(20000, 24.0, 2.1, seed=4200 + k) for k in range(6)]
    want = Expected(graphs)
    # measure one graph's footprint with its cache, then allow about two of them
    with ps.Context(0) as c:
        dg = c.load(graphs[0])
        dg.query(1, 2, 2, ps.SCAN_Q_BUILD_CACHE)
        one = c.device_bytes
    ctx = ps.scan_ctx_create(0, budget_bytes=int(2.3 * one))
    srv = ps.scan_server_create(ctx, max_inflight=4, use_cache=True)
    try:
        ids = [ps.scan_server_add_graph(srv, g) for g in graphs]
        reqs = requests(60, len(graphs), seed=11)
        tickets = [ps.scan_server_submit(srv, ids[gi], p, q, mu) for (gi, p, q, mu) in reqs]
        for t, r in zip(tickets, reqs):
            got, _ = ps.scan_server_wait(srv, t)
            assert_same(got, want(*r), f"{r}")
        st = ps.scan_server_stats(srv)
        assert st["completed"] == len(reqs)
        assert st["cache_evictions"] + st["graph_evictions"] > 0
        assert st["graph_loads"] > len({r[0] for r in reqs}) - 1
        assert st["device_bytes"] <= int(2.3 * one)
    finally:
        ps.scan_server_destroy(srv)
        ps.scan_ctx_destroy(ctx)


def test_a_request_that_can_never_fit_is_refused(ps):
    big = gg.chung_lu(50000, 30.0, 2.1, seed=9)
    small = gg.from_edges(3, [(0, 1), (1, 2)])
    ctx = ps.scan_ctx_create(0, budget_bytes=4 << 20)
    srv = ps.scan_server_create(ctx, max_inflight=2)
    try:
        gb = ps.scan_server_add_graph(srv, big)
        gs = ps.scan_server_add_graph(srv, small)
        t1 = ps.scan_server_submit(srv, gb, 1, 2, 3)
        t2 = ps.scan_server_submit(srv, gs, 1, 2, 2)
        with pytest.raises(ps.ScanError) as ei:
            ps.scan_server_wait(srv, t1)
        assert ei.value.status == ps.SCAN_EBUSY
        got, _ = ps.scan_server_wait(srv, t2)
        assert_same(got, oracle.scan(small, 1, 2, 2))
        with pytest.raises(ps.ScanError):
            ps.scan_server_submit(srv, 99, 1, 2, 2)
        with pytest.raises(ps.ScanError):
            ps.scan_server_submit(srv, gs, 3, 2, 2)
    finally:
        ps.scan_server_destroy(srv)
        ps.scan_ctx_destroy(ctx)


def test_poll(ps):
    g = gg.rmat(11, 16, seed=5)
    ctx = ps.scan_ctx_create(0)
    srv = ps.scan_server_create(ctx, max_inflight=2)
    try:
        gi = ps.scan_server_add_graph(srv, g)
        t = ps.scan_server_submit(srv, gi, 1, 2, 3)
        res = None
        for _ in range(200000):
            res = ps.scan_server_poll(srv, t)
            if res is not None:
                break
        assert res is not None
        assert_same(res[0], oracle.scan(g, 1, 2, 3))
    finally:
        ps.scan_server_destroy(srv)
        ps.scan_ctx_destroy(ctx)
