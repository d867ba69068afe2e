"""Batched clustering of many graphs (each with its own eps, mu) vs the oracle,
graph by graph, bit-exact, through the C ABI."""
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


@pytest.fixture(scope="module")
def ctx(ps):
    c = ps.Context(0)
    yield c
    c.close()


def small_batch(count=60, seed=3100):
    specs = gg.chung_lu_batch_specs(count, seed)
    graphs = []
    for s in specs:
        n = max(2, s["n"] // 20)  # scaled down so the oracle stays fast
        graphs.append(gg.chung_lu(n, s["avg_deg"], 2.1, s["seed"]))
    # degenerate members: an edgeless graph, a single edge, an empty graph
    graphs += [gg.from_edges(5, []), gg.from_edges(2, [(0, 1)]),
               gg.from_csr(np.zeros(1, np.int64), np.zeros(0, np.int32))]
    params = [(s["eps"][0], s["eps"][1], s["mu"]) for s in specs] + [(1, 2, 2), (1, 2, 2), (1, 2, 2)]
    return graphs, params


@pytest.mark.parametrize("mode", ["recompute", "plain", "cache"])
def test_batch_equals_each_graph_alone(ps, ctx, mode):
    graphs, params = small_batch()
    b = ps.scan_batch_load(ctx.handle, graphs)
    try:
        m = {"recompute": ps.SCAN_Q_RECOMPUTE, "plain": ps.SCAN_Q_PLAIN, "cache": ps.SCAN_Q_BUILD_CACHE}[mode]
        res = ps.scan_batch_query(b, params, m)
        if mode == "cache":  # second pass answered from the cached counts
            res = ps.scan_batch_query(b, params, ps.SCAN_Q_AUTO)
        assert len(res) == len(graphs)
        for j, (g, (p, q, mu), r) in enumerate(zip(graphs, params, res)):
            assert_same(r, oracle.scan(g, p, q, mu), f"batch member {j} (n={g.n}) eps={p}/{q} mu={mu}")
    finally:
        ps.scan_batch_free(b)


def test_batch_parameters_change_between_queries(ps, ctx):
    graphs, params = small_batch(30, seed=4200)
    b = ps.scan_batch_load(ctx.handle, graphs)
    try:
        rng = np.random.default_rng(0)
        for _ in range(3):
            new = [(int(rng.integers(4, 17)), 20, int(rng.integers(2, 9))) for _ in graphs]
            res = ps.scan_batch_query(b, new)
            for g, (p, q, mu), r in zip(graphs, new, res):
                assert_same(r, oracle.scan(g, p, q, mu))
    finally:
        ps.scan_batch_free(b)


def test_query_batch_over_loaded_graphs(ps, ctx):
    graphs, params = small_batch(12, seed=5300)
    handles = [ps.scan_graph_load(ctx.handle, g.n, g.offsets, g.adj) for g in graphs]
    try:
        res = ps.scan_query_batch(handles, params)
        for g, (p, q, mu), r in zip(graphs, params, res):
            assert_same(r, oracle.scan(g, p, q, mu))
    finally:
        for h in handles:
            ps.scan_graph_free(h)


def test_batch_larger_than_one_upload_block(ps, ctx):
    # 24 R-MAT graphs of about 1M edges: the union's adjacency (about 190 MB)
    # goes up in several pinned blocks, some graphs straddling two of them.
    # Each member must match the same graph queried alone (a path the oracle
    # checks at smaller sizes) and its counts must match the oracle on samples.
    graphs = [gg.rmat(16, 16, seed=600 + j) for j in range(24)]
    assert sum(g.adj.nbytes for g in graphs) > (128 << 20)
    params = [(1 + j % 4, 5, 2 + j % 5) for j in range(len(graphs))]
    b = ps.scan_batch_load(ctx.handle, graphs)
    try:
        res = ps.scan_batch_query(b, params)
        for j, (g, (p, q, mu), r) in enumerate(zip(graphs, params, res)):
            dg = ctx.load(g)
            try:
                assert_same(r, dg.query(p, q, mu, ps.SCAN_Q_RECOMPUTE), f"member {j}")
            finally:
                dg.free()
        # the union's counts, slot by slot, against the oracle on a sample
        cache = ps.scan_batch_query(b, params, ps.SCAN_Q_BUILD_CACHE)
        for r, want in zip(cache, res):
            assert_same(r, want)
        counts = ps.scan_graph_copy_counts(ps.scan_batch_union(b), sum(g.nnz for g in graphs))
        base = 0
        rng = np.random.default_rng(5)
        for g in graphs[:3]:
            slots = rng.integers(0, g.nnz, 2000)
            assert np.array_equal(counts[base + slots], oracle.counts_for_slots(g, slots))
            base += g.nnz
    finally:
        ps.scan_batch_free(b)


def test_batch_rejects_bad_members(ps, ctx):
    bad = gg.from_csr([0, 1, 2, 2], [1, 2])  # asymmetric
    with pytest.raises(ps.ScanError) as ei:
        ps.scan_batch_load(ctx.handle, [gg.from_edges(3, [(0, 1)]), bad])
    assert ei.value.status == ps.SCAN_EINVAL
    b = ps.scan_batch_load(ctx.handle, [gg.from_edges(3, [(0, 1)])])
    with pytest.raises(ps.ScanError):
        ps.scan_batch_query(b, [(0, 1, 2)])
    ps.scan_batch_free(b)


def test_replayed_batch_queries_follow_new_parameters(ps, ctx):
    # the second and later device queries on the same buffers replay a captured
    # CUDA graph; each must see its own parameters
    torch = pytest.importorskip("torch")
    graphs, _ = small_batch(20, seed=4300)
    b = ps.scan_batch_load(ctx.handle, graphs)
    try:
        n = sum(g.n for g in graphs)
        nnz = sum(g.nnz for g in graphs)
        core = torch.zeros(n, dtype=torch.uint8, device="cuda")
        cid = torch.zeros(n, dtype=torch.int32, device="cuda")
        label = torch.zeros(n, dtype=torch.uint8, device="cuda")
        pairs = torch.zeros(2 * max(nnz, 1), dtype=torch.int32, device="cuda")
        npairs = torch.zeros(1, dtype=torch.int64, device="cuda")
        rng = np.random.default_rng(7)
        for round_ in range(4):
            new = [(int(rng.integers(4, 17)), 20, int(rng.integers(2, 9))) for _ in graphs]
            before = ps.scan_ctx_kernel_launches(ctx.handle)
            ps.scan_batch_query_device(b, new, ps.SCAN_Q_RECOMPUTE, core.data_ptr(), cid.data_ptr(),
                                       label.data_ptr(), pairs.data_ptr(), nnz, npairs.data_ptr())
            ps.scan_ctx_sync(ctx.handle)
            assert ps.scan_ctx_kernel_launches(ctx.handle) > before  # replays count their kernels too
            base = 0
            got_core, got_cid = core.cpu().numpy(), cid.cpu().numpy()
            for g, (p, q, mu) in zip(graphs, new):
                want = oracle.scan(g, p, q, mu)
                assert np.array_equal(got_core[base:base + g.n], want["core"]), f"round {round_}"
                c = got_cid[base:base + g.n].astype(np.int64)
                c[c >= 0] -= base
                assert np.array_equal(c, want["cid"]), f"round {round_}"
                base += g.n
    finally:
        ps.scan_batch_free(b)


@pytest.mark.parametrize("mode", ["recompute", "cache"])
def test_packed_batch_result_equals_per_graph_results_and_oracle(ps, ctx, mode):
    # one result over the whole batch: each member's ranges hold its own ids
    graphs, params = small_batch(40, seed=6100)
    b = ps.scan_batch_load(ctx.handle, graphs)
    try:
        m = ps.SCAN_Q_RECOMPUTE if mode == "recompute" else ps.SCAN_Q_BUILD_CACHE
        packed = ps.scan_batch_query_packed(b, params, m)
        per = ps.scan_batch_query(b, params, ps.SCAN_Q_AUTO if mode == "cache" else m)
        assert len(packed) == len(per) == len(graphs)
        for j, (g, (p, q, mu)) in enumerate(zip(graphs, params)):
            assert packed[j]["core"].shape == (g.n,)
            assert_same(packed[j], per[j], f"packed vs per-graph member {j}")
            assert_same(packed[j], oracle.scan(g, p, q, mu), f"packed member {j} eps={p}/{q} mu={mu}")
        # the views outlive the batch
        keep = packed[3]
        ps.scan_batch_free(b)
        b = None
        assert_same(keep, oracle.scan(graphs[3], *params[3]), "kept view")
    finally:
        if b is not None:
            ps.scan_batch_free(b)
