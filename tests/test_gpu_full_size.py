"""Full-size parity on the benchmark workload: R-MAT scale 22 (4.19M vertices,
64.2M undirected edges), the 21-query eps x mu sweep, in the benchmark's launch
configuration (device-resident query, full recompute with degree pruning).

The oracle's per-slot counts are computed once (all host cores) and every
query is then answered by the oracle's remaining steps from those counts; the
GPU's counts are checked against them slot by slot first.
"""
import os

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
def s22():
    g = gg.rmat_s22()
    cn = oracle.common_counts(g, threads=os.cpu_count())
    return g, cn


@pytest.fixture(scope="module")
def loaded(ps, s22):
    pytest.importorskip("torch")
    g, _ = s22
    ctx = ps.Context(0)
    dg = ctx.load(g)
    yield ctx, dg
    ctx.close()


def test_counts_bit_exact(ps, s22, loaded):
    g, cn = s22
    ctx, dg = loaded
    dg.query(1, 2, 5, ps.SCAN_Q_BUILD_CACHE)
    got = dg.counts()
    bad = np.flatnonzero(got != cn)
    assert bad.size == 0, f"{bad.size} slots differ, first slot {bad[0]}: {got[bad[0]]} vs {cn[bad[0]]}"
    dg.drop_cache()


def test_sweep_bit_exact_device_resident(ps, s22, loaded):
    torch = pytest.importorskip("torch")
    g, cn = s22
    ctx, dg = loaded
    n = g.n
    core = torch.empty(n, dtype=torch.uint8, device="cuda")
    cid = torch.empty(n, dtype=torch.int32, device="cuda")
    label = torch.empty(n, dtype=torch.uint8, device="cuda")
    pairs = torch.empty(2 * g.nnz, dtype=torch.int32, device="cuda")
    npairs = torch.empty(1, dtype=torch.int64, device="cuda")
    for (p, q) in gg.EPS_SWEEP:
        for mu in gg.MU_SWEEP:
            ps.scan_query_device(dg.handle, p, q, mu, ps.SCAN_Q_RECOMPUTE, core.data_ptr(), cid.data_ptr(),
                                 label.data_ptr(), pairs.data_ptr(), g.nnz, npairs.data_ptr())
            ps.scan_ctx_sync(ctx.handle)
            k = int(npairs.item())
            got = {"core": core.cpu().numpy(), "cid": cid.cpu().numpy(), "label": label.cpu().numpy(),
                   "pairs": pairs[: 2 * k].cpu().numpy().reshape(k, 2)}
            assert_same(got, oracle.scan_from_counts(g, cn, p, q, mu), f"rmat_s22 eps={p}/{q} mu={mu}")


def test_plain_path_matches_on_one_query(ps, s22, loaded):
    g, cn = s22
    ctx, dg = loaded
    assert_same(dg.query(1, 2, 5, ps.SCAN_Q_PLAIN), oracle.scan_from_counts(g, cn, 1, 2, 5), "plain path")


def test_cached_queries_beyond_l2_match_recompute(ps):
    # a graph whose similarity array and count cache are larger than L2: the
    # cached answers must equal the recompute path's (checked against the
    # oracle above) on every array, and the cached counts the oracle's on
    # sampled slots
    g = gg.chung_lu(2_500_000, 64.0, 2.1, seed=9)
    assert g.nnz > (1 << 27)
    with ps.Context(0) as ctx:
        dg = ctx.load(g)
        first = dg.query(1, 2, 3, ps.SCAN_Q_BUILD_CACHE)
        assert_same(first, dg.query(1, 2, 3, ps.SCAN_Q_RECOMPUTE))
        for (p, q, mu) in [(1, 5, 2), (3, 5, 5), (4, 5, 10)]:
            assert_same(dg.query(p, q, mu, ps.SCAN_Q_AUTO), dg.query(p, q, mu, ps.SCAN_Q_RECOMPUTE),
                        f"eps={p}/{q} mu={mu}")
        counts = dg.counts()
    rng = np.random.default_rng(5)
    slots = np.sort(rng.choice(g.nnz, 20000, replace=False)).astype(np.int64)
    assert np.array_equal(counts[slots], oracle.counts_for_slots(g, slots))
