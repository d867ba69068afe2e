"""Full-size parity of the batched, serving and out-of-core workloads.

* 4,096 Chung-Lu graphs (exponent 2.1, n log-uniform in [100, 50,000], mean
  degree uniform in [4, 64]), each with its own (eps, mu), clustered as one
  batch: every member's result equals the oracle's, compared by digest (the
  oracle runs in spawned worker processes while the GPU works).
* The serving workload's big graph (Chung-Lu, 16M vertices, mean sampled
  degree 72): the cached per-slot counts against the oracle's on a uniform
  sample of slots, and the core flags of served queries against the oracle's
  on sampled vertices (each from the oracle's counts of its whole row). The
  whole count array and whole served answers are compared in the slow test.
* R-MAT scale 27 out of core under an 8 GB device budget (slow test): the
  partitioned result equals the resident one, array by array; the resident
  counts match the oracle's on sampled slots and the core flags on sampled
  vertices.
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

import graphgen as gg
import oracle
import oracle_pool
from scan_checks import assert_same

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ps():
    from paper_2311_12281_gb300 import _build
    _build.build()
    import paper_2311_12281_gb300 as mod
    return mod


def sampled_core_flags(g, verts, p, q, mu):
    """Core flags of the given vertices by the oracle: the closed counts of
    every slot of their rows (oracle_counts_for_slots), the exact eps-test in
    Python integers, and |N_eps[v]| = 1 + similar neighbours >= mu."""
    off = g.offsets
    deg = np.diff(off).astype(np.int64)
    rows = [np.arange(off[v], off[v + 1], dtype=np.int64) for v in verts]
    slots = np.concatenate(rows) if rows else np.zeros(0, np.int64)
    cn = oracle.counts_for_slots(g, slots, threads=os.cpu_count())
    out, k = [], 0
    for v, r in zip(verts, rows):
        c = cn[k:k + len(r)]
        k += len(r)
        nb = g.adj[r].astype(np.int64)
        sim = sum(1 for cc, w in zip(c.tolist(), nb.tolist())
                  if cc * cc * q * q >= p * p * (int(deg[v]) + 1) * (int(deg[w]) + 1))
        out.append(1 if 1 + sim >= mu else 0)
    return np.array(out, dtype=np.uint8)


def sample_vertices(g, count, seed):
    """Uniform vertices plus the highest-degree ones (a fixed few, so hub rows
    are covered), sorted."""
    rng = np.random.default_rng(seed)
    deg = np.diff(g.offsets)
    uni = rng.choice(g.n, size=min(count, g.n), replace=False)
    top = np.argsort(deg)[-8:]
    return np.unique(np.concatenate([uni, top]))


# ------------------------------------------------------------ 4,096 graphs
def test_batch_4096_full_size_every_member_equals_the_oracle(ps):
    specs = gg.chung_lu_batch_specs(4096)
    order = sorted(range(len(specs)), key=lambda i: -specs[i]["n"] * specs[i]["avg_deg"])
    pool = mp.get_context("spawn").Pool(os.cpu_count())
    try:
        pending = pool.map_async(oracle_pool.oracle_member_digest, [specs[i] for i in order], chunksize=4)
        graphs = [oracle_pool.chung_lu_member(s) for s in specs]
        params = [(s["eps"][0], s["eps"][1], s["mu"]) for s in specs]
        assert sum(g.m for g in graphs) > 500_000_000
        with ps.Context(0) as ctx:
            b = ps.scan_batch_load(ctx.handle, graphs)
            try:
                res = ps.scan_batch_query(b, params, ps.SCAN_Q_RECOMPUTE)
                got = [oracle_pool.digest(r) for r in res]
                del res
            finally:
                ps.scan_batch_free(b)
        want_ordered = pending.get(timeout=3000)
    finally:
        pool.terminate()
    want = [None] * len(specs)
    for i, d in zip(order, want_ordered):
        want[i] = d
    bad = [i for i in range(len(specs)) if got[i] != want[i]]
    if bad:
        i = bad[0]
        with ps.Context(0) as ctx:
            dg = ctx.load(graphs[i])
            assert_same(dg.query(*params[i], ps.SCAN_Q_RECOMPUTE), oracle.scan(graphs[i], *params[i]),
                        f"member {i} (n={graphs[i].n}) of {len(bad)} differing")
        raise AssertionError(f"{len(bad)} members differ in the batch, first {i}, which agrees alone")


# ------------------------------------------------------------ serving graph
@pytest.fixture(scope="module")
def big():
    return gg.chung_lu(16_000_000, 72.0, 2.1, seed=4)


SERVED = [(4, 20, 2), (10, 20, 5), (16, 20, 10)]


def test_serving_graph_counts_and_served_cores_on_samples(ps, big):
    g = big
    ctx = ps.scan_ctx_create(0)
    srv = ps.scan_server_create(ctx, max_inflight=4, use_cache=True)
    try:
        gid = ps.scan_server_add_graph(srv, g)
        answers = [ps.scan_server_wait(srv, ps.scan_server_submit(srv, gid, p, q, mu))[0] for (p, q, mu) in SERVED]
    finally:
        ps.scan_server_destroy(srv)
        ps.scan_ctx_destroy(ctx)
    with ps.Context(0) as c2:
        dg = c2.load(g)
        dg.query(1, 2, 2, ps.SCAN_Q_BUILD_CACHE)
        counts = dg.counts()
    rng = np.random.default_rng(44)
    slots = np.sort(rng.choice(g.nnz, 1_000_000, replace=False)).astype(np.int64)
    want = oracle.counts_for_slots(g, slots, threads=os.cpu_count())
    bad = np.flatnonzero(counts[slots] != want)
    assert bad.size == 0, f"{bad.size} sampled slots differ, first slot {slots[bad[0]]}"
    verts = sample_vertices(g, 3000, 45)
    for (p, q, mu), r in zip(SERVED, answers):
        assert r["core"].shape == (g.n,)
        got = r["core"][verts]
        exp = sampled_core_flags(g, verts, p, q, mu)
        diff = np.flatnonzero(got != exp)
        assert diff.size == 0, f"eps={p}/{q} mu={mu}: core of vertex {verts[diff[0]]} differs"


@pytest.mark.slow
def test_serving_graph_whole_counts_and_served_answers(ps, big):
    g = big
    want_cn = oracle.common_counts(g, threads=os.cpu_count())
    ctx = ps.scan_ctx_create(0)
    srv = ps.scan_server_create(ctx, max_inflight=4, use_cache=True)
    try:
        gid = ps.scan_server_add_graph(srv, g)
        for (p, q, mu) in SERVED:
            r = ps.scan_server_wait(srv, ps.scan_server_submit(srv, gid, p, q, mu))[0]
            assert_same(r, oracle.scan_from_counts(g, want_cn, p, q, mu), f"served eps={p}/{q} mu={mu}")
    finally:
        ps.scan_server_destroy(srv)
        ps.scan_ctx_destroy(ctx)
    with ps.Context(0) as c2:
        dg = c2.load(g)
        dg.query(1, 2, 2, ps.SCAN_Q_BUILD_CACHE)
        got = dg.counts()
    bad = np.flatnonzero(got != want_cn)
    assert bad.size == 0, f"{bad.size} slots differ, first {bad[0]}"


# ------------------------------------------------------------ out of core
@pytest.mark.slow
def test_out_of_core_scale_27_equals_resident_and_oracle_samples(ps):
    g = gg.rmat(27, 16, seed=5)
    p, q, mu = 1, 2, 5
    with ps.Context(0, budget_bytes=8 << 30) as ctx:
        dg = ctx.load_partitioned(g)
        assert dg.blocks > 1
        part = dg.query(p, q, mu)
        part = {k: np.array(v) for k, v in part.items()}
    with ps.Context(0) as c2:
        h = c2.load(g)
        res = h.query(p, q, mu, ps.SCAN_Q_BUILD_CACHE)
        assert_same(part, res, "partitioned vs resident")
        counts = h.counts()
    rng = np.random.default_rng(27)
    slots = np.sort(rng.choice(g.nnz, 200_000, replace=False)).astype(np.int64)
    want = oracle.counts_for_slots(g, slots, threads=os.cpu_count())
    bad = np.flatnonzero(counts[slots] != want)
    assert bad.size == 0, f"{bad.size} sampled slots differ, first slot {slots[bad[0]]}"
    verts = sample_vertices(g, 2000, 28)
    exp = sampled_core_flags(g, verts, p, q, mu)
    diff = np.flatnonzero(res["core"][verts] != exp)
    assert diff.size == 0, f"core of vertex {verts[diff[0]]} differs"
