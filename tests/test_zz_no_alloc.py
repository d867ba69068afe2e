"""The no-allocation counting entry point, for callers that cannot allocate
device memory (code running inside another framework's memory pool, under a
hard memory budget, or where a cudaMalloc/cudaFree would synchronise the
device at the wrong time).

Its counts are compared, slot by slot and with tolerance 0 (the counts are
integers), against the library's existing count path (a cache-building query
followed by scan_graph_copy_counts), on two calls in a row. The test
allocates its own device buffers with torch; the entry point allocates none.
The file name makes pytest collect it last.
"""
import numpy as np
import pytest

import graphgen as gg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ps():
    from paper_2311_12281_gb300 import _build
    _build.build()
    import paper_2311_12281_gb300 as mod
    return mod


def existing_counts(ps, g):
    with ps.Context(0) as ctx:
        dg = ctx.load(g)
        dg.query(1, 2, 2, ps.SCAN_Q_BUILD_CACHE)
        return dg.counts()


@pytest.mark.parametrize("which", ["rmat12", "chung_lu"])
def test_static_counts_match_the_existing_entry_point_twice(ps, which):
    torch = pytest.importorskip("torch")
    g = gg.rmat(12, 16, seed=7) if which == "rmat12" else gg.chung_lu(20000, 24.0, 2.1, seed=12)
    want = existing_counts(ps, g)
    off = torch.from_numpy(g.offsets).cuda()
    adj = torch.from_numpy(g.adj).cuda()
    stream = torch.cuda.Stream()
    for call in range(2):
        cn = torch.full((g.nnz,), -7, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        ps.scan_common_counts_static(off.data_ptr(), adj.data_ptr(), g.n, g.nnz, cn.data_ptr(), stream.cuda_stream)
        got = cn.cpu().numpy()
        bad = np.flatnonzero(got != want)
        assert bad.size == 0, f"call {call}: {bad.size} slots differ, first {bad[0]}: {got[bad[0]]} vs {want[bad[0]]}"


def test_static_counts_reject_too_large_and_malformed(ps):
    torch = pytest.importorskip("torch")
    # beyond the fixed scratch: rejected before any device work
    with pytest.raises(ps.ScanError) as ei:
        ps.scan_common_counts_static(16, 16, 1000, 20_000_000, 16, None)
    assert ei.value.status == ps.SCAN_EINVAL and "too large" in str(ei.value)
    # an asymmetric CSR is reported, and the next good call still works
    off = torch.tensor([0, 1, 2, 2], dtype=torch.int64, device="cuda")
    adj = torch.tensor([1, 2], dtype=torch.int32, device="cuda")
    cn = torch.zeros(2, dtype=torch.int32, device="cuda")
    with pytest.raises(ps.ScanError) as ei:
        ps.scan_common_counts_static(off.data_ptr(), adj.data_ptr(), 3, 2, cn.data_ptr(), None)
    assert ei.value.status == ps.SCAN_EINVAL
    g = gg.from_edges(4, [(0, 1), (1, 2), (0, 2), (2, 3)])
    off = torch.from_numpy(g.offsets).cuda()
    adj = torch.from_numpy(g.adj).cuda()
    cn = torch.zeros(g.nnz, dtype=torch.int32, device="cuda")
    ps.scan_common_counts_static(off.data_ptr(), adj.data_ptr(), g.n, g.nnz, cn.data_ptr(), None)
    assert np.array_equal(cn.cpu().numpy(), existing_counts(ps, g))
