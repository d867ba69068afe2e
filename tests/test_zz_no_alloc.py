"""The no-allocation counting entry point, for callers that cannot allocate
device memory (code running inside another framework's memory pool, under a
hard memory budget, or where a cudaMalloc/cudaFree would synchronise the
device at the wrong time).

Its counts are compared, slot by slot and with tolerance 0 (the counts are
integers), against the library's existing count path (a cache-building query
followed by scan_graph_copy_counts) and directly against the CPU oracle's
counts, on two calls in a row. Every input the entry point rejects is tried
once, each followed by a good call. The test allocates its own device
buffers with torch; the entry point allocates none. The file name makes
pytest collect it last.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle

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
    assert np.array_equal(want, oracle.common_counts(g))
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
        assert np.array_equal(got, oracle.common_counts(g)), f"call {call}: differs from the oracle"


# One case per rejection: (n, offsets, adj, the text the error must hold).
MALFORMED = {
    "odd nnz": (4, [0, 1, 1, 1, 1], [1], "bad sizes"),
    "offsets[0] != 0": (4, [1, 2, 3, 4, 4], [1, 0, 3, 2], "offsets"),
    "offsets decrease": (4, [0, 2, 1, 3, 4], [1, 2, 0, 0], "offsets"),
    "offsets[n] != nnz": (4, [0, 1, 2, 2, 2], [1, 0, 3, 2], "offsets"),
    "unsorted row": (4, [0, 2, 3, 4, 4], [2, 1, 0, 0], "slot 1 "),
    "duplicate in a row": (4, [0, 2, 4, 4, 4], [1, 1, 0, 0], "slot 1 "),
    "self-loop": (4, [0, 2, 4, 4, 4], [0, 1, 0, 1], "slot 0 "),
    "id out of range": (4, [0, 2, 4, 4, 4], [1, 9, 0, 9], "slot 1 "),
    "asymmetric": (3, [0, 1, 2, 2], [1, 2], "slot 0 "),
}


@pytest.mark.parametrize("case", sorted(MALFORMED))
def test_static_counts_reject_each_malformed_input(ps, case):
    torch = pytest.importorskip("torch")
    n, offs, adjs, text = MALFORMED[case]
    off = torch.tensor(offs, dtype=torch.int64, device="cuda")
    adj = torch.tensor(adjs, dtype=torch.int32, device="cuda")
    cn = torch.zeros(len(adjs), dtype=torch.int32, device="cuda")
    with pytest.raises(ps.ScanError) as ei:
        ps.scan_common_counts_static(off.data_ptr(), adj.data_ptr(), n, len(adjs), cn.data_ptr(), None)
    assert ei.value.status == ps.SCAN_EINVAL
    assert text in str(ei.value), f"{case}: {ei.value}"
    # the shared scratch carries nothing bad into the next good call
    g = gg.from_edges(5, [(0, 1), (1, 2), (0, 2), (2, 3), (3, 4), (2, 4)])
    off = torch.from_numpy(g.offsets).cuda()
    adj = torch.from_numpy(g.adj).cuda()
    cn = torch.full((g.nnz,), -1, dtype=torch.int32, device="cuda")
    ps.scan_common_counts_static(off.data_ptr(), adj.data_ptr(), g.n, g.nnz, cn.data_ptr(), None)
    assert np.array_equal(cn.cpu().numpy(), oracle.common_counts(g))


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
