"""The benchmark's byte accounting and the counting method's enumeration,
checked by brute force on small graphs (CPU only).

- The degree-oriented enumeration (each triangle a < b < c found once, at b,
  by looking for c in the part of out(a) after b) finds every triangle once:
  summed over edges, the open common counts from the oracle are three times
  the triangles it finds.
- The streamed-suffix term of the kernel's own bytes is that enumeration's
  candidate count, sum over a of d+(a)(d+(a)-1)/2.
- The degree prune in the per-edge byte count never contradicts the exact
  eps-test: an edge pruned as dissimilar is not similar and one pruned as
  similar is."""
import importlib.util
import os

import numpy as np

import graphgen as gg
import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_bytes_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _out_lists(g):
    deg = g.degrees()
    rank = {v: (int(deg[v]), v) for v in range(g.n)}
    out = []
    for a in range(g.n):
        row = g.adj[g.offsets[a]:g.offsets[a + 1]]
        out.append(sorted((int(b) for b in row if rank[int(b)] > rank[a]), key=lambda b: rank[b]))
    return out


def test_each_triangle_is_found_once_at_its_middle_vertex():
    for seed in (1, 2, 3):
        g = gg.rmat(9, 8, seed=seed)
        out = _out_lists(g)
        outset = [set(o) for o in out]
        found = 0
        for a in range(g.n):
            for i, b in enumerate(out[a]):
                found += sum(1 for c in out[a][i + 1:] if c in outset[b])
        assert found > 0
        cn = oracle.common_counts(g).astype(np.int64)
        # every slot holds |N[u] & N[v]| = open count + 2; each edge has two slots
        assert int((cn - 2).sum()) == 2 * 3 * found


def test_streamed_suffix_term_is_the_candidate_count():
    bench = _bench()
    g = gg.rmat(9, 8, seed=4)
    out = _out_lists(g)
    candidates = sum(len(o) * (len(o) - 1) // 2 for o in out)
    rest = 4.0 * g.m + 12.0 * g.nnz + 12.0 * g.m + 1.0 * g.m + 8.0 * (g.n + 1)
    assert bench.forward_bytes(g) == 4.0 * candidates + rest


def test_degree_prune_agrees_with_the_exact_test():
    bench = _bench()
    g = gg.chung_lu(2000, 12.0, 2.1, seed=5)
    cn = oracle.common_counts(g).astype(np.int64)
    deg = g.degrees()
    src = np.repeat(np.arange(g.n, dtype=np.int64), deg)
    dst = g.adj.astype(np.int64)
    d1, d2 = deg[src] + 1, deg[dst] + 1
    dmin, dmax = np.minimum(d1, d2), np.maximum(d1, d2)
    for (p, q) in [(1, 5), (3, 10), (1, 2), (7, 10), (4, 5)]:
        similar = cn * cn * q * q >= p * p * d1 * d2  # exact in int64 at these sizes
        never = dmin * q * q < p * p * dmax
        always = 4 * q * q >= p * p * dmin * dmax
        assert not (never & similar).any()
        assert similar[always].all()
        # the per-edge byte count drops exactly these edges' intersections
        dmin1, dmax1 = bench.oriented_dmin(g)
        live = ~(dmin1 * q * q < p * p * dmax1) & ~(4 * q * q >= p * p * dmin1 * dmax1)
        want = 4.0 * float((dmin1[live] - 1).sum()) + 5.0 * g.nnz + 8.0 * (g.n + 1)
        assert bench.algorithmic_bytes(g, dmin1, dmax1, p, q) == want
