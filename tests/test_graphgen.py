"""The seeded input generators: deterministic, simple, symmetric CSR (CPU only)."""
import numpy as np

import graphgen as gg
import oracle

# R-MAT sampling is integer-only, so this digest holds on every platform and
# for any thread count (scale 14, edge factor 8, (.57, .19, .19, .05), seed 1).
RMAT_S14_SHA256 = "9c08fbfa2ab09c175d1ba9b61ffa3e81f156b4b14d7a42b3bf9c2b8aca0fd669"


def test_rmat_s14_is_reproducible_and_valid():
    g = gg.rmat_s14()
    st = gg.stats(g)
    assert st["sha256"] == RMAT_S14_SHA256
    assert st["n"] == 16384 and st["m"] == 114036
    assert oracle.validate(g) == -1
    assert gg.stats(gg.rmat_s14())["sha256"] == RMAT_S14_SHA256


def test_chung_lu_and_edges_are_simple_graphs():
    for g in (gg.chung_lu(5000, 20.0, 2.1, seed=9), gg.rmat(9, 16, seed=4),
              gg.from_edges(5, [(0, 1), (1, 0), (2, 2), (3, 4), (4, 3), (1, 3)])):
        assert oracle.validate(g) == -1
    g = gg.from_edges(5, [(0, 1), (1, 0), (2, 2), (3, 4), (4, 3), (1, 3)])
    assert g.offsets.tolist() == [0, 1, 3, 3, 5, 6]
    assert g.adj.tolist() == [1, 0, 3, 1, 4, 3]


def test_batch_specs_follow_the_recipe():
    specs = gg.chung_lu_batch_specs(256)
    ns = np.array([s["n"] for s in specs])
    assert ns.min() >= 100 and ns.max() <= 50000
    assert all(4 <= s["avg_deg"] <= 64 for s in specs)
    assert all(s["eps"][1] == 20 and 4 <= s["eps"][0] <= 16 for s in specs)
    assert all(2 <= s["mu"] <= 8 for s in specs)
    assert specs == gg.chung_lu_batch_specs(256)
