"""Pins of the CPU oracle to facts outside itself (runs without a GPU).

Each test ties the oracle to something the paper or the mathematics fixes:
the worked values the paper prints (Examples 2.1, 3.1, 4.2, 4.3), closed
forms, the equality boundary of the eps-test, a library matrix product for
the common counts, a literal set-definition brute force, and invariants.
"""
import math
import os
import random

import numpy as np
import pytest
import scipy.sparse as sp

import graphgen as gg
import oracle
from conftest import load_golden
from scan_checks import CORE, BORDER, HUB, OUTLIER, assert_same, check_invariants


def fig1():
    gd = load_golden("fig1.txt")
    n = int(gd["n"][0])
    e = list(map(int, gd["edges"][0].split()))
    edges = list(zip(e[0::2], e[1::2]))
    return gd, n, edges


def test_fig1_roles_match_the_papers_statements():
    gd, n, edges = fig1()
    p, q = map(int, gd["eps"][0].split())
    mu = int(gd["mu"][0])
    g = gg.from_edges(n, edges)
    r = oracle.scan(g, p, q, mu)
    cores = set(map(int, gd["core"][0].split()))
    assert set(np.flatnonzero(r["core"]).tolist()) == cores
    for tok in gd["cid"][0].split():
        v, c = map(int, tok.split(":"))
        assert r["cid"][v] == c
    assert [tuple(x) for x in r["pairs"].tolist()] == [tuple(map(int, t.split(":"))) for t in gd["border"][0].split()]
    hubs = set(map(int, gd["hub"][0].split()))
    outl = set(map(int, gd["outlier"][0].split()))
    assert set(np.flatnonzero(r["label"] == HUB).tolist()) == hubs
    assert set(np.flatnonzero(r["label"] == OUTLIER).tolist()) == outl
    assert len(set(r["cid"][r["core"] == 1].tolist())) == 2  # two clusters


def test_worked_similarity_of_v0_v1():
    # Example 3.1 / 4.2: |N[v0] & N[v1]| = 2 + 3 = 5, |N[v0]| = 8, |N[v1]| = 5,
    # sigma = 5/sqrt(40) = 0.79 > 0.6
    gd, n, edges = fig1()
    g = gg.from_edges(n, edges)
    cn = oracle.common_counts(g)
    u, v, c = map(int, gd["common"][0].split())
    slot = int(g.offsets[u]) + int(np.searchsorted(g.adj[g.offsets[u]:g.offsets[u + 1]], v))
    assert cn[slot] == c == 5
    assert g.degrees()[0] + 1 == 8 and g.degrees()[1] + 1 == 5
    assert abs(c / math.sqrt(8 * 5) - 0.79) < 0.005
    # Example 3.1: N_eps[v0] = {v0, v1, v4, v7} at eps = 0.6
    want = set(map(int, gd["eps_neighbourhood"][0].split(":")[1].split()))
    row = g.adj[g.offsets[0]:g.offsets[1]]
    deg = g.degrees()
    got = {0} | {int(w) for k, w in enumerate(row)
                 if cn[g.offsets[0] + k] ** 2 * 25 >= 9 * (deg[0] + 1) * (deg[w] + 1)}
    assert got == want


def test_common_counts_equal_the_matrix_square():
    # |N[u] & N[v]| - 2 = (A^2)[u, v] for every edge (u, v): scipy's sparse product
    for seed in range(3):
        g = gg.chung_lu(600, 12.0, 2.1, seed=seed + 11)
        A = sp.csr_matrix((np.ones(g.nnz, dtype=np.int64), g.adj, g.offsets), shape=(g.n, g.n))
        A2 = (A @ A).tocsr()
        src = np.repeat(np.arange(g.n), g.degrees())
        want = np.asarray(A2[src, g.adj]).ravel() + 2
        assert np.array_equal(oracle.common_counts(g), want)
        assert np.array_equal(oracle.common_counts(g, threads=3), want)


def slot_pin_graphs():
    """Graphs for the per-slot counts: isolated vertices between non-empty
    rows (empty rows share their offset with the next row), and a hub whose
    degree is more than 32 times its neighbours' (the binary-search branch),
    with partner leaves so that those edges have common neighbours."""
    hub_edges = [(0, k) for k in range(1, 121)] + [(k, k + 1) for k in range(1, 120, 2)]
    sparse_edges = [(1, 5), (5, 9), (1, 9), (9, 14), (14, 20), (20, 5), (27, 28)]
    return [gg.from_edges(126, hub_edges + [(123, 124)]), gg.from_edges(30, sparse_edges),
            gg.chung_lu(500, 3.0, 2.1, seed=5), gg.rmat(9, 8, seed=3)]


def test_counts_for_slots_equal_the_matrix_square():
    # the sampled full-size checker: every slot, in a shuffled order, against
    # (A^2)[u, v] + 2 from scipy's sparse product
    rng = np.random.default_rng(0)
    for g in slot_pin_graphs():
        deg = g.degrees()
        assert (deg == 0).any()
        A = sp.csr_matrix((np.ones(g.nnz, dtype=np.int64), g.adj, g.offsets), shape=(g.n, g.n))
        src = np.repeat(np.arange(g.n), deg)
        want = np.asarray((A @ A).tocsr()[src, g.adj]).ravel() + 2
        slots = rng.permutation(g.nnz)
        assert np.array_equal(oracle.counts_for_slots(g, slots), want[slots])
        assert np.array_equal(oracle.counts_for_slots(g, slots, threads=3), want[slots])
    hub = slot_pin_graphs()[0]
    d = hub.degrees()
    assert d[0] == 120 and d[1] == 2 and d[0] // d[1] > 32  # the binary-search branch runs


def test_eps_equality_boundary_is_inclusive():
    # double star u=0 - v=1 with two leaves each: sigma(u, v) = 2/sqrt(4*4) = 1/2 exactly
    edges = [(0, 1), (0, 2), (0, 3), (1, 4), (1, 5)]
    g = gg.from_edges(6, edges)
    at = oracle.scan(g, 1, 2, 3)
    assert at["core"][:2].tolist() == [1, 1] and at["cid"][0] == at["cid"][1] == 0
    above = oracle.scan(g, 501, 1000, 3)
    assert above["core"][:2].tolist() == [1, 1] and above["cid"][1] == 1  # split in two
    # a rational equal to 1/2 in other terms gives the same answer (homogeneous test)
    assert_same(oracle.scan(g, 7, 14, 3), at)


def test_equality_grid_against_exact_rationals():
    # every (c, du, dv) with du, dv <= 24 that sits exactly on a sweep eps:
    # build the graph K_2 + (c-2) shared neighbours + private leaves and check S
    from fractions import Fraction
    cases = 0
    for (p, q) in gg.EPS_SWEEP:
        for du in range(2, 25):
            for dv in range(du, 25):
                for c in range(2, du + 1):
                    if Fraction(c * c, du * dv) != Fraction(p * p, q * q):
                        continue
                    shared = c - 2
                    lu, lv = du - 2 - shared, dv - 2 - shared
                    edges = [(0, 1)] + [(x, 2 + k) for k in range(shared) for x in (0, 1)]
                    nxt = 2 + shared
                    edges += [(0, nxt + k) for k in range(lu)]
                    nxt += lu
                    edges += [(1, nxt + k) for k in range(lv)]
                    g = gg.from_edges(nxt + lv, edges)
                    cn = oracle.common_counts(g)
                    slot = int(g.offsets[0])  # row 0 starts with vertex 1
                    assert g.adj[slot] == 1 and cn[slot] == c
                    # mu = 2: u is a core iff some neighbour is similar; the pair is
                    # in one cluster iff S(u, v) holds at the boundary (inclusive)
                    r = oracle.scan(g, p, q, 2)
                    assert r["core"][0] == 1 and r["core"][1] == 1 and r["cid"][1] == 0
                    cases += 1
    assert cases > 5


@pytest.mark.parametrize("n", [3, 5, 9])
def test_complete_graph_is_one_cluster(n):
    g = gg.from_edges(n, [(a, b) for a in range(n) for b in range(a + 1, n)])
    assert (oracle.common_counts(g) == n).all()  # sigma = n / sqrt(n * n) = 1
    for mu in range(2, n + 1):
        r = oracle.scan(g, 1, 1, mu)
        assert (r["core"] == 1).all() and (r["cid"] == 0).all() and len(r["pairs"]) == 0
    r = oracle.scan(g, 1, 1, n + 1)
    assert (r["label"] == OUTLIER).all()


@pytest.mark.parametrize("k", [1, 3, 7])
def test_star(k):
    # sigma(centre, leaf) = 2 / sqrt(2 (k + 1)); leaves have |N_eps| <= 2
    g = gg.from_edges(k + 1, [(0, i) for i in range(1, k + 1)])
    assert (oracle.common_counts(g) == 2).all()
    s2 = 4 / (2 * (k + 1))
    for (p, q) in [(1, 5), (1, 2), (7, 10), (1, 1)]:
        r = oracle.scan(g, p, q, 3)
        similar = s2 >= (p / q) ** 2
        if similar and k + 1 >= 3:
            assert r["core"][0] == 1 and (r["core"][1:] == 0).all()
            assert [tuple(x) for x in r["pairs"].tolist()] == [(i, 0) for i in range(1, k + 1)]
        else:
            assert (r["label"] == OUTLIER).all()


def test_path():
    # interior sigma = 2/3, end edges 2/sqrt(6)
    n = 7
    g = gg.from_edges(n, [(i, i + 1) for i in range(n - 1)])
    r = oracle.scan(g, 2, 3, 3)
    assert r["core"].tolist() == [0] + [1] * (n - 2) + [0]
    assert (r["cid"][1:n - 1] == 1).all()
    assert [tuple(x) for x in r["pairs"].tolist()] == [(0, 1), (n - 1, 1)]
    r = oracle.scan(g, 67, 100, 3)  # just above 2/3: no interior edge is similar
    assert (r["core"] == 0).all() and (r["label"] == OUTLIER).all()


def test_hub_through_a_border_in_two_clusters():
    # reading of Definition Hub: a degree-1 non-member whose only neighbour is a
    # border of two clusters is a hub (the union of memberships has 2 ids);
    # Algorithm 4's degree guard would call it an outlier. Two stars centred
    # on 0 and 9 share the border 2; vertex 7 hangs off 2.
    edges = [(0, 1), (0, 2), (0, 4), (0, 6), (2, 7), (2, 9), (3, 9), (5, 9), (8, 9)]
    g = gg.from_edges(10, edges)
    cn = oracle.common_counts(g)
    r = oracle.scan(g, 2, 5, 5)
    check_invariants(g, r, cn, 2, 5, 5)
    assert r["core"].tolist() == [1, 0, 0, 0, 0, 0, 0, 0, 0, 1]
    assert r["label"][2] == BORDER and [(2, 0), (2, 9)] == [tuple(x) for x in r["pairs"].tolist() if x[0] == 2]
    assert g.degrees()[7] == 1 and r["label"][7] == HUB
    assert_same(r, oracle.brute(10, edges, 2, 5, 5))


def test_isolated_vertices_are_outliers():
    g = gg.from_edges(5, [(1, 2)])
    r = oracle.scan(g, 1, 5, 2)
    assert r["label"][0] == OUTLIER and r["label"][3] == OUTLIER and r["label"][4] == OUTLIER
    g0 = gg.from_csr(np.zeros(1, np.int64), np.zeros(0, np.int32))
    assert len(oracle.scan(g0, 1, 2, 2)["core"]) == 0


def test_invalid_parameters_and_inputs_are_rejected():
    g = gg.from_edges(3, [(0, 1), (1, 2)])
    for (p, q, mu) in [(0, 1, 2), (1, 0, 2), (3, 2, 2), (1, 2, 1), (1, 2, 0)]:
        with pytest.raises(ValueError):
            oracle.scan(g, p, q, mu)
    assert oracle.validate(g) == -1
    bad = [
        gg.from_csr([0, 1, 2], [1, 1]),            # asymmetric
        gg.from_csr([0, 1, 1], [0]),               # self-loop
        gg.from_csr([0, 2, 3, 4], [2, 1, 0, 0]),   # unsorted row 0
        gg.from_csr([0, 2, 3, 4], [1, 1, 0, 0]),   # duplicate
        gg.from_csr([0, 1, 2], [5, 0]),            # out of range
    ]
    for b in bad:
        assert oracle.validate(b) >= 0


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_brute_force_every_small_graph(n):
    for (p, q) in [(1, 5), (1, 3), (1, 2), (3, 5), (2, 3), (3, 4), (4, 5), (1, 1)]:
        for mu in range(2, n + 2):
            bad, first = oracle.exhaustive(n, p, q, mu)
            assert bad == 0, f"n={n} eps={p}/{q} mu={mu}: {bad} graphs differ, first mask {first}"


@pytest.mark.parametrize("p,q,mu", [(1, 2, 2), (1, 2, 3), (3, 5, 3), (2, 3, 4), (1, 3, 5)])
def test_brute_force_every_graph_of_order_7(p, q, mu):
    bad, first = oracle.exhaustive(7, p, q, mu)
    assert bad == 0, f"first differing mask {first}"


@pytest.mark.slow
@pytest.mark.parametrize("p,q,mu", [(1, 2, 2), (1, 2, 3), (3, 5, 3)])
def test_brute_force_every_graph_of_order_8(p, q, mu):
    bad, first = oracle.exhaustive(8, p, q, mu)
    assert bad == 0, f"first differing mask {first}"


def test_brute_force_random_graphs_up_to_12():
    rng = random.Random(12)
    for trial in range(1500):
        n = rng.randint(8, 12)
        dens = rng.choice([0.15, 0.3, 0.5, 0.7])
        edges = [(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < dens]
        p, q = rng.choice([(1, 5), (1, 3), (1, 2), (3, 5), (2, 3), (3, 4), (4, 5), (1, 1)])
        mu = rng.randint(2, 6)
        g = gg.from_edges(n, edges)
        assert_same(oracle.scan(g, p, q, mu), oracle.brute(n, edges, p, q, mu), f"trial {trial}")


@pytest.mark.parametrize("which", ["rmat10", "chung_lu"])
def test_invariants_and_monotonicity(which):
    g = gg.rmat(10, 8, seed=7) if which == "rmat10" else gg.chung_lu(3000, 10.0, 2.1, seed=5)
    cn = oracle.common_counts(g)
    prev_eps = None
    for (p, q) in gg.EPS_SWEEP:
        prev_mu = None
        for mu in gg.MU_SWEEP:
            r = oracle.scan(g, p, q, mu)
            check_invariants(g, r, cn, p, q, mu)
            if prev_mu is not None:  # core set shrinks as mu grows
                assert not (r["core"] & ~prev_mu).any()
            prev_mu = r["core"]
            if mu == 2:
                if prev_eps is not None:  # and as eps grows
                    assert not (r["core"] & ~prev_eps).any()
                prev_eps = r["core"]


def test_relabelling_equivariance_and_disjoint_union():
    a = gg.chung_lu(400, 8.0, 2.1, seed=21)
    b = gg.rmat(8, 8, seed=3)
    ra, rb = oracle.scan(a, 2, 5, 3), oracle.scan(b, 2, 5, 3)
    u, base = gg.disjoint_union([a, b])
    ru = oracle.scan(u, 2, 5, 3)
    assert np.array_equal(ru["core"], np.concatenate([ra["core"], rb["core"]]))
    shift = lambda c, s: np.where(c >= 0, c + s, -1)
    assert np.array_equal(ru["cid"], np.concatenate([ra["cid"], shift(rb["cid"], a.n)]))
    assert np.array_equal(ru["label"], np.concatenate([ra["label"], rb["label"]]))
    assert np.array_equal(ru["pairs"], np.concatenate([ra["pairs"], rb["pairs"] + a.n]))

    perm = np.random.default_rng(5).permutation(a.n)
    rp = oracle.scan(gg.relabel(a, perm), 2, 5, 3)
    inv = np.argsort(perm)
    assert np.array_equal(rp["core"][perm], ra["core"])
    assert np.array_equal(rp["label"][perm], ra["label"])
    # cluster id = smallest permuted member id among the cluster's cores
    for c in set(ra["cid"][ra["cid"] >= 0].tolist()):
        members = np.flatnonzero(ra["cid"] == c)
        assert set(rp["cid"][perm[members]].tolist()) == {int(perm[members].min())}
    del inv
