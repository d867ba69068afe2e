"""Planted mistakes in a copy of the oracle must each fail a pin (CPU only).

The committed oracle is never modified: each mutant is a textual edit of a
temporary copy of ``oracle/scan_oracle.c``, compiled next to the brute force,
and run through a short battery of the pins (the reconstructed Figure-1
fixture, the matrix-square counts, the eps boundary, the brute force on every
graph of up to 5 vertices).

A mutant may read outside its arrays (a row search that runs past the last
row does), so each compiled copy runs its pins in a child process: exit 10 is
"every pin passed", exit 11 "a pin failed", and death by a signal is a failure
too. Any other exit (an exception in the harness exits 1) fails the test.
"""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest
import scipy.sparse as sp

import graphgen as gg
from conftest import ROOT, load_golden

MUTANTS = {
    "closed count drops a shared endpoint": ("cn[e] = (int32_t)(c + 2);", "cn[e] = (int32_t)(c + 1);"),
    "eps test exclusive": ("return lhs >= rhs;", "return lhs > rhs;"),
    "u not counted in N_eps[u]": ("int64_t e_u = 1;", "int64_t e_u = 0;"),
    "open size of v": ("off[v + 1] - off[v] + 1, p, q);", "off[v + 1] - off[v], p, q);"),
    "p and q transposed": ("(unsigned __int128)((uint64_t)p * (uint64_t)p) * ((uint64_t)du1",
                           "(unsigned __int128)((uint64_t)q * (uint64_t)q) * ((uint64_t)du1"),
    "BFS walks through non-cores": ("if (sim[e] && core[y] && cid[y] < 0)", "if (sim[e] && cid[y] < 0)"),
    "border from non-core neighbours": ("if (core[u] && sim[e]) b[k++] = cid[u];", "if (sim[e]) b[k++] = cid[u];"),
    "hub threshold off by one": ("label[u] = (uint8_t)(k >= 2 ? LABEL_HUB", "label[u] = (uint8_t)(k >= 1 ? LABEL_HUB"),
    "core threshold strict": ("core[u] = (uint8_t)(e_u >= (int64_t)mu);", "core[u] = (uint8_t)(e_u > (int64_t)mu);"),
    "mirror slot not written": ("cn[find_slot(off, adj, v, (int32_t)u)] = (int32_t)(c + 2);", ""),
    "slot row search overshoots into the next row": ("if (off[mid] <= s) lo = mid; else hi = mid;",
                                                      "if (off[mid] <= s + 1) lo = mid; else hi = mid;"),
    "slot row search skips one row too many": ("while (lo + 1 <= n && off[lo + 1] <= s) ++lo;",
                                               "while (lo + 1 <= n && off[lo + 1] <= s + 1) ++lo;"),
    "slot count drops a shared endpoint": ("out[i] = (int32_t)(c + 2);", "out[i] = (int32_t)(c + 1);"),
    "slot column taken from the row's first slot": ("int64_t u = lo, v = adj[s];", "int64_t u = lo, v = adj[off[lo]];"),
}


def _compile(tmp_path, name, src_text):
    src = tmp_path / f"{name}.c"
    src.write_text(src_text)
    so = tmp_path / f"lib{name}.so"
    subprocess.run(["gcc", "-O1", "-fopenmp", "-fPIC", "-shared", "-o", str(so), str(src),
                    os.path.join(ROOT, "oracle", "brute.c")], check=True)
    return str(so)


def _load(so):
    lib = ctypes.CDLL(so)
    vp, i64, u32, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint32, ctypes.c_int
    lib.oracle_common_counts.argtypes = [i64, vp, vp, vp, i32]
    lib.oracle_counts_for_slots.argtypes = [i64, vp, vp, vp, i64, vp, i32]
    lib.oracle_scan.restype = i32
    lib.oracle_scan.argtypes = [i64, vp, vp, u32, u32, u32, i32, vp, vp, vp, vp, vp, vp]
    lib.brute_exhaustive.restype = i64
    lib.brute_exhaustive.argtypes = [i32, u32, u32, u32, i64, i64, i32, vp]
    return lib


def _scan(lib, g, p, q, mu):
    core = np.zeros(max(g.n, 1), np.uint8)
    cid = np.zeros(max(g.n, 1), np.int32)
    label = np.zeros(max(g.n, 1), np.uint8)
    pairs = np.zeros(max(2 * g.nnz, 2), np.int32)
    npairs = np.zeros(1, np.int64)
    adj = g.adj if g.nnz else np.zeros(1, np.int32)
    lib.oracle_scan(g.n, g.offsets.ctypes.data, adj.ctypes.data, p, q, mu, 1, core.ctypes.data,
                    cid.ctypes.data, label.ctypes.data, pairs.ctypes.data, npairs.ctypes.data, None)
    k = int(npairs[0])
    return core[:g.n], cid[:g.n], label[:g.n], pairs[:2 * k].reshape(k, 2)


def _pins_pass(lib) -> bool:
    gd = load_golden("fig1.txt")
    e = list(map(int, gd["edges"][0].split()))
    g = gg.from_edges(int(gd["n"][0]), list(zip(e[0::2], e[1::2])))
    core, cid, label, pairs = _scan(lib, g, 3, 5, 3)
    if set(np.flatnonzero(core).tolist()) != set(map(int, gd["core"][0].split())):
        return False
    if set(np.flatnonzero(label == 2).tolist()) != {8} or set(np.flatnonzero(label == 3).tolist()) != {3, 5, 6}:
        return False
    if [tuple(x) for x in pairs.tolist()] != [(2, 0)]:
        return False
    h = gg.chung_lu(300, 10.0, 2.1, seed=4)
    A = sp.csr_matrix((np.ones(h.nnz, np.int64), h.adj, h.offsets), shape=(h.n, h.n))
    src = np.repeat(np.arange(h.n), h.degrees())
    cn = np.zeros(h.nnz, np.int32)
    lib.oracle_common_counts(h.n, h.offsets.ctypes.data, h.adj.ctypes.data, cn.ctypes.data, 1)
    if not np.array_equal(cn, np.asarray((A @ A)[src, h.adj]).ravel() + 2):
        return False
    # the per-slot checker on every slot: isolated vertices (empty rows) and a
    # hub 60 times its partners' degree (binary search)
    edges = [(0, k) for k in range(1, 121)] + [(k, k + 1) for k in range(1, 120, 2)] + [(130, 131)]
    for sg in (gg.from_edges(135, edges), gg.chung_lu(400, 3.0, 2.1, seed=5)):
        B = sp.csr_matrix((np.ones(sg.nnz, np.int64), sg.adj, sg.offsets), shape=(sg.n, sg.n))
        want = np.asarray((B @ B).tocsr()[np.repeat(np.arange(sg.n), sg.degrees()), sg.adj]).ravel() + 2
        slots = np.random.default_rng(1).permutation(sg.nnz).astype(np.int64)
        out = np.zeros(sg.nnz, np.int32)
        lib.oracle_counts_for_slots(sg.n, sg.offsets.ctypes.data, sg.adj.ctypes.data, slots.ctypes.data, sg.nnz,
                                    out.ctypes.data, 1)
        if not np.array_equal(out, want[slots]):
            return False
    ds = gg.from_edges(6, [(0, 1), (0, 2), (0, 3), (1, 4), (1, 5)])
    if _scan(lib, ds, 1, 2, 3)[1][1] != 0:
        return False
    first = np.zeros(1, np.int64)
    for n in range(2, 6):
        for (p, q, mu) in [(1, 2, 2), (1, 2, 3), (3, 5, 3), (2, 3, 4), (1, 5, 2)]:
            if lib.brute_exhaustive(n, p, q, mu, 0, 1 << (n * (n - 1) // 2), 1, first.ctypes.data) != 0:
                return False
    return True


def _pins_pass_in_child(so) -> bool:
    tests = os.path.dirname(os.path.abspath(__file__))
    code = ("import sys; sys.path[:0] = [{!r}, {!r}]; import test_oracle_mutants as t; "
            "sys.exit(10 if t._pins_pass(t._load({!r})) else 11)").format(ROOT, tests, so)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300,
                       env=dict(os.environ, OMP_NUM_THREADS="1"))
    if r.returncode in (10, 11) or r.returncode < 0:
        return r.returncode == 10
    raise AssertionError(f"pin harness failed (exit {r.returncode}):\n{r.stderr[-2000:]}")


def test_unmodified_copy_passes(tmp_path):
    text = open(os.path.join(ROOT, "oracle", "scan_oracle.c")).read()
    assert _pins_pass_in_child(_compile(tmp_path, "orig", text))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    text = open(os.path.join(ROOT, "oracle", "scan_oracle.c")).read()
    assert text.count(old) == 1, f"mutation site for '{name}' not found once"
    so = _compile(tmp_path, "mut", text.replace(old, new))
    assert not _pins_pass_in_child(so), f"planted mistake '{name}' passed every pin"
