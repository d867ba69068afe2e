"""Seeded synthetic graph inputs shared by the oracle, the tests and the benchmark.

Holds none of the clustering arithmetic: it samples R-MAT and Chung-Lu edge lists
and turns them into a simple undirected CSR (self-loops dropped, symmetrised,
rows sorted ascending, duplicates removed), with int64 offsets and int32 ids.

Workload recipes (the synthetic stand-ins for the paper's real datasets, whose
shapes -- power-law degrees, mean degree 16-105, millions of vertices -- are in
its Table 2):

* ``rmat_s14``: R-MAT scale 14, edge factor 8, (a,b,c,d)=(.57,.19,.19,.05), seed 1.
* ``rmat_s22``: R-MAT scale 22, edge factor 16, same probabilities, seed 2.
* ``rmat_s27``: R-MAT scale 27, edge factor 16, seed 5 (out-of-core size).
* ``chung_lu_batch``: 4,096 Chung-Lu graphs, exponent 2.1, vertex counts
  log-uniform in [100, 50,000], mean degree uniform in [4, 64], each with its own
  eps = p/20 (p uniform in 4..16) and mu uniform in 2..8.
"""
from __future__ import annotations

import ctypes
import hashlib
import math
import os
import subprocess
import tempfile
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libgraphgen.so")
_SRC = os.path.join(_HERE, "graphgen.c")
_lib_handle = None

RMAT_ABC = (0.57, 0.19, 0.19)


def build(force: bool = False) -> str:
    """Compile libgraphgen.so with gcc (OpenMP, no fp contraction)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    cmd = ["gcc", "-O3", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _lib():
    global _lib_handle
    if _lib_handle is None:
        build()
        lib = ctypes.CDLL(_SO)
        vp, i64, u64, dbl, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_int
        lib.gg_rmat.restype = vp
        lib.gg_rmat.argtypes = [i32, i64, dbl, dbl, dbl, u64, i32]
        lib.gg_chung_lu.restype = vp
        lib.gg_chung_lu.argtypes = [i64, dbl, dbl, u64, i32]
        lib.gg_from_edges.restype = vp
        lib.gg_from_edges.argtypes = [i64, i64, vp, vp]
        for fn in ("gg_n", "gg_nnz"):
            getattr(lib, fn).restype = i64
            getattr(lib, fn).argtypes = [vp]
        for fn in ("gg_offsets", "gg_adj"):
            getattr(lib, fn).restype = vp
            getattr(lib, fn).argtypes = [vp]
        lib.gg_free.restype = None
        lib.gg_free.argtypes = [vp]
        lib.gg_uniform_u64.restype = None
        lib.gg_uniform_u64.argtypes = [u64, u64, i64, vp]
        _lib_handle = lib
    return _lib_handle


class _Owner:
    """Keeps a C-allocated graph alive while numpy views of it exist."""

    def __init__(self, handle):
        self.handle = handle

    def __del__(self):
        if self.handle:
            _lib().gg_free(self.handle)
            self.handle = None


@dataclass
class Graph:
    """Simple undirected graph in CSR form (int64 offsets, int32 sorted rows)."""
    n: int
    offsets: np.ndarray
    adj: np.ndarray
    name: str = ""
    _owner: object = field(default=None, repr=False)

    @property
    def nnz(self) -> int:
        return int(self.offsets[-1]) if self.n > 0 else 0

    @property
    def m(self) -> int:
        """Undirected edge count."""
        return self.nnz // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.offsets).astype(np.int64)


def _wrap(handle, name: str) -> Graph:
    if not handle:
        raise MemoryError("graph generation failed (bad arguments or out of memory)")
    lib = _lib()
    n = lib.gg_n(handle)
    nnz = lib.gg_nnz(handle)
    owner = _Owner(handle)
    off = np.ctypeslib.as_array(ctypes.cast(lib.gg_offsets(handle), ctypes.POINTER(ctypes.c_int64)), shape=(n + 1,))
    if nnz > 0:
        adj = np.ctypeslib.as_array(ctypes.cast(lib.gg_adj(handle), ctypes.POINTER(ctypes.c_int32)), shape=(nnz,))
    else:
        adj = np.zeros(0, dtype=np.int32)
    return Graph(n=int(n), offsets=off, adj=adj, name=name, _owner=owner)


def rmat(scale: int, edge_factor: int, abc=RMAT_ABC, seed: int = 1, relabel: bool = True) -> Graph:
    a, b, c = abc
    h = _lib().gg_rmat(int(scale), int(edge_factor), float(a), float(b), float(c), int(seed), int(bool(relabel)))
    return _wrap(h, f"rmat_s{scale}_ef{edge_factor}_seed{seed}")


def chung_lu(n: int, avg_deg: float, gamma: float = 2.1, seed: int = 3, relabel: bool = True) -> Graph:
    h = _lib().gg_chung_lu(int(n), float(avg_deg), float(gamma), int(seed), int(bool(relabel)))
    return _wrap(h, f"chung_lu_n{n}_d{avg_deg:g}_g{gamma:g}_seed{seed}")


def from_edges(n: int, edges) -> Graph:
    """CSR of an undirected edge list [(u, v), ...]; drops loops/duplicates, symmetrises."""
    e = np.asarray(edges, dtype=np.int32).reshape(-1, 2)
    src = np.ascontiguousarray(e[:, 0])
    dst = np.ascontiguousarray(e[:, 1])
    h = _lib().gg_from_edges(int(n), int(len(e)), src.ctypes.data, dst.ctypes.data)
    return _wrap(h, f"edges_n{n}_m{len(e)}")


def from_csr(offsets, adj, name: str = "") -> Graph:
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    a = np.ascontiguousarray(adj, dtype=np.int32)
    return Graph(n=len(off) - 1, offsets=off, adj=a, name=name)


def uniform_u64(seed: int, stream: int, count: int) -> np.ndarray:
    out = np.empty(int(count), dtype=np.uint64)
    if count:
        _lib().gg_uniform_u64(int(seed), int(stream), int(count), out.ctypes.data)
    return out


def disjoint_union(graphs) -> tuple[Graph, np.ndarray]:
    """Concatenate graphs with shifted ids; returns the union and the vertex offsets."""
    vbase = [0]
    offs = [np.zeros(1, dtype=np.int64)]
    adjs = []
    ebase = 0
    for g in graphs:
        offs.append(g.offsets[1:] + ebase)
        adjs.append(g.adj.astype(np.int64) + vbase[-1])
        ebase += g.nnz
        vbase.append(vbase[-1] + g.n)
    off = np.concatenate(offs).astype(np.int64)
    adj = np.concatenate(adjs).astype(np.int32) if adjs else np.zeros(0, np.int32)
    return Graph(n=vbase[-1], offsets=off, adj=adj, name="union"), np.asarray(vbase, dtype=np.int64)


def relabel(g: Graph, perm: np.ndarray) -> Graph:
    """Graph with vertex v renamed perm[v]."""
    perm = np.asarray(perm, dtype=np.int64)
    deg = g.degrees()
    src = np.repeat(np.arange(g.n, dtype=np.int64), deg)
    edges = np.stack([perm[src], perm[g.adj.astype(np.int64)]], axis=1)
    return from_edges(g.n, edges)


def stats(g: Graph) -> dict:
    """Shape statistics: degrees, the smaller-side row sum of the (deg, id)
    orientation (the adjacency the per-edge intersection must read), sum deg^2,
    and a SHA-256 of the CSR bytes."""
    deg = g.degrees()
    src = np.repeat(np.arange(g.n, dtype=np.int64), deg)
    dst = g.adj.astype(np.int64)
    ds, dd = deg[src], deg[dst]
    dmin = np.minimum(ds, dd)
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(g.offsets).tobytes())
    h.update(np.ascontiguousarray(g.adj).tobytes())
    return {
        "n": g.n,
        "m": g.m,
        "nnz": g.nnz,
        "d_max": int(deg.max()) if g.n else 0,
        "isolated": int((deg == 0).sum()),
        "sum_dmin": int(dmin.sum() // 2),
        "sum_deg_sq": int((deg.astype(np.float64) ** 2).sum()),
        "sha256": h.hexdigest(),
    }


# ------------------------------------------------------------------ recipes
def rmat_s14() -> Graph:
    return rmat(14, 8, RMAT_ABC, seed=1)


def rmat_s22() -> Graph:
    return rmat(22, 16, RMAT_ABC, seed=2)


def rmat_s27() -> Graph:
    return rmat(27, 16, RMAT_ABC, seed=5)


EPS_SWEEP = [(1, 5), (3, 10), (2, 5), (1, 2), (3, 5), (7, 10), (4, 5)]
MU_SWEEP = [2, 5, 10]


def chung_lu_batch_specs(count: int = 4096, seed: int = 3000):
    """Per-graph (n, mean degree, seed, eps_num, eps_den, mu) for the batched workload."""
    specs = []
    lo, hi = math.log(100.0), math.log(50000.0)
    for k in range(count):
        r = uniform_u64(seed + k, 7, 4)
        u0 = float(r[0] >> np.uint64(11)) / 9007199254740992.0
        u1 = float(r[1] >> np.uint64(11)) / 9007199254740992.0
        n = int(round(math.exp(lo + (hi - lo) * u0)))
        d = 4.0 + 60.0 * u1
        p = 4 + int(r[2] % np.uint64(13))
        mu = 2 + int(r[3] % np.uint64(7))
        specs.append({"n": n, "avg_deg": d, "seed": seed + k, "eps": (p, 20), "mu": mu})
    return specs


def chung_lu_batch(count: int = 4096, seed: int = 3000):
    specs = chung_lu_batch_specs(count, seed)
    graphs = [chung_lu(s["n"], s["avg_deg"], 2.1, s["seed"]) for s in specs]
    return graphs, specs
