"""CPU oracle for exact SCAN -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The product library never does, and the
two share no code: the oracle is plain C written from Section 2.1 of the paper
(``scan_oracle.c``), pinned by a literal set-definition brute force
(``brute.c``), worked values the paper prints, closed forms and invariants.

Result format (shared with the product API so results compare field by field):
``core`` uint8[n], ``cid`` int32[n] (smallest core id of the cluster, -1 for a
non-core), ``label`` uint8[n] (0 core, 1 border, 2 hub, 3 outlier) and
``pairs`` int32[k, 2] -- every (vertex, cluster id) membership of a non-core
vertex, ascending.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRCS = [os.path.join(_HERE, f) for f in ("scan_oracle.c", "brute.c")]
_lib_handle = None

CORE, BORDER, HUB, OUTLIER = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (OpenMP only splits the common-count loop)."""
    newest = max(os.path.getmtime(s) for s in _SRCS)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, *_SRCS], check=True)
    os.replace(tmp, _SO)
    return _SO


def _lib():
    global _lib_handle
    if _lib_handle is None:
        build()
        lib = ctypes.CDLL(_SO)
        vp, i64, u32, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint32, ctypes.c_int
        lib.oracle_validate.restype = i32
        lib.oracle_validate.argtypes = [i64, vp, vp, i64, vp]
        lib.oracle_common_counts.restype = None
        lib.oracle_common_counts.argtypes = [i64, vp, vp, vp, i32]
        lib.oracle_scan.restype = i32
        lib.oracle_scan.argtypes = [i64, vp, vp, u32, u32, u32, i32, vp, vp, vp, vp, vp, vp]
        lib.oracle_scan_from_counts.restype = i32
        lib.oracle_scan_from_counts.argtypes = [i64, vp, vp, vp, u32, u32, u32, vp, vp, vp, vp, vp]
        lib.oracle_counts_for_slots.restype = None
        lib.oracle_counts_for_slots.argtypes = [i64, vp, vp, vp, i64, vp, i32]
        lib.brute_scan.restype = i32
        lib.brute_scan.argtypes = [i32, vp, u32, u32, u32, vp, vp, vp, vp, vp]
        lib.brute_exhaustive.restype = i64
        lib.brute_exhaustive.argtypes = [i32, u32, u32, u32, i64, i64, i32, vp]
        _lib_handle = lib
    return _lib_handle


def _csr(graph):
    off = np.ascontiguousarray(graph.offsets, dtype=np.int64)
    adj = np.ascontiguousarray(graph.adj, dtype=np.int32)
    if adj.size == 0:
        adj = np.zeros(1, dtype=np.int32)
    return off, adj


def validate(graph) -> int:
    """-1 if the CSR is a valid simple undirected graph, else the first bad slot
    (or -2 for a malformed offsets array)."""
    off, adj = _csr(graph)
    bad = np.zeros(1, dtype=np.int64)
    rc = _lib().oracle_validate(graph.n, off.ctypes.data, adj.ctypes.data, int(off[-1]), bad.ctypes.data)
    if rc == 0:
        return -1
    return int(bad[0]) if bad[0] >= 0 else -2


def common_counts(graph, threads: int = 0) -> np.ndarray:
    """Per-slot closed common-neighbour count |N[u] & N[v]| (Definition 2.2)."""
    off, adj = _csr(graph)
    cn = np.zeros(max(int(off[-1]), 1), dtype=np.int32)
    _lib().oracle_common_counts(graph.n, off.ctypes.data, adj.ctypes.data, cn.ctypes.data, int(threads))
    return cn[: int(off[-1])]


def counts_for_slots(graph, slots, threads: int = 0) -> np.ndarray:
    """|N[u] & N[v]| for the given slots only, each computed independently."""
    off, adj = _csr(graph)
    sl = np.ascontiguousarray(slots, dtype=np.int64)
    out = np.zeros(max(len(sl), 1), dtype=np.int32)
    if len(sl):
        _lib().oracle_counts_for_slots(graph.n, off.ctypes.data, adj.ctypes.data, sl.ctypes.data, len(sl),
                                       out.ctypes.data, int(threads))
    return out[: len(sl)]


def scan(graph, eps_num: int, eps_den: int, mu: int, threads: int = 0, want_cn: bool = False) -> dict:
    """SCAN(eps = eps_num/eps_den, mu) by the plain definition."""
    off, adj = _csr(graph)
    n, nnz = graph.n, int(off[-1])
    core = np.zeros(max(n, 1), dtype=np.uint8)
    cid = np.zeros(max(n, 1), dtype=np.int32)
    label = np.zeros(max(n, 1), dtype=np.uint8)
    pairs = np.zeros(max(2 * nnz, 2), dtype=np.int32)
    npairs = np.zeros(1, dtype=np.int64)
    cn = np.zeros(max(nnz, 1), dtype=np.int32) if want_cn else None
    rc = _lib().oracle_scan(n, off.ctypes.data, adj.ctypes.data, int(eps_num), int(eps_den), int(mu),
                            int(threads), core.ctypes.data, cid.ctypes.data, label.ctypes.data,
                            pairs.ctypes.data, npairs.ctypes.data, cn.ctypes.data if want_cn else None)
    if rc != 0:
        raise ValueError(f"oracle_scan rejected the input (code {rc})")
    k = int(npairs[0])
    out = {"core": core[:n], "cid": cid[:n], "label": label[:n], "pairs": pairs[: 2 * k].reshape(k, 2)}
    if want_cn:
        out["cn"] = cn[:nnz]
    return out


def scan_from_counts(graph, cn: np.ndarray, eps_num: int, eps_den: int, mu: int) -> dict:
    """SCAN given the per-slot closed common counts (from common_counts)."""
    off, adj = _csr(graph)
    n, nnz = graph.n, int(off[-1])
    c = np.ascontiguousarray(cn, dtype=np.int32)
    if c.size == 0:
        c = np.zeros(1, np.int32)
    core = np.zeros(max(n, 1), dtype=np.uint8)
    cid = np.zeros(max(n, 1), dtype=np.int32)
    label = np.zeros(max(n, 1), dtype=np.uint8)
    pairs = np.zeros(max(2 * nnz, 2), dtype=np.int32)
    npairs = np.zeros(1, dtype=np.int64)
    rc = _lib().oracle_scan_from_counts(n, off.ctypes.data, adj.ctypes.data, c.ctypes.data, int(eps_num),
                                        int(eps_den), int(mu), core.ctypes.data, cid.ctypes.data,
                                        label.ctypes.data, pairs.ctypes.data, npairs.ctypes.data)
    if rc != 0:
        raise ValueError(f"oracle_scan_from_counts rejected the input (code {rc})")
    k = int(npairs[0])
    return {"core": core[:n], "cid": cid[:n], "label": label[:n], "pairs": pairs[: 2 * k].reshape(k, 2)}


def brute(n: int, edges, eps_num: int, eps_den: int, mu: int) -> dict:
    """Literal set-definition SCAN for n <= 32 (bitmask sets)."""
    nbr = np.zeros(32, dtype=np.uint32)
    for u, v in edges:
        if u != v:
            nbr[u] |= np.uint32(1 << v)
            nbr[v] |= np.uint32(1 << u)
    core = np.zeros(32, np.uint8)
    cid = np.zeros(32, np.int32)
    label = np.zeros(32, np.uint8)
    pairs = np.zeros(2 * 32 * 32, np.int32)
    npairs = np.zeros(1, np.int64)
    rc = _lib().brute_scan(int(n), nbr.ctypes.data, int(eps_num), int(eps_den), int(mu), core.ctypes.data,
                           cid.ctypes.data, label.ctypes.data, pairs.ctypes.data, npairs.ctypes.data)
    if rc != 0:
        raise ValueError(f"brute_scan failed (code {rc})")
    k = int(npairs[0])
    return {"core": core[:n], "cid": cid[:n], "label": label[:n], "pairs": pairs[: 2 * k].reshape(k, 2)}


def exhaustive(n: int, eps_num: int, eps_den: int, mu: int, lo: int = 0, hi: int | None = None,
               threads: int = 0) -> tuple[int, int]:
    """Oracle vs brute force on every graph of order n with edge mask in [lo, hi).
    Returns (number of disagreeing graphs, first disagreeing mask or -1)."""
    if hi is None:
        hi = 1 << (n * (n - 1) // 2)
    first = np.zeros(1, dtype=np.int64)
    bad = _lib().brute_exhaustive(int(n), int(eps_num), int(eps_den), int(mu), int(lo), int(hi), int(threads),
                                  first.ctypes.data)
    return int(bad), int(first[0])
