"""Exact SCAN structural graph clustering on one GB300 -- Python binding.

A thin ctypes binding of ``libscan.so`` (declared in ``include/scan.h``): the
functions below carry the C names and only marshal arguments. Every step of a
query runs in the library's CUDA kernels; there is no CPU fallback, and
importing this package fails loudly if the library has not been built
(``paper_2311_12281_gb300._build.build()``).

Results compare field by field with the CPU oracle: ``core`` uint8[n],
``cid`` int32[n] (smallest core id of the cluster, -1 for non-cores), ``label``
uint8[n] (0 core, 1 border, 2 hub, 3 outlier), ``pairs`` int32[k, 2] of
(vertex, cluster id) memberships of non-core vertices, ascending.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libscan.so")

SCAN_OK, SCAN_EINVAL, SCAN_ENOMEM, SCAN_EBUDGET, SCAN_ECUDA, SCAN_ETIMEOUT, SCAN_EBUSY = range(7)
SCAN_CORE, SCAN_BORDER, SCAN_HUB, SCAN_OUTLIER = range(4)
SCAN_LOAD_DEVICE_PTRS = 0x1
SCAN_LOAD_PINNED_BORROW = 0x2
SCAN_Q_AUTO, SCAN_Q_RECOMPUTE, SCAN_Q_PLAIN, SCAN_Q_BUILD_CACHE = 0x0, 0x1, 0x2, 0x4

_STATUS = {1: "SCAN_EINVAL", 2: "SCAN_ENOMEM", 3: "SCAN_EBUDGET", 4: "SCAN_ECUDA", 5: "SCAN_ETIMEOUT",
           6: "SCAN_EBUSY"}


class ScanError(RuntimeError):
    def __init__(self, status: int, detail: str):
        super().__init__(f"{_STATUS.get(status, status)}: {detail}")
        self.status = status


class scan_ctx_opts(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("budget_bytes", ctypes.c_uint64), ("stream", ctypes.c_void_p)]


class scan_params(ctypes.Structure):
    _fields_ = [("eps_num", ctypes.c_uint32), ("eps_den", ctypes.c_uint32), ("mu", ctypes.c_uint32)]


class scan_server_opts(ctypes.Structure):
    _fields_ = [("max_inflight", ctypes.c_int32), ("use_cache", ctypes.c_int32)]


class scan_server_report(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_uint64), ("rejected", ctypes.c_uint64), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double), ("throughput_rps", ctypes.c_double),
                ("cache_builds", ctypes.c_uint64), ("cache_evictions", ctypes.c_uint64),
                ("graph_loads", ctypes.c_uint64), ("graph_evictions", ctypes.c_uint64),
                ("max_inflight", ctypes.c_int32), ("device_bytes", ctypes.c_uint64)]


class scan_device_out(ctypes.Structure):
    _fields_ = [("core", ctypes.c_void_p), ("cid", ctypes.c_void_p), ("label", ctypes.c_void_p),
                ("pairs", ctypes.c_void_p), ("pairs_cap", ctypes.c_int64), ("npairs", ctypes.c_void_p)]


# C signatures: name -> (restype, argtypes)
_VP, _I32, _U32, _I64, _U64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_int64, ctypes.c_uint64
_PP = ctypes.POINTER(ctypes.c_void_p)
SIGNATURES = {
    "scan_last_error": (ctypes.c_char_p, []),
    "scan_ctx_create": (ctypes.c_int, [ctypes.POINTER(scan_ctx_opts), _PP]),
    "scan_ctx_destroy": (None, [_VP]),
    "scan_ctx_device_bytes": (_U64, [_VP]),
    "scan_ctx_kernel_launches": (_U64, [_VP]),
    "scan_ctx_sync": (ctypes.c_int, [_VP]),
    "scan_ctx_profile": (ctypes.c_int, [_VP, _I32]),
    "scan_ctx_set_loop_limit": (ctypes.c_int, [_VP, ctypes.c_uint32]),
    "scan_ctx_stage_time": (ctypes.c_int, [_VP, _I32, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_int64)]),
    "scan_graph_load": (ctypes.c_int, [_VP, _I32, _VP, _VP, _I64, _U32, _PP]),
    "scan_graph_free": (None, [_VP]),
    "scan_graph_load_partitioned": (ctypes.c_int, [_VP, _I32, _VP, _VP, _I64, _I64, _PP]),
    "scan_graph_blocks": (_I32, [_VP]),
    "scan_graph_transfer_bytes": (_U64, [_VP]),
    "scan_graph_set_zero_copy": (ctypes.c_int, [_VP, _I32]),
    "scan_plan_edge_extended": (ctypes.c_int, [_I32, _VP, _VP, _I64, _U64, ctypes.POINTER(ctypes.c_int64),
                                               ctypes.POINTER(ctypes.c_uint64)]),
    "scan_plan_triangle_blocks": (ctypes.c_int, [_I32, _VP, _VP, _I64, _U64, ctypes.POINTER(ctypes.c_int32),
                                                   ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_uint64)]),
    "scan_graph_n": (_I32, [_VP]),
    "scan_graph_nnz": (_I64, [_VP]),
    "scan_graph_device_bytes": (_U64, [_VP]),
    "scan_graph_drop_cache": (ctypes.c_int, [_VP]),
    "scan_graph_has_cache": (_I32, [_VP]),
    "scan_graph_copy_counts": (ctypes.c_int, [_VP, _VP]),
    "scan_graph_set_strategy": (ctypes.c_int, [_VP, _I32]),
    "scan_graph_strategy": (_I32, [_VP]),
    "scan_graph_autotune": (ctypes.c_int, [_VP, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int32),
                                           ctypes.POINTER(ctypes.c_double)]),
    "scan_query": (ctypes.c_int, [_VP, _U32, _U32, _U32, _PP]),
    "scan_query_ex": (ctypes.c_int, [_VP, ctypes.POINTER(scan_params), _U32, _PP]),
    "scan_query_sweep": (ctypes.c_int, [_VP, _VP, ctypes.c_int32, _U32, _VP]),
    "scan_query_device": (ctypes.c_int, [_VP, ctypes.POINTER(scan_params), _U32, ctypes.POINTER(scan_device_out)]),
    "scan_batch_load": (ctypes.c_int, [_VP, _I32, _VP, _VP, _VP, _U32, _PP]),
    "scan_batch_size": (_I32, [_VP]),
    "scan_batch_union": (_VP, [_VP]),
    "scan_batch_query": (ctypes.c_int, [_VP, _VP, _U32, _VP]),
    "scan_batch_query_packed": (ctypes.c_int, [_VP, _VP, _U32, _PP, _VP, _VP]),
    "scan_batch_query_device": (ctypes.c_int, [_VP, _VP, _U32, ctypes.POINTER(scan_device_out)]),
    "scan_batch_free": (None, [_VP]),
    "scan_query_batch": (ctypes.c_int, [_VP, _VP, _I32, _VP]),
    "scan_common_counts_static": (ctypes.c_int, [_VP, _VP, _I32, _I64, _VP, _VP]),
    "scan_server_create": (ctypes.c_int, [_VP, ctypes.POINTER(scan_server_opts), _PP]),
    "scan_server_add_graph": (ctypes.c_int, [_VP, _I32, _VP, _VP, _I64, ctypes.POINTER(ctypes.c_int32)]),
    "scan_server_submit": (ctypes.c_int, [_VP, _I32, ctypes.POINTER(scan_params), ctypes.POINTER(ctypes.c_uint64)]),
    "scan_server_wait": (ctypes.c_int, [_VP, _U64, _PP, ctypes.POINTER(ctypes.c_double)]),
    "scan_server_poll": (ctypes.c_int, [_VP, _U64, _PP, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_int32)]),
    "scan_server_stats": (ctypes.c_int, [_VP, ctypes.POINTER(scan_server_report)]),
    "scan_server_reset_stats": (ctypes.c_int, [_VP]),
    "scan_server_destroy": (None, [_VP]),
    "scan_result_n": (_I32, [_VP]),
    "scan_result_core": (_VP, [_VP]),
    "scan_result_cluster": (_VP, [_VP]),
    "scan_result_label": (_VP, [_VP]),
    "scan_result_border_count": (_I64, [_VP]),
    "scan_result_border_pairs": (_VP, [_VP]),
    "scan_result_free": (None, [_VP]),
}

_lib = None


def lib() -> ctypes.CDLL:
    """The loaded libscan.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libscan.so not built at {LIB_PATH}; run paper_2311_12281_gb300._build.build()")
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def _check(status: int):
    if status != SCAN_OK:
        raise ScanError(status, (lib().scan_last_error() or b"").decode())


# ----------------------------------------------------------- same-name calls
def scan_last_error() -> str:
    return (lib().scan_last_error() or b"").decode()


def scan_ctx_create(device: int = 0, budget_bytes: int = 0, stream: int | None = None) -> int:
    opts = scan_ctx_opts(device, budget_bytes, stream or None)
    out = ctypes.c_void_p()
    _check(lib().scan_ctx_create(ctypes.byref(opts), ctypes.byref(out)))
    return out.value


def scan_ctx_destroy(ctx: int):
    lib().scan_ctx_destroy(ctx)


def scan_ctx_device_bytes(ctx: int) -> int:
    return int(lib().scan_ctx_device_bytes(ctx))


def scan_ctx_kernel_launches(ctx: int) -> int:
    return int(lib().scan_ctx_kernel_launches(ctx))


def scan_ctx_sync(ctx: int):
    _check(lib().scan_ctx_sync(ctx))


SCAN_STAGE_SIMILARITY, SCAN_STAGE_CORE, SCAN_STAGE_CLUSTER, SCAN_STAGE_BORDER, SCAN_STAGE_LABEL = range(5)
STAGE_NAMES = ("similarity", "core", "cluster", "border", "label")


def scan_ctx_profile(ctx: int, enable: bool):
    _check(lib().scan_ctx_profile(ctx, 1 if enable else 0))


def scan_ctx_set_loop_limit(ctx: int, limit: int):
    _check(lib().scan_ctx_set_loop_limit(ctx, ctypes.c_uint32(int(limit))))


def scan_ctx_stage_time(ctx: int, stage: int) -> tuple[float, int]:
    """(summed milliseconds, number of timed intervals) of one stage."""
    ms = ctypes.c_double()
    cnt = ctypes.c_int64()
    _check(lib().scan_ctx_stage_time(ctx, stage, ctypes.byref(ms), ctypes.byref(cnt)))
    return ms.value, cnt.value


def scan_graph_load(ctx: int, n: int, offsets, adj, nnz: int | None = None, flags: int = 0) -> int:
    """offsets/adj: numpy arrays (host) or integer device addresses with
    flags |= SCAN_LOAD_DEVICE_PTRS."""
    out = ctypes.c_void_p()
    if flags & SCAN_LOAD_DEVICE_PTRS:
        po, pa = int(offsets), int(adj)
        assert nnz is not None
    else:
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        adj = np.ascontiguousarray(adj, dtype=np.int32)
        nnz = int(adj.size) if nnz is None else nnz
        po = offsets.ctypes.data if offsets.size else None
        pa = adj.ctypes.data if adj.size else None
    _check(lib().scan_graph_load(ctx, int(n), po, pa, int(nnz), int(flags), ctypes.byref(out)))
    return out.value


def scan_graph_free(g: int):
    lib().scan_graph_free(g)


def scan_graph_load_partitioned(ctx: int, n: int, offsets: np.ndarray, adj: np.ndarray,
                                block_slots: int = 0) -> int:
    """Out-of-core graph: offsets/adj are host arrays that must stay alive and
    unchanged until scan_graph_free (the caller keeps a reference)."""
    assert offsets.dtype == np.int64 and adj.dtype == np.int32
    assert offsets.flags["C_CONTIGUOUS"] and adj.flags["C_CONTIGUOUS"]
    out = ctypes.c_void_p()
    _check(lib().scan_graph_load_partitioned(ctx, int(n), offsets.ctypes.data, adj.ctypes.data if adj.size else None,
                                             int(adj.size), int(block_slots), ctypes.byref(out)))
    return out.value


def scan_graph_blocks(g: int) -> int:
    return int(lib().scan_graph_blocks(g))


def scan_graph_transfer_bytes(g: int) -> int:
    return int(lib().scan_graph_transfer_bytes(g))


def scan_graph_set_zero_copy(g: int, enable: bool):
    _check(lib().scan_graph_set_zero_copy(g, 1 if enable else 0))


def scan_plan_edge_extended(n: int, offsets: np.ndarray, adj: np.ndarray, device_bytes: int) -> tuple[int, int]:
    """(subgraphs, bytes) of the paper's edge extended subgraph partition (host only)."""
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    a = np.ascontiguousarray(adj, dtype=np.int32)
    k = ctypes.c_int64()
    b = ctypes.c_uint64()
    _check(lib().scan_plan_edge_extended(int(n), off.ctypes.data, a.ctypes.data if a.size else None, int(a.size),
                                         int(device_bytes), ctypes.byref(k), ctypes.byref(b)))
    return k.value, b.value


def scan_plan_triangle_blocks(n: int, offsets: np.ndarray, adj: np.ndarray, device_bytes: int) -> tuple[int, int, int]:
    """(blocks, pairs with work, bytes) of triangle counting over block pairs out of core (host only)."""
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    a = np.ascontiguousarray(adj, dtype=np.int32)
    nb = ctypes.c_int32()
    npairs = ctypes.c_int64()
    b = ctypes.c_uint64()
    _check(lib().scan_plan_triangle_blocks(int(n), off.ctypes.data, a.ctypes.data if a.size else None, int(a.size),
                                           int(device_bytes), ctypes.byref(nb), ctypes.byref(npairs), ctypes.byref(b)))
    return nb.value, npairs.value, b.value


def scan_graph_n(g: int) -> int:
    return int(lib().scan_graph_n(g))


def scan_graph_nnz(g: int) -> int:
    return int(lib().scan_graph_nnz(g))


def scan_graph_device_bytes(g: int) -> int:
    return int(lib().scan_graph_device_bytes(g))


def scan_graph_drop_cache(g: int):
    _check(lib().scan_graph_drop_cache(g))


def scan_graph_has_cache(g: int) -> bool:
    return bool(lib().scan_graph_has_cache(g))


SCAN_STRATEGY_FORWARD, SCAN_STRATEGY_OWNER, SCAN_STRATEGY_BSEARCH, SCAN_STRATEGY_FORWARD_LEAN = 0, 1, 2, 3
SCAN_STRATEGY_PROGRESSIVE = 4


def scan_graph_set_strategy(g: int, strategy: int):
    _check(lib().scan_graph_set_strategy(g, int(strategy)))


def scan_graph_strategy(g: int) -> int:
    return int(lib().scan_graph_strategy(g))


def scan_graph_autotune(g: int, cache_path: str | None = None) -> tuple[int, float]:
    """Time the kernel families on this graph, keep the fastest; returns (strategy, ms)."""
    st = ctypes.c_int32()
    ms = ctypes.c_double()
    path = cache_path.encode() if cache_path else None
    _check(lib().scan_graph_autotune(g, path, ctypes.byref(st), ctypes.byref(ms)))
    return st.value, ms.value


def scan_graph_copy_counts(g: int, nnz: int) -> np.ndarray:
    """Per-slot closed common counts from the graph's cache (int32[nnz])."""
    out = np.zeros(max(nnz, 1), dtype=np.int32)
    _check(lib().scan_graph_copy_counts(g, out.ctypes.data))
    return out[:nnz]


class _ResultOwner:
    """Holds one scan_result; it is freed when the last array viewing it goes."""

    __slots__ = ("r",)

    def __init__(self, r: int):
        self.r = r

    def __del__(self):
        if self.r:
            try:
                lib().scan_result_free(self.r)
            except Exception:  # interpreter shutdown: the process frees it
                pass
            self.r = None


def _result_to_numpy(r: int) -> dict:
    """The result's arrays as numpy views of its own (pinned) buffers: no host
    copy; the result is released once every array is gone."""
    L = lib()
    n = L.scan_result_n(r)
    k = L.scan_result_border_count(r)
    owner = _ResultOwner(r)

    def arr(ptr, dtype, count):
        if count == 0:
            return np.zeros(0, dtype=dtype)
        buf = (ctypes.c_char * (count * np.dtype(dtype).itemsize)).from_address(ptr)
        buf._owner = owner  # the view's base keeps the result alive
        return np.frombuffer(buf, dtype=dtype, count=count)

    return {
        "core": arr(L.scan_result_core(r), np.uint8, n),
        "cid": arr(L.scan_result_cluster(r), np.int32, n),
        "label": arr(L.scan_result_label(r), np.uint8, n),
        "pairs": arr(L.scan_result_border_pairs(r), np.int32, 2 * k).reshape(k, 2),
    }


def scan_query(g: int, eps_num: int, eps_den: int, mu: int) -> dict:
    out = ctypes.c_void_p()
    _check(lib().scan_query(g, eps_num, eps_den, mu, ctypes.byref(out)))
    return _result_to_numpy(out.value)


def scan_query_ex(g: int, eps_num: int, eps_den: int, mu: int, mode: int = SCAN_Q_AUTO) -> dict:
    out = ctypes.c_void_p()
    p = scan_params(eps_num, eps_den, mu)
    _check(lib().scan_query_ex(g, ctypes.byref(p), mode, ctypes.byref(out)))
    return _result_to_numpy(out.value)


def scan_query_sweep(g: int, params, mode: int = SCAN_Q_AUTO) -> list:
    """params: [(eps_num, eps_den, mu)]; one result dict per query, in order
    (each result's copy to the host overlaps the next query)."""
    k = len(params)
    outs = (ctypes.c_void_p * max(k, 1))()
    _check(lib().scan_query_sweep(g, _params_array(params) if k else None, k, mode, outs))
    return [_result_to_numpy(outs[j]) for j in range(k)]


def scan_query_device(g: int, eps_num: int, eps_den: int, mu: int, mode: int, core: int, cid: int, label: int,
                      pairs: int, pairs_cap: int, npairs: int):
    """Device-resident query into caller-owned device buffers (addresses)."""
    p = scan_params(eps_num, eps_den, mu)
    o = scan_device_out(core, cid, label, pairs, pairs_cap, npairs)
    _check(lib().scan_query_device(g, ctypes.byref(p), mode, ctypes.byref(o)))


def _params_array(params):
    arr = (scan_params * len(params))()
    for j, (p, q, mu) in enumerate(params):
        arr[j] = scan_params(int(p), int(q), int(mu))
    return arr


def scan_batch_load(ctx: int, graphs, flags: int = 0) -> int:
    """graphs: objects with n, offsets (int64), adj (int32) host arrays."""
    k = len(graphs)
    offs = [np.ascontiguousarray(g.offsets, dtype=np.int64) for g in graphs]
    adjs = [np.ascontiguousarray(g.adj, dtype=np.int32) for g in graphs]
    ns = np.asarray([g.n for g in graphs], dtype=np.int32)
    po = (ctypes.c_void_p * k)(*[o.ctypes.data for o in offs])
    pa = (ctypes.c_void_p * k)(*[a.ctypes.data if a.size else None for a in adjs])
    out = ctypes.c_void_p()
    _check(lib().scan_batch_load(ctx, k, ns.ctypes.data, po, pa, int(flags), ctypes.byref(out)))
    return out.value


def scan_batch_size(b: int) -> int:
    return int(lib().scan_batch_size(b))


def scan_batch_union(b: int) -> int:
    return lib().scan_batch_union(b)


def scan_batch_free(b: int):
    lib().scan_batch_free(b)


def scan_batch_query(b: int, params, mode: int = SCAN_Q_RECOMPUTE) -> list:
    """params: [(eps_num, eps_den, mu)] per graph; returns one result dict per graph."""
    k = scan_batch_size(b)
    assert len(params) == k
    outs = (ctypes.c_void_p * k)()
    _check(lib().scan_batch_query(b, _params_array(params), mode, outs))
    return [_result_to_numpy(outs[j]) for j in range(k)]


def scan_batch_query_packed(b: int, params, mode: int = SCAN_Q_RECOMPUTE) -> list:
    """The same answers as scan_batch_query from one packed result: each
    graph's dict holds numpy views into the one result's arrays."""
    k = scan_batch_size(b)
    assert len(params) == k
    out = ctypes.c_void_p()
    voff = np.zeros(k + 1, np.int64)
    poff = np.zeros(k + 1, np.int64)
    _check(lib().scan_batch_query_packed(b, _params_array(params), mode, ctypes.byref(out), voff.ctypes.data,
                                         poff.ctypes.data))
    whole = _result_to_numpy(out.value)
    core, cid, label, pairs = whole["core"], whole["cid"], whole["label"], whole["pairs"]
    return [{"core": core[voff[j]:voff[j + 1]], "cid": cid[voff[j]:voff[j + 1]],
             "label": label[voff[j]:voff[j + 1]], "pairs": pairs[poff[j]:poff[j + 1]]} for j in range(k)]


def scan_batch_query_device(b: int, params, mode: int, core: int, cid: int, label: int, pairs: int,
                            pairs_cap: int, npairs: int):
    o = scan_device_out(core, cid, label, pairs, pairs_cap, npairs)
    _check(lib().scan_batch_query_device(b, _params_array(params), mode, ctypes.byref(o)))


def scan_query_batch(graphs, params) -> list:
    """graphs: scan_graph handles of one context; one full-recompute result per graph."""
    k = len(graphs)
    gs = (ctypes.c_void_p * k)(*graphs)
    outs = (ctypes.c_void_p * k)()
    _check(lib().scan_query_batch(gs, _params_array(params), k, outs))
    return [_result_to_numpy(outs[j]) for j in range(k)]


def scan_common_counts_static(offsets: int, adj: int, n: int, nnz: int, cn: int, stream: int | None = None):
    """Per-slot closed common counts into the caller's device array `cn`,
    allocating nothing (all arguments are device addresses). For callers that
    cannot allocate device memory; see include/scan.h for the size limit."""
    _check(lib().scan_common_counts_static(offsets, adj, int(n), int(nnz), cn, stream))


def scan_server_create(ctx: int, max_inflight: int = 8, use_cache: bool | int = True) -> int:
    """use_cache: True/1 cached counts, False/0 recompute every query, 2 the plain comparator path."""
    out = ctypes.c_void_p()
    opts = scan_server_opts(int(max_inflight), int(use_cache))
    _check(lib().scan_server_create(ctx, ctypes.byref(opts), ctypes.byref(out)))
    return out.value


def scan_server_add_graph(srv: int, graph) -> int:
    off = np.ascontiguousarray(graph.offsets, dtype=np.int64)
    adj = np.ascontiguousarray(graph.adj, dtype=np.int32)
    gid = ctypes.c_int32()
    _check(lib().scan_server_add_graph(srv, int(graph.n), off.ctypes.data, adj.ctypes.data if adj.size else None,
                                       int(adj.size), ctypes.byref(gid)))
    return gid.value


def scan_server_submit(srv: int, graph_id: int, eps_num: int, eps_den: int, mu: int) -> int:
    t = ctypes.c_uint64()
    p = scan_params(int(eps_num), int(eps_den), int(mu))
    _check(lib().scan_server_submit(srv, int(graph_id), ctypes.byref(p), ctypes.byref(t)))
    return t.value


def scan_server_wait(srv: int, ticket: int, keep: bool = True) -> tuple[dict | None, float]:
    """(result, latency_ms); with keep=False the result is released unread (None)."""
    out = ctypes.c_void_p()
    lat = ctypes.c_double()
    _check(lib().scan_server_wait(srv, ctypes.c_uint64(ticket), ctypes.byref(out), ctypes.byref(lat)))
    if not keep:
        lib().scan_result_free(out.value)
        return None, lat.value
    return _result_to_numpy(out.value), lat.value


def scan_server_poll(srv: int, ticket: int):
    """None while running, else (result, latency_ms)."""
    out = ctypes.c_void_p()
    lat = ctypes.c_double()
    ready = ctypes.c_int32()
    _check(lib().scan_server_poll(srv, ctypes.c_uint64(ticket), ctypes.byref(out), ctypes.byref(lat),
                                  ctypes.byref(ready)))
    if not ready.value:
        return None
    return _result_to_numpy(out.value), lat.value


def scan_server_stats(srv: int) -> dict:
    r = scan_server_report()
    _check(lib().scan_server_stats(srv, ctypes.byref(r)))
    return {name: getattr(r, name) for name, _ in scan_server_report._fields_}


def scan_server_reset_stats(srv: int):
    _check(lib().scan_server_reset_stats(srv))


def scan_server_destroy(srv: int):
    lib().scan_server_destroy(srv)


# --------------------------------------------------------------- convenience
class Context:
    """Owns a scan_ctx; graphs loaded through it are freed with it."""

    def __init__(self, device: int = 0, budget_bytes: int = 0, stream: int | None = None):
        self.handle = scan_ctx_create(device, budget_bytes, stream)
        self._graphs = []

    def load(self, graph, flags: int = 0) -> "Graph":
        off = np.ascontiguousarray(graph.offsets, dtype=np.int64)
        adj = np.ascontiguousarray(graph.adj, dtype=np.int32)
        g = Graph(self, scan_graph_load(self.handle, graph.n, off, adj, None, flags), graph.n)
        if flags & SCAN_LOAD_PINNED_BORROW:
            g._host = (off, adj)  # borrowed by the library until free
        self._graphs.append(g)
        return g

    def load_partitioned(self, graph, block_slots: int = 0) -> "Graph":
        """Out-of-core load: the graph's host arrays stay referenced by the
        returned object until it is freed (the library streams from them)."""
        off = np.ascontiguousarray(graph.offsets, dtype=np.int64)
        adj = np.ascontiguousarray(graph.adj, dtype=np.int32)
        g = Graph(self, scan_graph_load_partitioned(self.handle, graph.n, off, adj, block_slots), graph.n)
        g._host = (off, adj)
        self._graphs.append(g)
        return g

    @property
    def kernel_launches(self) -> int:
        return scan_ctx_kernel_launches(self.handle)

    @property
    def device_bytes(self) -> int:
        return scan_ctx_device_bytes(self.handle)

    def sync(self):
        scan_ctx_sync(self.handle)

    def close(self):
        for g in self._graphs:
            g.free()
        self._graphs = []
        if self.handle:
            scan_ctx_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Graph:
    def __init__(self, ctx: Context, handle: int, n: int):
        self.ctx, self.handle, self.n = ctx, handle, n
        self._host = None

    def query(self, eps_num: int, eps_den: int, mu: int, mode: int = SCAN_Q_AUTO) -> dict:
        return scan_query_ex(self.handle, eps_num, eps_den, mu, mode)

    def sweep(self, params, mode: int = SCAN_Q_AUTO) -> list:
        return scan_query_sweep(self.handle, params, mode)

    def drop_cache(self):
        scan_graph_drop_cache(self.handle)

    def set_strategy(self, strategy: int):
        scan_graph_set_strategy(self.handle, strategy)

    def counts(self) -> np.ndarray:
        return scan_graph_copy_counts(self.handle, int(lib().scan_graph_nnz(self.handle)))

    @property
    def has_cache(self) -> bool:
        return scan_graph_has_cache(self.handle)

    @property
    def blocks(self) -> int:
        return scan_graph_blocks(self.handle)

    @property
    def transfer_bytes(self) -> int:
        return scan_graph_transfer_bytes(self.handle)

    def set_zero_copy(self, enable: bool):
        scan_graph_set_zero_copy(self.handle, enable)

    def free(self):
        if self.handle:
            scan_graph_free(self.handle)
            self.handle = None
        self._host = None
