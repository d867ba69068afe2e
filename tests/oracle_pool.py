"""Oracle work run in worker processes (started with ``spawn``) for the
full-size GPU parity tests, and the digests they compare.

Test infrastructure only: each worker regenerates its graphs from their
seeds and runs the CPU oracle on them, one graph per call, single-threaded.
"""
from __future__ import annotations

import hashlib

import numpy as np


def digest(res: dict) -> str:
    """SHA-256 over a SCAN result's arrays (core, cid, label, border pairs),
    each in its fixed dtype, so results of any origin compare by digest."""
    h = hashlib.sha256()
    for key, dt in (("core", np.uint8), ("cid", np.int32), ("label", np.uint8), ("pairs", np.int32)):
        a = np.ascontiguousarray(np.asarray(res[key]), dtype=dt).reshape(-1)
        h.update(key.encode())
        h.update(np.int64(a.size).tobytes())
        h.update(a.tobytes())
    return h.hexdigest()


def chung_lu_member(spec: dict):
    import graphgen as gg

    return gg.chung_lu(spec["n"], spec["avg_deg"], 2.1, spec["seed"])


def oracle_member_digest(spec: dict) -> str:
    """The oracle's answer for one member of the Chung-Lu batch, by digest."""
    import oracle

    g = chung_lu_member(spec)
    p, q = spec["eps"]
    return digest(oracle.scan(g, p, q, spec["mu"], threads=1))
