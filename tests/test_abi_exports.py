"""The C-ABI library builds, loads and exports every symbol include/*.h
declares (no GPU needed: nothing here calls into the device)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

from conftest import ROOT


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(scan_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libscan():
    from paper_2311_12281_gb300 import _build
    path = _build.build()
    return path


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("scan_ctx_create", "scan_graph_load", "scan_query", "scan_query_device",
                     "scan_result_border_pairs", "scan_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(libscan):
    lib = ctypes.CDLL(libscan)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"
    out = subprocess.run(["nm", "-D", "--defined-only", libscan], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert set(declared_functions()) <= exported


def test_binding_covers_the_boundary(libscan):
    import paper_2311_12281_gb300 as ps
    for n in declared_functions():
        assert n in ps.SIGNATURES, f"{n} has no binding signature"
        assert hasattr(ps, n) or n.startswith("scan_result_"), f"{n} has no same-name wrapper"
    ps.lib()  # loads without touching the device
