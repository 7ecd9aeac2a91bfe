"""The C-ABI library builds for sm_103a, loads and exports every function
declared in include/*.h (no GPU needed; no compute calls)."""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*\b(mantra_[a-z0-9_]+)\s*\(", src,
                             flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2304_08356_gb300 import build as B
    B.build()
    from paper_2304_08356_gb300 import mantra
    return mantra


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert {"mantra_graph_load", "mantra_estimate", "mantra_temporal_stats", "mantra_sample_paths"} <= names
    L = lib.lib()
    for nm in sorted(names):
        assert hasattr(L, nm), nm
    assert set(lib.EXPORTS) == names


def test_host_side_argument_checks(lib):
    L = lib.lib()
    out = C.c_void_p()
    u = np.zeros(1, np.uint32)
    # NULL output handle and NULL edge arrays are rejected before any device call
    assert L.mantra_graph_load(u.ctypes.data_as(C.POINTER(C.c_uint32)), u.ctypes.data_as(C.POINTER(C.c_uint32)),
                               u.ctypes.data_as(C.POINTER(C.c_uint32)), 1, 2, None) == 1
    assert L.mantra_graph_load(None, None, None, 5, 2, C.byref(out)) == 1
    assert L.mantra_estimate(None, 0, 0.1, 0.1, 1, None, None, None, None) == 1
    assert L.mantra_temporal_stats(None, 0, 0.1, 1, 0, 0.9, None, None, 0) == 1
    assert lib.strerror(0) == "ok" and "128" in lib.strerror(3)
