"""C-ABI checks that need no GPU: the library builds for sm_103a, loads, exports
every function include/pa.h declares, and rejects invalid input on the host
before touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2510_21105_gb300 import binding as B
from paper_2510_21105_gb300 import build as build_mod
from paper_2510_21105_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build_mod.build()
    return B.lib()


def _declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(pa_\w+)\s*\(", src, flags=re.M):
            if "typedef" not in m.group(0):
                names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported(lib):
    declared = _declared_functions()
    assert len(declared) >= 20
    missing = [n for n in declared if not hasattr(lib, n)]
    assert not missing, missing
    assert set(B.exported_symbols()) <= declared


def test_host_only_calls(lib):
    assert B.lib().pa_version() >= 10000
    assert B.strerror(B.PA_EINVAL) == "invalid argument"
    o = B.pa_default_opts()
    assert o.field_bits == 0 and o.nlm_period == 0 and o.adaptive == 0 and o.variant == B.PA_VARIANT_AUTO


def _bad(n, rp, col, w=None):
    out = C.c_void_p()
    rp = np.ascontiguousarray(rp, np.uint32)
    col = np.ascontiguousarray(col, np.uint16)
    w = None if w is None else np.ascontiguousarray(w, np.int8)
    return B.lib().pa_create(C.byref(out), n, rp.ctypes.data, col.ctypes.data if len(col) else None,
                             None if w is None else w.ctypes.data)


def test_create_rejects_invalid_graphs_on_host(lib):
    # 0-1, 1-2 stored symmetrically is valid; each case breaks one rule.
    assert _bad(0, [0], []) == B.PA_EINVAL                                   # n < 1
    assert _bad(2, [0, 1, 1], [1]) == B.PA_EINVAL                            # asymmetric
    assert _bad(2, [0, 1, 2], [0, 0]) == B.PA_EINVAL                         # self loop
    assert _bad(2, [0, 2, 4], [1, 1, 0, 0]) == B.PA_EINVAL                   # duplicate
    assert _bad(2, [0, 1, 2], [5, 0]) == B.PA_EINVAL                         # index >= n
    assert _bad(2, [0, 1, 2], [1, 0], [2, 2]) == B.PA_EINVAL                 # |w| != 1
    assert _bad(2, [0, 1, 2], [1, 0], [1, -1]) == B.PA_EINVAL                # unequal weights
    assert _bad(3, [0, 2, 1, 2], [1, 2, 0, 0]) == B.PA_EINVAL                # row_ptr decreasing
    assert _bad(70000, np.zeros(70001), []) == B.PA_EINVAL                   # n > 65536


def test_graph_generators_produce_valid_symmetric_csr():
    for g in [wl.gnp(300, 0.05, 1), wl.gnm(400, 1500, 2), wl.torus(10, 3), wl.delaunay(200, 4)]:
        i, j, w = g.edges()
        rows = np.repeat(np.arange(g.n), np.diff(g.rp))
        assert np.all(rows != g.col)
        fw = {(a, b): c for a, b, c in zip(rows.tolist(), g.col.tolist(),
                                           (g.w if g.w is not None else np.ones(len(rows))).tolist())}
        assert all(fw[(b, a)] == c for (a, b), c in fw.items())
    g = wl.gnm(7000, 41459, seed=0)
    assert g.n == 7000 and g.m == 41459
    t = wl.torus(100, seed=0)
    assert t.m == 20000 and set(np.unique(t.w).tolist()) == {-1, 1}


def test_product_path_has_no_oracle_dependency():
    pkg = os.path.join(ROOT, "paper_2510_21105_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "pamc_oracle" not in src, f
