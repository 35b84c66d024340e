"""Host-side checks of the CUDA library that need no GPU: it was built for
sm_103a, loads, exports every entry point the public headers declare, and
rejects bad arguments before touching the device."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(hamls_[a-z_0-9]+)\s*\(", src))
    return names


def test_library_loads_and_exports_all_declared_symbols():
    import paper_2609_39200_b300 as h
    L = h.lib()
    declared = _declared()
    assert {"hamls_plan", "hamls_fit", "hamls_destroy", "hamls_sync"} <= declared
    for name in declared:
        assert hasattr(L, name), name
    assert declared == set(h.EXPORTS)


def test_library_is_built_for_sm103a_only():
    from paper_2609_39200_b300 import build as b
    assert b.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert not b.needs_build()


def test_default_params_and_status_strings():
    import paper_2609_39200_b300 as h
    p = h.default_params()
    assert (p.n_target, p.eps, p.chi_target, p.chi_full, p.sobolev_s, p.aux_radius) == (0, 0.05, 16.0, 32.0, 1.0, 3.0)
    for code in range(9):
        assert h.lib().hamls_status_string(code)


def test_status_codes_agree_between_header_binding_and_library():
    # every hamls_status of the public header has a name in the binding and a
    # distinct text in the library; the Voronoi calls report code 9
    import paper_2609_39200_b300 as h
    src = open(os.path.join(ROOT, "include", "hamls.h")).read()
    enum = src[src.index("typedef enum {"):src.index("} hamls_status;")]
    codes = {name: int(v) for name, v in re.findall(r"(HAMLS_(?:OK|ERR_[A-Z_]+))\s*=\s*(\d+)", enum)}
    assert codes["HAMLS_ERR_VORONOI"] == 9
    assert set(codes.values()) == set(h.STATUS)
    texts = {h.lib().hamls_status_string(c) for c in codes.values()}
    assert len(texts) == len(codes) and b"unknown status" not in texts


def test_bad_arguments_rejected_on_host():
    import numpy as np
    import paper_2609_39200_b300 as h
    L = h.lib()
    hnd = ctypes.c_void_p()
    x = np.zeros((100, 3))
    p = h.default_params()
    # K out of range, N out of range, too few nodes, bad parameters: no device work happens
    assert L.hamls_plan(ctypes.byref(hnd), x.ctypes.data, None, 100, 8, 9, ctypes.byref(p), None) == 1
    assert L.hamls_plan(ctypes.byref(hnd), x.ctypes.data, None, 100, 0, 2, ctypes.byref(p), None) == 1
    assert L.hamls_plan(ctypes.byref(hnd), x.ctypes.data, None, 5, 8, 2, ctypes.byref(p), None) == 1
    bad = h.default_params(chi_full=10.0)
    assert L.hamls_plan(ctypes.byref(hnd), x.ctypes.data, None, 100, 8, 2, ctypes.byref(bad), None) == 1
    assert L.hamls_plan(None, x.ctypes.data, None, 100, 8, 2, ctypes.byref(p), None) == 1
    assert L.hamls_fit(None, None, None, None) == 1
    assert L.hamls_destroy(None) == 1


def test_product_has_no_path_to_the_oracle_and_fails_loudly_without_the_library(monkeypatch):
    # the package never imports the CPU oracle, and with its CUDA library
    # missing it raises instead of computing anything another way
    pkg = os.path.join(ROOT, "paper_2609_39200_b300")
    for f in glob.glob(os.path.join(pkg, "*.py")):
        src = open(f).read()
        assert not re.search(r"^\s*(import|from)\s+oracle\b", src, flags=re.M), f
        assert "hamls_oracle" not in src, f
    import paper_2609_39200_b300 as h
    monkeypatch.setattr(h, "_lib", None)
    monkeypatch.setattr(h, "LIB_PATH", os.path.join(pkg, "missing-libhamls.so"))
    with pytest.raises(ImportError):
        h.lib()
