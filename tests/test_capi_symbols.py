"""The C-ABI library builds, loads without a GPU, and exports every entry
point that include/hm.h declares; the Python binding covers each of them."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "hm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hm_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libhm():
    from paper_1706_09384_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    syms = declared_symbols()
    for need in ("hm_build", "hm_matvec", "hm_gmres", "hm_stats", "hm_free", "hm_import",
                 "hm_green_eval", "hm_matvec_host"):
        assert need in syms


def test_library_exports_every_declared_symbol(libhm):
    missing = [s for s in declared_symbols() if not hasattr(libhm, s)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    from paper_1706_09384_gb300 import hm
    assert sorted(hm.SIGNATURES) == declared_symbols()


def test_status_strings_and_defaults_without_gpu(libhm):
    from paper_1706_09384_gb300 import hm
    hm.lib()
    assert hm.lib().hm_status_string(0).decode() == "ok"
    o = hm.hm_opts_default()
    assert o.storage == hm.HM_STORE_FP32 and o.recompress == 1 and o.diag_value == 1.0


def test_argument_errors_without_gpu():
    """Argument checks run before any CUDA call and report HM_ERR_ARG."""
    import numpy as np
    from paper_1706_09384_gb300 import hm
    L = hm.lib()
    h = ctypes.c_void_p()
    pts = np.zeros((4, 3))
    st = L.hm_build(pts.ctypes.data_as(ctypes.c_void_p), None, 0, 1.0, 2.0, 1.0, 1.0, 0, 1e-4,
                    3.0, 32, None, None, ctypes.byref(h))
    assert st == hm.HM_ERR_ARG and not h.value
    st = L.hm_build(pts.ctypes.data_as(ctypes.c_void_p), None, 4, 1.0, 2.0, 1.0, 1.0, 1, 1e-4,
                    3.0, 32, None, None, ctypes.byref(h))  # T without normals
    assert st == hm.HM_ERR_ARG
    pts[1, 2] = float("nan")
    st = L.hm_build(pts.ctypes.data_as(ctypes.c_void_p), None, 4, 1.0, 2.0, 1.0, 1.0, 0, 1e-4,
                    3.0, 32, None, None, ctypes.byref(h))
    assert st == hm.HM_ERR_ARG
    assert b"non-finite" in L.hm_last_error()
    assert L.hm_matvec(None, 1, None, None, None) == hm.HM_ERR_ARG
