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
    return sorted(set(re.findall(r"\b(hm_[a-z0-9_]+)\s*\(", text)))


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


def test_binding_constants_match_header():
    """Every #define of include/hm.h that the binding mirrors has the same value,
    and the binding's structures have the header's sizes (checked field by field
    through the offsets the C compiler would give: all fields are 8-byte or
    4-byte scalars in declaration order)."""
    from paper_1706_09384_gb300 import hm
    text = open(os.path.join(ROOT, "include", "hm.h")).read()
    defines = dict(re.findall(r"#define\s+(HM_[A-Z0-9_]+)\s+(\d+)", text))
    for name in ("HM_NOALLOC_MAX_POINTS", "HM_RANK_MODEL_PARAMS", "HM_NRHS_BLOCK"):
        assert name in defines, name
        assert getattr(hm, name) == int(defines[name]), name
    # points, normals, n_c | rho, lambda, mu, omega | kernel, pad_ | eta, leaf_size, weights
    assert ctypes.sizeof(hm.hm_problem) == 3 * 8 + 4 * 8 + 2 * 4 + 3 * 8
    # storage, aca_fp32 | diag_value, fp64_switch_ksr | recompress, aca_max_rank |
    # workspace_bytes | verbose, pad_ | weights, rank_model, tune_cache
    assert ctypes.sizeof(hm.hm_opts) == 2 * 4 + 2 * 8 + 2 * 4 + 8 + 2 * 4 + 3 * 8
    assert "tune_cache" in text


def test_batch_argument_errors_without_gpu():
    from paper_1706_09384_gb300 import hm
    L = hm.lib()
    outs = (ctypes.c_void_p * 2)()
    assert L.hm_build_batch(0, None, 1e-4, None, None, outs) == hm.HM_ERR_ARG
    assert L.hm_gmres_multi(None, 2, None, None, 50, 1e-6, 100, None, None, None) == hm.HM_ERR_ARG


def test_noalloc_binding_refuses_undersized_output_without_a_gpu():
    """The allocation-free entry point writes (3m + 3n) cap complex128 entries
    through a raw pointer: the binding refuses a smaller buffer (or a mistyped
    or strided one) itself, before the library is called."""
    torch = pytest.importorskip("torch")
    from paper_1706_09384_gb300 import hm
    x = torch.zeros((10, 3), dtype=torch.float64)
    y = torch.ones((8, 3), dtype=torch.float64)
    cap = 12
    need = (3 * 10 + 3 * 8) * cap
    bad = [
        (x, y, torch.zeros(need - 1, dtype=torch.complex128), "holds"),
        (x, y, torch.zeros(need, dtype=torch.complex64), "complex128"),
        (x.t().contiguous().t(), y, torch.zeros(need, dtype=torch.complex128), "contiguous"),
        (x, y, torch.zeros(need, dtype=torch.complex128), "cuda"),  # right sizes, host memory
    ]
    for xx, yy, uv, words in bad:
        with pytest.raises(hm.HmError) as e:
            hm.hm_aca_block_noalloc(hm.HM_KERNEL_U, 1.0, 2.0, 1.0, 4.0, xx, yy, None, 1e-4, cap,
                                    uv)
        assert e.value.status == hm.HM_ERR_ARG and words in str(e.value)


def test_build_options_are_checked_without_a_gpu():
    """Options the library does not implement are refused, not ignored:
    aca_fp32 must be 0 (the ACA residuals run in double-float arithmetic) and
    fp64_switch_ksr must be positive (+inf: always FP64)."""
    import numpy as np
    from paper_1706_09384_gb300 import hm
    L = hm.lib()
    pts = np.random.default_rng(0).standard_normal((4, 3))
    h = ctypes.c_void_p()
    for kw in ({"aca_fp32": 1}, {"fp64_switch_ksr": 0.0}, {"fp64_switch_ksr": float("nan")},
               {"fp64_switch_ksr": -1.0}):
        o = hm.hm_opts_default(**kw)
        st = L.hm_build(pts.ctypes.data_as(ctypes.c_void_p), None, 4, 1.0, 2.0, 1.0, 1.0, 0,
                        1e-4, 3.0, 32, ctypes.byref(o), None, ctypes.byref(h))
        assert st == hm.HM_ERR_ARG, kw
        assert h.value is None
    o = hm.hm_opts_default()
    assert o.aca_fp32 == 0 and o.fp64_switch_ksr == float("inf")
