"""The C-ABI library builds, loads without a GPU and exports every entry point
declared in include/lsrn.h; without a GPU every compute call fails loudly."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(lsrn_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1109_5981_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("lsrn_plan", "lsrn_sketch", "lsrn_precond", "lsrn_solve_lsqr",
                     "lsrn_solve_cs", "lsrn_submit", "lsrn_poll"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_default_options_and_status_strings():
    import paper_1109_5981_gb300 as L
    o = L.default_options()
    assert o.gamma == 2.0 and o.tol == 1e-14 and o.lambda_ == 0.0 and o.refine_max == 1
    assert o.rcond < 0 and o.cs_alpha < 0 and o.max_iter < 0
    assert L.status_string(L.LSRN_ERR_DIVERGED) == "LSRN_ERR_DIVERGED"
    assert L.status_string(L.LSRN_OK) == "LSRN_OK"


def test_binding_rejects_bad_options():
    import paper_1109_5981_gb300 as L
    with pytest.raises(TypeError):
        L.default_options(no_such_option=1)


def test_no_cpu_fallback_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1109_5981_gb300 as L
    with pytest.raises(L.LsrnError) as e:
        L.solve(np.ones((20, 4)), np.ones(20))
    assert e.value.status in (L.LSRN_ERR_CUDA,)


def test_server_needs_a_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1109_5981_gb300 as L
    with pytest.raises(L.LsrnError) as e:
        L.lsrn_server_create(1 << 30, 2)
    assert e.value.status == L.LSRN_ERR_CUDA
    with pytest.raises(L.LsrnError) as e:
        L.lsrn_server_create(0, 2)
    assert e.value.status == L.LSRN_ERR_INVALID_ARG


def test_inspection_calls_reject_a_null_plan():
    # argument checks come before any device call, so they hold without a GPU
    import paper_1109_5981_gb300 as L
    lib = L.load_library()
    rows, cols = ctypes.c_int64(), ctypes.c_int64()
    scale = ctypes.c_double()
    assert lib.lsrn_plan_get_sketch(None, None, ctypes.byref(rows), ctypes.byref(cols)) == \
        L.LSRN_ERR_INVALID_ARG
    assert lib.lsrn_plan_get_precond(None, None, None, ctypes.byref(rows)) == L.LSRN_ERR_INVALID_ARG
    assert lib.lsrn_plan_get_planes(None, None, None, None, ctypes.byref(rows), ctypes.byref(cols),
                                    ctypes.byref(scale)) == L.LSRN_ERR_INVALID_ARG
