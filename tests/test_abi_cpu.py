"""CPU checks of the C-ABI boundary: the library loads without a GPU, exports every
function include/fepa.h declares with the binding's signature, and the product code
never reaches the oracle."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "fepa.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?(?:int|void|int64_t|int32_t|char)\s*\*?\s*(fepa_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2402_15940_b300 import build
    build.build()
    from paper_2402_15940_b300 import fepa
    return fepa.load_library()


def test_header_symbols_exported(lib):
    from paper_2402_15940_b300 import fepa
    names = header_functions()
    assert len(names) >= 20
    bound = {n for n, _, _ in fepa.SIGNATURES}
    for n in names:
        assert hasattr(lib, n), n          # exported by the .so
        assert n in bound, n                # declared in the binding
    assert bound == set(names)


def test_exports_are_plain_c(lib):
    out = os.popen("nm -D --defined-only %s" % os.path.join(ROOT, "paper_2402_15940_b300", "libfepa.so")).read()
    exported = set(re.findall(r" T (fepa_\w+)", out))
    assert set(header_functions()) <= exported


def test_version_and_error_strings(lib):
    assert b"sm_103a" in lib.fepa_version()
    assert isinstance(lib.fepa_last_error(), bytes)
    assert lib.fepa_launch_count() >= 0


def test_argument_errors_need_no_gpu(lib):
    import ctypes
    from paper_2402_15940_b300 import fepa
    h = ctypes.c_void_p()
    # invalid order / form / null pointers are rejected before any device work
    assert lib.fepa_op_create(1, 1, 1, None, 2, 0, 1, None, ctypes.byref(h)) == fepa.ERR_ARG
    import numpy as np
    v = np.zeros((8, 3))
    assert lib.fepa_op_create(1, 1, 1, v.ctypes.data_as(ctypes.c_void_p), 9, 0, 1, None, ctypes.byref(h)) == fepa.ERR_UNSUPPORTED
    assert lib.fepa_op_create(1, 1, 1, v.ctypes.data_as(ctypes.c_void_p), 2, 7, 1, None, ctypes.byref(h)) == fepa.ERR_UNSUPPORTED
    assert lib.fepa_op_create(0, 1, 1, v.ctypes.data_as(ctypes.c_void_p), 2, 0, 1, None, ctypes.byref(h)) == fepa.ERR_ARG
    assert lib.fepa_op_create(1, 1, 1, v.ctypes.data_as(ctypes.c_void_p), 2, 0, 5, None, ctypes.byref(h)) == fepa.ERR_ARG
    assert b"unknown form" in lib.fepa_last_error()
    assert lib.fepa_cg_solve(None, None, None, 1e-10, 10, 1, None) == fepa.ERR_ARG
    assert lib.fepa_op_set_fused_dot(None, 1) == fepa.ERR_ARG
    assert lib.fepa_op_apply_f32_dot(None, None, None, None) == fepa.ERR_ARG
    st = fepa.SolverState()
    assert lib.fepa_mg_solver_start(None, None, None, 1e-10, 10) == fepa.ERR_ARG
    assert lib.fepa_mg_solver_advance(None, 1) == fepa.ERR_ARG
    assert lib.fepa_mg_solver_poll(None, 0, ctypes.byref(st)) == fepa.ERR_ARG
    assert lib.fepa_batch_group_info(None, 0, None, None, None, None, None) == fepa.ERR_ARG


def test_product_code_never_imports_oracle():
    pkg = os.path.join(ROOT, "paper_2402_15940_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".hpp", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", txt, re.M), f
                assert "fem_oracle" not in txt, f
