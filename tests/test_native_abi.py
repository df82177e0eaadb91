"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, exports every function declared in include/gnaosc.h, the
binding declares each of them, and the product path refuses to run without
a CUDA device instead of falling back to the CPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gnaosc.h")


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(gna_[a-z0-9_]+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1804_07682_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_abi():
    fns = header_functions()
    for name in ["gna_oscprob_ee", "gna_plan_create", "gna_chain_eval", "gna_chain_eval_host", "gna_chain_eval_plain",
                 "gna_fit_batch", "gna_gl_nodes", "gna_plan_status", "gna_plan_autotune"]:
        assert name in fns


def test_library_exports_every_header_function(lib):
    missing = [f for f in header_functions() if not hasattr(lib, f)]
    assert not missing, missing


def test_binding_declares_every_header_function():
    from paper_1804_07682_gb300 import _native

    assert sorted(_native.SIGNATURES) == header_functions()


def test_strerror_is_host_only(lib):
    lib.gna_strerror.restype = ctypes.c_char_p
    assert lib.gna_strerror(0) == b"ok"
    assert lib.gna_strerror(5).startswith(b"bounded device wait")
    assert lib.gna_strerror(99) == b"unknown status"


def test_argument_errors_return_before_any_device_work(lib):
    # NULL plan / NULL arguments are rejected on the host
    assert lib.gna_plan_destroy(None) == 0
    assert lib.gna_plan_status(None) == 1
    assert lib.gna_chain_eval(None, None, None, ctypes.c_double(0), None, 0, None, None) == 1
    out = ctypes.c_void_p()
    assert lib.gna_plan_create(ctypes.byref(out), None, None) == 1
    assert lib.gna_gl_nodes(0, ctypes.c_void_p(1), ctypes.c_void_p(1), None) == 2
    assert lib.gna_gl_nodes(8, None, None, None) == 1
    # n = 0 OscProb is a no-op; bad nL is a shape error
    lib.gna_oscprob_ee.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                   ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    L = (ctypes.c_double * 1)(52.5)
    p = (ctypes.c_double * 4)(0.307, 0.0218, 7.53e-5, 2.44e-3)
    assert lib.gna_oscprob_ee(None, 0, L, 1, p, 0, None, None) == 0
    assert lib.gna_oscprob_ee(None, 10, L, 17, p, 0, None, None) == 2
    assert lib.gna_oscprob_ee(None, -1, L, 1, p, 0, None, None) == 2
    assert lib.gna_oscprob_ee(None, 10, L, 1, p, 7, None, None) == 1


def test_product_path_refuses_cpu():
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1804_07682_gb300 import api

    with pytest.raises(RuntimeError):
        api.Plan([1.0, 2.0], [1.0], nodes_per_bin=4)
    with pytest.raises(RuntimeError):
        api.oscprob(torch.ones(4, dtype=torch.float64), [1.0], (0.3, 0.02, 7e-5, 2e-3))
