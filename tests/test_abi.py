"""The C ABI without a GPU: the library loads, exports every function that
include/*.h declares, and rejects bad arguments before touching CUDA."""
import ctypes as C
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def gs():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2504_06598_gb300 as m
    return m


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(gs_[a-z0-9_]+)\s*\(", text))
    return names


def test_exports_every_declared_symbol(gs):
    names = _declared()
    assert {"gs_build_bvh", "gs_trace_stochastic", "gs_bvh_free"} <= names
    lib = C.CDLL(gs.LIB_PATH)
    for n in sorted(names):
        assert hasattr(lib, n), n
    # the binding knows every declared function
    assert names <= set(gs._SIGNATURES)


def test_status_strings(gs):
    L = gs.lib()
    for code in range(8):
        assert L.gs_status_string(code)
    assert L.gs_status_string(99) == b"unknown status"


def test_argument_errors_before_cuda(gs):
    L = gs.lib()
    h = C.c_void_p()
    assert L.gs_build_bvh(None, C.byref(h), None) == 1
    g = gs._Gaussians(0, 0, 0, 0, 0, 10, 3, 0)
    assert L.gs_build_bvh(C.byref(g), C.byref(h), None) == 1
    assert b"NULL" in L.gs_last_error()
    g = gs._Gaussians(16, 16, 16, 16, 16, -1, 3, 0)
    assert L.gs_build_bvh(C.byref(g), C.byref(h), None) == 1
    g = gs._Gaussians(16, 16, 16, 16, 16, 10, 4, 0)
    assert L.gs_build_bvh(C.byref(g), C.byref(h), None) == 1
    g = gs._Gaussians(16, 16, 16, 16, 16, 10, 3, 7)
    assert L.gs_build_bvh(C.byref(g), C.byref(h), None) == 1
    assert L.gs_bvh_rebuild(None, C.byref(g), None) == 1
    assert L.gs_bvh_sync_status(None, None) == 1
    assert L.gs_bvh_free(None) == 0
    assert L.gs_trace_stochastic(None, None, None, None, None, None, None, None) == 1
    assert L.gs_trace_stochastic_keys(None, None, None, None, None, None, None) == 1
    assert L.gs_trace_backward_keys(*([None] * 12)) == 1


def test_keys_struct_layout():
    """gs_sample_key is {float tc, float tau, uint32 gid}: 12 bytes, and the
    binding's int32 [..., 3] buffer has the same layout."""
    text = open(os.path.join(ROOT, "include", "gsrt.h")).read()
    body = re.search(r"typedef struct gs_sample_key \{(.*?)\} gs_sample_key;", text, re.S).group(1)
    fields = re.findall(r"\b(float|uint32_t)\s+(\w+);", body)
    assert fields == [("float", "tc"), ("float", "tau"), ("uint32_t", "gid")]


def test_no_device_is_reported(gs):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    L = gs.lib()
    h = C.c_void_p()
    g = gs._Gaussians(16, 16, 16, 16, 16, 10, 3, 0)
    assert L.gs_build_bvh(C.byref(g), C.byref(h), None) == 7
