"""gs_build_bvh_noalloc: the hierarchy build for callers that cannot call
cudaMalloc (a thread that must never trigger an allocation's implicit
synchronisation, or an application that owns all device memory through its
own pool). Its scratch is a static device array of the library; the test
checks that it writes exactly what gs_build_bvh writes, on two calls in a
row with different inputs (so the shared scratch's leftovers from the first
call cannot leak into the second), and that it rejects sizes above its
limit. This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

import scenes

torch = pytest.importorskip("torch")

MAX_M = 65536


@pytest.fixture(scope="module")
def gs():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2504_06598_gb300 as m
    return m


def _noalloc(gs, g):
    M = g.M
    nodes = torch.zeros(max(M - 1, 1) * 64, dtype=torch.uint8, device="cuda")
    prims = torch.zeros(M * 64, dtype=torch.uint8, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    gstruct = g.struct()
    st = gs.lib().gs_build_bvh_noalloc(C.byref(gstruct), C.c_void_p(nodes.data_ptr()),
                                        C.c_void_p(prims.data_ptr()),
                                        C.c_void_p(status.data_ptr()),
                                        C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, gs.lib().gs_last_error()
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    return nodes.cpu().numpy().view(np.uint32).reshape(-1, 16), \
        prims.cpu().numpy().view(np.uint32).reshape(-1, 16)


@pytest.mark.gpu
def test_noalloc_matches_build(gs):
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    clouds = [scenes.shell_cloud(4, M=20000), scenes.tiny_cloud(9, M=7001)]
    for cloud in clouds:
        g = gs.Gaussians.from_cloud(cloud)
        bvh = gs.build_bvh(g)
        ref = bvh.export()
        bvh.sync_status()
        bvh.free()
        nodes, prims = _noalloc(gs, g)
        assert np.array_equal(nodes, ref["nodes"])
        assert np.array_equal(prims, ref["prims"])


@pytest.mark.gpu
def test_noalloc_rejects_oversize(gs):
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    g = gs._Gaussians(16, 16, 16, 16, 16, MAX_M + 1, 3, 0)
    st = gs.lib().gs_build_bvh_noalloc(C.byref(g), None, None, None, None)
    assert st == 1
    assert b"exceeds" in gs.lib().gs_last_error()
