"""gs_build_bvh_noalloc: the hierarchy build for callers that cannot call
cudaMalloc (a thread that must never trigger an allocation's implicit
synchronisation, or an application that owns all device memory through its
own pool). Its scratch is a static device array of the library; the test
checks that it writes exactly what gs_build_bvh writes, on two calls in a
row with different inputs (so the shared scratch's leftovers from the first
call cannot leak into the second), at the size limit (where the fixed
histogram and scan pieces are filled exactly) and at one Gaussian; that a
warmed-up call leaves the device's free memory unchanged; that it reports a
non-finite parameter through the caller's status word; and that it rejects
sizes above its limit and a missing status word. This file is collected
last on purpose."""
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


def _buffers(M):
    nodes = torch.zeros(max(M - 1, 1) * 64, dtype=torch.uint8, device="cuda")
    prims = torch.zeros(M * 64, dtype=torch.uint8, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    return nodes, prims, status


def _call(gs, g, nodes, prims, status):
    gstruct = g.struct()
    return gs.lib().gs_build_bvh_noalloc(C.byref(gstruct), C.c_void_p(nodes.data_ptr()),
                                         C.c_void_p(prims.data_ptr()),
                                         C.c_void_p(status.data_ptr()),
                                         C.c_void_p(torch.cuda.current_stream().cuda_stream))


def _noalloc(gs, g, expect_status=0):
    nodes, prims, status = _buffers(g.M)
    st = _call(gs, g, nodes, prims, status)
    assert st == 0, gs.lib().gs_last_error()
    torch.cuda.synchronize()
    assert int(status.item()) == expect_status
    return nodes.cpu().numpy().view(np.uint32).reshape(-1, 16), \
        prims.cpu().numpy().view(np.uint32).reshape(-1, 16)


@pytest.mark.gpu
def test_noalloc_matches_build(gs):
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    clouds = [scenes.shell_cloud(4, M=20000), scenes.tiny_cloud(9, M=7001),
              scenes.shell_cloud(5, M=MAX_M), scenes.tiny_cloud(2, M=1)]
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


@pytest.mark.gpu
def test_noalloc_keeps_free_memory(gs):
    """After a warm-up call (which loads the module and resolves the array's
    address), a call changes the device's free memory by nothing."""
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    g = gs.Gaussians.from_cloud(scenes.shell_cloud(6, M=30000))
    nodes, prims, status = _buffers(g.M)
    assert _call(gs, g, nodes, prims, status) == 0, gs.lib().gs_last_error()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        assert _call(gs, g, nodes, prims, status) == 0, gs.lib().gs_last_error()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert int(status.item()) == 0


@pytest.mark.gpu
def test_noalloc_reports_nonfinite(gs):
    """A non-finite parameter sets the caller's status word; the next clean
    call, with the word cleared, leaves it at zero."""
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    bad = scenes.tiny_cloud(3, M=500)
    bad.means[17, 1] = np.nan
    _noalloc(gs, gs.Gaussians.from_cloud(bad), expect_status=4)
    _noalloc(gs, gs.Gaussians.from_cloud(scenes.tiny_cloud(3, M=500)), expect_status=0)


@pytest.mark.gpu
def test_noalloc_rejects_missing_status(gs):
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    g = gs.Gaussians.from_cloud(scenes.tiny_cloud(1, M=100))
    nodes, prims, _ = _buffers(g.M)
    gstruct = g.struct()
    st = gs.lib().gs_build_bvh_noalloc(C.byref(gstruct), C.c_void_p(nodes.data_ptr()),
                                        C.c_void_p(prims.data_ptr()), None, None)
    assert st == 1
    assert b"status_out" in gs.lib().gs_last_error()
