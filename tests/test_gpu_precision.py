"""Precision form: 4-wide hierarchies with FP32 and 8-bit quantised child
boxes, and the 8-bit form of the 8/16/32-wide copies that groups of lanes
traverse, give exactly the FP32 binary traversal's samples (conservative
boxes only prune), decoded 8-bit boxes contain the FP32 boxes, and SH
stored in FP16 / BF16 shades within 1e-5 of the FP64 oracle fed the same
rounded coefficients."""
import numpy as np
import pytest

import oracle
import scenes
from tests import _parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gs():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2504_06598_gb300 as m
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for gpu tests")
    return m


def _trace(gs, g, cam, fmt, **kw):
    bvh = gs.build_bvh(g, node_format=fmt)
    rgb, hid, ht = gs.trace_stochastic(bvh, g, cam, want_hits=True, **kw)
    bvh.sync_status()
    out = (rgb.cpu().numpy(), hid.cpu().numpy(), ht.cpu().numpy())
    bvh.free()
    return out


@pytest.mark.parametrize("which", ["tiny", "shell", "one", "coincident"])
@pytest.mark.parametrize("n_hits,spp", [(1, 4), (4, 2)])
def test_wide_formats_match_binary(gs, which, n_hits, spp):
    if which == "tiny":
        cloud, cam = scenes.tiny_cloud(0), scenes.default_camera(64, 48)
    elif which == "shell":
        cloud, cam = scenes.shell_cloud(1, M=50000), scenes.default_camera(120, 90)
    elif which == "one":
        cloud, cam = scenes.tiny_cloud(2, M=1), scenes.default_camera(16, 16)
        cloud.means[:] = 0.0
        cloud.log_scales[:] = -1.0
    else:
        cloud, cam = scenes.tiny_cloud(3, M=700), scenes.default_camera(24, 24)
        cloud.means[:] = 0.02
        cloud.log_scales[:] += 1.5
    g = gs.Gaussians.from_cloud(cloud)
    ref = _trace(gs, g, cam, "binary", seed=3, spp=spp, n_hits=n_hits)
    for fmt in ("wide4", "wide4_q8"):
        got = _trace(gs, g, cam, fmt, seed=3, spp=spp, n_hits=n_hits)
        for a, b in zip(ref, got):
            assert np.array_equal(a, b), fmt


# (n_hits, spp, samples per lane): 8-, 16- and 32-lane groups with one
# sample per lane, then the library's own layouts (32 lanes x 2 samples at
# spp 64, 16 lanes x 4 slots at N=4 spp 16, 4-lane packets at spp 16)
@pytest.mark.parametrize("which", ["tiny", "shell", "one", "coincident"])
@pytest.mark.parametrize("n_hits,spp,spl", [(1, 8, 1), (1, 16, 1), (1, 32, 1), (1, 64, 0),
                                            (4, 16, 0), (1, 16, 0), (2, 8, 1)])
def test_binary_q8_groups_match_binary(gs, which, n_hits, spp, spl):
    if which == "tiny":
        cloud, cam = scenes.tiny_cloud(0), scenes.default_camera(40, 30)
    elif which == "shell":
        cloud, cam = scenes.shell_cloud(1, M=50000), scenes.default_camera(72, 40)
    elif which == "one":
        cloud, cam = scenes.tiny_cloud(2, M=1), scenes.default_camera(16, 16)
        cloud.means[:] = 0.0
        cloud.log_scales[:] = -1.0
    else:
        cloud, cam = scenes.tiny_cloud(3, M=700), scenes.default_camera(24, 24)
        cloud.means[:] = 0.02
        cloud.log_scales[:] += 1.5
    g = gs.Gaussians.from_cloud(cloud)
    kw = dict(seed=3, spp=spp, n_hits=n_hits, samples_per_lane=spl)
    ref = _trace(gs, g, cam, "binary", **kw)
    got = _trace(gs, g, cam, "binary_q8", **kw)
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)


def test_binary_q8_full_size_3m(gs):
    """3M-Gaussian shell, 1080p, N=1 spp 64 (the precision form's launch):
    every sample's hit and depth from the 8-bit 32-wide records equals the
    FP32 records'; the image is bit-identical."""
    cloud = scenes.shell_cloud(0, M=3_000_000)
    cam = scenes.default_camera(1920, 1080)
    g = gs.Gaussians.from_cloud(cloud, sh_dtype=torch.float16)
    out = {}
    for fmt in ("binary", "binary_q8"):
        bvh = gs.build_bvh(g, node_format=fmt)
        out[fmt] = gs.trace_stochastic(bvh, g, cam, seed=0, spp=64, want_hits=True)
        bvh.sync_status()
        bvh.free()
    for a, b in zip(out["binary"], out["binary_q8"]):
        assert torch.equal(a, b)
    assert (out["binary"][1] >= 0).float().mean().item() > 0.05


def _decode_q8(words):
    """Decode NodeQ4 words [n,16] to FP32 boxes [n,4,6] the way the kernel
    does: plane = float32(origin + q * 2^e)."""
    n = len(words)
    cut = lambda a, b: np.ascontiguousarray(words[:, a:b])  # noqa: E731
    origin = cut(0, 3).view(np.float32)
    meta = cut(3, 4).view(np.uint8).reshape(n, 4)
    e = np.ascontiguousarray(meta[:, :3]).view(np.int8).astype(np.int32)
    used = meta[:, 3]
    qlo = cut(4, 7).view(np.uint8).reshape(n, 3, 4).astype(np.float32)
    qhi = cut(7, 10).view(np.uint8).reshape(n, 3, 4).astype(np.float32)
    scale = np.ldexp(np.float32(1.0), e).astype(np.float32)[:, :, None]
    lo = (origin[:, :, None] + (qlo * scale).astype(np.float32)).astype(np.float32)
    hi = (origin[:, :, None] + (qhi * scale).astype(np.float32)).astype(np.float32)
    child = words[:, 10:14]
    return lo, hi, used, child


def test_q8_boxes_contain_fp32_boxes(gs):
    cloud = scenes.shell_cloud(4, M=60000)
    g = gs.Gaussians.from_cloud(cloud)
    b32 = gs.build_bvh(g, node_format="wide4")
    b8 = gs.build_bvh(g, node_format="wide4_q8")
    w32 = b32.export_wide()
    w8 = b8.export_wide()
    b32.free()
    b8.free()
    assert len(w32) == len(w8) > 0
    lo32 = np.ascontiguousarray(w32[:, 0:12]).view(np.float32).reshape(-1, 3, 4)
    hi32 = np.ascontiguousarray(w32[:, 12:24]).view(np.float32).reshape(-1, 3, 4)
    c32 = w32[:, 24:28]
    lo8, hi8, used, c8 = _decode_q8(w8)
    assert np.array_equal(c32, c8)
    for k in range(4):
        m = ((used >> k) & 1).astype(bool)
        assert np.array_equal(m, c32[:, k] != 0xFFFFFFFF)
        assert np.all(lo8[m, :, k] <= lo32[m, :, k]) and np.all(hi8[m, :, k] >= hi32[m, :, k])
    # quantisation is tight: mean slack below 2% of the node extent
    ext = np.maximum(hi32.max(2) - lo32.min(2), 1e-12)[:, :, None]
    slack = ((lo32 - lo8) + (hi8 - hi32)) / ext
    assert np.nanmean(np.where(np.isfinite(slack), slack, np.nan)[np.repeat(
        ((used[:, None] >> np.arange(4)) & 1).astype(bool)[:, None, :], 3, 1)]) < 0.02
    # every leaf exactly once, every wide node reachable exactly once
    leaves = c32[(c32 != 0xFFFFFFFF) & ((c32 & 0x80000000) != 0)] & 0x7FFFFFFF
    assert np.array_equal(np.sort(leaves), np.arange(cloud.M))
    inner = c32[(c32 != 0xFFFFFFFF) & ((c32 & 0x80000000) == 0)]
    assert np.array_equal(np.sort(inner), np.arange(1, len(w32)))


@pytest.mark.parametrize("dtype", ["float16", "bfloat16"])
def test_half_precision_sh_parity(gs, dtype):
    cloud = scenes.shell_cloud(5, M=20000)
    cam = scenes.default_camera(80, 60)
    tdt = getattr(torch, dtype)
    g = gs.Gaussians.from_cloud(cloud, sh_dtype=tdt)
    g32 = gs.Gaussians.from_cloud(cloud)
    rgb, ids, _ = _trace(gs, g, cam, "wide4_q8", seed=2, spp=4)
    _, ids32, _ = _trace(gs, g32, cam, "binary", seed=2, spp=4)
    assert np.array_equal(ids, ids32)  # SH never changes acceptance
    rounded = scenes.GaussianCloud(cloud.means, cloud.log_scales, cloud.quats,
                                   cloud.opacity_logits,
                                   torch.from_numpy(cloud.sh).to(tdt).float().numpy(), 3)
    S = 4
    ids_p = ids.reshape(S, -1).T
    ref = oracle.render_pinhole(rounded, cam, scenes.TraceSettings(seed=2, spp=S))
    agree, classes, det = _parity.compare(rounded, cam, 2, ids_p, ref, np.arange(80 * 60))
    assert agree >= 0.9999 and set(classes) <= {"i"}, (agree, classes)
    same = np.all(ids_p == ref["hit_id"], axis=1)
    assert _parity.colour_check(rgb.reshape(-1, 3), ref["est"], same) <= 0.0
