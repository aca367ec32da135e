"""GPU hierarchy build checked on the host: sorted keys, a valid binary tree
over every Gaussian, parent boxes that contain their children, leaf boxes
that contain each Gaussian's exact ellipsoid box (Eq. 2), and records that
match the oracle's activation (Eq. 1)."""
import numpy as np
import pytest

import oracle
import scenes

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


def _export(gs, cloud):
    g = gs.Gaussians.from_cloud(cloud)
    bvh = gs.build_bvh(g)
    bvh.sync_status()
    ex = bvh.export()
    bvh.free()
    return ex


def _check_tree(ex, M):
    codes, order, nodes = ex["codes"], ex["order"], ex["nodes"]
    assert np.all(codes[1:] >= codes[:-1])
    # stable: equal keys keep increasing Gaussian ids
    eq = codes[1:] == codes[:-1]
    assert np.all(order[1:][eq] > order[:-1][eq])
    assert np.array_equal(np.sort(order), np.arange(M, dtype=np.uint32))
    n = len(nodes)
    assert n == max(M - 1, 1)
    boxes = nodes[:, :12].copy().view(np.float32).reshape(n, 2, 6)
    child = nodes[:, 12:14]
    leaf = (child & 0x80000000) != 0
    idx = child & 0x7FFFFFFF
    if M == 1:
        assert np.all(leaf) and np.all(idx == 0)
        return boxes, child
    # every internal node but the root and every leaf referenced exactly once
    internal_refs = np.sort(idx[~leaf])
    assert np.array_equal(internal_refs, np.arange(1, n))
    assert np.array_equal(np.sort(idx[leaf]), np.arange(M))
    # each node covers a contiguous leaf range: the left child's, then the right's
    rng = nodes[:, 14:16].astype(np.int64)
    assert rng[0, 0] == 0 and rng[0, 1] == M - 1
    lo_of = lambda s: np.where(leaf[:, s], idx[:, s], rng[idx[:, s] * (~leaf[:, s]), 0])  # noqa: E731
    hi_of = lambda s: np.where(leaf[:, s], idx[:, s], rng[idx[:, s] * (~leaf[:, s]), 1])  # noqa: E731
    assert np.array_equal(lo_of(0), rng[:, 0]) and np.array_equal(hi_of(1), rng[:, 1])
    assert np.array_equal(hi_of(0) + 1, lo_of(1))
    # parent slot box contains the child's own box (the union of its slots)
    for i in range(n):
        for s in range(2):
            if not leaf[i, s]:
                c = idx[i, s]
                own_lo = np.minimum(boxes[c, 0, :3], boxes[c, 1, :3])
                own_hi = np.maximum(boxes[c, 0, 3:], boxes[c, 1, 3:])
                assert np.all(boxes[i, s, :3] <= own_lo) and np.all(boxes[i, s, 3:] >= own_hi)
    # every node reachable from the root
    seen = np.zeros(n, bool)
    stack = [0]
    while stack:
        i = stack.pop()
        assert not seen[i]
        seen[i] = True
        stack += [int(idx[i, s]) for s in range(2) if not leaf[i, s]]
    assert seen.all()
    return boxes, child


@pytest.mark.parametrize("which", ["tiny", "shell", "one", "two", "coincident"])
def test_tree_structure_and_boxes(gs, which):
    if which == "tiny":
        cloud = scenes.tiny_cloud(0)
    elif which == "shell":
        cloud = scenes.shell_cloud(5, M=30000)
    elif which == "one":
        cloud = scenes.tiny_cloud(1, M=1)
    elif which == "two":
        cloud = scenes.tiny_cloud(2, M=2)
    else:
        cloud = scenes.tiny_cloud(3, M=3000)
        cloud.means[:] = cloud.means[0]  # every centroid equal: keys tie
    M = cloud.M
    ex = _export(gs, cloud)
    boxes, child = _check_tree(ex, M)
    # leaf boxes contain the exact FP64 box of the ellipsoid |M(x-mu)| <= 2 sqrt 2
    _, R, _ = oracle.activate(cloud)
    s = np.exp(cloud.log_scales.astype(np.float64))
    half = 2 * np.sqrt(2) * np.sqrt(np.einsum("gik,gk->gi", R ** 2, s ** 2))
    mu = cloud.means.astype(np.float64)
    leaf_box = np.zeros((M, 6))
    n = len(ex["nodes"])
    for i in range(n):
        for sl in range(2):
            if child[i, sl] & 0x80000000:
                pos = child[i, sl] & 0x7FFFFFFF
                leaf_box[ex["order"][pos]] = boxes[i, sl]
    assert np.all(leaf_box[:, :3] <= mu - half) and np.all(leaf_box[:, 3:] >= mu + half)
    # boxes are tight up to the documented padding (2^-10 relative + 2^-18 abs)
    assert np.all(leaf_box[:, :3] >= mu - half * (1 + 2e-3) - 1e-4)


def test_records_match_activation(gs):
    cloud = scenes.shell_cloud(6, M=5000)
    ex = _export(gs, cloud)
    rec = ex["prims"].view(np.float32)
    gid = ex["prims"][:, 13]
    assert np.array_equal(gid, ex["order"])
    op, R, _ = oracle.activate(cloud)
    inv_s = np.exp(-cloud.log_scales.astype(np.float64))
    Mref = inv_s[:, :, None] * np.transpose(R, (0, 2, 1))  # S^-1 R_q^T
    assert np.array_equal(rec[:, :3], cloud.means[gid])
    assert np.allclose(rec[:, 3], op[gid], rtol=1e-6)
    Mgpu = rec[:, 4:13].reshape(-1, 3, 3).astype(np.float64)
    scale = np.abs(Mref[gid]).max(axis=2, keepdims=True)
    assert np.all(np.abs(Mgpu - Mref[gid]) <= 2e-6 * scale)


def test_rebuild_equals_fresh_build(gs):
    a = scenes.shell_cloud(7, M=9000)
    b = scenes.shell_cloud(8, M=6000)
    ga, gb = gs.Gaussians.from_cloud(a), gs.Gaussians.from_cloud(b)
    bvh = gs.build_bvh(ga)
    bvh.rebuild(gb)
    bvh.sync_status()
    ex = bvh.export()
    bvh.free()
    ref = _export(gs, b)
    for k in ("nodes", "prims", "codes", "order"):
        assert np.array_equal(ex[k], ref[k]), k
