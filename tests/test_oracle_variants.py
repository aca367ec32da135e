"""Pins of the oracle's variants: the projected-centre depth of Sec. 4.1
(depth order of two Gaussians where the 1D-mean order and the centre order
differ, composited by hand), and the trigonometric hash draw of Eq. 8-9
(its coefficients against the values the paper prints; range, uniformity,
per-sample variation, approximate unbiasedness). The composition
r2(p_xy + r1(p_z)) itself is pinned only statistically: the paper prints no
hash values to compare with."""
import json
import os

import numpy as np
from scipy.spatial.transform import Rotation

import scenes


def _two_gaussians():
    # A: centre at the origin, long along (1,0,1)/sqrt2, seen by a ray along
    # -z at x = 0.2, whose 1D mean sits near z = 0.2 (depth 2.8) while the
    # centre's depth is 3.0. B: small, on the ray at z = 0.1 (depth 2.9).
    q = Rotation.from_rotvec([0, -np.pi / 4, 0]).as_quat()  # maps x to (1,0,1)/sqrt2
    quats = np.array([[q[3], q[0], q[1], q[2]], [1, 0, 0, 0]], np.float32)
    means = np.array([[0.0, 0.0, 0.0], [0.2, 0.0, 0.1]], np.float32)
    ls = np.log(np.array([[0.6, 0.08, 0.08], [0.05, 0.05, 0.05]], np.float32))
    logits = np.array([0.5, 1.0], np.float32)
    sh = np.array([[[1, 0, 0]], [[0, 1, 0]]], np.float32)
    return scenes.GaussianCloud(means, ls.astype(np.float32), quats, logits, sh, 0)


def test_centre_depth_changes_the_order(oracle_lib):
    cloud = _two_gaussians()
    cam = scenes.Pinhole(width=1, height=1, eye=(0.2, 0.0, 3.0), look_at=(0.2, 0.0, 0.0))
    o, d, _ = oracle_lib.camera_ray(cam, 0, 0)
    tA, qA, aA, vA = oracle_lib.eval_pair(cloud, 0, o, d)
    tB, qB, aB, vB = oracle_lib.eval_pair(cloud, 1, o, d)
    assert vA and vB
    assert tA < tB  # 1D-mean order: A first
    cA, cB = np.array([1.0, 0, 0]), np.array([0, 1.0, 0])
    mean_mode = oracle_lib.render_pinhole(cloud, cam, scenes.TraceSettings(depth_mode=0))
    centre_mode = oracle_lib.render_pinhole(cloud, cam, scenes.TraceSettings(depth_mode=1))
    assert np.allclose(mean_mode["blend"][0], aA * cA + (1 - aA) * aB * cB, atol=1e-12)
    assert np.allclose(centre_mode["blend"][0], aB * cB + (1 - aB) * aA * cA, atol=1e-12)


def test_hash_constants_match_the_paper(oracle_lib):
    path = os.path.join(os.path.dirname(__file__), "golden", "trig_hash_constants.json")
    gold = json.load(open(path))
    got = oracle_lib.hash_constants()
    assert got["a1"] == gold["a1"] and got["b1"] == gold["b1"]
    assert got["a2"] == gold["a2"] and got["b2"] == gold["b2"]


def test_hash_draws(oracle_lib):
    rng = np.random.default_rng(0)
    pts = rng.uniform(-1, 1, (20000, 3))
    xi = np.array([oracle_lib.hash_xi(p, 3) for p in pts])
    assert xi.min() >= 0 and xi.max() < 1
    h, _ = np.histogram(xi, bins=20, range=(0, 1))
    chi2 = ((h - 1000) ** 2 / 1000).sum()
    assert chi2 < 43.8
    # different samples of one point differ
    same_p = np.array([oracle_lib.hash_xi(pts[0], s) for s in range(64)])
    assert len(np.unique(same_p)) > 60


def test_hash_estimator_is_nearly_unbiased(oracle_lib):
    cloud = scenes.tiny_cloud(0)
    cam = scenes.default_camera(16, 16)
    r = oracle_lib.render_pinhole(cloud, cam, scenes.TraceSettings(spp=2048, rng_mode=1))
    hit = r["n_valid"] > 0
    err = r["est"][hit] - r["blend"][hit]
    sd = np.sqrt(np.maximum(r["blend2"][hit] - r["blend"][hit] ** 2, 1e-12) / 2048)
    z = err / sd
    assert abs(z.mean()) < 0.25
    assert np.mean(np.abs(z) > 4) < 0.02
