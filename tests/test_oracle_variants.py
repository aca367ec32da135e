"""Pins of the oracle's variants: the projected-centre depth of Sec. 4.1
(depth order of two Gaussians where the 1D-mean order and the centre order
differ, composited by hand), and the trigonometric hash draw of Eq. 8-9
(its coefficients against the values the paper prints; its composition
r2(p_xy + r1(p_z)) through special points where the sines are 0 or 1, so
the draw is a known fraction, and through invariances the composition
implies; range, uniformity, per-sample variation, approximate
unbiasedness)."""
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


def _xi_at(oracle_lib, q):
    """The hash of the point q itself: sample 0 moves the point by -5e-4 on
    every axis, so hash the point q + 5e-4."""
    return oracle_lib.hash_xi(np.asarray(q, np.float64) + 5e-4, 0)


def test_hash_composition_special_points(oracle_lib):
    """Closed forms of Eq. 8-9 at points where every sine is 0 or 1:
    sin(a1 q_z) = 0 gives r1 = 0; sin(a1 q_z) = 1 gives r1 = fract(b1);
    a2 . (q_xy + r1) = pi/2 gives xi = fract(b2); a zero argument gives 0.
    Adding r1 to only one component, a swapped coefficient or a missing
    fract fails one of them."""
    c = oracle_lib.hash_constants()
    a1, b1 = c["a1"], c["b1"]
    (a2x, a2y), b2 = c["a2"], c["b2"][0]
    fb1, fb2 = b1 - np.floor(b1), b2 - np.floor(b2)
    assert abs(_xi_at(oracle_lib, (0.0, 0.0, 0.0))) < 1e-12
    # r1 = 0, argument pi/2
    assert abs(_xi_at(oracle_lib, (np.pi / 2 / a2x, 0.0, 0.0)) - fb2) < 1e-9
    assert abs(_xi_at(oracle_lib, (0.0, np.pi / 2 / a2y, 0.0)) - fb2) < 1e-9
    # r1 = fract(b1) enters both components: pick q_x so the argument is pi/2
    qz = np.pi / 2 / a1
    qx = (np.pi / 2 - a2y * fb1) / a2x - fb1
    assert abs(_xi_at(oracle_lib, (qx, 0.0, qz)) - fb2) < 1e-9
    qy = (np.pi / 2 - a2x * fb1) / a2y - fb1
    assert abs(_xi_at(oracle_lib, (0.0, qy, qz)) - fb2) < 1e-9


def test_hash_composition_invariances(oracle_lib):
    """The draw depends on q_xy only through a2 . q_xy (moving along
    (a2y, -a2x) keeps it), is periodic in that argument with period 2 pi,
    and r1 acts as the same shift of both components: xi(q_x, q_y,
    pi / (2 a1)) = xi(q_x + fract(b1), q_y + fract(b1), 0). (Periodicity in
    q_z is not testable in float64: the chain of large coefficients turns a
    1e-16 rounding of sin(a1 q_z) into 1e-4 of the draw.)"""
    c = oracle_lib.hash_constants()
    a1, b1 = c["a1"], c["b1"]
    a2x, a2y = c["a2"]
    fb1 = b1 - np.floor(b1)
    rng = np.random.default_rng(3)
    for _ in range(20):
        q = rng.uniform(-0.5, 0.5, 3)
        base = _xi_at(oracle_lib, q)
        t = rng.uniform(-0.01, 0.01)
        moved = q + np.array([a2y * t, -a2x * t, 0.0])
        assert abs(_xi_at(oracle_lib, moved) - base) < 1e-7
        assert abs(_xi_at(oracle_lib, q + [2 * np.pi / a2x, 0.0, 0.0]) - base) < 1e-7
        lhs = _xi_at(oracle_lib, (q[0], q[1], np.pi / 2 / a1))
        rhs = _xi_at(oracle_lib, (q[0] + fb1, q[1] + fb1, 0.0))
        assert abs(lhs - rhs) < 1e-7


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
