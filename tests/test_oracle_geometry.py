"""Pins of the oracle's activation and 1D-Gaussian arithmetic (Eq. 1-2,
Sec. 3.1, Alg. 1 range and negligibility tests) against library routines
(scipy rotations and sigmoid, numpy inverse, scipy scalar minimisation)
and closed forms."""
import json
import os

import numpy as np
import pytest
from scipy.optimize import minimize_scalar
from scipy.spatial.transform import Rotation
from scipy.special import expit

import scenes

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _cloud(means, log_scales, quats, logits):
    means = np.asarray(means, np.float32).reshape(-1, 3)
    M = len(means)
    return scenes.GaussianCloud(means, np.asarray(log_scales, np.float32).reshape(M, 3),
                                np.asarray(quats, np.float32).reshape(M, 4),
                                np.asarray(logits, np.float32).reshape(M),
                                np.full((M, 1, 3), 0.5, np.float32), 0)


def test_activation_matches_scipy(oracle_lib):
    cl = scenes.tiny_cloud(5, M=64)
    op, R, Si = oracle_lib.activate(cl)
    q = cl.quats.astype(np.float64)
    Rs = Rotation.from_quat(q[:, [1, 2, 3, 0]]).as_matrix()  # scipy is scalar-last
    assert np.allclose(R, Rs, atol=1e-12)
    assert np.allclose(op, expit(cl.opacity_logits.astype(np.float64)), rtol=1e-14)
    for g in range(64):
        assert np.allclose(R[g] @ R[g].T, np.eye(3), atol=1e-12)
        assert abs(np.linalg.det(R[g]) - 1.0) < 1e-12
        S2 = np.diag(np.exp(2.0 * cl.log_scales[g].astype(np.float64)))
        Sigma = Rs[g] @ S2 @ Rs[g].T
        assert np.allclose(Si[g], np.linalg.inv(Sigma), rtol=1e-9, atol=1e-9 * np.abs(Si[g]).max())


def test_quaternion_sign_and_scale_invariance(oracle_lib):
    cl = scenes.tiny_cloud(6, M=8)
    _, R1, _ = oracle_lib.activate(cl)
    cl2 = scenes.tiny_cloud(6, M=8)
    cl2.quats = (-3.0 * cl2.quats).astype(np.float32)
    _, R2, _ = oracle_lib.activate(cl2)
    assert np.allclose(R1, R2, atol=1e-12)


@pytest.mark.parametrize("axis", [0, 1])
def test_axis_aligned_closed_form(oracle_lib, axis):
    """Gaussian at the origin, scales sigma; ray along -z offset by b on one
    axis: t* = 5, q = b^2/sigma_axis^2, alpha = o exp(-q/2)."""
    sig = np.array([0.3, 0.7, 0.2])
    logit = 0.4
    cl = _cloud([0, 0, 0], np.log(sig), [1, 0, 0, 0], [logit])
    o_f = float(expit(np.float64(np.float32(logit))))
    for b in [0.0, 0.1, 0.25, 0.5]:
        o = np.zeros(3)
        o[axis] = b
        o[2] = 5.0
        t, q, a, valid = oracle_lib.eval_pair(cl, 0, o, [0, 0, -1])
        s_ax = float(np.exp(np.float64(np.float32(np.log(sig[axis])))))
        assert t == pytest.approx(5.0, abs=1e-12)
        assert q == pytest.approx(b * b / s_ax**2, rel=1e-9, abs=1e-12)
        assert a == pytest.approx(o_f * np.exp(-0.5 * b * b / s_ax**2), rel=1e-10)
        assert valid == (q <= 8.0)


def test_negligibility_cutoff(oracle_lib):
    gold = json.load(open(os.path.join(GOLD, "negligibility_cutoff.json")))
    s = gold["s"]
    assert s * s == pytest.approx(gold["s_squared"], rel=1e-15)
    sig = 0.25
    cl = _cloud([0, 0, 0], np.log([sig] * 3), [1, 0, 0, 0], [0.0])
    sig_f = float(np.exp(np.float64(np.float32(np.log(sig)))))
    inside = oracle_lib.eval_pair(cl, 0, [s * sig_f * (1 - 1e-9), 0, 4], [0, 0, -1])
    outside = oracle_lib.eval_pair(cl, 0, [s * sig_f * (1 + 1e-9), 0, 4], [0, 0, -1])
    assert inside[3] and not outside[3]
    # at the boundary alpha = o exp(-s^2/2) = o e^-4
    assert inside[2] == pytest.approx(0.5 * np.exp(-4.0), rel=1e-6)


def test_range_tests(oracle_lib):
    """Alg. 1: culled when t* <= t_min or t* >= t_max; behind the origin."""
    cl = _cloud([0, 0, 0], np.log([0.2] * 3), [1, 0, 0, 0], [0.0])
    assert not oracle_lib.eval_pair(cl, 0, [0, 0, -1], [0, 0, -1])[3]  # behind
    assert oracle_lib.eval_pair(cl, 0, [0, 0, 1], [0, 0, -1])[3]
    assert not oracle_lib.eval_pair(cl, 0, [0, 0, 1], [0, 0, -1], t_min=1.0)[3]
    assert not oracle_lib.eval_pair(cl, 0, [0, 0, 1], [0, 0, -1], t_max=1.0)[3]
    assert oracle_lib.eval_pair(cl, 0, [0, 0, 1], [0, 0, -1], t_min=0.999, t_max=1.001)[3]


def test_rotation_invariance(oracle_lib):
    """Rotating the Gaussian and the ray together leaves t*, q, alpha."""
    rng = np.random.default_rng(3)
    for _ in range(10):
        q0 = rng.normal(size=4)
        cl = _cloud([0.1, -0.2, 0.3], rng.normal(-1.5, 0.3, 3), q0, [0.3])
        o = np.array([0.2, 0.1, 4.0])
        d = np.array([0.05, -0.02, -1.0])
        d /= np.linalg.norm(d)
        ref = oracle_lib.eval_pair(cl, 0, o, d)
        rot = Rotation.random(random_state=int(rng.integers(1 << 30)))
        qr = rot.as_quat()  # x,y,z,w
        qg = Rotation.from_quat(np.asarray(q0)[[1, 2, 3, 0]])
        qn = (rot * qg).as_quat()
        mu = rot.apply(cl.means[0].astype(np.float64))
        cl2 = _cloud(mu.astype(np.float32), cl.log_scales, np.asarray(qn)[[3, 0, 1, 2]], [0.3])
        # float32 rounding of the rotated mean moves it by ~1e-8
        mu32 = cl2.means[0].astype(np.float64)
        o2 = rot.apply(o) + (mu32 - mu)
        got = oracle_lib.eval_pair(cl2, 0, o2, rot.apply(d))
        assert got[0] == pytest.approx(ref[0], rel=1e-6)
        assert got[1] == pytest.approx(ref[1], rel=1e-5, abs=1e-6)
        assert got[2] == pytest.approx(ref[2], rel=1e-5)
        del qr


def test_mean_and_peak_by_minimisation(oracle_lib):
    """t* and q equal the argmin and minimum of the Mahalanobis quadratic
    form along the ray, found by scipy's bounded scalar minimiser with Sigma
    built from scipy's rotation and inverted by numpy."""
    cl = scenes.tiny_cloud(11, M=40)
    rng = np.random.default_rng(4)
    for g in range(40):
        mu = cl.means[g].astype(np.float64)
        o = np.array([0.0, 0.0, 3.0])
        target = mu + rng.normal(0, 0.03, 3)
        d = (target - o) / np.linalg.norm(target - o)
        t, q, a, valid = oracle_lib.eval_pair(cl, g, o, d)
        Rq = Rotation.from_quat(cl.quats[g].astype(np.float64)[[1, 2, 3, 0]]).as_matrix()
        Sigma = Rq @ np.diag(np.exp(2 * cl.log_scales[g].astype(np.float64))) @ Rq.T
        Si = np.linalg.inv(Sigma)
        f = lambda tt: float((o + tt * d - mu) @ Si @ (o + tt * d - mu))  # noqa: E731
        res = minimize_scalar(f, bounds=(0.0, 10.0), method="bounded",
                              options={"xatol": 1e-12, "maxiter": 1000})
        assert t == pytest.approx(res.x, abs=1e-5)
        assert q == pytest.approx(f(t), rel=1e-7, abs=1e-9)
        assert q <= res.fun * (1 + 1e-9) + 1e-12
        op = expit(np.float64(cl.opacity_logits[g]))
        assert a == pytest.approx(op * np.exp(-0.5 * q), rel=1e-12)
