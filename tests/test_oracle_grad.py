"""Pins of the oracle's gradients (differentiable rendering, Sec. 6): the
analytic gradient of the exact blend against central finite differences of
the oracle's own blend, a closed form for one Gaussian, and the stochastic
estimator's gradient converging to the blend gradient (unbiasedness)."""
import numpy as np
import pytest
from scipy.special import expit

import scenes

PARAMS = ["means", "log_scales", "quats", "opacity_logits", "sh"]


def _cluster(seed=0, M=40, sh_degree=1):
    rng = np.random.default_rng(seed)
    means = np.stack([rng.uniform(-0.15, 0.15, M), rng.uniform(-0.15, 0.15, M),
                      rng.uniform(-0.4, 0.4, M)], 1)
    K = (sh_degree + 1) ** 2
    sh = np.concatenate([rng.uniform(0.1, 1.0, (M, 1, 3)), rng.normal(0, 0.3, (M, K - 1, 3))], 1)
    f = lambda a: np.ascontiguousarray(a, np.float32)  # noqa: E731
    return scenes.GaussianCloud(f(means), f(rng.normal(-2.3, 0.3, (M, 3))),
                                f(rng.normal(size=(M, 4))), f(rng.normal(0.5, 1.0, M)), f(sh),
                                sh_degree)


def _camera():
    return scenes.Pinhole(width=6, height=6, fov_y_deg=9.0)


def _G(oracle_lib, cloud, cam, st, g):
    r = oracle_lib.render_pinhole(cloud, cam, st, want_hits=False)
    return float(np.sum(r["blend"] * g))


def _perturbed(cloud, name, idx, delta):
    c = scenes.GaussianCloud(cloud.means.copy(), cloud.log_scales.copy(), cloud.quats.copy(),
                             cloud.opacity_logits.copy(), cloud.sh.copy(), cloud.sh_degree)
    arr = getattr(c, name)
    v = arr[idx]
    new = np.float32(np.float64(v) + delta)
    arr[idx] = new
    return c, float(np.float64(new) - np.float64(v))


def _fd(oracle_lib, cloud, cam, st, g, name, idx, h):
    """Central difference; a depth-order swap inside the step (not
    differentiated on purpose) shows as disagreement between h and h/2, in
    which case the step shrinks."""
    def one(hh):
        cp, hp = _perturbed(cloud, name, idx, +hh)
        cm, hm = _perturbed(cloud, name, idx, -hh)
        return (_G(oracle_lib, cp, cam, st, g) - _G(oracle_lib, cm, cam, st, g)) / (hp - hm)
    for _ in range(4):
        a, b = one(h), one(h / 2)
        if abs(a - b) <= 1e-3 * max(abs(a), abs(b)) + 1e-9:
            return b
        h /= 10
    return b


def test_blend_gradient_matches_finite_differences(oracle_lib):
    cloud = _cluster()
    cam = _camera()
    st = scenes.TraceSettings(bg=(0.2, 0.1, 0.4))
    rng = np.random.default_rng(1)
    g = rng.normal(size=(cam.width * cam.height, 3))
    an = oracle_lib.grad_pinhole(cloud, cam, st, g, mode="blend")
    # the Gaussians that matter most
    weight = np.abs(an["opacity_logits"]) + np.abs(an["means"]).sum(1)
    top = np.argsort(-weight)[:6]
    assert weight[top[0]] > 0
    checked = 0
    for gi in top:
        for name, shape in [("means", 3), ("log_scales", 3), ("quats", 4), ("opacity_logits", 1)]:
            for k in range(shape):
                idx = (gi, k) if shape > 1 else gi
                base = np.float64(getattr(cloud, name)[idx])
                fd = _fd(oracle_lib, cloud, cam, st, g, name, idx, 3e-5 * max(abs(base), 0.05))
                a = an[name][idx]
                scale = np.abs(an[name]).max()
                assert abs(fd - a) <= 1e-4 * scale + 1e-7, (name, gi, k, fd, a)
                checked += 1
        for k in range(cloud.sh.shape[1]):
            for ch in range(3):
                idx = (gi, k, ch)
                cp, hp = _perturbed(cloud, "sh", idx, +0.01)
                cm, hm = _perturbed(cloud, "sh", idx, -0.01)
                fd = (_G(oracle_lib, cp, cam, st, g) - _G(oracle_lib, cm, cam, st, g)) / (hp - hm)
                assert abs(fd - an["sh"][idx]) <= 1e-6 * np.abs(an["sh"]).max() + 1e-9
    assert checked == 6 * 11


def test_single_gaussian_closed_form(oracle_lib):
    """One isotropic Gaussian on the pixel's axis: q = 0, alpha = o, and
    L = o c + (1 - o) bg, so dG/dlogit = g . (c - bg) o (1 - o) and
    dG/dk0 = g o."""
    cloud = scenes.GaussianCloud(np.array([[0, 0, 0]], np.float32),
                                 np.full((1, 3), -1.5, np.float32),
                                 np.array([[1, 0, 0, 0]], np.float32), np.array([0.3], np.float32),
                                 np.array([[[0.7, 0.2, 0.5]]], np.float32), 0)
    cam = scenes.Pinhole(width=1, height=1)
    bg = np.array([0.1, 0.3, 0.2])
    g = np.array([[0.5, -1.0, 2.0]])
    an = oracle_lib.grad_pinhole(cloud, cam, scenes.TraceSettings(bg=tuple(bg)), g, mode="blend")
    o = expit(np.float64(np.float32(0.3)))
    c = np.array([0.7, 0.2, 0.5], np.float32).astype(np.float64)
    assert an["opacity_logits"][0] == pytest.approx(float(g[0] @ (c - bg)) * o * (1 - o), rel=1e-12)
    assert np.allclose(an["sh"][0, 0], g[0] * o, rtol=1e-12)
    # on the axis through the centre the mean gradient is zero (q is at its minimum)
    assert np.allclose(an["means"][0], 0.0, atol=1e-12)


@pytest.mark.slow
def test_estimator_gradient_is_unbiased(oracle_lib):
    cloud = _cluster(seed=3, M=25, sh_degree=0)
    cam = scenes.Pinhole(width=4, height=4, fov_y_deg=6.0)
    rng = np.random.default_rng(2)
    g = rng.normal(size=(16, 3))
    st = scenes.TraceSettings(seed=5, spp=20000, bg=(0.3, 0.3, 0.3))
    est = oracle_lib.grad_pinhole(cloud, cam, st, g, mode="estimator")
    ref = oracle_lib.grad_pinhole(cloud, cam, st, g, mode="blend")
    a = np.concatenate([est[k].ravel() for k in PARAMS])
    b = np.concatenate([ref[k].ravel() for k in PARAMS])
    cos = a @ b / np.linalg.norm(a) / np.linalg.norm(b)
    assert cos > 0.995
    assert np.linalg.norm(a - b) < 0.1 * np.linalg.norm(b)
