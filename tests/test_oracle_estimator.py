"""Pins of the oracle's estimator (Eq. 4-7, Alg. 1) and exact blend (Eq. 3):
the worked example of Fig. 2, hand-computed two-Gaussian expectations,
exhaustive enumeration of acceptance outcomes, per-sample properties of the
rendered winners, and the statistical convergence of the estimator."""
import itertools
import json
import os

import numpy as np
import pytest
from scipy.special import expit

import scenes

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_fig2_order_independence(oracle_lib):
    gold = json.load(open(os.path.join(GOLD, "fig2_binary_opacity.json")))
    acc = np.array(gold["binary_opacity"], np.uint8)
    t = np.array([1.0, 1.5, 2.0, 2.6, 3.1, 4.0])
    gid = np.array([40, 7, 22, 3, 15, 9], np.int32)
    want = gold["winner_one_based"] - 1
    for perm in itertools.permutations(range(6)):
        assert oracle_lib.closest_accepted(t, gid, acc, np.array(perm)) == want


def test_equal_depth_tie_goes_to_smaller_id(oracle_lib):
    t = np.array([2.0, 2.0, 2.0])
    gid = np.array([9, 4, 6], np.int32)
    acc = np.array([1, 1, 0], np.uint8)
    for perm in itertools.permutations(range(3)):
        assert oracle_lib.closest_accepted(t, gid, acc, np.array(perm)) == 1


def test_two_gaussians_hand_computed(oracle_lib):
    """E[L] = a1 c1 + (1-a1) a2 c2 + (1-a1)(1-a2) bg.
    a1 = 0.3, a2 = 0.6, c1 = red, c2 = green, bg = blue:
    E = (0.3, 0.7*0.6, 0.7*0.4) = (0.3, 0.42, 0.28)."""
    want = np.array([0.3, 0.42, 0.28])
    rgb = np.array([[1, 0, 0], [0, 1, 0]], float)
    got = oracle_lib.blend([1.0, 2.0], [0, 1], [0.3, 0.6], rgb, bg=(0, 0, 1))
    assert np.allclose(got, want, atol=1e-15)
    # order of the input arrays does not matter, depth does
    got = oracle_lib.blend([2.0, 1.0], [1, 0], [0.6, 0.3], rgb[::-1], bg=(0, 0, 1))
    assert np.allclose(got, want, atol=1e-15)
    assert np.allclose(oracle_lib.enumerate_expectation([0.3, 0.6], rgb, (0, 0, 1)), want, atol=1e-15)


def test_two_gaussians_rendered(oracle_lib):
    """Two isotropic Gaussians on the optical axis of pixel (0,0) of a 1x1
    camera: the ray passes through both centres, so alpha_i = sigmoid(logit_i)
    exactly and the blend is the hand formula above."""
    cam = scenes.Pinhole(width=1, height=1)
    means = np.array([[0, 0, 1.0], [0, 0, -1.0]], np.float32)
    logits = np.array([np.log(0.3 / 0.7), np.log(0.6 / 0.4)], np.float32)
    cl = scenes.GaussianCloud(means, np.full((2, 3), -2.0, np.float32),
                              np.tile(np.array([1, 0, 0, 0], np.float32), (2, 1)), logits,
                              np.array([[[1, 0, 0]], [[0, 1, 0]]], np.float32), 0)
    a1, a2 = expit(logits.astype(np.float64))
    want = np.array([a1, (1 - a1) * a2, (1 - a1) * (1 - a2) * 0.5])
    r = oracle_lib.render_pinhole(cl, cam, scenes.TraceSettings(spp=2000, bg=(0, 0, 0.5)))
    assert np.allclose(r["blend"][0], want, atol=1e-12)
    assert r["n_valid"][0] == 2
    # every sample's winner is the front Gaussian, the back one, or none
    ids = r["hit_id"][0]
    assert set(np.unique(ids)) <= {-1, 0, 1}
    f0 = np.mean(ids == 0)
    assert abs(f0 - a1) < 4 * np.sqrt(a1 * (1 - a1) / 2000)


def test_enumeration_equals_blend(oracle_lib):
    """Eq. 5 => Eq. 3: summing P(acceptance vector) * colour of the closest
    accepted candidate over all 2^n vectors gives the sorted blend."""
    rng = np.random.default_rng(0)
    for n in [1, 3, 7, 12]:
        alpha = rng.uniform(0, 1, n)
        rgb = rng.uniform(0, 1, (n, 3))
        bg = rng.uniform(0, 1, 3)
        t = np.sort(rng.uniform(1, 5, n))
        want = oracle_lib.enumerate_expectation(alpha, rgb, bg)
        perm = rng.permutation(n)
        got = oracle_lib.blend(t[perm], np.arange(n, dtype=np.int32)[perm], alpha[perm], rgb[perm], bg)
        assert np.allclose(got, want, atol=1e-12)


def test_second_moment_by_enumeration(oracle_lib):
    """E[L^2] of one sample: the 2^n enumeration with squared colours equals
    the composite of squared colours returned beside the blend."""
    rng = np.random.default_rng(5)
    for n in [1, 4, 9]:
        alpha = rng.uniform(0, 1, n)
        rgb = rng.uniform(0, 1, (n, 3))
        bg = rng.uniform(0, 1, 3)
        t = rng.uniform(1, 5, n)
        want = oracle_lib.enumerate_expectation(alpha[np.argsort(t)], rgb[np.argsort(t)] ** 2, bg ** 2)
        _, got = oracle_lib.blend(t, np.arange(n, dtype=np.int32), alpha, rgb, bg, second_moment=True)
        assert np.allclose(got, want, atol=1e-12)


def _tiny_setup(spp):
    cl = scenes.tiny_cloud(0)
    cam = scenes.default_camera(16, 16)
    return cl, cam, scenes.TraceSettings(seed=7, spp=spp)


def test_winners_are_closest_accepted(oracle_lib):
    """Per sample: the winner was accepted (xi < alpha) and no candidate
    closer in (t, gid) order was accepted; an empty sample accepted none."""
    cl, cam, st = _tiny_setup(spp=8)
    pix = np.arange(0, 256, 5)
    r = oracle_lib.render_pinhole(cl, cam, st, pixels=pix)
    checked = 0
    for i, p in enumerate(pix):
        o, d, rid = oracle_lib.camera_ray(cam, p % 16, p // 16)
        c = oracle_lib.ray_candidates(cl, o, d)
        for s in range(8):
            xi = np.array([oracle_lib.xi(st.seed, rid, g, s) for g in c["gid"]])
            acc = xi < c["alpha"]
            w = r["hit_id"][i, s]
            if w < 0:
                assert not acc.any()
                continue
            k = int(np.nonzero(c["gid"] == w)[0][0])
            assert acc[k]
            closer = (c["t"] < c["t"][k]) | ((c["t"] == c["t"][k]) & (c["gid"] < w))
            assert not (acc & closer).any()
            assert r["hit_t"][i, s] == c["t"][k]
            checked += 1
    assert checked > 20


def test_samples_by_passes_and_hits_are_the_same_draws(oracle_lib):
    cl, cam, _ = _tiny_setup(1)
    pix = np.arange(0, 256, 3)
    a = oracle_lib.render_pinhole(cl, cam, scenes.TraceSettings(seed=3, spp=8, n_hits=1), pixels=pix)
    b = oracle_lib.render_pinhole(cl, cam, scenes.TraceSettings(seed=3, spp=2, n_hits=4), pixels=pix)
    assert np.array_equal(a["hit_id"], b["hit_id"])
    assert np.allclose(a["est"], b["est"], atol=1e-15)


def test_blend_matches_candidates(oracle_lib):
    cl, cam, st = _tiny_setup(1)
    pix = np.arange(0, 256, 7)
    r = oracle_lib.render_pinhole(cl, cam, st, pixels=pix)
    for i, p in enumerate(pix):
        o, d, _ = oracle_lib.camera_ray(cam, p % 16, p // 16)
        c = oracle_lib.ray_candidates(cl, o, d)
        assert len(c["t"]) == r["n_valid"][i]
        want = oracle_lib.blend(c["t"], c["gid"], c["alpha"], c["rgb"])
        assert np.allclose(r["blend"][i], want, atol=1e-14)


@pytest.mark.slow
def test_estimator_converges_to_blend(oracle_lib):
    """Unbiasedness (Eq. 5): the 4096-sample mean is within a few standard
    errors of the exact blend; z-scores pool to mean ~0, variance ~1. The
    sample variance also matches the exact one (blend2 - blend^2)."""
    cl = scenes.tiny_cloud(0)
    cam = scenes.default_camera(32, 32)
    st = scenes.TraceSettings(seed=1, spp=4096)
    pix = np.arange(0, 1024, 2)
    r = oracle_lib.render_pinhole(cl, cam, st, pixels=pix)
    zs = []
    for i, p in enumerate(pix):
        if r["n_valid"][i] == 0:
            assert np.all(r["est"][i] == 0) and np.all(r["blend"][i] == 0)
            continue
        o, d, _ = oracle_lib.camera_ray(cam, p % 32, p // 32)
        c = oracle_lib.ray_candidates(cl, o, d)
        lut = {int(g): c["rgb"][k] for k, g in enumerate(c["gid"])}
        cols = np.array([lut[int(g)] if g >= 0 else np.zeros(3) for g in r["hit_id"][i]])
        se = cols.std(axis=0, ddof=1) / np.sqrt(len(cols))
        var_exact = r["blend2"][i] - r["blend"][i] ** 2
        assert np.all(np.abs(cols.var(axis=0, ddof=1) - var_exact) <= 0.15 * var_exact + 2e-3)
        for ch in range(3):
            if se[ch] == 0:
                assert r["est"][i, ch] == pytest.approx(r["blend"][i, ch], abs=1e-12)
            else:
                zs.append((r["est"][i, ch] - r["blend"][i, ch]) / se[ch])
    zs = np.array(zs)
    assert len(zs) > 300
    assert abs(zs.mean()) < 4.0 / np.sqrt(len(zs))
    assert 0.8 < zs.var() < 1.2
    assert np.mean(np.abs(zs) > 3) < 0.0027 + 3 * np.sqrt(0.0027 / len(zs)) + 1e-9


def test_inverted_acceptance_would_be_biased(oracle_lib):
    """Guard on the reading of the acceptance test: accepting on xi >= alpha
    (the inverted Alg. 1 test) gives the blend of 1-alpha, which differs."""
    alpha = np.array([0.2, 0.7])
    rgb = np.array([[1, 0, 0], [0, 1, 0]], float)
    good = oracle_lib.enumerate_expectation(alpha, rgb)
    bad = oracle_lib.enumerate_expectation(1 - alpha, rgb)
    assert not np.allclose(good, bad)
    cl = scenes.tiny_cloud(0)
    cam = scenes.default_camera(8, 8)
    r = oracle_lib.render_pinhole(cl, cam, scenes.TraceSettings(seed=2, spp=512))
    hit = r["n_valid"] > 0
    err = np.abs(r["est"][hit] - r["blend"][hit]).mean()
    assert err < 0.02
