"""Pins of the oracle's batched scene renderer (ground, point lights, one
diffuse bounce): reduction to the pinned pinhole estimator, the bounce
directions' cosine-lobe moments, shadow visibility averaging to the exact
transmittance of the segment (Eq. 5 for transmittance), and the closed-form
ground radiance of an empty scene."""
import numpy as np
import pytest

import scenes


def test_reduces_to_pinhole_estimator(oracle_lib):
    cloud = scenes.tiny_cloud(0, M=400)
    cam = scenes.default_camera(12, 10, ray_id_offset=77)
    st = scenes.TraceSettings(seed=4, spp=6)
    items = [(0, p) for p in range(120)]
    r = oracle_lib.render_scene(cloud, [cam], scenes.SceneExtras(), st, items)
    ref = oracle_lib.render_pinhole(cloud, cam, st)
    assert np.allclose(r["est"], ref["est"], atol=1e-14)
    assert np.array_equal(r["diag"][:, :, 0], ref["hit_id"])


def test_bounce_directions_are_cosine_weighted(oracle_lib):
    d = np.array([oracle_lib.bounce_dir(3, rid, s) for rid in range(400) for s in range(10)],
                 np.float64)
    n = len(d)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-6)
    assert np.all(d[:, 1] >= 0)
    # cosine lobe about +y: E[cos] = 2/3, E[cos^2] = 1/2, E[x] = E[z] = 0
    se = 1 / np.sqrt(n)
    assert abs(d[:, 1].mean() - 2 / 3) < 5 * 0.24 * se
    assert abs((d[:, 1] ** 2).mean() - 0.5) < 5 * 0.3 * se
    assert abs(d[:, 0].mean()) < 5 * 0.6 * se and abs(d[:, 2].mean()) < 5 * 0.6 * se


def test_shadow_visibility_is_the_transmittance(oracle_lib):
    """One light straight above a ground point covered by a few Gaussians:
    the fraction of samples that see the light equals prod (1 - alpha_i)
    over the valid Gaussians on the segment."""
    rng = np.random.default_rng(0)
    M = 6
    means = np.stack([rng.uniform(-0.05, 0.05, M), np.linspace(-0.8, 0.4, M),
                      rng.uniform(-0.05, 0.05, M)], 1).astype(np.float32)
    cloud = scenes.GaussianCloud(means, np.full((M, 3), -2.0, np.float32),
                                 np.tile(np.array([1, 0, 0, 0], np.float32), (M, 1)),
                                 rng.normal(0, 1, M).astype(np.float32),
                                 np.full((M, 1, 3), 0.5, np.float32), 0)
    light = ((0.0, 2.0, 0.0), (1.0, 1.0, 1.0))
    ex = scenes.SceneExtras(lights=[light], has_ground=True, ground_y=-1.0, ground_half_extent=5,
                            bounce=False)
    # a camera looking straight down at the ground point below the column
    cam = scenes.Pinhole(width=1, height=1, eye=(0.0, -0.999, 0.0), look_at=(0.0, -5.0, 0.0),
                         up=(1.0, 0.0, 0.0), fov_y_deg=10.0)
    S = 20000
    r = oracle_lib.render_scene(cloud, [cam], ex, scenes.TraceSettings(seed=1, spp=S), [(0, 0)])
    vis = (r["diag"][0, :, 2] & 1).astype(float)
    assert np.all(r["diag"][0, :, 0] == -2)
    o = np.array([0.0, -1.0, 0.0])
    c = oracle_lib.ray_candidates(cloud, o, np.array([0.0, 1.0, 0.0]), t_min=1e-4, t_max=3.0)
    T = np.prod(1 - c["alpha"])
    assert len(c["alpha"]) >= 3
    assert abs(vis.mean() - T) < 4 * np.sqrt(T * (1 - T) / S)


def test_empty_scene_ground_radiance(oracle_lib):
    """No Gaussians, white background: a ground point gets
    albedo/pi * I cos / r^2 from each light plus albedo * bg from the
    bounce (every bounce ray escapes)."""
    cloud = scenes.tiny_cloud(0, M=0)
    light = ((1.0, 2.0, 0.5), (3.0, 2.0, 1.0))
    ex = scenes.SceneExtras(lights=[light], has_ground=True, ground_y=-1.0, ground_half_extent=5,
                            ground_albedo=(0.5, 0.25, 1.0), bounce=True)
    cam = scenes.Pinhole(width=1, height=1, eye=(0.0, 1.0, 0.0), look_at=(0.0, -1.0, 0.0),
                         up=(1.0, 0.0, 0.0), fov_y_deg=10.0)
    r = oracle_lib.render_scene(cloud, [cam], ex, scenes.TraceSettings(spp=3, bg=(1.0, 1.0, 1.0)),
                                [(0, 0)])
    p = np.array([0.0, -1.0, 0.0])
    w = np.array(light[0]) - p
    cosv = w[1] / np.linalg.norm(w)
    want = np.array(ex.ground_albedo) / np.pi * np.array(light[1]) * cosv / (w @ w) \
        + np.array(ex.ground_albedo) * 1.0
    assert np.allclose(r["est"][0], want, rtol=1e-6)


def _winner(oracle_lib, cloud, o, d, rid, s, seed, tag, t_min, t_max, any_hit=False):
    c = oracle_lib.ray_candidates(cloud, o, d, t_min=t_min, t_max=t_max)
    acc = [(t, int(g)) for t, g, a in zip(c["t"], c["gid"], c["alpha"])
           if oracle_lib.xi(seed, rid, int(g), s, tag) < a]
    if not acc:
        return -1, np.inf
    t, g = min(acc)
    return g, t


def test_sample_rays_reproduce_the_renderers_outcomes(oracle_lib):
    """The exported per-sample rays (used to classify GPU mismatches) are
    the renderer's own: re-deciding each sample from them with the pinned
    candidate list and draws gives the renderer's camera hit, bounce hit
    and visible-light bits; a planted wrong outcome is classified 'other'."""
    from tests import _parity
    cloud = scenes.shell_cloud(7, M=3000)
    cams = scenes.wavefront_views(2, seed=2, res_range=((9, 7), (14, 10)))
    ex = scenes.ground_and_lights(4, seed=1)
    st = scenes.TraceSettings(seed=5, spp=3)
    items = [(v, p) for v, c in enumerate(cams) for p in range(c.width * c.height)]
    diag = oracle_lib.render_scene(cloud, cams, ex, st, items)["diag"]
    n_ground = 0
    for i, (v, p) in enumerate(items):
        for s in range(st.spp):
            cam = cams[v]
            r = oracle_lib.scene_sample_rays(cam, ex, st, p % cam.width, p // cam.width, s)
            g, t = _winner(oracle_lib, cloud, r["o"], r["d"], r["ray_id"], s, st.seed, 0,
                           st.t_min, np.inf)
            ground = r["ground"] and not (g >= 0 and t < r["tq"])
            cam_out = -2 if ground else g
            bounce, bits = -1, 0
            if ground:
                n_ground += 1
                bounce, _ = _winner(oracle_lib, cloud, r["p"], r["bounce_d"], r["ray_id"], s,
                                    st.seed, 9, ex.shadow_eps, np.inf)
                for l, lr in enumerate(r["lights"]):
                    if lr is not None:
                        blk, _ = _winner(oracle_lib, cloud, r["p"], lr[0], r["ray_id"], s, st.seed,
                                         1 + l, ex.shadow_eps, lr[1])
                        bits |= (blk < 0) << l
            assert (cam_out, bounce, bits) == tuple(diag[i, s]), (v, p, s)
    assert n_ground > 20
    # a planted mistake: a sample's camera hit replaced by an unrelated id
    i = next(i for i in range(len(items)) if diag[i, 0, 0] >= 0)
    wrong = diag[i, 0].copy()
    wrong[0] = (wrong[0] + 1234) % cloud.M
    v, p = items[i]
    k = _parity.classify_scene_sample(cloud, cams[v], ex, st, p, 0, wrong, diag[i, 0])
    assert k == "other"
