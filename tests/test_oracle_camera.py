"""Pins of the oracle's pinhole rays: pixel-centre directions against the
closed form of a 60-degree vertical field of view (to float32 rounding),
float32 exactness of the defined rays, row 0 at the top."""
import numpy as np
import pytest

import scenes


def test_default_camera_closed_form(oracle_lib):
    W, H = 64, 48
    cam = scenes.default_camera(W, H, ray_id_offset=100)
    th = np.tan(np.radians(30.0))
    for x, y in [(0, 0), (63, 47), (31, 20), (5, 40)]:
        o, d, rid = oracle_lib.camera_ray(cam, x, y)
        assert np.array_equal(o, [0, 0, 3])
        ux = (2 * x + 1 - W) / H * th
        uy = (H - 1 - 2 * y) / H * th
        want = np.array([ux, uy, -1.0])
        want /= np.linalg.norm(want)
        assert np.allclose(d, want, atol=3e-7)
        assert np.all(d.astype(np.float32).astype(np.float64) == d)
        assert abs(np.linalg.norm(d) - 1) < 3e-7
        assert rid == 100 + y * W + x
    # row 0 is the top of the image
    assert oracle_lib.camera_ray(cam, 10, 0)[1][1] > 0


def test_general_camera_axes(oracle_lib):
    cam = scenes.Pinhole(width=101, height=51, eye=(1.0, 2.0, -2.0), look_at=(0.2, -0.1, 0.3),
                         up=(0.0, 1.0, 0.0), fov_y_deg=45.0)
    eye = np.array(cam.eye)
    fwd = np.array(cam.look_at) - eye
    fwd /= np.linalg.norm(fwd)
    _, dc, _ = oracle_lib.camera_ray(cam, 50, 25)  # exact centre pixel
    assert np.allclose(dc, fwd, atol=3e-7)
    _, dt, _ = oracle_lib.camera_ray(cam, 50, 0)
    _, db, _ = oracle_lib.camera_ray(cam, 50, 50)
    # top and bottom centre rays span the field of view minus one pixel
    span = np.degrees(np.arccos(np.clip(dt @ db, -1, 1)))
    th = np.tan(np.radians(22.5))
    want = 2 * np.degrees(np.arctan(50 / 51 * th))
    assert span == pytest.approx(want, abs=1e-4)
    assert dt[1] > db[1]
