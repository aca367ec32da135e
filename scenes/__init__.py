"""Seeded synthetic inputs: Gaussian clouds and pinhole cameras.

This module only draws random parameters and lays out camera descriptions.
It holds none of the rendering arithmetic (no activation, no ray generation,
no intersection, no random draw of the method): both the FP64 CPU oracle and
the CUDA path consume exactly the arrays produced here.

The paper measures on reconstructed 3DGS scenes and object assets (Sec. 5),
none of which is available; the clouds below are seeded stand-ins with the
sizes and structure of those workloads:

* ``tiny``:    1,000 Gaussians, means uniform in [-1,1]^3, log-scales
  N(-3, 0.5), quaternions N(0,1)^4 (uniform on SO(3) after normalisation),
  opacity logits N(0, 1.5), SH degree 0 colour U[0,1].
* ``shell``:   M Gaussians (1M by default) in 64 clusters whose centres are
  uniform on the unit sphere; members offset by N(0, 0.05^2 I); log-scales
  N(-4.5, 0.6); opacity logits N(0, 2); SH degree 3 with DC U[0,1] and the
  other 15x3 coefficients N(0, 0.2).

Parameters are float32, row-major, in the layout the C ABI takes:
means [M,3], log_scales [M,3], quats [M,4] as (w,x,y,z) (not normalised),
opacity_logits [M], sh [M,K,3] with K = (deg+1)^2.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class GaussianCloud:
    means: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray
    opacity_logits: np.ndarray
    sh: np.ndarray
    sh_degree: int

    @property
    def M(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "GaussianCloud":
        idx = np.asarray(idx)
        return GaussianCloud(self.means[idx].copy(), self.log_scales[idx].copy(),
                             self.quats[idx].copy(), self.opacity_logits[idx].copy(),
                             self.sh[idx].copy(), self.sh_degree)


@dataclass
class Pinhole:
    """A pinhole camera description (pure data).

    ``eye`` looks at ``look_at`` with ``up`` as the approximate up vector,
    ``fov_y_deg`` is the vertical field of view, row 0 is the top row, and
    ray ``y*width + x + ray_id_offset`` goes through the centre of pixel
    (x, y)."""
    width: int
    height: int
    eye: tuple = (0.0, 0.0, 3.0)
    look_at: tuple = (0.0, 0.0, 0.0)
    up: tuple = (0.0, 1.0, 0.0)
    fov_y_deg: float = 60.0
    ray_id_offset: int = 0

    @property
    def n_rays(self) -> int:
        return self.width * self.height


@dataclass
class TraceSettings:
    seed: int = 0
    spp: int = 1
    n_hits: int = 1
    t_min: float = 0.0
    t_max: float = float("inf")
    bg: tuple = (0.0, 0.0, 0.0)
    stream_tag: int = 0
    depth_mode: int = 0  # 0: mean of the 1D Gaussian, 1: projected centre
    rng_mode: int = 0    # 0: Philox, 1: trigonometric hash of the hit position
    extra: dict = field(default_factory=dict)


@dataclass
class SceneExtras:
    """Ground quad, point lights and the diffuse bounce of the batched
    wavefront form (pure data)."""
    lights: list = field(default_factory=list)  # [(position, intensity), ...]
    has_ground: bool = False
    ground_y: float = -1.3
    ground_half_extent: float = 3.0
    ground_albedo: tuple = (0.5, 0.5, 0.5)
    bounce: bool = False
    shadow_eps: float = 1e-4


def ground_and_lights(n_lights: int = 4, seed: int = 0, intensity: float = 4.0) -> SceneExtras:
    """A ground quad below the unit shell and point lights above it."""
    rng = np.random.default_rng(seed)
    lights = []
    for _ in range(n_lights):
        a = rng.uniform(0, 2 * np.pi)
        pos = (float(2.5 * np.cos(a)), float(rng.uniform(2.0, 3.0)), float(2.5 * np.sin(a)))
        lights.append((pos, (intensity, intensity, intensity)))
    return SceneExtras(lights=lights, has_ground=True, ground_y=-1.3, ground_half_extent=3.0,
                       ground_albedo=(0.5, 0.5, 0.5), bounce=True, shadow_eps=1e-4)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def tiny_cloud(seed: int = 0, M: int = 1000) -> GaussianCloud:
    """Small uniform cloud: 1,000 Gaussians, SH degree 0."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-1.0, 1.0, size=(M, 3))
    log_scales = rng.normal(-3.0, 0.5, size=(M, 3))
    quats = rng.normal(0.0, 1.0, size=(M, 4))
    logits = rng.normal(0.0, 1.5, size=(M,))
    sh = rng.uniform(0.0, 1.0, size=(M, 1, 3))
    return GaussianCloud(_f32(means), _f32(log_scales), _f32(quats), _f32(logits), _f32(sh), 0)


def shell_cloud(seed: int = 0, M: int = 1_000_000, n_clusters: int = 64,
                sh_degree: int = 3) -> GaussianCloud:
    """Clustered shell cloud: 64 anisotropic clusters on the unit sphere."""
    rng = np.random.default_rng(seed)
    centres = rng.normal(0.0, 1.0, size=(n_clusters, 3))
    centres /= np.linalg.norm(centres, axis=1, keepdims=True)
    which = rng.integers(0, n_clusters, size=M)
    means = centres[which] + rng.normal(0.0, 0.05, size=(M, 3))
    log_scales = rng.normal(-4.5, 0.6, size=(M, 3))
    quats = rng.normal(0.0, 1.0, size=(M, 4))
    logits = rng.normal(0.0, 2.0, size=(M,))
    K = (sh_degree + 1) ** 2
    sh = np.empty((M, K, 3), dtype=np.float32)
    sh[:, 0, :] = rng.uniform(0.0, 1.0, size=(M, 3))
    if K > 1:
        sh[:, 1:, :] = rng.normal(0.0, 0.2, size=(M, K - 1, 3))
    return GaussianCloud(_f32(means), _f32(log_scales), _f32(quats), _f32(logits), sh, sh_degree)


def default_camera(width: int, height: int, ray_id_offset: int = 0) -> Pinhole:
    """Eye at distance 3 on +z looking at the origin, 60 degree vertical FOV."""
    return Pinhole(width=width, height=height, ray_id_offset=ray_id_offset)


def orbit_cameras(n_views: int, seed: int = 0, radius: float = 3.0,
                  res_range=((256, 256), (1920, 1080)),
                  fixed_res=None) -> list:
    """Cameras on a sphere of the given radius looking at the origin.

    Resolutions are drawn uniformly between the two corners of ``res_range``
    (width and height independently) unless ``fixed_res`` is given. Ray ids
    are offset so that every ray of the batch has a unique id."""
    rng = np.random.default_rng(seed)
    cams = []
    offset = 0
    for _ in range(n_views):
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        eye = tuple(float(x) for x in (radius * v))
        up = (0.0, 1.0, 0.0) if abs(v[1]) < 0.95 else (1.0, 0.0, 0.0)
        if fixed_res is None:
            (w0, h0), (w1, h1) = res_range
            w = int(rng.integers(w0, w1 + 1))
            h = int(rng.integers(h0, h1 + 1))
        else:
            w, h = fixed_res
        cams.append(Pinhole(width=w, height=h, eye=eye, up=up, ray_id_offset=offset))
        offset += w * h
    return cams


def wavefront_views(n_views: int = 16, seed: int = 0, radius: float = 3.0,
                    res_range=((256, 256), (1920, 1080)), fixed_res=None) -> list:
    """Views of the batched form: eyes on the upper part of a sphere of the
    given radius (elevation 15-60 degrees, above the ground), looking at the
    origin, resolutions uniform between the corners of ``res_range``."""
    rng = np.random.default_rng(seed)
    cams = []
    offset = 0
    for _ in range(n_views):
        az = rng.uniform(0, 2 * np.pi)
        el = np.radians(rng.uniform(15.0, 60.0))
        eye = (float(radius * np.cos(el) * np.cos(az)), float(radius * np.sin(el)),
               float(radius * np.cos(el) * np.sin(az)))
        if fixed_res is None:
            (w0, h0), (w1, h1) = res_range
            w = int(rng.integers(w0, w1 + 1))
            h = int(rng.integers(h0, h1 + 1))
        else:
            w, h = fixed_res
        cams.append(Pinhole(width=w, height=h, eye=eye, ray_id_offset=offset))
        offset += w * h
    return cams


def pixel_subset(width: int, height: int, n: int, seed: int = 1234) -> np.ndarray:
    """A fixed seeded subset of linear pixel indices y*width + x (sorted)."""
    rng = np.random.default_rng(seed)
    n = min(n, width * height)
    return np.sort(rng.choice(width * height, size=n, replace=False)).astype(np.int64)
