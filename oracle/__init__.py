"""FP64 CPU oracle for stochastic ray tracing of transparent 3D Gaussians.

TEST INFRASTRUCTURE. Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package. The CUDA path
never calls it; the two share no code.

The C source (``gs_oracle.c``) brute-forces every ray against every Gaussian
in double precision and computes both the stochastic estimator (Eq. 4-7,
Alg. 1) with the same keyed Philox draws as the GPU path, and its
expectation, the exact depth-sorted blend (Eq. 3). This module only builds
that file with gcc and marshals numpy arrays through ctypes.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libgs_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP when available). Returns the path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    # -ffp-contract=off: no fused multiply-add, so the float32 camera-ray
    # definition rounds after every operation on every architecture.
    # a temporary of this process, renamed atomically: processes that build
    # at the same time do not write the same file
    tmp = "%s.%d.tmp" % (_LIB_PATH, os.getpid())
    base = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared",
            "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True, text=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True, text=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Scene(C.Structure):
    _fields_ = [("M", C.c_int64), ("means", C.c_void_p), ("log_scales", C.c_void_p),
                ("quats", C.c_void_p), ("opacity_logits", C.c_void_p), ("sh", C.c_void_p),
                ("sh_degree", C.c_int32), ("pad", C.c_int32)]


class _Pinhole(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("look_at", C.c_float * 3), ("up", C.c_float * 3),
                ("fov_y_deg", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("ray_id_offset", C.c_uint32), ("pad", C.c_int32)]


class _Params(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("spp", C.c_int32), ("n_hits", C.c_int32),
                ("t_min", C.c_double), ("t_max", C.c_double), ("bg", C.c_double * 3),
                ("stream_tag", C.c_uint32), ("depth_mode", C.c_int32), ("rng_mode", C.c_int32),
                ("pad", C.c_int32)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.c_void_p
            lib.orc_philox4x32_10.argtypes = [P, P, P]
            lib.orc_xi.restype = C.c_double
            lib.orc_xi.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32]
            lib.orc_activate.argtypes = [P, P, P, P]
            lib.orc_eval_pair.argtypes = [P, C.c_int64, P, P, C.c_double, C.c_double, P]
            lib.orc_sh_basis.argtypes = [C.c_int, P, P]
            lib.orc_camera_ray.argtypes = [P, C.c_int32, C.c_int32, P, P, P]
            lib.orc_closest_accepted.restype = C.c_int64
            lib.orc_closest_accepted.argtypes = [C.c_int64, P, P, P, P]
            lib.orc_blend.argtypes = [C.c_int64, P, P, P, P, P, P, P]
            lib.orc_enumerate_expectation.restype = C.c_int
            lib.orc_enumerate_expectation.argtypes = [C.c_int, P, P, P, P]
            lib.orc_ray_candidates.restype = C.c_int64
            lib.orc_ray_candidates.argtypes = [P, P, P, C.c_double, C.c_double, C.c_int64,
                                               P, P, P, P, P]
            lib.orc_max_threads.restype = C.c_int
            lib.orc_render_pinhole.restype = C.c_int
            lib.orc_render_pinhole.argtypes = [P, P, P, C.c_int64, P, P, P, P, P, P, P, C.c_int]
            lib.orc_grad_pinhole.restype = C.c_int
            lib.orc_grad_pinhole.argtypes = [P, P, P, C.c_int64, P, P, C.c_int, P, P, P, P, P,
                                             C.c_int]
            lib.orc_bounce_dir.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, P]
            lib.orc_hash_xi.restype = C.c_double
            lib.orc_hash_xi.argtypes = [P, C.c_uint32]
            lib.orc_hash_constants.restype = None
            lib.orc_hash_constants.argtypes = [P]
            lib.orc_render_scene.restype = C.c_int
            lib.orc_render_scene.argtypes = [P, P, C.c_int32, P, P, C.c_int64, P, P, P, P, C.c_int]
            lib.orc_scene_sample_rays.restype = C.c_int
            lib.orc_scene_sample_rays.argtypes = [P, P, P, C.c_int32, C.c_int32, C.c_uint32, P]
            lib.orc_render_rays.restype = C.c_int
            lib.orc_render_rays.argtypes = [P, P, C.c_int64, P, P, P, P, P, P, P, P, P, C.c_int]
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


class _SceneHandle:
    """Keeps the float32 arrays alive for the lifetime of the C struct."""

    def __init__(self, cloud):
        self.arrays = [_c(cloud.means, np.float32), _c(cloud.log_scales, np.float32),
                       _c(cloud.quats, np.float32), _c(cloud.opacity_logits, np.float32),
                       _c(cloud.sh, np.float32)]
        m, ls, q, lo, sh = self.arrays
        self.struct = _Scene(int(m.shape[0]), m.ctypes.data, ls.ctypes.data, q.ctypes.data,
                             lo.ctypes.data, sh.ctypes.data, int(cloud.sh_degree), 0)

    @property
    def ref(self):
        return C.byref(self.struct)


def _pinhole(cam):
    s = _Pinhole()
    s.eye[:] = [float(v) for v in cam.eye]
    s.look_at[:] = [float(v) for v in cam.look_at]
    s.up[:] = [float(v) for v in cam.up]
    s.fov_y_deg = float(cam.fov_y_deg)
    s.width, s.height = int(cam.width), int(cam.height)
    s.ray_id_offset = int(cam.ray_id_offset)
    return s


def _params(st):
    p = _Params()
    p.seed = int(st.seed)
    p.spp = int(st.spp)
    p.n_hits = int(st.n_hits)
    p.t_min = float(st.t_min)
    p.t_max = float(st.t_max)
    p.bg[:] = [float(v) for v in st.bg]
    p.stream_tag = int(st.stream_tag)
    p.depth_mode = int(getattr(st, "depth_mode", 0))
    p.rng_mode = int(getattr(st, "rng_mode", 0))
    return p


# ---------------------------------------------------------------- primitives

def philox4x32_10(ctr, key):
    """Philox-4x32-10 of one 4-word counter under a 2-word key."""
    lib = _load()
    c = _c(ctr, np.uint32)
    k = _c(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib.orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def xi(seed, ray_id, gid, sample, stream_tag=0) -> float:
    return float(_load().orc_xi(int(seed), int(ray_id), int(gid), int(sample), int(stream_tag)))


def activate(cloud):
    """(opacity [M], R_q [M,3,3] local-to-world, Sigma^-1 [M,3,3]) in FP64."""
    lib = _load()
    h = _SceneHandle(cloud)
    M = cloud.M
    op = np.zeros(M)
    R = np.zeros((M, 3, 3))
    Si = np.zeros((M, 3, 3))
    lib.orc_activate(h.ref, _ptr(op), _ptr(R), _ptr(Si))
    return op, R, Si


def eval_pair(cloud, g, o, d, t_min=0.0, t_max=np.inf):
    """(t*, q, alpha, valid) for Gaussian g and the ray o + t d."""
    lib = _load()
    h = _SceneHandle(cloud)
    o = _c(o, np.float64)
    d = _c(d, np.float64)
    out = np.zeros(4)
    lib.orc_eval_pair(h.ref, int(g), _ptr(o), _ptr(d), float(t_min), float(t_max), _ptr(out))
    return float(out[0]), float(out[1]), float(out[2]), bool(out[3])


def sh_basis(deg, d):
    lib = _load()
    d = _c(d, np.float64)
    Y = np.zeros((deg + 1) ** 2)
    lib.orc_sh_basis(int(deg), _ptr(d), _ptr(Y))
    return Y


def camera_ray(cam, x, y):
    """(origin, unit direction, ray_id) of pixel (x, y); float32-valued."""
    lib = _load()
    s = _pinhole(cam)
    o = np.zeros(3)
    d = np.zeros(3)
    rid = C.c_uint32(0)
    lib.orc_camera_ray(C.byref(s), int(x), int(y), _ptr(o), _ptr(d), C.byref(rid))
    return o, d, int(rid.value)


def closest_accepted(t, gid, accepted, order=None) -> int:
    lib = _load()
    t = _c(t, np.float64)
    g = _c(gid, np.int32)
    a = _c(accepted, np.uint8)
    o = None if order is None else _c(order, np.int64)
    return int(lib.orc_closest_accepted(len(t), _ptr(t), _ptr(g), _ptr(a), _ptr(o)))


def blend(t, gid, alpha, rgb, bg=(0.0, 0.0, 0.0), second_moment=False):
    """Eq. 3 (with background); optionally also E[L^2] of one sample."""
    lib = _load()
    t = _c(t, np.float64)
    g = _c(gid, np.int32)
    a = _c(alpha, np.float64)
    c = _c(rgb, np.float64).reshape(-1, 3)
    b = _c(bg, np.float64)
    out = np.zeros(3)
    out2 = np.zeros(3)
    lib.orc_blend(len(t), _ptr(t), _ptr(g), _ptr(a), _ptr(c), _ptr(b), _ptr(out), _ptr(out2))
    return (out, out2) if second_moment else out


def enumerate_expectation(alpha, rgb, bg=(0.0, 0.0, 0.0)):
    lib = _load()
    a = _c(alpha, np.float64)
    c = _c(rgb, np.float64).reshape(-1, 3)
    b = _c(bg, np.float64)
    out = np.zeros(3)
    if lib.orc_enumerate_expectation(len(a), _ptr(a), _ptr(c), _ptr(b), _ptr(out)) != 0:
        raise ValueError("at most 24 candidates")
    return out


def ray_candidates(cloud, o, d, t_min=0.0, t_max=np.inf):
    """All valid candidates of one ray, in Gaussian-id order, as a dict."""
    lib = _load()
    h = _SceneHandle(cloud)
    o = _c(o, np.float64)
    d = _c(d, np.float64)
    n = int(lib.orc_ray_candidates(h.ref, _ptr(o), _ptr(d), float(t_min), float(t_max), 0,
                                   None, None, None, None, None))
    t = np.zeros(n)
    q = np.zeros(n)
    a = np.zeros(n)
    g = np.zeros(n, np.int32)
    c = np.zeros((n, 3))
    lib.orc_ray_candidates(h.ref, _ptr(o), _ptr(d), float(t_min), float(t_max), n,
                           _ptr(t), _ptr(q), _ptr(a), _ptr(g), _ptr(c))
    return {"t": t, "q": q, "alpha": a, "gid": g, "rgb": c}


def max_threads() -> int:
    return int(_load().orc_max_threads())


# ---------------------------------------------------------------- rendering

def render_pinhole(cloud, cam, settings, pixels=None, want_hits=True, n_threads=0):
    """Brute-force render of the listed linear pixel indices (all by default).

    Returns a dict with ``blend`` [n,3], ``blend2`` [n,3] (second moment of
    one sample, so the per-sample variance is blend2 - blend^2), ``est`` [n,3],
    ``hit_id`` [n,S],
    ``hit_t`` [n,S] (S = spp * n_hits, sample s = pass * n_hits + k),
    ``n_valid`` [n] and ``threads``."""
    lib = _load()
    h = _SceneHandle(cloud)
    if pixels is None:
        pixels = np.arange(cam.width * cam.height, dtype=np.int64)
    pix = _c(pixels, np.int64)
    n = len(pix)
    S = int(settings.spp) * int(settings.n_hits)
    blend_o = np.zeros((n, 3))
    blend2 = np.zeros((n, 3))
    est = np.zeros((n, 3))
    hid = np.zeros((n, S), np.int32) if want_hits else None
    ht = np.zeros((n, S)) if want_hits else None
    nv = np.zeros(n, np.int64)
    cs = _pinhole(cam)
    ps = _params(settings)
    used = lib.orc_render_pinhole(h.ref, C.byref(cs), C.byref(ps), n, _ptr(pix), _ptr(blend_o),
                                  _ptr(blend2), _ptr(est), _ptr(hid), _ptr(ht), _ptr(nv),
                                  int(n_threads))
    return {"blend": blend_o, "blend2": blend2, "est": est, "hit_id": hid, "hit_t": ht,
            "n_valid": nv, "threads": int(used)}


def render_rays(cloud, origins, dirs, ray_ids, settings, want_hits=True, n_threads=0):
    """Brute-force render of explicit float32 rays (same outputs as above)."""
    lib = _load()
    h = _SceneHandle(cloud)
    o = _c(origins, np.float32).reshape(-1, 3)
    d = _c(dirs, np.float32).reshape(-1, 3)
    rid = _c(ray_ids, np.uint32)
    n = len(rid)
    S = int(settings.spp) * int(settings.n_hits)
    blend_o = np.zeros((n, 3))
    blend2 = np.zeros((n, 3))
    est = np.zeros((n, 3))
    hid = np.zeros((n, S), np.int32) if want_hits else None
    ht = np.zeros((n, S)) if want_hits else None
    nv = np.zeros(n, np.int64)
    ps = _params(settings)
    used = lib.orc_render_rays(h.ref, C.byref(ps), n, _ptr(o), _ptr(d), _ptr(rid),
                               _ptr(blend_o), _ptr(blend2), _ptr(est), _ptr(hid), _ptr(ht),
                               _ptr(nv), int(n_threads))
    return {"blend": blend_o, "blend2": blend2, "est": est, "hit_id": hid, "hit_t": ht,
            "n_valid": nv, "threads": int(used)}


# ---------------------------------------------------------------- gradients

def grad_pinhole(cloud, cam, settings, d_rgb, pixels=None, mode="blend", n_threads=0):
    """Gradient of sum_p d_rgb[p] . L_p w.r.t. every parameter (FP64).

    mode "blend": exact sorted blend (Eq. 3); mode "estimator": the
    stochastic estimate averaged over the spp * n_hits samples of each pixel
    with the same draws as rendering. Returns a dict of arrays shaped like
    the parameters (means, log_scales, quats, opacity_logits, sh)."""
    lib = _load()
    h = _SceneHandle(cloud)
    if pixels is None:
        pixels = np.arange(cam.width * cam.height, dtype=np.int64)
    pix = _c(pixels, np.int64)
    g = _c(d_rgb, np.float64).reshape(-1, 3)
    assert len(g) == len(pix)
    M = cloud.M
    out = {"means": np.zeros((M, 3)), "log_scales": np.zeros((M, 3)), "quats": np.zeros((M, 4)),
           "opacity_logits": np.zeros(M), "sh": np.zeros(cloud.sh.shape)}
    cs = _pinhole(cam)
    ps = _params(settings)
    lib.orc_grad_pinhole(h.ref, C.byref(cs), C.byref(ps), len(pix), _ptr(pix), _ptr(g),
                         0 if mode == "blend" else 1, _ptr(out["means"]), _ptr(out["log_scales"]),
                         _ptr(out["quats"]), _ptr(out["opacity_logits"]), _ptr(out["sh"]),
                         int(n_threads))
    return out


# ---------------------------------------------------------------- scenes

class _Light(C.Structure):
    _fields_ = [("position", C.c_float * 3), ("intensity", C.c_float * 3)]


class _Extras(C.Structure):
    _fields_ = [("n_lights", C.c_int32), ("lights", _Light * 8), ("has_ground", C.c_int32),
                ("ground_y", C.c_float), ("ground_half_extent", C.c_float),
                ("ground_albedo", C.c_float * 3), ("bounce", C.c_int32),
                ("shadow_eps", C.c_float)]


def _extras(ex):
    e = _Extras()
    e.n_lights = len(ex.lights)
    for i, (pos, inten) in enumerate(ex.lights):
        e.lights[i].position[:] = [float(v) for v in pos]
        e.lights[i].intensity[:] = [float(v) for v in inten]
    e.has_ground = int(ex.has_ground)
    e.ground_y = float(ex.ground_y)
    e.ground_half_extent = float(ex.ground_half_extent)
    e.ground_albedo[:] = [float(v) for v in ex.ground_albedo]
    e.bounce = int(ex.bounce)
    e.shadow_eps = float(ex.shadow_eps)
    return e


def render_scene(cloud, cams, extras, settings, items, want_diag=True, n_threads=0):
    """Ground, lights and bounce (see gs_oracle.c). items: list of
    (view index, linear pixel). Returns est [n,3] and diag [n,spp,3]."""
    lib = _load()
    h = _SceneHandle(cloud)
    arr = (_Pinhole * len(cams))(*[_pinhole(c) for c in cams])
    items = np.asarray(items, np.int64).reshape(-1, 2)
    v = _c(items[:, 0], np.int32)
    px = _c(items[:, 1], np.int64)
    n = len(items)
    est = np.zeros((n, 3))
    diag = np.zeros((n, int(settings.spp), 3), np.int32) if want_diag else None
    ex = _extras(extras)
    ps = _params(settings)
    lib.orc_render_scene(h.ref, arr, len(cams), C.byref(ex), C.byref(ps), n, _ptr(v), _ptr(px),
                         _ptr(est), _ptr(diag), int(n_threads))
    return {"est": est, "diag": diag}


def scene_sample_rays(cam, extras, settings, x, y, sample):
    """The float32 rays of one sample of the scene renderer: camera ray,
    ground hit, shadow rays to each light and the bounce direction."""
    out = np.zeros(46, np.float32)
    ps = _params(settings)
    cs = _pinhole(cam)
    ex = _extras(extras)
    ground = _load().orc_scene_sample_rays(C.byref(cs), C.byref(ex), C.byref(ps), int(x), int(y),
                                           int(sample), _ptr(out))
    lights = []
    for l in range(len(extras.lights)):
        v = out[14 + 4 * l: 18 + 4 * l]
        lights.append(None if v[3] < 0 else (v[:3].copy(), float(v[3])))
    return {"o": out[0:3].copy(), "d": out[3:6].copy(), "ray_id": int(out[6:7].view(np.uint32)[0]),
            "ground": bool(ground), "tq": float(out[7]), "p": out[8:11].copy(),
            "bounce_d": out[11:14].copy(), "lights": lights}


def bounce_dir(seed, ray_id, sample):
    lib = _load()
    d = np.zeros(3, np.float32)
    lib.orc_bounce_dir(int(seed), int(ray_id), int(sample), _ptr(d))
    return d


def hash_xi(p, sample):
    """The trigonometric hash draw (Eq. 8-9) of hit position p for a sample."""
    q = _c(p, np.float64)
    return float(_load().orc_hash_xi(_ptr(q), int(sample)))


def hash_constants():
    """The coefficients of Eq. 8-9 the oracle's hash uses:
    {"a1", "b1", "a2": [2], "b2": [2]}."""
    out = np.zeros(6, np.float64)
    _load().orc_hash_constants(_ptr(out))
    return {"a1": float(out[0]), "b1": float(out[1]), "a2": [float(out[2]), float(out[3])],
            "b2": [float(out[4]), float(out[5])]}
