"""Stochastic ray tracing of transparent 3D Gaussians on GB300 (sm_103a).

Thin Python binding over the C ABI of ``include/gsrt.h`` (``libgsrt.so``):
argument marshalling only. PyTorch provides device memory and streams; every
step of the rendering path runs in the library's CUDA kernels. There is no
CPU fallback: if the library has not been built, importing the binding's
entry points raises.

Entry points mirror the C names: :func:`build_bvh` (``gs_build_bvh``),
:meth:`Bvh.rebuild` (``gs_bvh_rebuild``), :func:`trace_stochastic`
(``gs_trace_stochastic``).
"""

from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgsrt.so")

GS_OK = 0
STATUS_NAMES = {0: "GS_OK", 1: "GS_ERR_INVALID_ARG", 2: "GS_ERR_CUDA", 3: "GS_ERR_OOM",
                4: "GS_ERR_STACK_OVERFLOW", 5: "GS_ERR_STEP_LIMIT", 6: "GS_ERR_NONFINITE",
                7: "GS_ERR_NO_DEVICE"}
SH_F32, SH_F16, SH_BF16 = 0, 1, 2
_SH_DTYPES = {torch.float32: SH_F32, torch.float16: SH_F16, torch.bfloat16: SH_BF16}


class GsError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status


class _Gaussians(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logits", C.c_void_p), ("sh", C.c_void_p), ("M", C.c_int64),
                ("sh_degree", C.c_int32), ("sh_dtype", C.c_int32)]


class _Pinhole(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("look_at", C.c_float * 3), ("up", C.c_float * 3),
                ("fov_y_deg", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("ray_id_offset", C.c_uint32), ("reserved", C.c_int32)]


class _TraceParams(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("spp", C.c_int32), ("n_hits", C.c_int32),
                ("t_min", C.c_float), ("t_max", C.c_float), ("bg", C.c_float * 3),
                ("depth_mode", C.c_int32), ("stack_depth", C.c_int32),
                ("stream_tag", C.c_uint32), ("rng_mode", C.c_int32),
                ("samples_per_lane", C.c_int32), ("counters", C.c_void_p)]


class _BvhInfo(C.Structure):
    _fields_ = [("M", C.c_int64), ("n_nodes", C.c_int64), ("capacity", C.c_int64),
                ("device_bytes", C.c_int64), ("node_bytes", C.c_int32),
                ("prim_bytes", C.c_int32), ("node_format", C.c_int32),
                ("wide_node_bytes", C.c_int32)]


class _BuildOptions(C.Structure):
    _fields_ = [("node_format", C.c_int32), ("reserved", C.c_int32 * 7)]


NODES_BINARY, NODES_WIDE4, NODES_WIDE4_Q8, NODES_BINARY_Q8 = 0, 1, 2, 3
NODE_FORMATS = {"binary": NODES_BINARY, "wide4": NODES_WIDE4, "wide4_q8": NODES_WIDE4_Q8,
                "binary_q8": NODES_BINARY_Q8}


_lib = None
_lib_lock = threading.Lock()

# Every function the header declares, with its ctypes signature.
_SIGNATURES = {
    "gs_build_bvh": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "gs_build_bvh_ex": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "gs_bvh_export_wide": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "gs_bvh_rebuild": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "gs_bvh_free": (C.c_int, [C.c_void_p]),
    "gs_bvh_get_info": (C.c_int, [C.c_void_p, C.c_void_p]),
    "gs_bvh_sync_status": (C.c_int, [C.c_void_p, C.c_void_p]),
    "gs_bvh_export": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "gs_trace_stochastic": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "gs_trace_stochastic_keys": (C.c_int, [C.c_void_p] * 7),
    "gs_trace_backward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_void_p, C.c_void_p]),
    "gs_trace_backward_keys": (C.c_int, [C.c_void_p] * 12),
    "gs_build_bvh_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_void_p]),
    "gs_render_views": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p,
                                  C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p]),
    "gs_graph_capture_views": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p,
                                         C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                         C.c_void_p, C.c_void_p, C.c_void_p]),
    "gs_graph_launch": (C.c_int, [C.c_void_p, C.c_void_p]),
    "gs_graph_free": (C.c_int, [C.c_void_p]),
    "gs_trace_layout": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "gs_probe_copy": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p]),
    "gs_status_string": (C.c_char_p, [C.c_int]),
    "gs_last_error": (C.c_char_p, []),
}


def lib():
    """The loaded ``libgsrt.so``. Raises if it has not been built."""
    global _lib
    with _lib_lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libgsrt.so is not built (%s); run "
                                   "paper_2504_06598_gb300.build.build() first" % LIB_PATH)
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in _SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(status: int):
    if status != GS_OK:
        raise GsError(status, lib().gs_last_error().decode(errors="replace"))


def _stream_handle(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


# ---------------------------------------------------------------- data


class Gaussians:
    """Device-resident Gaussian parameters in the layout of ``gs_gaussians``."""

    def __init__(self, means, log_scales, quats, opacity_logits, sh, sh_degree: int):
        def dev(t, dtype=torch.float32):
            t = torch.as_tensor(t)
            if not t.is_cuda:
                t = t.to("cuda")
            return t.to(dtype).contiguous()

        self.means = dev(means)
        self.log_scales = dev(log_scales)
        self.quats = dev(quats)
        self.opacity_logits = dev(opacity_logits)
        sh = torch.as_tensor(sh)
        self.sh = dev(sh, sh.dtype if sh.dtype in _SH_DTYPES else torch.float32)
        self.sh_degree = int(sh_degree)
        self.M = int(self.means.shape[0])

    @classmethod
    def from_cloud(cls, cloud, sh_dtype=torch.float32):
        return cls(torch.from_numpy(cloud.means), torch.from_numpy(cloud.log_scales),
                   torch.from_numpy(cloud.quats), torch.from_numpy(cloud.opacity_logits),
                   torch.from_numpy(cloud.sh).to(sh_dtype), cloud.sh_degree)

    def struct(self) -> _Gaussians:
        return _Gaussians(self.means.data_ptr(), self.log_scales.data_ptr(),
                          self.quats.data_ptr(), self.opacity_logits.data_ptr(),
                          self.sh.data_ptr(), self.M, self.sh_degree, _SH_DTYPES[self.sh.dtype])


@dataclass
class Camera:
    width: int
    height: int
    eye: tuple = (0.0, 0.0, 3.0)
    look_at: tuple = (0.0, 0.0, 0.0)
    up: tuple = (0.0, 1.0, 0.0)
    fov_y_deg: float = 60.0
    ray_id_offset: int = 0

    def struct(self) -> _Pinhole:
        s = _Pinhole()
        s.eye[:] = [float(v) for v in self.eye]
        s.look_at[:] = [float(v) for v in self.look_at]
        s.up[:] = [float(v) for v in self.up]
        s.fov_y_deg = float(self.fov_y_deg)
        s.width, s.height = int(self.width), int(self.height)
        s.ray_id_offset = int(self.ray_id_offset)
        return s

    @classmethod
    def of(cls, cam):
        return cls(cam.width, cam.height, tuple(cam.eye), tuple(cam.look_at), tuple(cam.up),
                   float(cam.fov_y_deg), int(cam.ray_id_offset))


def _params(seed=0, spp=1, n_hits=1, t_min=0.0, t_max=float("inf"), bg=(0.0, 0.0, 0.0),
            stack_depth=0, stream_tag=0, counters=None, depth_mode=0,
            rng_mode=0, samples_per_lane=0) -> _TraceParams:
    p = _TraceParams()
    p.seed = int(seed)
    p.spp = int(spp)
    p.n_hits = int(n_hits)
    p.t_min = float(t_min)
    p.t_max = float(t_max)
    p.bg[:] = [float(v) for v in bg]
    p.depth_mode = int(depth_mode)
    p.stack_depth = int(stack_depth)
    p.stream_tag = int(stream_tag)
    p.rng_mode = int(rng_mode)
    p.samples_per_lane = int(samples_per_lane)
    p.counters = None if counters is None else counters.data_ptr()
    return p


# ---------------------------------------------------------------- hierarchy


class Bvh:
    """Owns a ``gs_bvh`` handle (released on :meth:`free` or collection)."""

    def __init__(self, handle: C.c_void_p, M: int):
        self._h = handle
        self.M = M

    @property
    def handle(self):
        return self._h

    def rebuild(self, g: Gaussians, stream=None):
        gs = g.struct()
        _check(lib().gs_bvh_rebuild(self._h, C.byref(gs), _stream_handle(stream)))
        self.M = g.M

    def info(self) -> dict:
        i = _BvhInfo()
        _check(lib().gs_bvh_get_info(self._h, C.byref(i)))
        return {k: getattr(i, k) for k, _ in _BvhInfo._fields_}

    def sync_status(self, stream=None):
        _check(lib().gs_bvh_sync_status(self._h, _stream_handle(stream)))

    def export(self) -> dict:
        info = self.info()
        nn, M = info["n_nodes"], info["M"]
        nodes = np.zeros((max(nn, 0), 16), np.uint32)
        prims = np.zeros((max(M, 0), 16), np.uint32)
        codes = np.zeros(max(M, 0), np.uint64)
        order = np.zeros(max(M, 0), np.uint32)
        ptr = lambda a: a.ctypes.data_as(C.c_void_p) if a.size else None  # noqa: E731
        _check(lib().gs_bvh_export(self._h, ptr(nodes), ptr(prims), ptr(codes), ptr(order)))
        return {"nodes": nodes, "prims": prims, "codes": codes, "order": order}

    def export_wide(self) -> np.ndarray:
        """Wide nodes as raw uint32 words [n, wide_node_bytes/4]."""
        info = self.info()
        n = C.c_int64(0)
        _check(lib().gs_bvh_export_wide(self._h, None, 0, C.byref(n)))
        out = np.zeros((n.value, info["wide_node_bytes"] // 4), np.uint32)
        if n.value:
            _check(lib().gs_bvh_export_wide(self._h, out.ctypes.data_as(C.c_void_p), n.value,
                                            C.byref(n)))
        return out

    def free(self):
        if self._h is not None and _lib is not None:
            lib().gs_bvh_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def build_bvh(g: Gaussians, stream=None, node_format="binary") -> Bvh:
    """``gs_build_bvh`` / ``gs_build_bvh_ex``: hierarchy over the Gaussians'
    bounding boxes; ``node_format`` is "binary", "wide4" or "wide4_q8"."""
    h = C.c_void_p()
    gs = g.struct()
    fmt = NODE_FORMATS[node_format] if isinstance(node_format, str) else int(node_format)
    if fmt == NODES_BINARY:
        _check(lib().gs_build_bvh(C.byref(gs), C.byref(h), _stream_handle(stream)))
    else:
        opt = _BuildOptions()
        opt.node_format = fmt
        _check(lib().gs_build_bvh_ex(C.byref(gs), C.byref(opt), C.byref(h),
                                     _stream_handle(stream)))
    return Bvh(h, g.M)


# ---------------------------------------------------------------- tracing


def sample_keys(cam, spp=1, n_hits=1, device="cuda"):
    """A buffer for every sample's payload (``gs_sample_key``: the depth key
    tc, tau and the Gaussian id of its closest accepted hit), filled by
    ``trace_stochastic(..., keys=)`` and read by ``trace_backward(...,
    keys=)``: int32 [H, W, spp * n_hits, 3], the float fields as their bits.
    12 bytes per sample."""
    cam = cam if isinstance(cam, Camera) else Camera.of(cam)
    return torch.empty((int(cam.height), int(cam.width), spp * n_hits, 3), dtype=torch.int32,
                       device=device)


def decode_keys(keys):
    """(tc, tau, gid) of a ``sample_keys`` buffer: float32, float32, int64
    (-1 where the sample accepted nothing)."""
    tc = keys[..., 0].contiguous().view(torch.float32)
    tau = keys[..., 1].contiguous().view(torch.float32)
    return tc, tau, keys[..., 2].to(torch.int64)


def _check_keys(keys, cam, spp, n_hits, dev):
    H, W = int(cam.height), int(cam.width)
    if (keys.dtype != torch.int32 or tuple(keys.shape) != (H, W, spp * n_hits, 3)
            or not keys.is_contiguous() or keys.device != dev):
        raise ValueError("keys must be a contiguous int32 tensor [%d, %d, %d, 3] on %s "
                         "(sample_keys)" % (H, W, spp * n_hits, dev))


def trace_stochastic(bvh: Bvh, g: Gaussians, cam, seed=0, spp=1, n_hits=1, t_min=0.0,
                     t_max=float("inf"), bg=(0.0, 0.0, 0.0), stack_depth=0, stream_tag=0,
                     want_hits=False, counters=None, out=None, stream=None, depth_mode=0,
                     rng_mode=0, samples_per_lane=0, keys=None):
    """``gs_trace_stochastic``: render one pinhole view.

    Returns ``rgb`` [H, W, 3] float32 (and ``hit_id``, ``hit_t`` of shape
    [spp, n_hits, H, W] when ``want_hits``), all on the current CUDA device.
    With ``keys`` (a ``sample_keys`` buffer) the call is
    ``gs_trace_stochastic_keys`` and also stores every sample's payload
    there, for ``trace_backward(..., keys=keys)``."""
    cam = cam if isinstance(cam, Camera) else Camera.of(cam)
    H, W = int(cam.height), int(cam.width)
    dev = g.means.device
    rgb = out if out is not None else torch.empty((H, W, 3), dtype=torch.float32, device=dev)
    gs = g.struct()
    cs = cam.struct()
    ps = _params(seed, spp, n_hits, t_min, t_max, bg, stack_depth, stream_tag, counters,
                 depth_mode, rng_mode, samples_per_lane)
    if keys is not None:
        if want_hits:
            raise ValueError("keys and want_hits are separate calls")
        _check_keys(keys, cam, spp, n_hits, dev)
        _check(lib().gs_trace_stochastic_keys(
            bvh.handle, C.byref(gs), C.byref(cs), C.byref(ps), C.c_void_p(rgb.data_ptr()),
            C.c_void_p(keys.data_ptr()), _stream_handle(stream)))
        return rgb
    hit_id = hit_t = None
    if want_hits:
        hit_id = torch.empty((spp, n_hits, H, W), dtype=torch.int32, device=dev)
        hit_t = torch.empty((spp, n_hits, H, W), dtype=torch.float32, device=dev)
    _check(lib().gs_trace_stochastic(
        bvh.handle, C.byref(gs), C.byref(cs), C.byref(ps), C.c_void_p(rgb.data_ptr()),
        None if hit_id is None else C.c_void_p(hit_id.data_ptr()),
        None if hit_t is None else C.c_void_p(hit_t.data_ptr()), _stream_handle(stream)))
    if want_hits:
        return rgb, hit_id, hit_t
    return rgb


def trace_layout(bvh: Bvh, spp=1, n_hits=1, samples_per_lane=0) -> dict:
    """``gs_trace_layout``: how a trace with these options maps samples to
    lanes (samples per lane, lanes per pixel, passes of n_hits * S slots,
    grouped)."""
    ps = _params(0, spp, n_hits, samples_per_lane=samples_per_lane)
    out = (C.c_int32 * 4)()
    _check(lib().gs_trace_layout(bvh.handle, C.byref(ps), out))
    return {"samples_per_lane": out[0], "lanes_per_pixel": out[1], "passes": out[2],
            "grouped": bool(out[3])}


def probe_copy(src, dst, repeats=1, stream=None):
    """``gs_probe_copy``: enqueue a copy of ``src`` into ``dst`` (device
    tensors of equal byte size) repeated ``repeats`` times in one kernel."""
    nbytes = src.numel() * src.element_size()
    assert dst.numel() * dst.element_size() == nbytes
    _check(lib().gs_probe_copy(C.c_void_p(src.data_ptr()), C.c_void_p(dst.data_ptr()),
                               nbytes, int(repeats), _stream_handle(stream)))


def trace_backward(bvh: Bvh, g: Gaussians, cam, d_rgb, seed=0, spp=1, n_hits=1, t_min=0.0,
                   t_max=float("inf"), bg=(0.0, 0.0, 0.0), stack_depth=0, stream_tag=0,
                   grads=None, stream=None, samples_per_lane=0, keys=None):
    """``gs_trace_backward``: stochastic gradients of sum(d_rgb * rgb).

    Returns (and accumulates into, if given) a dict of float32 gradients
    shaped like the parameters. With ``keys`` (filled by
    ``trace_stochastic(..., keys=)`` with the same options) the call is
    ``gs_trace_backward_keys``: the winners are read instead of traced."""
    cam = cam if isinstance(cam, Camera) else Camera.of(cam)
    dev = g.means.device
    if grads is None:
        grads = {"means": torch.zeros_like(g.means), "log_scales": torch.zeros_like(g.log_scales),
                 "quats": torch.zeros_like(g.quats),
                 "opacity_logits": torch.zeros_like(g.opacity_logits),
                 "sh": torch.zeros(g.sh.shape, dtype=torch.float32, device=dev)}
    d_rgb = d_rgb.to(device=dev, dtype=torch.float32).contiguous()
    gs_ = g.struct()
    cs = cam.struct()
    ps = _params(seed, spp, n_hits, t_min, t_max, bg, stack_depth, stream_tag, None,
                 samples_per_lane=samples_per_lane)
    outs = [C.c_void_p(d_rgb.data_ptr()),
            C.c_void_p(grads["means"].data_ptr()), C.c_void_p(grads["log_scales"].data_ptr()),
            C.c_void_p(grads["quats"].data_ptr()), C.c_void_p(grads["opacity_logits"].data_ptr()),
            C.c_void_p(grads["sh"].data_ptr()), _stream_handle(stream)]
    if keys is not None:
        _check_keys(keys, cam, spp, n_hits, dev)
        _check(lib().gs_trace_backward_keys(bvh.handle, C.byref(gs_), C.byref(cs), C.byref(ps),
                                            C.c_void_p(keys.data_ptr()), *outs))
    else:
        _check(lib().gs_trace_backward(bvh.handle, C.byref(gs_), C.byref(cs), C.byref(ps),
                                       *outs))
    return grads


class StochasticRender(torch.autograd.Function):
    """Differentiable stochastic rendering of one view.

    forward(means, log_scales, quats, opacity_logits, sh, sh_degree, cam,
    options) -> rgb [H, W, 3]; backward returns the unbiased stochastic
    gradients of gs_trace_backward (same seed, same samples). With
    ``keep_keys`` (the default) the forward stores every sample's payload
    (12 bytes per sample) and the backward reads it instead of tracing
    again (gs_trace_backward_keys)."""

    @staticmethod
    def forward(ctx, means, log_scales, quats, opacity_logits, sh, sh_degree, cam, options):
        options = dict(options)
        shared = options.pop("bvh", None)
        rebuild = options.pop("rebuild", True)
        keep_keys = options.pop("keep_keys", True)
        g = Gaussians(means.detach(), log_scales.detach(), quats.detach(),
                      opacity_logits.detach(), sh.detach(), sh_degree)
        if shared is not None:
            if rebuild:
                shared.rebuild(g)  # reuse the caller's handle: no allocation
            bvh = shared
        else:
            bvh = build_bvh(g)
        keys = None
        if keep_keys:
            keys = sample_keys(cam, options.get("spp", 1), options.get("n_hits", 1),
                               device=means.device)
        rgb = trace_stochastic(bvh, g, cam, keys=keys, **options)
        ctx.state = (bvh, shared is None, g, cam, options, keys)
        return rgb

    @staticmethod
    def backward(ctx, d_rgb):
        bvh, owned, g, cam, options, keys = ctx.state
        grads = trace_backward(bvh, g, cam, d_rgb, keys=keys, **options)
        if owned:
            bvh.free()
        ctx.state = None
        return (grads["means"], grads["log_scales"], grads["quats"], grads["opacity_logits"],
                grads["sh"].to(g.sh.dtype), None, None, None)


def render_differentiable(means, log_scales, quats, opacity_logits, sh, sh_degree, cam, **options):
    """Autograd entry point: rgb = StochasticRender.apply(...).

    ``bvh=`` (optional) is a handle to rebuild in place instead of building
    a new one per call; its backward must run before the next forward that
    uses the same handle. ``rebuild=False`` uses that handle as it is: the
    caller has already rebuilt it from these same parameters (several views
    of one parameter state share one rebuild). ``keep_keys=False`` stores
    nothing between forward and backward: the backward traces the winners
    again; with gradients disabled (``torch.no_grad``) nothing is stored."""
    if not torch.is_grad_enabled():
        options = dict(options, keep_keys=False)
    return StochasticRender.apply(means, log_scales, quats, opacity_logits, sh, sh_degree, cam,
                                  options)


# ---------------------------------------------------------------- batched form


class _Light(C.Structure):
    _fields_ = [("position", C.c_float * 3), ("intensity", C.c_float * 3)]


class _SceneExtras(C.Structure):
    _fields_ = [("n_lights", C.c_int32), ("lights", _Light * 8), ("has_ground", C.c_int32),
                ("ground_y", C.c_float), ("ground_half_extent", C.c_float),
                ("ground_albedo", C.c_float * 3), ("bounce", C.c_int32),
                ("shadow_eps", C.c_float)]


class _LaunchOptions(C.Structure):
    _fields_ = [("block_threads", C.c_int32), ("stack_entries", C.c_int32),
                ("reserved", C.c_int32 * 6)]


def _extras_struct(ex):
    e = _SceneExtras()
    if ex is None:
        return e
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


def _views_args(cams, extras, block_threads, stack_entries, seed, spp, t_min, t_max, bg,
                stack_depth, stream_tag):
    cams = [c if isinstance(c, Camera) else Camera.of(c) for c in cams]
    arr = (_Pinhole * len(cams))(*[c.struct() for c in cams])
    ex = _extras_struct(extras)
    opt = _LaunchOptions()
    opt.block_threads = int(block_threads)
    opt.stack_entries = int(stack_entries)
    ps = _params(seed, spp, 1, t_min, t_max, bg, stack_depth, stream_tag, None)
    total = sum(c.width * c.height for c in cams)
    return cams, arr, ex, opt, ps, total


def render_views(bvh: Bvh, g: Gaussians, cams, extras=None, seed=0, spp=1, t_min=0.0,
                 t_max=float("inf"), bg=(0.0, 0.0, 0.0), stack_depth=0, stream_tag=0,
                 block_threads=0, stack_entries=0, counters=None, want_samples=False, out=None,
                 stream=None):
    """``gs_render_views``: all views in one persistent launch.

    Returns the packed image [total pixels, 3] (view v starts after the
    pixels of views < v), and the per-sample diagnostics [spp, total, 3]
    when ``want_samples``."""
    cams, arr, ex, opt, ps, total = _views_args(cams, extras, block_threads, stack_entries, seed,
                                                 spp, t_min, t_max, bg, stack_depth, stream_tag)
    dev = g.means.device
    rgb = out if out is not None else torch.empty((total, 3), dtype=torch.float32, device=dev)
    samples = torch.empty((spp, total, 3), dtype=torch.int32, device=dev) if want_samples else None
    gs_ = g.struct()
    _check(lib().gs_render_views(
        bvh.handle, C.byref(gs_), arr, len(cams), C.byref(ex), C.byref(ps), C.byref(opt),
        C.c_void_p(rgb.data_ptr()), None if counters is None else C.c_void_p(counters.data_ptr()),
        None if samples is None else C.c_void_p(samples.data_ptr()), _stream_handle(stream)))
    return (rgb, samples) if want_samples else rgb


def split_views(packed, cams):
    """Packed [total, 3] image -> list of [H, W, 3] views."""
    out, o = [], 0
    for c in cams:
        n = c.width * c.height
        out.append(packed[o:o + n].reshape(c.height, c.width, 3))
        o += n
    return out


class FrameGraph:
    """``gs_graph_capture_views``: one frame (optional rebuild + the batched
    render) captured as a CUDA graph on a side stream; ``replay()`` runs it."""

    def __init__(self, bvh: Bvh, g: Gaussians, cams, extras=None, rebuild=True, out=None,
                 stream=None, **kw):
        self.stream = stream or torch.cuda.Stream()
        opts = dict(seed=0, spp=1, t_min=0.0, t_max=float("inf"), bg=(0.0, 0.0, 0.0),
                    stack_depth=0, stream_tag=0, block_threads=0, stack_entries=0)
        opts.update(kw)
        cams, arr, ex, opt, ps, total = _views_args(cams, extras, **{
            k: opts[k] for k in ("block_threads", "stack_entries", "seed", "spp", "t_min",
                                 "t_max", "bg", "stack_depth", "stream_tag")})
        self.rgb = out if out is not None else torch.empty((total, 3), dtype=torch.float32,
                                                           device=g.means.device)
        self._keep = (bvh, g, arr, ex, opt, ps)
        gs_ = g.struct()
        self._gs = gs_
        h = C.c_void_p()
        torch.cuda.synchronize()
        _check(lib().gs_graph_capture_views(
            bvh.handle, C.byref(gs_), int(bool(rebuild)), arr, len(cams), C.byref(ex),
            C.byref(ps), C.byref(opt), C.c_void_p(self.rgb.data_ptr()),
            C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self._h = h

    def replay(self, stream=None):
        _check(lib().gs_graph_launch(self._h, _stream_handle(stream or self.stream)))
        return self.rgb

    def free(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            lib().gs_graph_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def render(g: Gaussians, cam, stream=None, **kw):
    """Build a hierarchy and trace one view (convenience for one-off use)."""
    bvh = build_bvh(g, stream)
    try:
        res = trace_stochastic(bvh, g, cam, stream=stream, **kw)
        bvh.sync_status(stream)
        return res
    finally:
        bvh.free()
