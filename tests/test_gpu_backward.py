"""GPU gradients (gs_trace_backward) against the FP64 oracle: the same
stochastic estimator with the same draws (parity), its mean against the
analytic gradient of the sorted blend (unbiasedness) on a 2,000-Gaussian
subset of the shell cloud, finite differences of the oracle blend for a few
parameters, and the autograd path."""
import numpy as np
import pytest

import oracle
import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEYS = ["means", "log_scales", "quats", "opacity_logits", "sh"]


@pytest.fixture(scope="module")
def gs():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2504_06598_gb300 as m
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for gpu tests")
    return m


def _cluster(seed=0, M=60, sh_degree=1):
    rng = np.random.default_rng(seed)
    means = np.stack([rng.uniform(-0.15, 0.15, M), rng.uniform(-0.15, 0.15, M),
                      rng.uniform(-0.4, 0.4, M)], 1)
    K = (sh_degree + 1) ** 2
    sh = np.concatenate([rng.uniform(0.1, 1.0, (M, 1, 3)), rng.normal(0, 0.3, (M, K - 1, 3))], 1)
    f = lambda a: np.ascontiguousarray(a, np.float32)  # noqa: E731
    return scenes.GaussianCloud(f(means), f(rng.normal(-2.3, 0.3, (M, 3))),
                                f(rng.normal(size=(M, 4))), f(rng.normal(0.5, 1.0, M)), f(sh),
                                sh_degree)


def _gpu_grads(gs, cloud, cam, d_rgb, node_format="binary", keys=False, fwd_samples_per_lane=0,
               **opts):
    """Gradients of gs_trace_backward, or with keys=True of
    gs_trace_backward_keys fed by a gs_trace_stochastic_keys rendering
    (its own samples_per_lane, automatic by default)."""
    g = gs.Gaussians.from_cloud(cloud)
    bvh = gs.build_bvh(g, node_format=node_format)
    d = torch.from_numpy(np.ascontiguousarray(d_rgb, np.float32)).cuda().reshape(cam.height, cam.width, 3)
    kb = None
    if keys:
        kb = gs.sample_keys(cam, opts.get("spp", 1), opts.get("n_hits", 1))
        fwd = {k: v for k, v in opts.items() if k != "samples_per_lane"}
        gs.trace_stochastic(bvh, g, cam, keys=kb, samples_per_lane=fwd_samples_per_lane, **fwd)
    grads = gs.trace_backward(bvh, g, cam, d, keys=kb, **opts)
    bvh.sync_status()
    bvh.free()
    return {k: v.cpu().numpy().astype(np.float64) for k, v in grads.items()}


# the library's choice of samples per lane: per-lane packets at spp 2-4
# (four slots), grouped traversals (8 or 16 lanes on one pixel, two slots)
# at spp 16 and 40
# keys: the winners read from the rendering's stored payloads instead of
# traced again
@pytest.mark.parametrize("keys", [False, True])
@pytest.mark.parametrize("spp,n_hits", [(4, 1), (2, 4), (3, 2), (40, 1), (16, 1), (8, 2)])
def test_estimator_parity(gs, spp, n_hits, keys):
    cloud = _cluster()
    cam = scenes.Pinhole(width=16, height=12, fov_y_deg=9.0)
    rng = np.random.default_rng(spp)
    d_rgb = rng.normal(size=(cam.width * cam.height, 3))
    bg = (0.2, 0.1, 0.4)
    gpu = _gpu_grads(gs, cloud, cam, d_rgb, keys=keys, seed=7, spp=spp, n_hits=n_hits, bg=bg)
    ref = oracle.grad_pinhole(cloud, cam, scenes.TraceSettings(seed=7, spp=spp, n_hits=n_hits, bg=bg),
                              d_rgb, mode="estimator")
    for k in KEYS:
        scale = np.abs(ref[k]).max()
        assert scale > 0, k
        err = np.abs(gpu[k] - ref[k]).max()
        assert err <= 1e-4 * scale + 1e-6, (k, err, scale)


def test_mean_gradient_matches_blend_gradient(gs):
    """2,000 Gaussians of the shell generator around one cluster; the GPU
    estimate at 4096 samples per pixel against the oracle's analytic FP64
    gradient of the sorted blend."""
    full = scenes.shell_cloud(3, M=128000, sh_degree=3)
    centre = full.means[0]
    near = np.argsort(np.linalg.norm(full.means - centre, axis=1))[:2000]
    cloud = full.subset(near)
    eye = tuple(float(v) for v in 3.0 * centre / np.linalg.norm(centre))
    cam = scenes.Pinhole(width=24, height=24, eye=eye, look_at=tuple(float(v) for v in centre),
                         fov_y_deg=3.0)
    rng = np.random.default_rng(0)
    d_rgb = rng.normal(size=(cam.width * cam.height, 3))
    gpu = _gpu_grads(gs, cloud, cam, d_rgb, seed=1, spp=1024, n_hits=4)
    ref = oracle.grad_pinhole(cloud, cam, scenes.TraceSettings(), d_rgb, mode="blend")
    a = np.concatenate([gpu[k].ravel() for k in KEYS])
    b = np.concatenate([ref[k].ravel() for k in KEYS])
    cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b))
    assert cos > 0.99, cos
    assert np.linalg.norm(a - b) < 0.15 * np.linalg.norm(b)
    # and the analytic gradient itself against FP64 finite differences of
    # the oracle blend, for the most influential opacity logits
    top = np.argsort(-np.abs(ref["opacity_logits"]))[:4]
    st = scenes.TraceSettings()
    for gi in top:
        def G(delta):
            c = cloud.subset(np.arange(cloud.M))
            v = np.float32(np.float64(c.opacity_logits[gi]) + delta)
            c.opacity_logits[gi] = v
            r = oracle.render_pinhole(c, cam, st, want_hits=False)
            return float(np.sum(r["blend"] * d_rgb)), float(v)
        gp, vp = G(1e-3)
        gm, vm = G(-1e-3)
        fd = (gp - gm) / (vp - vm)
        assert abs(fd - ref["opacity_logits"][gi]) <= 1e-3 * abs(ref["opacity_logits"][gi]) + 1e-6


def test_autograd_and_fit(gs):
    """render_differentiable gives the trace_backward gradients, and a few
    Adam steps on perturbed parameters reduce the L2 loss to a target image."""
    cloud = _cluster(seed=4, M=80, sh_degree=1)
    cam = scenes.Pinhole(width=32, height=32, fov_y_deg=9.0)
    opts = dict(seed=0, spp=16, n_hits=4)
    p = {k: torch.from_numpy(getattr(cloud, k)).cuda() for k in KEYS}
    with torch.no_grad():
        target = gs.render_differentiable(p["means"], p["log_scales"], p["quats"],
                                          p["opacity_logits"], p["sh"], cloud.sh_degree, cam,
                                          **dict(opts, spp=256))
    def render(params, seed):
        return gs.render_differentiable(params["means"], params["log_scales"], params["quats"],
                                        params["opacity_logits"], params["sh"], cloud.sh_degree,
                                        cam, **dict(opts, seed=seed))
    # Monte-Carlo noise floor: the loss of the true parameters at this spp
    with torch.no_grad():
        floor = float(np.mean([float(((render(p, 100 + s) - target) ** 2).sum()) for s in range(5)]))
    rng = np.random.default_rng(1)
    q = {k: v.clone() for k, v in p.items()}
    q["means"] += torch.from_numpy(rng.normal(0, 0.01, q["means"].shape).astype(np.float32)).cuda()
    q["opacity_logits"] += torch.from_numpy(rng.normal(0, 0.5, q["opacity_logits"].shape).astype(np.float32)).cuda()
    for v in q.values():
        v.requires_grad_(True)
    opt = torch.optim.Adam(q.values(), lr=5e-3)
    losses = []
    for it in range(30):
        opt.zero_grad()
        loss = ((render(q, it) - target) ** 2).sum()
        loss.backward()
        opt.step()
        losses.append(float(loss.detach()))
    assert all(np.isfinite(losses))
    assert losses[0] > 1.5 * floor
    # most of the excess over the noise floor is gone
    assert np.mean(losses[-5:]) - floor < 0.3 * (losses[0] - floor), (floor, losses)


def test_grouped_and_packet_gradients_agree(gs):
    """Samples 0..15 by 16 lanes on one pixel (grouped traversals) and by 2
    lanes x 8 slots (per-lane packets): the same per-sample hits, so the same
    gradients up to the order of the float sums."""
    cloud = scenes.shell_cloud(8, M=20000)
    cam = scenes.default_camera(48, 36)
    rng = np.random.default_rng(5)
    d_rgb = rng.normal(size=(cam.width * cam.height, 3))
    a = _gpu_grads(gs, cloud, cam, d_rgb, seed=2, spp=16, n_hits=1)
    b = _gpu_grads(gs, cloud, cam, d_rgb, seed=2, spp=2, n_hits=8)
    for k in KEYS:
        scale = np.abs(b[k]).max()
        assert scale > 0, k
        assert np.abs(a[k] - b[k]).max() <= 1e-5 * scale, k


@pytest.mark.parametrize("spp,n_hits", [(16, 1), (8, 4), (32, 1)])
def test_binary_q8_gradients_match_binary(gs, spp, n_hits):
    """The grouped backward on the 8-bit wide copies re-traces the same hits
    and enumerates the same Gaussians: gradients equal the FP32 copies' up
    to the order of the atomic float sums."""
    cloud = scenes.shell_cloud(8, M=20000)
    cam = scenes.default_camera(48, 36)
    rng = np.random.default_rng(6)
    d_rgb = rng.normal(size=(cam.width * cam.height, 3))
    a = _gpu_grads(gs, cloud, cam, d_rgb, seed=2, spp=spp, n_hits=n_hits)
    b = _gpu_grads(gs, cloud, cam, d_rgb, node_format="binary_q8", seed=2, spp=spp,
                   n_hits=n_hits)
    for k in KEYS:
        scale = np.abs(a[k]).max()
        assert scale > 0, k
        assert np.abs(a[k] - b[k]).max() <= 1e-5 * scale, k


@pytest.mark.parametrize("spp,n_hits", [(16, 1), (5, 1), (8, 2), (64, 1)])
def test_samples_per_lane_gradients_agree(gs, spp, n_hits):
    """A lane carrying S consecutive samples (unused slots past the last
    sample) re-traces the same per-sample hits: gradients equal one sample
    per lane's up to the order of the float sums."""
    cloud = scenes.shell_cloud(8, M=20000)
    cam = scenes.default_camera(40, 30)
    rng = np.random.default_rng(7)
    d_rgb = rng.normal(size=(cam.width * cam.height, 3))
    a = _gpu_grads(gs, cloud, cam, d_rgb, seed=3, spp=spp, n_hits=n_hits, samples_per_lane=1)
    for S in (0, 2, 4):
        if S * n_hits > 8:
            continue
        b = _gpu_grads(gs, cloud, cam, d_rgb, seed=3, spp=spp, n_hits=n_hits, samples_per_lane=S)
        for k in KEYS:
            scale = np.abs(a[k]).max()
            assert scale > 0, k
            assert np.abs(a[k] - b[k]).max() <= 1e-5 * scale, (S, k)


@pytest.mark.parametrize("spp,n_hits,S", [(1, 1, 0), (16, 1, 0), (16, 1, 1), (64, 1, 0),
                                          (5, 1, 4), (4, 4, 0), (8, 2, 2), (2, 8, 0)])
def test_keys_match_hits(gs, spp, n_hits, S):
    """gs_trace_stochastic_keys renders the same image as gs_trace_stochastic
    and stores each sample's payload: gid is the sample's hit id, tc + tau
    (one float32 add) its hit depth, bit for bit."""
    cloud = scenes.shell_cloud(8, M=20000)
    cam = scenes.default_camera(45, 31)  # ragged against every tile shape
    g = gs.Gaussians.from_cloud(cloud)
    bvh = gs.build_bvh(g)
    rgb, hid, ht = gs.trace_stochastic(bvh, g, cam, seed=4, spp=spp, n_hits=n_hits,
                                       samples_per_lane=S, want_hits=True)
    kb = gs.sample_keys(cam, spp, n_hits)
    rgb2 = gs.trace_stochastic(bvh, g, cam, seed=4, spp=spp, n_hits=n_hits, samples_per_lane=S,
                               keys=kb)
    bvh.sync_status()
    bvh.free()
    assert torch.equal(rgb, rgb2)
    tc, tau, gid = gs.decode_keys(kb)
    # keys are [H, W, sample], hits [sample pass, slot, H, W]
    hid = hid.reshape(spp * n_hits, cam.height, cam.width).permute(1, 2, 0).to(torch.int64)
    ht = ht.reshape(spp * n_hits, cam.height, cam.width).permute(1, 2, 0)
    assert torch.equal(gid, hid)
    assert torch.equal((tc + tau)[gid >= 0], ht[gid >= 0])
    assert bool(torch.isinf(tc[gid < 0]).all()) and bool((tau[gid < 0] == 0).all())
    assert float((gid >= 0).float().mean()) > 0.05  # the view holds hits at all


@pytest.mark.parametrize("spp,n_hits,fwd_S,bwd_S,fmt", [
    (16, 1, 0, 0, "binary"), (16, 1, 1, 2, "binary"), (4, 4, 0, 0, "binary"),
    (64, 1, 0, 0, "binary"), (7, 1, 8, 1, "binary"), (8, 2, 0, 4, "binary"),
    (16, 1, 0, 0, "binary_q8"), (4, 1, 0, 0, "wide4_q8")])
def test_keys_gradients_match_retrace(gs, spp, n_hits, fwd_S, bwd_S, fmt):
    """Gradients from stored payloads equal those of tracing the winners
    again, for any pair of rendering and gradient layouts, up to the order
    of the atomic float sums."""
    cloud = scenes.shell_cloud(8, M=20000)
    cam = scenes.default_camera(40, 30)
    rng = np.random.default_rng(11)
    d_rgb = rng.normal(size=(cam.width * cam.height, 3))
    a = _gpu_grads(gs, cloud, cam, d_rgb, node_format=fmt, seed=5, spp=spp, n_hits=n_hits,
                   samples_per_lane=bwd_S)
    b = _gpu_grads(gs, cloud, cam, d_rgb, node_format=fmt, keys=True, fwd_samples_per_lane=fwd_S,
                   seed=5, spp=spp, n_hits=n_hits, samples_per_lane=bwd_S)
    for k in KEYS:
        scale = np.abs(a[k]).max()
        assert scale > 0, k
        assert np.abs(a[k] - b[k]).max() <= 1e-5 * scale, k


def test_keys_with_unknown_gaussian_are_reported(gs):
    """A key naming no Gaussian of the handle is checked before use: that
    sample counts as no hit and gs_bvh_sync_status reports
    GS_ERR_INVALID_ARG; the other samples' gradients are unchanged."""
    cloud = scenes.shell_cloud(8, M=20000)
    cam = scenes.default_camera(32, 24)
    g = gs.Gaussians.from_cloud(cloud)
    bvh = gs.build_bvh(g)
    kb = gs.sample_keys(cam, 4, 1)
    gs.trace_stochastic(bvh, g, cam, seed=1, spp=4, keys=kb)
    d = torch.zeros((cam.height, cam.width, 3), device="cuda")
    d[5:9, 7:12] = 1.0
    ref = gs.trace_backward(bvh, g, cam, d, seed=1, spp=4, keys=kb)
    bvh.sync_status()
    bad = kb.clone()
    bad[20, 3, 2, 2] = cloud.M + 5  # a pixel outside the weighted window
    out = gs.trace_backward(bvh, g, cam, d, seed=1, spp=4, keys=bad)
    with pytest.raises(gs.GsError) as e:
        bvh.sync_status()
    assert e.value.status == 1
    bvh.sync_status()  # cleared
    for k in KEYS:
        scale = float(ref[k].abs().max())
        assert float((ref[k] - out[k]).abs().max()) <= 1e-5 * scale, k
    bvh.free()


def test_keys_full_size(gs):
    """1M-Gaussian shell at 1080p, N=1 spp 16 as the gradient benchmark
    launches it (automatic layouts: eight samples per lane in the rendering,
    two in the gradient launch): stored payloads and tracing the winners
    again give the same gradients up to the atomics' summation order."""
    cloud = scenes.shell_cloud(0, M=1_000_000)
    cam = scenes.default_camera(1920, 1080)
    g = gs.Gaussians.from_cloud(cloud)
    bvh = gs.build_bvh(g)
    gen = torch.Generator(device="cuda").manual_seed(3)
    d = torch.randn((1080, 1920, 3), device="cuda", generator=gen)
    kb = gs.sample_keys(cam, 16, 1)
    gs.trace_stochastic(bvh, g, cam, seed=0, spp=16, keys=kb)
    a = gs.trace_backward(bvh, g, cam, d, seed=0, spp=16)
    b = gs.trace_backward(bvh, g, cam, d, seed=0, spp=16, keys=kb)
    bvh.sync_status()
    bvh.free()
    for k in KEYS:
        scale = float(a[k].abs().max())
        assert scale > 0, k
        assert float((a[k] - b[k]).abs().max()) <= 1e-4 * scale, k
