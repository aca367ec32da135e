"""Comparison of GPU hit ids and colours with the oracle, with every
mismatch classified by its cause.

Classes of a mismatched (ray, sample):
  i    a candidate whose acceptance differs has |alpha - xi| < 1e-6
       (float32 vs float64 alpha at the threshold; the allowed class)
  ii   a candidate at the ellipsoid edge, |q - 8| < 1e-5 * 8
  iii  the two winners are accepted by the oracle and their depths agree
       to 1e-6 relative
  iv   a candidate within 1e-6 of t_min
  other  anything else (a bug)
The batched form's samples (camera hit or ground, bounce hit, visible-light
bits) are classified the same way on the ray whose outcome differs: the
camera ray (stream tag 0), the bounce ray from the ground point (tag 9) or
the shadow ray to light l (tag 1 + l, any accepted Gaussian on the segment
blocks it)."""
import numpy as np

import oracle

ALPHA_TOL = 1e-6


def classify(cloud, o, d, ray_id, s, g_gpu, g_orc, seed, t_min=0.0, stream_tag=0):
    c = oracle.ray_candidates(cloud, o, d, t_min=t_min)
    by = {int(g): k for k, g in enumerate(c["gid"])}
    xi = lambda g: oracle.xi(seed, ray_id, int(g), s, stream_tag)  # noqa: E731
    # class i: a winner (either side) sits at the acceptance threshold, or a
    # closer candidate does
    for g in (g_gpu, g_orc):
        if g >= 0 and g in by and abs(c["alpha"][by[g]] - xi(g)) < ALPHA_TOL:
            return "i"
    t_ref = min([c["t"][by[g]] for g in (g_gpu, g_orc) if g >= 0 and g in by] or [np.inf])
    for k, g in enumerate(c["gid"]):
        if c["t"][k] <= t_ref and abs(c["alpha"][k] - xi(g)) < ALPHA_TOL:
            return "i"
    if g_gpu >= 0 and g_gpu not in by:
        t, q, a, _ = oracle.eval_pair(cloud, g_gpu, o, d, t_min=t_min)
        if abs(q - 8.0) < 8e-5:
            return "ii"
        if abs(t - t_min) < 1e-6 * max(1.0, abs(t)):
            return "iv"
        return "other"
    if g_gpu >= 0 and g_orc >= 0:
        ta, tb = c["t"][by[g_gpu]], c["t"][by[g_orc]]
        if abs(ta - tb) < 1e-6 * abs(tb):
            return "iii"
    for k in range(len(c["t"])):
        if c["t"][k] <= t_ref and abs(c["q"][k] - 8.0) < 8e-5:
            return "ii"
    return "other"


def compare(cloud, cam, seed, gpu_ids, ref, pixels, n_hits=1, stream_tag=0):
    """gpu_ids [n_pix, S] for the listed pixels; ref from oracle.render_*.

    Returns (agreement, {class: count}, list of mismatch tuples)."""
    ref_ids = ref["hit_id"]
    mism = np.argwhere(gpu_ids != ref_ids)
    classes = {}
    details = []
    for i, s in mism:
        p = int(pixels[i])
        o, d, rid = oracle.camera_ray(cam, p % cam.width, p // cam.width)
        k = classify(cloud, o, d, rid, int(s), int(gpu_ids[i, s]), int(ref_ids[i, s]), seed,
                     stream_tag=stream_tag)
        classes[k] = classes.get(k, 0) + 1
        details.append((p, int(s), int(gpu_ids[i, s]), int(ref_ids[i, s]), k))
    agree = 1.0 - len(mism) / max(1, gpu_ids.size)
    return agree, classes, details


def colour_check(gpu_rgb, ref_est, same_rows, rel=1e-5, abs_floor=1e-6):
    """Max violation of |gpu - ref| <= rel*|ref| + abs_floor on pixels whose
    samples all agree (<= 0 means pass)."""
    g = gpu_rgb[same_rows]
    r = ref_est[same_rows]
    if g.size == 0:
        return -1.0
    return float(np.max(np.abs(g - r) - (rel * np.abs(r) + abs_floor)))


def _classify_any_hit(cloud, o, d, ray_id, s, seed, t_min, t_max, stream_tag):
    """A visibility flip: some candidate on the segment must sit at the
    acceptance threshold (class i)."""
    c = oracle.ray_candidates(cloud, o, d, t_min=t_min, t_max=t_max)
    for k, g in enumerate(c["gid"]):
        if abs(c["alpha"][k] - oracle.xi(seed, ray_id, int(g), s, stream_tag)) < ALPHA_TOL:
            return "i"
    for k in range(len(c["t"])):
        if abs(c["q"][k] - 8.0) < 8e-5:
            return "ii"
        if abs(c["t"][k] - t_min) < 1e-6 * max(1.0, abs(c["t"][k])):
            return "iv"
    return "other"


def classify_scene_sample(cloud, cam, extras, settings, pixel, s, gpu, orc):
    """Class of one mismatched sample of the scene renderer; gpu and orc are
    its (camera hit, bounce hit, light bits) triples."""
    x, y = pixel % cam.width, pixel // cam.width
    r = oracle.scene_sample_rays(cam, extras, settings, x, y, s)
    seed, rid = settings.seed, r["ray_id"]
    eps = extras.shadow_eps
    if gpu[0] != orc[0]:
        gg, go = (int(v) if v >= 0 else -1 for v in (gpu[0], orc[0]))
        if -2 in (gpu[0], orc[0]) and max(gg, go) >= 0:
            # ground against a Gaussian: a tie in depth with the quad
            t, _, _, _ = oracle.eval_pair(cloud, max(gg, go), r["o"], r["d"])
            if abs(t - r["tq"]) < 1e-6 * abs(r["tq"]):
                return "iii"
        return classify(cloud, r["o"], r["d"], rid, s, gg, go, seed, t_min=settings.t_min)
    if gpu[1] != orc[1]:
        return classify(cloud, r["p"], r["bounce_d"], rid, s, int(gpu[1]), int(orc[1]), seed,
                        t_min=eps, stream_tag=9)
    worst = "i"
    for l, lr in enumerate(r["lights"]):
        if ((int(gpu[2]) ^ int(orc[2])) >> l) & 1:
            if lr is None:
                return "other"
            k = _classify_any_hit(cloud, r["p"], lr[0], rid, s, seed, eps, lr[1], 1 + l)
            if k != "i":
                worst = k
    return worst


def compare_scene(cloud, cams, extras, settings, items, gpu_smp, orc_diag):
    """gpu_smp and orc_diag [n_items, spp, 3] for the (view, pixel) items.

    Returns (agreement over sample slots, {class: count}, mismatch tuples)."""
    mism = np.argwhere(np.any(gpu_smp != orc_diag, axis=2))
    classes, details = {}, []
    for i, s in mism:
        v, p = items[int(i)]
        k = classify_scene_sample(cloud, cams[v], extras, settings, int(p), int(s),
                                  gpu_smp[i, s], orc_diag[i, s])
        classes[k] = classes.get(k, 0) + 1
        details.append((int(v), int(p), int(s), tuple(gpu_smp[i, s]), tuple(orc_diag[i, s]), k))
    agree = 1.0 - len(mism) / max(1, gpu_smp.shape[0] * gpu_smp.shape[1])
    return agree, classes, details
