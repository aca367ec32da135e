"""Comparison of GPU hit ids and colours with the oracle, with every
mismatch classified by its cause.

Classes of a mismatched (ray, sample):
  i    a candidate whose acceptance differs has |alpha - xi| < 1e-6
       (float32 vs float64 alpha at the threshold; the allowed class)
  ii   a candidate at the ellipsoid edge, |q - 8| < 1e-5 * 8
  iii  the two winners are accepted by the oracle and their depths agree
       to 1e-6 relative
  iv   a candidate within 1e-6 of t_min
  other  anything else (a bug)"""
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
