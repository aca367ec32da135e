"""Autotuner for the batched wavefront form.

Picks the hierarchy node format (binary with FP32 or 8-bit wide copies,
4-wide FP32, 4-wide 8-bit), the
traversal stack capacity and the threads per block of gs_render_views by
timing each combination on the caller's own workload (CUDA events on the
launching stream, after a warm-up launch). The choice can be cached in a JSON
file keyed by the workload's shape, so later runs skip the search.
"""

from __future__ import annotations

import itertools
import json
import os

import torch

from . import Bvh, Gaussians, build_bvh, render_views

FORMATS = ("binary", "binary_q8", "wide4", "wide4_q8")
STACKS = (48, 96)
BLOCKS = (64, 128, 256)


def workload_key(g: Gaussians, cams, extras, spp: int) -> str:
    px = sum(c.width * c.height for c in cams)
    n_l = len(extras.lights) if extras is not None else 0
    bounce = int(bool(extras.bounce)) if extras is not None else 0
    return "M%d_deg%d_sh%s_v%d_px%d_spp%d_l%d_b%d" % (
        g.M, g.sh_degree, str(g.sh.dtype).replace("torch.", ""), len(cams), px, spp, n_l, bounce)


def _time(fn, repeats):
    fn()  # warm-up
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(repeats):
        fn()
    e1.record(s)
    e1.synchronize()
    return e0.elapsed_time(e1) / repeats


def autotune(g: Gaussians, cams, extras=None, spp=1, seed=0, formats=FORMATS, stacks=STACKS,
             blocks=BLOCKS, repeats=2, cache_path=None):
    """Return {"node_format", "stack_entries", "block_threads", "ms", "trials"}."""
    key = workload_key(g, cams, extras, spp)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if key in cache:
            return dict(cache[key], cached=True)
    trials = []
    out = torch.empty((sum(c.width * c.height for c in cams), 3), dtype=torch.float32,
                      device=g.means.device)
    for fmt in formats:
        bvh: Bvh = build_bvh(g, node_format=fmt)
        for stack, block in itertools.product(stacks, blocks):
            ms = _time(lambda: render_views(bvh, g, cams, extras, seed=seed, spp=spp,
                                            block_threads=block, stack_entries=stack, out=out),
                       repeats)
            trials.append({"node_format": fmt, "stack_entries": stack, "block_threads": block,
                           "ms": ms})
        bvh.sync_status()
        bvh.free()
    best = min(trials, key=lambda t: t["ms"])
    result = dict(best, key=key, trials=trials)
    if cache_path:
        cache[key] = {k: v for k, v in result.items() if k != "trials"}
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return result
