"""Fitting Gaussians to images with the stochastic renderer's gradients.

The differentiation workload: a 500k-Gaussian shell cloud seen from 16
views at 800x800; target images are rendered from the true parameters; the
means, log-scales and opacity logits are perturbed (N(0, 0.01), N(0, 0.1),
N(0, 0.5)); every step renders all views stochastically, takes the L2 loss
to the targets and its unbiased gradient (gs_trace_backward, through
torch.autograd), and applies one Adam update. Checkpoints (parameters,
optimiser state, step) are written with torch.save and can be resumed.

    python -m paper_2504_06598_gb300.fit --steps 200 --spp 4 --out fit.json
"""

from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import paper_2504_06598_gb300 as gs  # noqa: E402
import scenes  # noqa: E402

KEYS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def make_problem(M=500_000, views=16, res=800, seed=0, target_spp=64):
    cloud = scenes.shell_cloud(seed, M=M)
    cams = scenes.orbit_cameras(views, seed=seed + 1, fixed_res=(res, res))
    true = {k: torch.from_numpy(getattr(cloud, k)).cuda() for k in KEYS}
    bvh = gs.build_bvh(gs.Gaussians(**{k: true[k] for k in KEYS}, sh_degree=cloud.sh_degree))
    targets = []
    with torch.no_grad():
        for v, cam in enumerate(cams):
            targets.append(gs.render_differentiable(
                true["means"], true["log_scales"], true["quats"], true["opacity_logits"],
                true["sh"], cloud.sh_degree, cam, bvh=bvh, seed=10_000 + v, spp=target_spp,
                n_hits=4).clone())
    rng = np.random.default_rng(seed + 2)
    init = {k: v.clone() for k, v in true.items()}
    for k, sd in (("means", 0.01), ("log_scales", 0.1), ("opacity_logits", 0.5)):
        init[k] += torch.from_numpy(rng.normal(0, sd, init[k].shape).astype(np.float32)).cuda()
    return cloud, cams, true, init, targets, bvh


def fit(steps=200, spp=4, n_hits=1, lr=None, M=500_000, views=16, res=800, seed=0,
        checkpoint=None, resume=False, log_every=10):
    cloud, cams, true, init, targets, bvh = make_problem(M, views, res, seed)
    params = {k: v.clone().requires_grad_(True) for k, v in init.items()}
    # Adam moves each parameter by about lr per step whatever the gradient's
    # noise, so the rates are kept small enough for 4-sample gradients
    lrs = lr or {"means": 2e-5, "log_scales": 1e-3, "quats": 2e-4, "opacity_logits": 5e-3,
                 "sh": 5e-4}
    opt = torch.optim.Adam([{"params": [params[k]], "lr": lrs[k]} for k in KEYS])
    start = 0
    if resume and checkpoint and os.path.exists(checkpoint):
        ck = torch.load(checkpoint, map_location="cuda")
        with torch.no_grad():
            for k in KEYS:
                params[k].copy_(ck["params"][k])
        opt.load_state_dict(ck["opt"])
        start = int(ck["step"])

    def eval_loss(eval_spp=32):
        """Image loss with many samples and fixed seeds (low noise)."""
        with torch.no_grad():
            tot = 0.0
            for v, cam in enumerate(cams):
                img = gs.render_differentiable(params["means"], params["log_scales"],
                                               params["quats"], params["opacity_logits"],
                                               params["sh"], cloud.sh_degree, cam, bvh=bvh,
                                               seed=20_000 + v, spp=eval_spp, n_hits=4)
                tot += float(((img - targets[v]) ** 2).mean())
            return tot / len(cams)

    def param_error():
        with torch.no_grad():
            return {k: float((params[k] - true[k]).abs().mean()) for k in ("means", "log_scales",
                                                                            "opacity_logits")}

    history = []
    t_step = []
    err0 = param_error()
    eval0 = eval_loss()
    for step in range(start, steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        opt.zero_grad()
        total = 0.0
        # one hierarchy rebuild per parameter state, shared by all views
        bvh.rebuild(gs.Gaussians(*(params[k].detach() for k in KEYS), cloud.sh_degree))
        for v, cam in enumerate(cams):
            img = gs.render_differentiable(params["means"], params["log_scales"], params["quats"],
                                           params["opacity_logits"], params["sh"],
                                           cloud.sh_degree, cam, bvh=bvh, rebuild=False,
                                           seed=step * len(cams) + v, spp=spp, n_hits=n_hits)
            loss = ((img - targets[v]) ** 2).mean()
            loss.backward()
            total += float(loss.detach())
        opt.step()
        torch.cuda.synchronize()
        t_step.append(time.perf_counter() - t0)
        history.append(total / len(cams))
        if log_every and (step % log_every == 0 or step == steps - 1):
            print("step %4d  loss %.6f  %.3f s" % (step, history[-1], t_step[-1]), flush=True)
        if checkpoint and (step + 1) % 50 == 0:
            torch.save({"params": {k: params[k].detach() for k in KEYS},
                        "opt": opt.state_dict(), "step": step + 1}, checkpoint)
    eval1 = eval_loss()
    bvh.sync_status()
    bvh.free()
    return {"eval_loss_initial": eval0, "eval_loss_final": eval1, "steps": steps, "spp": spp, "n_hits": n_hits, "gaussians": M, "views": views,
            "res": res, "loss_first": history[0] if history else None,
            "loss_last": history[-1] if history else None, "loss_history": history,
            "param_error_initial": err0, "param_error_final": param_error(),
            "seconds_per_step": float(np.median(t_step)) if t_step else None}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--spp", type=int, default=4)
    ap.add_argument("--n-hits", type=int, default=1)
    ap.add_argument("--gaussians", type=int, default=500_000)
    ap.add_argument("--views", type=int, default=16)
    ap.add_argument("--res", type=int, default=800)
    ap.add_argument("--checkpoint", default=None)
    ap.add_argument("--resume", action="store_true")
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    from . import build as gbuild
    gbuild.build()
    res = fit(a.steps, a.spp, a.n_hits, None, a.gaussians, a.views, a.res,
              checkpoint=a.checkpoint, resume=a.resume)
    line = json.dumps({k: v for k, v in res.items() if k != "loss_history"})
    print(line)
    if a.out:
        with open(a.out, "w") as f:
            json.dump(res, f)


if __name__ == "__main__":
    main()
