"""The optimisation loop of the method's second stage, on the library: Adam on a scene's
material textures and environment map against target images, a few random views per step
(the workload's config 4: the config-2 scene, 300 steps at lr 1e-2, 8 views of 800 x 800 per
step, 4 bounces, 8 samples per pixel, from a flat start: albedo 0.5, roughness 0.5, env 1.0).

Every step renders the chosen views with the batched launch through MirresRender (the
PRIMARY-mode adjoint as its backward) and takes the L2 image loss (Eq. loss_pbr). The loop can
checkpoint its parameters and Adam state with torch.save and resume from them.

  python -m paper_2406_16360_gb300.optimize [--steps 300] [--res 800] [--views 8] [--out curve.json]
"""
from __future__ import annotations

import argparse
import copy
import json
import os
import time

import numpy as np
import torch

from . import mirres as M
from . import synth
from .renderer import GpuWorkload, MirresRender, scene_params

TRAINED = ("albedo", "roughness", "env")  # the textures and env map the loop optimises


class Loop:
    """Adam on the textures and env map of `init` (a synth.Scene) against renders of `truth`
    from a pool of cameras; `views_per_step` of them drawn per step from a seeded generator."""

    def __init__(self, truth, init, pool, views_per_step, lr, ris_m, seed=0, ctx=None, device=0):
        self.pool = list(pool)
        self.views_per_step = views_per_step
        self.seed = seed
        self.ris_m = ris_m
        self.own_ctx = ctx is None
        self.ctx = ctx or M.mirres_context_create(device)
        # targets: the ground truth rendered once per pool camera (another random stream)
        tw = synth.Workload("truth", [truth], self.pool, ris_m, seed=seed + 1_000_003)
        tgw = GpuWorkload(tw, device, ctx=self.ctx)
        imgs, _ = tgw.render(launch=1)
        self.targets = [im.clone() for im in imgs]
        for s in tgw.scenes:
            s.close()
        chosen = self.pool[:views_per_step]
        self.gw = GpuWorkload(synth.Workload("opt", [copy.deepcopy(init)], chosen, ris_m, seed=seed), device,
                              ctx=self.ctx)
        self.scene = self.gw.scenes[0]
        self.params = [getattr(self.scene, k) for k in TRAINED]
        for p in self.params:
            p.requires_grad_(True)
        self.opt = torch.optim.Adam(self.params, lr=lr)
        self.step_no = 0
        self.curve = []

    def choose(self, step):
        rng = np.random.Generator(np.random.PCG64([self.seed, step]))
        return np.sort(rng.choice(len(self.pool), size=self.views_per_step, replace=False))

    def step(self):
        idx = self.choose(self.step_no)
        self.gw.views = [self.pool[i] for i in idx]
        self.opt.zero_grad()
        img = MirresRender.apply(self.gw, 1, self.seed + self.step_no, *scene_params(self.gw))
        tgt = torch.stack([self.targets[i] for i in idx])
        loss = ((img - tgt) ** 2).sum()
        loss.backward()
        self.opt.step()
        with torch.no_grad():
            # keep the materials in their valid range and the env non-negative
            self.scene.albedo.clamp_(0.0, 1.0)
            self.scene.roughness.clamp_(0.02, 1.0)
            self.scene.env.clamp_(min=0.0)
        # (the env texels changed in place: the next forward's refresh rebuilds the env tables)
        self.curve.append(float(loss.detach()))
        self.step_no += 1
        return self.curve[-1]

    @torch.no_grad()
    def eval_loss(self, n_views=None, seed=12345):
        """the L2 image loss of the current parameters on a fixed set of cameras (the first
        `n_views` of the pool, default views_per_step) with a fixed random stream: comparable
        across steps, free of the per-step camera choice"""
        chosen = self.gw.views
        idx = list(range(min(n_views or self.views_per_step, len(self.pool))))
        self.gw.views = [self.pool[i] for i in idx]
        images, _ = self.gw.render(launch=1, seed=seed)
        tot = 0.0
        for i, im in zip(idx, images):
            tot += float(((im - self.targets[i]) ** 2).sum())
        self.gw.views = chosen
        return tot

    def save(self, path):
        torch.save({"step": self.step_no, "curve": self.curve, "opt": self.opt.state_dict(),
                    "params": {k: getattr(self.scene, k).detach().clone() for k in TRAINED}}, path)

    def load(self, path):
        ck = torch.load(path, map_location=self.scene.albedo.device)
        with torch.no_grad():
            for k in TRAINED:
                getattr(self.scene, k).copy_(ck["params"][k])
        self.opt.load_state_dict(ck["opt"])
        self.step_no = int(ck["step"])
        self.curve = list(ck["curve"])
        M.mirres_bvh_refit(self.scene.handle)

    def close(self):
        for p in self.params:
            p.requires_grad_(False)
        for s in self.gw.scenes:
            s.close()
        if self.own_ctx:
            self.ctx.close()


def config4_setup(res=800, spp=8, bounces=4, pool=32, seed=0):
    """the config-4 problem: the config-2 scene as ground truth, a flat start, a pool of cameras
    on the upper hemisphere at res x res"""
    truth = synth.config2(seed=seed).scenes[0]
    init = copy.deepcopy(truth)
    init.albedo[:] = 0.5
    init.roughness[:] = 0.5
    init.env[:] = 1.0
    views = synth.hemisphere_views(pool, res, spp, bounces, seed + 7)
    return truth, init, views


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--res", type=int, default=800)
    ap.add_argument("--views", type=int, default=8, help="views per step")
    ap.add_argument("--pool", type=int, default=32, help="cameras the views are drawn from")
    ap.add_argument("--spp", type=int, default=8)
    ap.add_argument("--bounces", type=int, default=4)
    ap.add_argument("--lr", type=float, default=1e-2)
    ap.add_argument("--checkpoint", default=None, help="torch.save path, written every --every steps")
    ap.add_argument("--every", type=int, default=50)
    ap.add_argument("--resume", action="store_true")
    ap.add_argument("--out", default=None, help="JSON file for the loss curve")
    args = ap.parse_args()
    truth, init, views = config4_setup(args.res, args.spp, args.bounces, args.pool)
    loop = Loop(truth, init, views, args.views, args.lr, synth.config2().ris_m)
    if args.resume and args.checkpoint and os.path.exists(args.checkpoint):
        loop.load(args.checkpoint)
    eval0 = loop.eval_loss()
    t0 = time.perf_counter()
    while loop.step_no < args.steps:
        loop.step()
        if args.checkpoint and loop.step_no % args.every == 0:
            loop.save(args.checkpoint)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    out = {"steps": loop.step_no, "res": args.res, "views_per_step": args.views, "spp": args.spp,
           "bounces": args.bounces, "lr": args.lr, "seconds": dt, "eval_loss": [eval0, loop.eval_loss()],
           "curve": loop.curve}
    if args.out:
        with open(args.out, "w") as f:
            json.dump(out, f)
    print(json.dumps({k: v for k, v in out.items() if k != "curve"} | {"first": loop.curve[:3], "last": loop.curve[-3:]}))
    loop.close()


if __name__ == "__main__":
    main()
