"""PyTorch-facing helpers over the C ABI: device-resident scenes and an autograd Function.

PyTorch supplies device memory and streams only; every step of the path runs in libmirres.
"""
from __future__ import annotations

import json
import os

import torch

from . import mirres as M


def _dev(a, dtype, device):
    return torch.as_tensor(a).to(device=device, dtype=dtype).contiguous()


class DeviceScene:
    """Scene inputs as CUDA tensors plus the library scene handle (LBVH and env tables built)."""

    def __init__(self, ctx: M.Context, scene, device="cuda", builder=M.MIRRES_BVH_LBVH,
                 normals=M.MIRRES_NORMALS_FACE, traversal=M.MIRRES_TRAVERSAL_BINARY):
        self.device = torch.device(device)
        self.verts = _dev(scene.verts, torch.float32, self.device)
        self.tris = _dev(scene.tris, torch.int32, self.device)
        self.tri_uv = _dev(scene.tri_uv, torch.float32, self.device)
        self.albedo = _dev(scene.albedo, torch.float32, self.device)
        self.roughness = _dev(scene.roughness, torch.float32, self.device)
        self.metallic = _dev(scene.metallic, torch.float32, self.device)
        self.env = _dev(scene.env, torch.float32, self.device)
        self.handle = M.mirres_scene_create(ctx, self.verts, self.tris, self.tri_uv, self.albedo, self.roughness,
                                            self.metallic, self.env)
        M.mirres_bvh_set_builder(self.handle, builder)
        M.mirres_scene_set_normals(self.handle, normals)
        M.mirres_scene_set_traversal(self.handle, traversal)
        M.mirres_bvh_build(self.handle)
        self._versions = self._param_versions()

    def _param_versions(self):
        return (self.verts._version, self.env._version)

    def refresh(self):
        """Refit the LBVH and rebuild the env tables if vertices or env changed in place."""
        v = self._param_versions()
        if v != self._versions:
            M.mirres_bvh_refit(self.handle)
            self._versions = v

    def params(self):
        return dict(albedo=self.albedo, roughness=self.roughness, metallic=self.metallic, env=self.env,
                    verts=self.verts)

    def close(self):
        self.handle.close()


class GpuWorkload:
    """A synthetic workload resident on one GPU."""

    def __init__(self, workload, device=0, ctx=None, builder=M.MIRRES_BVH_LBVH, normals=M.MIRRES_NORMALS_FACE,
                 traversal=M.MIRRES_TRAVERSAL_BINARY):
        self.workload = workload
        self.ctx = ctx or M.mirres_context_create(device)
        self.device = torch.device("cuda", device)
        self.scenes = [DeviceScene(self.ctx, s, self.device, builder=builder, normals=normals, traversal=traversal)
                       for s in workload.scenes]
        self.views = list(workload.views)
        self.samples = workload.samples

    def new_images(self):
        return [torch.empty((v.height, v.width, 3), device=self.device, dtype=torch.float32) for v in self.views]

    def new_tape(self, grad_mode=0):
        n = M.mirres_tape_bytes_mode(self.views, grad_mode)
        return torch.empty(n // 4, device=self.device, dtype=torch.int32)

    def params(self, launch=0, seed=None, block=0, blocks_per_sm=0, flags=0, grad_mode=0, reuse=(0, 0), temporal=0,
               temporal_cap=20, history=None, max_visits=0):
        s = self.workload.seed if seed is None else seed
        return M.make_params(self.workload.ris_m, s, launch, block, blocks_per_sm, grad_mode=grad_mode, flags=flags,
                             reuse=reuse, temporal=temporal, temporal_cap=temporal_cap, history=history,
                             max_visits=max_visits)

    def new_history(self):
        """reservoir history for temporal reuse (kept across renders of the same views)"""
        return torch.zeros(M.mirres_reuse_history_bytes(self.views) // 4, device=self.device, dtype=torch.int32)

    def render(self, launch=0, images=None, tape=None, seed=None, block=0, blocks_per_sm=0, flags=0, stream=None,
               grad_mode=0, reuse=(0, 0), temporal=0, temporal_cap=20, history=None, max_visits=0):
        """Forward render; grad_mode 1 (FULL) also records every vertex for the FULL adjoint;
        reuse = (neighbours, radius) turns on spatial reuse at the primary vertex; temporal = 1
        records the reservoir history into `history`, 2 merges it first. Scenes whose vertices
        or env were changed in place are refitted (and their env tables rebuilt) first."""
        for s in self.scenes:
            s.refresh()
        images = images if images is not None else self.new_images()
        tape = tape if tape is not None else self.new_tape(grad_mode)
        M.mirres_render(self.ctx, [s.handle for s in self.scenes], self.views,
                        self.params(launch, seed, block, blocks_per_sm, flags, grad_mode, reuse, temporal,
                                    temporal_cap, history, max_visits), images, tape, stream)
        return images, tape

    def tune_key(self):
        v = self.views
        return "|".join([torch.cuda.get_device_name(self.device), self.workload.name, f"{len(v)} views",
                         f"{len(self.scenes)} scenes", f"{self.samples} samples", f"M={self.workload.ris_m}"])

    def autotune(self, tape=None, budget=32_000_000, cache=None):
        """Pick the launch shapes of the batched launches: from the JSON cache if this (GPU,
        workload shape) was tuned before, else by timing them -- the persistent kernel's compiled
        variants and chunk (mirres_autotune) and the wavefront's wave size and per-stage block
        shape (mirres_autotune_wave) -- and caching both."""
        path = cache or os.environ.get("MIRRES_TUNE_CACHE") or os.path.join(
            os.path.dirname(os.path.abspath(__file__)), "_build", "tune_cache.json")
        key = self.tune_key()
        data = {}
        if os.path.exists(path):
            try:
                data = json.load(open(path))
            except (OSError, ValueError):
                data = {}
        if key in data and "wave" in data[key]:
            e = data[key]
            M.mirres_set_launch(self.ctx, e["block"], e["blocks_per_sm"], e["chunk"])
            M.mirres_set_wave_shape(self.ctx, e["wave"])
            return dict(e, cached=True)
        tape = tape if tape is not None else self.new_tape()
        scenes = [s.handle for s in self.scenes]
        res = M.mirres_autotune(self.ctx, scenes, self.views, self.params(1), tape, budget)
        wave = M.mirres_autotune_wave(self.ctx, scenes, self.views, self.params(1), tape, budget)
        res["wave_ms"] = wave.pop("ms")
        res["wave"] = wave
        data[key] = res
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1)
        os.replace(tmp, path)
        return dict(res, cached=False)

    def zero_grads(self):
        out = []
        for s in self.scenes:
            out.append({k: torch.zeros_like(t) for k, t in s.params().items()})
        return out

    def backward(self, d_images, tape, grads=None, launch=0, seed=None, stream=None, grad_mode=0):
        """Adjoint from the tape of a render with the same seed (and grad_mode)."""
        grads = grads if grads is not None else self.zero_grads()
        M.mirres_backward(self.ctx, [s.handle for s in self.scenes], self.views,
                          self.params(launch, seed, grad_mode=grad_mode), d_images, tape, grads, stream)
        return grads

    def light_demod(self, tape, launch=0, seed=None, grad_mode=0, demod=None, stream=None):
        """demodulated lighting c_d + c_s and coverage per pixel ([H][W][4] per view) of the
        render that wrote `tape` (the monochrome light regulariser's input)"""
        demod = demod if demod is not None else [
            torch.empty((v.height, v.width, 4), device=self.device, dtype=torch.float32) for v in self.views]
        M.mirres_light_demod(self.ctx, [s.handle for s in self.scenes], self.views,
                             self.params(launch, seed, grad_mode=grad_mode), tape, demod, stream)
        return demod

    def light_loss(self, demod, refs, weight=1.0, loss=None, stream=None):
        """adds weight * L_light to loss[0]; returns (loss, d_demod per view)"""
        loss = loss if loss is not None else torch.zeros(1, device=self.device, dtype=torch.float32)
        d = [torch.empty((v.height, v.width, 3), device=self.device, dtype=torch.float32) for v in self.views]
        M.mirres_light_loss(self.ctx, self.views, demod, refs, weight, loss, d, stream)
        return loss, d

    def light_backward(self, d_demod, tape, grads=None, launch=0, seed=None, grad_mode=0, stream=None):
        grads = grads if grads is not None else self.zero_grads()
        M.mirres_light_backward(self.ctx, [s.handle for s in self.scenes], self.views,
                                self.params(launch, seed, grad_mode=grad_mode), d_demod, tape, grads, stream)
        return grads

    def close(self):
        for s in self.scenes:
            s.close()
        self.ctx.close()


class MirresRender(torch.autograd.Function):
    """images = MirresRender.apply(gw, launch, seed, *params)

    params = (albedo, roughness, metallic, env, verts) of every scene of the GpuWorkload, scene
    after scene: the tensors the scenes borrow (updated in place by the optimiser). Returns the
    images of all views stacked when they share one size, else concatenated flat ([sum H W, 3]).
    Backward is the PRIMARY-mode adjoint of the paper (indirect rays detached), replayed from the
    tape the forward wrote, for every scene at once.
    """

    NAMES = ("albedo", "roughness", "metallic", "env", "verts")

    @staticmethod
    def forward(ctx, gw, launch, seed, *params):
        if len(params) != 5 * len(gw.scenes):
            raise ValueError("expected (albedo, roughness, metallic, env, verts) for every scene")
        for si, scene in enumerate(gw.scenes):
            for k, name in enumerate(MirresRender.NAMES):
                if params[5 * si + k].data_ptr() != getattr(scene, name).data_ptr():
                    raise ValueError(f"scene {si}: {name} is not the tensor the scene borrows")
            scene.refresh()
        images, tape = gw.render(launch=launch, seed=seed)
        ctx.gw, ctx.launch, ctx.seed, ctx.tape = gw, launch, seed, tape
        ctx.shapes = [tuple(im.shape) for im in images]
        if len(set(ctx.shapes)) == 1:
            ctx.stacked = True
            return torch.stack(images)
        ctx.stacked = False
        return torch.cat([im.reshape(-1, 3) for im in images])

    @staticmethod
    def backward(ctx, grad_images):
        gw = ctx.gw
        if ctx.stacked:
            d = [grad_images[i].contiguous() for i in range(grad_images.shape[0])]
        else:
            d, off = [], 0
            for shp in ctx.shapes:
                n = shp[0] * shp[1]
                d.append(grad_images[off:off + n].reshape(shp).contiguous())
                off += n
        g = gw.backward(d, ctx.tape, launch=ctx.launch, seed=ctx.seed)
        out = [None, None, None]
        for gs in g:
            out += [gs[name] for name in MirresRender.NAMES]
        return tuple(out)


def scene_params(gw):
    """the flat parameter list MirresRender.apply expects after (gw, launch, seed)"""
    return [getattr(s, name) for s in gw.scenes for name in MirresRender.NAMES]
