"""Thin Python binding of libmirres (include/mirres.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no arithmetic of the
method: tensors are passed as device pointers, views / params as the C structs. Streams
default to PyTorch's current stream. Importing this module never falls back to anything: if
the shared library is missing, calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import torch

from . import build as _build

__all__ = ["MirresError", "Context", "Scene", "View", "Params", "Grads", "make_view", "make_params",
           "mirres_context_create", "mirres_context_destroy", "mirres_scene_create", "mirres_scene_destroy",
           "mirres_scene_validate", "mirres_scene_set_traversal", "MIRRES_TRAVERSAL_BINARY", "MIRRES_TRAVERSAL_WIDE",
           "mirres_bvh_build", "mirres_bvh_refit", "mirres_bvh_set_builder", "MIRRES_BVH_LBVH", "MIRRES_BVH_PLOC",
           "mirres_scene_set_normals", "MIRRES_NORMALS_FACE", "MIRRES_NORMALS_INTERPOLATED", "mirres_tape_bytes", "mirres_tape_bytes_mode",
           "mirres_reuse_history_bytes", "mirres_render",
           "mirres_render_noalloc",
           "mirres_autotune", "mirres_set_launch", "mirres_stage_times", "mirres_stage_trace", "mirres_backward",
           "WaveShape", "mirres_set_wave_shape", "mirres_get_wave_shape", "mirres_autotune_wave",
           "mirres_l2_loss", "mirres_trace", "mirres_bvh_export", "mirres_env_export", "mirres_env_export_flat",
           "mirres_get_counters",
           "mirres_get_work_counters", "EawtParams", "mirres_eawt_record_bytes", "mirres_gbuffer", "mirres_eawt",
           "mirres_eawt_backward", "mirres_eawt_batch", "mirres_eawt_batch_backward", "mirres_mesh_regularizers", "LkParams", "mirres_material_smoothness",
           "mirres_light_demod", "mirres_light_loss", "mirres_light_backward",
           "mirres_reset_counters", "mirres_last_error", "library_path", "mirres_peak_fp32", "mirres_peak_l2"]

# limits of mirres_render_noalloc (include/mirres.h)
MIRRES_TAPE_BYTES_PER_SAMPLE = 68  # 17 words per path sample, one array per word
TAPE_WORDS = MIRRES_TAPE_BYTES_PER_SAMPLE // 4
MIRRES_TAPE_BYTES_PER_VERTEX = 36  # FULL mode: 9 words per later vertex
MIRRES_FULL_MAX_BOUNCES = 16
GRAD_PRIMARY, GRAD_FULL = 0, 1
MIRRES_BVH_LBVH, MIRRES_BVH_PLOC = 0, 1
MIRRES_NORMALS_FACE, MIRRES_NORMALS_INTERPOLATED = 0, 1
MIRRES_FLAG_STAGE_EVENTS, MIRRES_FLAG_COUNT_WORK, MIRRES_FLAG_RASTER, MIRRES_FLAG_BIN = 1, 2, 4, 8
MIRRES_TRAVERSAL_BINARY, MIRRES_TRAVERSAL_WIDE = 0, 1
MIRRES_NOALLOC_SCRATCH_BYTES = 512 * 1024
MIRRES_NOALLOC_MAX_VIEWS = 4096
MIRRES_NOALLOC_MAX_SCENES = 256

STATUS = {0: "MIRRES_OK", 1: "MIRRES_ERR_ARG", 2: "MIRRES_ERR_CUDA", 3: "MIRRES_ERR_OOM", 4: "MIRRES_ERR_TIMEOUT",
          5: "MIRRES_ERR_STATE"}


class MirresError(RuntimeError):
    def __init__(self, call, status, message):
        super().__init__(f"{call} -> {STATUS.get(status, status)}: {message}")
        self.status = status


class SceneDesc(C.Structure):
    _fields_ = [("verts", C.c_void_p), ("n_verts", C.c_int32), ("tris", C.c_void_p), ("n_tris", C.c_int32),
                ("tri_uv", C.c_void_p), ("albedo", C.c_void_p), ("roughness", C.c_void_p),
                ("metallic", C.c_void_p), ("tex_w", C.c_int32), ("tex_h", C.c_int32), ("env", C.c_void_p),
                ("env_w", C.c_int32), ("env_h", C.c_int32)]


class View(C.Structure):
    _fields_ = [("K", C.c_float * 4), ("c2w", C.c_float * 12), ("width", C.c_int32), ("height", C.c_int32),
                ("spp", C.c_int32), ("bounces", C.c_int32), ("scene", C.c_int32)]


class Params(C.Structure):
    _fields_ = [("ris_m", C.c_int32), ("seed_lo", C.c_uint32), ("seed_hi", C.c_uint32), ("grad_mode", C.c_int32),
                ("launch", C.c_int32), ("block", C.c_int32), ("blocks_per_sm", C.c_int32),
                ("flags", C.c_int32), ("reuse_k", C.c_int32), ("reuse_radius", C.c_int32),
                ("temporal", C.c_int32), ("temporal_cap", C.c_int32), ("reuse_history", C.c_void_p),
                ("reuse_history_bytes", C.c_uint64), ("max_visits", C.c_int32)]


class WaveShape(C.Structure):
    _fields_ = [("wave_log2", C.c_int32), ("block", C.c_int32 * 4), ("blocks_per_sm", C.c_int32 * 4),
                ("branches", C.c_int32)]


WAVE_STAGES = ("closest", "shade", "shadow", "raygen")  # index order of WaveShape.block / blocks_per_sm


def _shape_dict(w: WaveShape):
    return dict(wave_log2=int(w.wave_log2), block=[int(x) for x in w.block],
                blocks_per_sm=[int(x) for x in w.blocks_per_sm], branches=int(w.branches))


def _shape_struct(d):
    return WaveShape(int(d["wave_log2"]), (C.c_int32 * 4)(*[int(x) for x in d["block"]]),
                     (C.c_int32 * 4)(*[int(x) for x in d["blocks_per_sm"]]), int(d.get("branches", 1)))


class EawtParams(C.Structure):
    _fields_ = [("sigma_rt", C.c_float), ("sigma_n", C.c_float), ("sigma_x", C.c_float), ("levels", C.c_int32)]


class LkParams(C.Structure):
    _fields_ = [("sigma", C.c_float), ("w_albedo", C.c_float), ("w_roughness", C.c_float), ("seed_lo", C.c_uint32),
                ("seed_hi", C.c_uint32), ("w_normal", C.c_float)]


class Grads(C.Structure):
    _fields_ = [("albedo", C.c_void_p), ("roughness", C.c_void_p), ("metallic", C.c_void_p), ("env", C.c_void_p),
                ("verts", C.c_void_p)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_build.LIB):
                raise RuntimeError("libmirres.so is not built (run __graft_entry__.build()); there is no fallback")
            L = C.CDLL(_build.LIB)
            vp, i32, i64, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t
            st = C.c_int
            sig = {
                "mirres_context_create": (st, [i32, C.POINTER(vp)]),
                "mirres_context_destroy": (st, [vp]),
                "mirres_scene_create": (st, [vp, C.POINTER(SceneDesc), C.POINTER(vp)]),
                "mirres_scene_destroy": (st, [vp]),
                "mirres_scene_validate": (st, [vp, vp]),
                "mirres_bvh_build": (st, [vp, vp]),
                "mirres_bvh_refit": (st, [vp, vp]),
                "mirres_bvh_set_builder": (st, [vp, i32]),
                "mirres_scene_set_traversal": (st, [vp, i32]),
                "mirres_scene_set_normals": (st, [vp, i32]),
                "mirres_tape_bytes": (sz, [C.POINTER(View), i32]),
                "mirres_tape_bytes_mode": (sz, [C.POINTER(View), i32, i32]),
                "mirres_reuse_history_bytes": (sz, [C.POINTER(View), i32]),
                "mirres_render": (st, [vp, C.POINTER(vp), i32, C.POINTER(View), i32, C.POINTER(Params),
                                       C.POINTER(vp), vp, sz, vp]),
                "mirres_autotune": (st, [vp, C.POINTER(vp), i32, C.POINTER(View), i32, C.POINTER(Params), vp, sz,
                                         C.c_uint64, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32),
                                         C.POINTER(C.c_float), vp]),
                "mirres_set_launch": (st, [vp, i32, i32, i32]),
                "mirres_set_wave_shape": (st, [vp, C.POINTER(WaveShape)]),
                "mirres_get_wave_shape": (st, [vp, C.POINTER(WaveShape)]),
                "mirres_autotune_wave": (st, [vp, C.POINTER(vp), i32, C.POINTER(View), i32, C.POINTER(Params), vp,
                                              sz, C.c_uint64, C.POINTER(WaveShape), C.POINTER(C.c_float), vp]),
                "mirres_stage_times": (st, [vp, C.POINTER(C.c_double), C.POINTER(i32)]),
                "mirres_stage_trace": (st, [vp, i32, C.POINTER(C.c_float), C.POINTER(i32), C.POINTER(i32),
                                            C.POINTER(i32)]),
                "mirres_render_noalloc": (st, [C.POINTER(vp), i32, C.POINTER(View), i32, C.POINTER(Params),
                                               C.POINTER(vp), vp, sz, vp]),
                "mirres_backward": (st, [vp, C.POINTER(vp), i32, C.POINTER(View), i32, C.POINTER(Params),
                                         C.POINTER(vp), vp, sz, C.POINTER(Grads), vp]),
                "mirres_l2_loss": (st, [vp, vp, i64, vp, vp, vp]),
                "mirres_trace": (st, [vp, vp, vp, vp, i64, i32, vp, vp, vp]),
                "mirres_eawt_record_bytes": (sz, [i32, i32, i32]),
                "mirres_gbuffer": (st, [vp, vp, C.POINTER(View), vp, vp, vp]),
                "mirres_eawt": (st, [vp, vp, vp, vp, i32, i32, C.POINTER(EawtParams), vp, vp, sz, vp]),
                "mirres_eawt_backward": (st, [vp, vp, vp, vp, i32, i32, C.POINTER(EawtParams), vp, sz, vp, vp]),
                "mirres_eawt_batch": (st, [vp, i32, vp, vp, vp, i32, i32, C.POINTER(EawtParams), vp, vp, sz, vp]),
                "mirres_eawt_batch_backward": (st, [vp, i32, vp, vp, vp, i32, i32, C.POINTER(EawtParams), vp, sz, vp,
                                                    vp]),
                "mirres_mesh_regularizers": (st, [vp, vp, vp, C.c_float, C.c_float, vp, vp, vp]),
                "mirres_material_smoothness": (st, [vp, vp, C.POINTER(View), i32, C.POINTER(LkParams), vp, vp, vp,
                                                    vp, vp]),
                "mirres_light_demod": (st, [vp, C.POINTER(vp), i32, C.POINTER(View), i32, C.POINTER(Params), vp,
                                            sz, C.POINTER(vp), vp]),
                "mirres_light_loss": (st, [vp, C.POINTER(View), i32, C.POINTER(vp), C.POINTER(vp), C.c_float, vp,
                                           C.POINTER(vp), vp]),
                "mirres_light_backward": (st, [vp, C.POINTER(vp), i32, C.POINTER(View), i32, C.POINTER(Params),
                                               C.POINTER(vp), vp, sz, C.POINTER(Grads), vp]),
                "mirres_bvh_export": (st, [vp, vp, vp, vp, vp, vp, vp, vp]),
                "mirres_env_export": (st, [vp, vp, vp, vp, vp, vp]),
                "mirres_env_export_flat": (st, [vp, vp, vp]),
                "mirres_get_counters": (st, [vp, C.POINTER(C.c_uint64)]),
                "mirres_get_work_counters": (st, [vp, C.POINTER(C.c_uint64)]),
                "mirres_reset_counters": (st, [vp]),
                "mirres_last_error": (C.c_char_p, []),
                "mirres_peak_fp32": (C.c_int, [i32, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
                "mirres_peak_l2": (C.c_int, [C.c_uint64, i32, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def mirres_last_error() -> str:
    return lib().mirres_last_error().decode()


def _check(call, status):
    if status != 0:
        raise MirresError(call, status, mirres_last_error())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


class Context:
    def __init__(self, handle, device):
        self.handle = handle
        self.device = device

    def close(self):
        if self.handle:
            _check("mirres_context_destroy", lib().mirres_context_destroy(self.handle))
            self.handle = None


class Scene:
    """A scene handle plus references to the borrowed tensors (kept alive here)."""

    def __init__(self, ctx, handle, tensors):
        self.ctx = ctx
        self.handle = handle
        self.tensors = tensors

    def close(self):
        if self.handle:
            _check("mirres_scene_destroy", lib().mirres_scene_destroy(self.handle))
            self.handle = None


def make_view(K, c2w, width, height, spp, bounces, scene=0) -> View:
    return View((C.c_float * 4)(*[float(x) for x in K]), (C.c_float * 12)(*[float(x) for x in c2w]), int(width),
                int(height), int(spp), int(bounces), int(scene))


def make_params(ris_m, seed=0, launch=0, block=0, blocks_per_sm=0, grad_mode=0, flags=0, reuse=(0, 0), temporal=0,
                temporal_cap=20, history=None, max_visits=0) -> Params:
    """reuse = (neighbours, radius) of the spatial reuse at the primary vertex, (0, 0) = off;
    temporal = 1 records the reservoir history into `history` (a CUDA tensor of
    mirres_reuse_history_bytes), 2 merges it first; max_visits = iteration cap of one ray
    traversal (0 = the library's default)"""
    hb = 0 if history is None else history.numel() * history.element_size()
    return Params(int(ris_m), seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF, int(grad_mode), int(launch), int(block),
                  int(blocks_per_sm), int(flags), int(reuse[0]), int(reuse[1]), int(temporal), int(temporal_cap),
                  None if history is None else history.data_ptr(), int(hb), int(max_visits))


def _views(views):
    arr = (View * len(views))()
    for i, v in enumerate(views):
        arr[i] = v if isinstance(v, View) else make_view(v.K, v.c2w, v.width, v.height, v.spp, v.bounces,
                                                         getattr(v, "scene", 0))
    return arr


def mirres_context_create(device: int = 0) -> Context:
    h = C.c_void_p()
    _check("mirres_context_create", lib().mirres_context_create(int(device), C.byref(h)))
    return Context(h, device)


def mirres_context_destroy(ctx: Context):
    ctx.close()


def mirres_scene_create(ctx: Context, verts, tris, tri_uv, albedo, roughness, metallic, env) -> Scene:
    ts = dict(verts=verts, tris=tris, tri_uv=tri_uv, albedo=albedo, roughness=roughness, metallic=metallic, env=env)
    for k, t in ts.items():
        want = torch.int32 if k == "tris" else torch.float32
        if t.dtype != want:
            raise ValueError(f"{k} must be {want}")
    d = SceneDesc(_ptr(verts), verts.shape[0], _ptr(tris), tris.shape[0], _ptr(tri_uv), _ptr(albedo),
                  _ptr(roughness), _ptr(metallic), albedo.shape[1], albedo.shape[0], _ptr(env), env.shape[1],
                  env.shape[0])
    h = C.c_void_p()
    _check("mirres_scene_create", lib().mirres_scene_create(ctx.handle, C.byref(d), C.byref(h)))
    return Scene(ctx, h, ts)


def mirres_scene_destroy(scene: Scene):
    scene.close()


def mirres_scene_validate(scene: Scene, stream=None):
    _check("mirres_scene_validate", lib().mirres_scene_validate(scene.handle, _stream(stream)))


def mirres_bvh_build(scene: Scene, stream=None):
    _check("mirres_bvh_build", lib().mirres_bvh_build(scene.handle, _stream(stream)))


def mirres_bvh_refit(scene: Scene, stream=None):
    _check("mirres_bvh_refit", lib().mirres_bvh_refit(scene.handle, _stream(stream)))


def mirres_scene_set_traversal(scene: Scene, mode: int):
    _check("mirres_scene_set_traversal", lib().mirres_scene_set_traversal(scene.handle, int(mode)))


def mirres_bvh_set_builder(scene: Scene, builder: int):
    _check("mirres_bvh_set_builder", lib().mirres_bvh_set_builder(scene.handle, int(builder)))


def mirres_scene_set_normals(scene: Scene, mode: int):
    _check("mirres_scene_set_normals", lib().mirres_scene_set_normals(scene.handle, int(mode)))


def mirres_tape_bytes(views) -> int:
    vs = _views(views)
    return int(lib().mirres_tape_bytes(vs, len(vs)))


def mirres_reuse_history_bytes(views) -> int:
    vs = _views(views)
    return int(lib().mirres_reuse_history_bytes(vs, len(vs)))


def mirres_tape_bytes_mode(views, grad_mode) -> int:
    vs = _views(views)
    return int(lib().mirres_tape_bytes_mode(vs, len(vs), int(grad_mode)))


def mirres_render(ctx: Context, scenes, views, params: Params, images, tape=None, stream=None):
    vs = _views(views)
    sc = (C.c_void_p * len(scenes))(*[s.handle.value for s in scenes])
    im = (C.c_void_p * len(images))(*[_ptr(t).value for t in images])
    nbytes = 0 if tape is None else tape.numel() * tape.element_size()
    _check("mirres_render", lib().mirres_render(ctx.handle, sc, len(scenes), vs, len(vs), C.byref(params), im,
                                                _ptr(tape), nbytes, _stream(stream)))


def mirres_autotune(ctx: Context, scenes, views, params: Params, tape, budget_samples=0, stream=None):
    """Returns dict(block, blocks_per_sm, chunk, ms) of the fastest persistent launch."""
    vs = _views(views)
    sc = (C.c_void_p * len(scenes))(*[s.handle.value for s in scenes])
    b, m, c, ms = C.c_int32(), C.c_int32(), C.c_int32(), C.c_float()
    nbytes = tape.numel() * tape.element_size()
    _check("mirres_autotune", lib().mirres_autotune(ctx.handle, sc, len(scenes), vs, len(vs), C.byref(params),
                                                    _ptr(tape), nbytes, int(budget_samples), C.byref(b), C.byref(m),
                                                    C.byref(c), C.byref(ms), _stream(stream)))
    return dict(block=b.value, blocks_per_sm=m.value, chunk=c.value, ms=ms.value)


def mirres_set_launch(ctx: Context, block, blocks_per_sm, chunk):
    _check("mirres_set_launch", lib().mirres_set_launch(ctx.handle, int(block), int(blocks_per_sm), int(chunk)))


def mirres_set_wave_shape(ctx: Context, shape=None):
    """shape = dict(wave_log2, block[4], blocks_per_sm[4], branches=1) (stages in WAVE_STAGES order),
    None = default"""
    w = None if shape is None else C.byref(_shape_struct(shape))
    _check("mirres_set_wave_shape", lib().mirres_set_wave_shape(ctx.handle, w))


def mirres_get_wave_shape(ctx: Context):
    w = WaveShape()
    _check("mirres_get_wave_shape", lib().mirres_get_wave_shape(ctx.handle, C.byref(w)))
    return _shape_dict(w)


def mirres_autotune_wave(ctx: Context, scenes, views, params: Params, tape, budget_samples=0, stream=None):
    """Tunes the batched wavefront's launch shape; returns dict(wave_log2, block, blocks_per_sm,
    branches, ms)."""
    vs = _views(views)
    sc = (C.c_void_p * len(scenes))(*[s.handle.value for s in scenes])
    w, ms = WaveShape(), C.c_float()
    nbytes = tape.numel() * tape.element_size()
    _check("mirres_autotune_wave", lib().mirres_autotune_wave(ctx.handle, sc, len(scenes), vs, len(vs),
                                                              C.byref(params), _ptr(tape), nbytes,
                                                              int(budget_samples), C.byref(w), C.byref(ms),
                                                              _stream(stream)))
    return dict(_shape_dict(w), ms=ms.value)


def mirres_stage_times(ctx: Context):
    """(ms, launches) per stage of the last event-recording batched render: closest, shade, shadow, raygen."""
    ms = (C.c_double * 4)()
    n = (C.c_int32 * 4)()
    _check("mirres_stage_times", lib().mirres_stage_times(ctx.handle, ms, n))
    names = ("closest", "shade", "shadow", "raygen")
    return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(names)}


def mirres_stage_trace(ctx: Context):
    """every stage launch of the last event-recording batched render, in issue order:
    list of (stage name, bounce (-1: ray generation), ms)"""
    n = C.c_int32()
    lib().mirres_stage_trace(ctx.handle, 0, None, None, None, C.byref(n))
    cap = n.value
    ms, stg, bnc = (C.c_float * max(cap, 1))(), (C.c_int32 * max(cap, 1))(), (C.c_int32 * max(cap, 1))()
    _check("mirres_stage_trace", lib().mirres_stage_trace(ctx.handle, cap, ms, stg, bnc, C.byref(n)))
    names = ("closest", "shade", "shadow", "raygen")
    return [(names[stg[i]], int(bnc[i]), float(ms[i])) for i in range(min(cap, n.value))]


def mirres_render_noalloc(scenes, views, params: Params, images, tape, stream=None):
    vs = _views(views)
    sc = (C.c_void_p * len(scenes))(*[s.handle.value for s in scenes])
    im = (C.c_void_p * len(images))(*[_ptr(t).value for t in images])
    nbytes = 0 if tape is None else tape.numel() * tape.element_size()
    _check("mirres_render_noalloc", lib().mirres_render_noalloc(sc, len(scenes), vs, len(vs), C.byref(params), im,
                                                                _ptr(tape), nbytes, _stream(stream)))


def mirres_backward(ctx: Context, scenes, views, params: Params, d_images, tape, grads, stream=None):
    """grads: list (one per scene) of dicts with optional albedo/roughness/metallic/env/verts tensors."""
    vs = _views(views)
    sc = (C.c_void_p * len(scenes))(*[s.handle.value for s in scenes])
    di = (C.c_void_p * len(d_images))(*[_ptr(t).value for t in d_images])
    ga = (Grads * len(scenes))()
    for i, g in enumerate(grads):
        ga[i] = Grads(*[_ptr(g.get(k)) for k in ("albedo", "roughness", "metallic", "env", "verts")])
    nbytes = tape.numel() * tape.element_size()
    _check("mirres_backward", lib().mirres_backward(ctx.handle, sc, len(scenes), vs, len(vs), C.byref(params), di,
                                                    _ptr(tape), nbytes, ga, _stream(stream)))


def mirres_light_demod(ctx: Context, scenes, views, params: Params, tape, demod, stream=None):
    """demodulated lighting of the render that wrote `tape`: demod[v] float32 [H][W][4] CUDA tensors"""
    vs = _views(views)
    sc = (C.c_void_p * len(scenes))(*[s.handle.value for s in scenes])
    out = (C.c_void_p * len(demod))(*[_ptr(t).value for t in demod])
    nbytes = tape.numel() * tape.element_size()
    _check("mirres_light_demod", lib().mirres_light_demod(ctx.handle, sc, len(scenes), vs, len(vs), C.byref(params),
                                                          _ptr(tape), nbytes, out, _stream(stream)))


def mirres_light_loss(ctx: Context, views, demod, ref_images, weight=1.0, loss=None, d_demod=None, stream=None):
    """L_light from the demodulated lighting: adds weight * L_light to loss[0] and writes d_demod[v] [H][W][3]"""
    vs = _views(views)
    c = (C.c_void_p * len(demod))(*[_ptr(t).value for t in demod])
    r = (C.c_void_p * len(ref_images))(*[_ptr(t).value for t in ref_images])
    d = None if d_demod is None else (C.c_void_p * len(d_demod))(*[_ptr(t).value for t in d_demod])
    _check("mirres_light_loss", lib().mirres_light_loss(ctx.handle, vs, len(vs), c, r, float(weight), _ptr(loss), d,
                                                        _stream(stream)))


def mirres_light_backward(ctx: Context, scenes, views, params: Params, d_demod, tape, grads, stream=None):
    """adjoint of the demodulated lighting; grads as for mirres_backward (accumulated)"""
    vs = _views(views)
    sc = (C.c_void_p * len(scenes))(*[s.handle.value for s in scenes])
    di = (C.c_void_p * len(d_demod))(*[_ptr(t).value for t in d_demod])
    ga = (Grads * len(scenes))()
    for i, g in enumerate(grads):
        ga[i] = Grads(*[_ptr(g.get(k)) for k in ("albedo", "roughness", "metallic", "env", "verts")])
    nbytes = tape.numel() * tape.element_size()
    _check("mirres_light_backward", lib().mirres_light_backward(ctx.handle, sc, len(scenes), vs, len(vs),
                                                                C.byref(params), di, _ptr(tape), nbytes, ga,
                                                                _stream(stream)))


def mirres_l2_loss(image, ref, d_image=None, loss=None, stream=None):
    _check("mirres_l2_loss", lib().mirres_l2_loss(_ptr(image), _ptr(ref), image.numel(), _ptr(d_image), _ptr(loss),
                                                  _stream(stream)))


def mirres_trace(ctx: Context, scene: Scene, rays, hit_tri, hit_tuv=None, skip=None, any_hit=False, stream=None):
    _check("mirres_trace", lib().mirres_trace(ctx.handle, scene.handle, _ptr(rays), _ptr(skip), rays.shape[0],
                                              1 if any_hit else 0, _ptr(hit_tri), _ptr(hit_tuv), _stream(stream)))


def mirres_eawt_record_bytes(width, height, levels) -> int:
    return int(lib().mirres_eawt_record_bytes(int(width), int(height), int(levels)))


def mirres_gbuffer(ctx: Context, scene: Scene, view, normal, position, stream=None):
    """pixel-centre G-buffer of one view into [H][W][3] float32 CUDA tensors"""
    vs = _views([view])
    _check("mirres_gbuffer", lib().mirres_gbuffer(ctx.handle, scene.handle, vs, _ptr(normal), _ptr(position),
                                                  _stream(stream)))


def mirres_eawt(ctx: Context, image, normal, position, params: EawtParams, out, record, stream=None):
    H, W = image.shape[0], image.shape[1]
    _check("mirres_eawt", lib().mirres_eawt(ctx.handle, _ptr(image), _ptr(normal), _ptr(position), W, H,
                                            C.byref(params), _ptr(out), _ptr(record),
                                            record.numel() * record.element_size(), _stream(stream)))


def mirres_eawt_backward(ctx: Context, d_out, normal, position, params: EawtParams, record, d_image, stream=None):
    H, W = d_out.shape[0], d_out.shape[1]
    _check("mirres_eawt_backward", lib().mirres_eawt_backward(ctx.handle, _ptr(d_out), _ptr(normal), _ptr(position),
                                                              W, H, C.byref(params), _ptr(record),
                                                              record.numel() * record.element_size(), _ptr(d_image),
                                                              _stream(stream)))


def mirres_eawt_batch(ctx: Context, images, normal, position, params: EawtParams, out, record, stream=None):
    """the denoiser over a stack [N][H][W][3] of images of one size, one launch per level"""
    N, H, W = images.shape[0], images.shape[1], images.shape[2]
    _check("mirres_eawt_batch", lib().mirres_eawt_batch(ctx.handle, N, _ptr(images), _ptr(normal), _ptr(position), W,
                                                        H, C.byref(params), _ptr(out), _ptr(record),
                                                        record.numel() * record.element_size(), _stream(stream)))


def mirres_eawt_batch_backward(ctx: Context, d_out, normal, position, params: EawtParams, record, d_image,
                               stream=None):
    N, H, W = d_out.shape[0], d_out.shape[1], d_out.shape[2]
    _check("mirres_eawt_batch_backward", lib().mirres_eawt_batch_backward(
        ctx.handle, N, _ptr(d_out), _ptr(normal), _ptr(position), W, H, C.byref(params), _ptr(record),
        record.numel() * record.element_size(), _ptr(d_image), _stream(stream)))


def mirres_mesh_regularizers(ctx: Context, scene: Scene, rest_verts, w_smooth, w_offset, loss, grad_verts,
                             stream=None):
    """adds w_smooth L_smooth + w_offset L_offset of the scene's current vertices to loss[0] and its
    gradient to grad_verts (float32 CUDA tensors; either may be None)"""
    _check("mirres_mesh_regularizers", lib().mirres_mesh_regularizers(ctx.handle, scene.handle, _ptr(rest_verts),
                                                                      float(w_smooth), float(w_offset), _ptr(loss),
                                                                      _ptr(grad_verts), _stream(stream)))


def mirres_material_smoothness(ctx: Context, scene: Scene, view, view_index, params: LkParams, loss=None,
                               grad_albedo=None, grad_roughness=None, grad_verts=None, stream=None):
    """adds w_albedo L_albedo + w_roughness L_roughness + w_normal L_normal of one view's
    pixel-centre hits to loss[0] and its gradient to the texture and vertex gradients (float32
    CUDA tensors; any may be None)"""
    vs = _views([view])
    _check("mirres_material_smoothness", lib().mirres_material_smoothness(
        ctx.handle, scene.handle, vs, int(view_index), C.byref(params), _ptr(loss), _ptr(grad_albedo),
        _ptr(grad_roughness), _ptr(grad_verts), _stream(stream)))


def mirres_bvh_export(scene: Scene, keys=None, left=None, right=None, parent=None, lo=None, hi=None, stream=None):
    _check("mirres_bvh_export", lib().mirres_bvh_export(scene.handle, _ptr(keys), _ptr(left), _ptr(right),
                                                        _ptr(parent), _ptr(lo), _ptr(hi), _stream(stream)))


def mirres_env_export_flat(scene: Scene, thresholds, stream=None):
    _check("mirres_env_export_flat", lib().mirres_env_export_flat(scene.handle, _ptr(thresholds), _stream(stream)))


def mirres_env_export(scene: Scene, marg=None, cond=None, texel=None, total=None, stream=None):
    _check("mirres_env_export", lib().mirres_env_export(scene.handle, _ptr(marg), _ptr(cond), _ptr(texel),
                                                        _ptr(total), _stream(stream)))


def mirres_get_counters(ctx: Context):
    out = (C.c_uint64 * 8)()
    _check("mirres_get_counters", lib().mirres_get_counters(ctx.handle, out))
    return [int(x) for x in out]


def mirres_get_work_counters(ctx: Context):
    """[closest-hit box tests, closest-hit triangle tests, shadow box tests, shadow triangle tests]"""
    out = (C.c_uint64 * 4)()
    _check("mirres_get_work_counters", lib().mirres_get_work_counters(ctx.handle, out))
    return [int(x) for x in out]


def mirres_reset_counters(ctx: Context):
    _check("mirres_reset_counters", lib().mirres_reset_counters(ctx.handle))


def mirres_peak_fp32(iters: int = 1 << 18):
    """measured FP32 FMA rate of the current device: (FLOP/s, ms of the timed launch)"""
    f, ms = C.c_double(), C.c_double()
    e = lib().mirres_peak_fp32(int(iters), C.byref(f), C.byref(ms))
    if e != 0:
        raise RuntimeError(f"mirres_peak_fp32: CUDA error {e}")
    return f.value, ms.value


def mirres_peak_l2(nbytes: int = 32 << 20, passes: int = 400):
    """measured bandwidth of loads served by L2 on the current device: (bytes/s, ms)"""
    b, ms = C.c_double(), C.c_double()
    e = lib().mirres_peak_l2(int(nbytes), int(passes), C.byref(b), C.byref(ms))
    if e != 0:
        raise RuntimeError(f"mirres_peak_l2: CUDA error {e}")
    return b.value, ms.value
