"""ctypes wrapper around the FP64 CPU oracle (mirres_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the benchmark's
CPU-baseline / reference leg. The product (the CUDA library and its binding) never imports
this module.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mirres_oracle.c")
HDR = os.path.join(HERE, "mirres_oracle.h")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle.so")

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain C11, -ffp-contract=off, pthreads)."""
    os.makedirs(BUILD, exist_ok=True)
    stale = (not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(SRC), os.path.getmtime(HDR)))
    if force or stale:
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
               "-Wall", "-Wno-unused-function", "-o", tmp, SRC, "-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


class SceneDesc(C.Structure):
    _fields_ = [("verts", C.c_void_p), ("n_verts", C.c_int32), ("tris", C.c_void_p), ("n_tris", C.c_int32),
                ("tri_uv", C.c_void_p), ("albedo", C.c_void_p), ("roughness", C.c_void_p),
                ("metallic", C.c_void_p), ("tex_w", C.c_int32), ("tex_h", C.c_int32),
                ("env", C.c_void_p), ("env_w", C.c_int32), ("env_h", C.c_int32)]


class View(C.Structure):
    _fields_ = [("K", C.c_double * 4), ("c2w", C.c_double * 12), ("width", C.c_int32), ("height", C.c_int32),
                ("spp", C.c_int32), ("bounces", C.c_int32), ("view_index", C.c_int32)]


class Params(C.Structure):
    _fields_ = [("ris_m", C.c_int32), ("seed_lo", C.c_uint32), ("seed_hi", C.c_uint32),
                ("brdf_kind", C.c_int32), ("threads", C.c_int32), ("want_margin", C.c_int32),
                ("grad_mode", C.c_int32), ("reuse_k", C.c_int32), ("reuse_radius", C.c_int32),
                ("temporal", C.c_int32), ("temporal_cap", C.c_int32), ("history_in", C.c_void_p),
                ("history_out", C.c_void_p)]


GRAD_FIELDS = ("albedo", "roughness", "metallic", "env", "verts", "albedo_abs", "roughness_abs", "metallic_abs",
               "env_abs", "verts_abs", "albedo_sens", "roughness_sens", "metallic_sens", "verts_sens")


class Grads(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in GRAD_FIELDS]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            vp, i32, dbl = C.c_void_p, C.c_int32, C.c_double
            L.orc_scene_new.restype = vp
            L.orc_scene_new.argtypes = [C.POINTER(SceneDesc)]
            L.orc_scene_free.argtypes = [vp]
            L.orc_scene_tmin.restype = dbl
            L.orc_scene_tmin.argtypes = [vp]
            L.orc_scene_set_normals.argtypes = [vp, i32]
            L.orc_vertex_normals.argtypes = [vp, vp]
            L.orc_render.argtypes = [vp, C.POINTER(View), C.POINTER(Params), vp, i32, vp, vp, vp, vp]
            L.orc_render_samples.argtypes = [vp, C.POINTER(View), C.POINTER(Params), vp, i32, vp, vp, vp, vp, vp,
                                             vp]
            L.orc_sample_record.argtypes = [vp, C.POINTER(View), C.POINTER(Params), i32, i32, i32, vp]
            L.orc_backward.argtypes = [vp, C.POINTER(View), C.POINTER(Params), vp, i32, vp, C.POINTER(Grads), vp]
            L.orc_render_detached.argtypes = [vp, vp, C.POINTER(View), C.POINTER(Params), vp, i32, vp]
            L.orc_light_demod.argtypes = [vp, C.POINTER(View), C.POINTER(Params), vp, i32, vp, vp, vp]
            L.orc_light_backward.argtypes = [vp, C.POINTER(View), C.POINTER(Params), vp, i32, vp, C.POINTER(Grads),
                                             vp]
            L.orc_light_demod_detached.argtypes = [vp, vp, C.POINTER(View), C.POINTER(Params), vp, i32, vp]
            L.orc_trace.argtypes = [vp, vp, vp, i32, i32, vp, vp, vp]
            L.orc_lbvh.argtypes = [vp, vp, i32, vp, vp, vp, vp, vp, vp]
            L.orc_env_tables.restype = dbl
            L.orc_env_tables.argtypes = [vp, vp, vp, vp]
            L.orc_env_flat.argtypes = [vp, vp]
            L.orc_philox4x32_10.argtypes = [vp, vp, vp]
            L.orc_uniform.restype = dbl
            L.orc_uniform.argtypes = [C.c_uint32]
            L.orc_brdf_cos.argtypes = [vp, vp, vp, vp, dbl, dbl, i32, vp]
            L.orc_brdf_cos_grad.argtypes = [vp, vp, vp, vp, dbl, dbl, i32, vp, vp]
            L.orc_ggx_d.restype = dbl
            L.orc_ggx_d.argtypes = [dbl, dbl]
            L.orc_smith_g1.restype = dbl
            L.orc_smith_g1.argtypes = [dbl, dbl]
            L.orc_vndf_sample.argtypes = [vp, vp, dbl, dbl, dbl, vp]
            L.orc_vndf_pdf.restype = dbl
            L.orc_vndf_pdf.argtypes = [vp, vp, vp, dbl]
            L.orc_sample_continuation.restype = dbl
            L.orc_sample_continuation.argtypes = [vp, vp, vp, vp, dbl, dbl, i32, vp, vp]
            L.orc_pdf_continuation.restype = dbl
            L.orc_pdf_continuation.argtypes = [vp, vp, vp, vp, dbl, dbl, i32, vp]
            L.orc_env_sample.restype = dbl
            L.orc_env_sample.argtypes = [vp, vp, vp, vp]
            L.orc_env_pdf.restype = dbl
            L.orc_env_pdf.argtypes = [vp, vp]
            L.orc_env_texel.restype = i32
            L.orc_env_texel.argtypes = [vp, vp]
            L.orc_wrs.restype = i32
            L.orc_wrs.argtypes = [vp, vp, i32, vp]
            L.orc_taps_reach.restype = i32
            L.orc_taps_reach.argtypes = [i32, i32, dbl, dbl, dbl, dbl, vp]
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def _f64(x):
    return np.ascontiguousarray(x, dtype=np.float64)


class OracleScene:
    """FP64 copy of a scene plus the oracle's own median-split BVH and env tables."""

    def __init__(self, scene, normals=0):
        """normals: 0 face normals, 1 interpolated (area-weighted vertex normals)"""
        L = lib()
        self._keep = [np.ascontiguousarray(a) for a in (scene.verts, scene.tris, scene.tri_uv, scene.albedo,
                                                         scene.roughness, scene.metallic, scene.env)]
        v, t, uv, al, ro, me, env = self._keep
        d = SceneDesc(v.ctypes.data, v.shape[0], t.ctypes.data, t.shape[0], uv.ctypes.data, al.ctypes.data,
                      ro.ctypes.data, me.ctypes.data, al.shape[1], al.shape[0], env.ctypes.data, env.shape[1],
                      env.shape[0])
        self.h = L.orc_scene_new(C.byref(d))
        if not self.h:
            raise ValueError("oracle rejected the scene description")
        self.scene = scene
        self.normals = int(normals)
        L.orc_scene_set_normals(self.h, self.normals)
        self.tmin = L.orc_scene_tmin(self.h)

    def vertex_normals(self):
        out = np.zeros((self.scene.verts.shape[0], 3))
        lib().orc_vertex_normals(self.h, _p(out))
        return out

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_scene_free(self.h)
            self.h = None

    def env_tables(self):
        s = self.scene
        eh, ew = s.env.shape[:2]
        cond = np.zeros((eh, ew + 1))
        marg = np.zeros(eh + 1)
        prob = np.zeros((eh, ew))
        total = lib().orc_env_tables(self.h, _p(cond), _p(marg), _p(prob))
        return cond, marg, prob, total

    def env_flat(self):
        """the CDF over all texels (row-major) that the env draw inverts, [h w + 1]"""
        eh, ew = self.scene.env.shape[:2]
        out = np.zeros(eh * ew + 1)
        lib().orc_env_flat(self.h, _p(out))
        return out


def make_view(view, index):
    return View((C.c_double * 4)(*[float(x) for x in view.K]), (C.c_double * 12)(*[float(x) for x in view.c2w]),
                int(view.width), int(view.height), int(view.spp), int(view.bounces), int(index))


def make_params(ris_m, seed=0, threads=None, brdf_kind=0, want_margin=1, grad_mode=0, reuse=(0, 0), temporal=0,
                temporal_cap=20, history_in=None, history_out=None):
    if threads is None:
        threads = os.cpu_count() or 1
    return Params(int(ris_m), seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF, int(brdf_kind), int(threads),
                  int(want_margin), int(grad_mode), int(reuse[0]), int(reuse[1]), int(temporal), int(temporal_cap),
                  _p(history_in), _p(history_out))


def render(osc, view, index, ris_m, seed=0, pixels=None, threads=None, brdf_kind=0, margins=True,
           prim=False, reuse=(0, 0), temporal=0, temporal_cap=20, history=None):
    """Render pixels of one view. Returns dict(rgb [n,3], margin [n], prim [n,spp], counts [8]).
    With temporal reuse (1: record, 2: merge then record) also `history` [samples][5], the
    reservoir history of the view (input for 2; the output is a new array, unrendered
    samples copied from the input)."""
    L = lib()
    n = view.width * view.height if pixels is None else len(pixels)
    pix = None if pixels is None else np.ascontiguousarray(pixels, dtype=np.int32)
    rgb = np.zeros((n, 3))
    mg = np.zeros((n, 2)) if margins else None
    pr = np.zeros((n, view.spp), dtype=np.int32) if prim else None
    cnt = np.zeros(8, dtype=np.int64)
    v = make_view(view, index)
    hin = None if history is None else _f64(history).reshape(-1, 5)
    hout = None
    if temporal:
        hout = np.zeros((view.width * view.height * view.spp, 5)) if hin is None else hin.copy()
    p = make_params(ris_m, seed, threads, brdf_kind, int(margins), reuse=reuse, temporal=temporal,
                    temporal_cap=temporal_cap, history_in=hin, history_out=hout)
    rc = L.orc_render(osc.h, C.byref(v), C.byref(p), _p(pix), n, _p(rgb), _p(mg), _p(pr), _p(cnt))
    if rc:
        raise ValueError("orc_render rejected its arguments")
    return dict(rgb=rgb, margin=None if mg is None else mg[:, 0],
                kind=None if mg is None else mg[:, 1].astype(np.int32), prim=pr, counts=cnt, history=hout)


def sample_record(osc, view, index, ris_m, pixel, sample, seed=0):
    """one sample's path record: dict(prim_tri, sel, WV, Lind, rgb, y_texel, y, wc, p_ind, vertices
    [nv][12]: triangle, u, v, sel, texel, WV, wc (3), p_ind, has continuation, t)"""
    L = lib()
    out = np.zeros(18 + 12 * 16)
    v = make_view(view, index)
    p = make_params(ris_m, seed, 1, 0, 0)
    if L.orc_sample_record(osc.h, C.byref(v), C.byref(p), int(pixel % view.width), int(pixel // view.width),
                           int(sample), _p(out)):
        raise ValueError("orc_sample_record rejected its arguments")
    nv = int(out[17])
    return dict(prim_tri=int(out[0]), sel=int(out[1]), WV=out[2], Lind=out[3:6], rgb=out[6:9], y_texel=int(out[9]),
                y=out[10:13], wc=out[13:16], p_ind=out[16], vertices=out[18:18 + 12 * nv].reshape(nv, 12))


def render_samples(osc, view, index, ris_m, seed=0, pixels=None, threads=None, reuse=(0, 0)):
    """Render pixels of one view with every sample's own radiance, decision margin and FP32
    sensitivity: dict(rgb [n,3], margin [n], sample_rgb [n,spp,3], sample_margin [n,spp],
    sample_sens [n,spp], sens [n] = the mean of the samples'). reuse = (neighbours, radius) as
    for render (spatial reuse at the primary vertex)."""
    L = lib()
    n = view.width * view.height if pixels is None else len(pixels)
    pix = None if pixels is None else np.ascontiguousarray(pixels, dtype=np.int32)
    rgb = np.zeros((n, 3))
    mg = np.zeros((n, 2))
    srgb = np.zeros((n, view.spp, 3))
    smg = np.zeros((n, view.spp))
    sse = np.zeros((n, view.spp))
    cnt = np.zeros(8, dtype=np.int64)
    v = make_view(view, index)
    p = make_params(ris_m, seed, threads, 0, 1, reuse=reuse)
    if L.orc_render_samples(osc.h, C.byref(v), C.byref(p), _p(pix), n, _p(rgb), _p(mg), _p(srgb), _p(smg), _p(sse),
                            _p(cnt)):
        raise ValueError("orc_render_samples rejected its arguments")
    return dict(rgb=rgb, margin=mg[:, 0], sample_rgb=srgb, sample_margin=smg, sample_sens=sse,
                sens=sse.mean(axis=1), counts=cnt)


def backward(osc, view, index, ris_m, d_rgb, seed=0, pixels=None, threads=None, brdf_kind=0, want_abs=True,
             grad_mode=0, reuse=(0, 0), temporal=0, temporal_cap=20, history=None):
    """Adjoint of the listed pixels (grad_mode 0 PRIMARY, 1 FULL); returns dict of FP64
    gradients (and abs-sums)."""
    L = lib()
    s = osc.scene
    n = view.width * view.height if pixels is None else len(pixels)
    pix = None if pixels is None else np.ascontiguousarray(pixels, dtype=np.int32)
    d = _f64(d_rgb).reshape(n, 3)
    out = dict(albedo=np.zeros(s.albedo.shape), roughness=np.zeros(s.roughness.shape),
               metallic=np.zeros(s.metallic.shape), env=np.zeros(s.env.shape), verts=np.zeros(s.verts.shape))
    if want_abs:
        for k in list(out):
            out[k + "_abs"] = np.zeros(out[k].shape)
        for k in ("albedo", "roughness", "metallic", "verts"):
            out[k + "_sens"] = np.zeros(out[k].shape)
    g = Grads(*[_p(out.get(k)) for k in GRAD_FIELDS])
    cnt = np.zeros(8, dtype=np.int64)
    v = make_view(view, index)
    hin = None if history is None else _f64(history).reshape(-1, 5)
    p = make_params(ris_m, seed, threads, brdf_kind, 0, grad_mode, reuse, temporal, temporal_cap, hin, None)
    rc = L.orc_backward(osc.h, C.byref(v), C.byref(p), _p(pix), n, _p(d), C.byref(g), _p(cnt))
    if rc:
        raise ValueError("orc_backward rejected its arguments")
    out["counts"] = cnt
    return out


def render_detached(frozen, evaled, view, index, ris_m, seed=0, pixels=None, threads=None, brdf_kind=0,
                    grad_mode=0, reuse=(0, 0)):
    L = lib()
    n = view.width * view.height if pixels is None else len(pixels)
    pix = None if pixels is None else np.ascontiguousarray(pixels, dtype=np.int32)
    rgb = np.zeros((n, 3))
    v = make_view(view, index)
    p = make_params(ris_m, seed, threads, brdf_kind, 0, grad_mode, reuse)
    rc = L.orc_render_detached(frozen.h, evaled.h, C.byref(v), C.byref(p), _p(pix), n, _p(rgb))
    if rc:
        raise ValueError("orc_render_detached rejected its arguments")
    return rgb


def _grad_out(s, want_abs):
    out = dict(albedo=np.zeros(s.albedo.shape), roughness=np.zeros(s.roughness.shape),
               metallic=np.zeros(s.metallic.shape), env=np.zeros(s.env.shape), verts=np.zeros(s.verts.shape))
    if want_abs:
        for k in list(out):
            out[k + "_abs"] = np.zeros(out[k].shape)
        for k in ("albedo", "roughness", "metallic", "verts"):
            out[k + "_sens"] = np.zeros(out[k].shape)
    return out


def light_demod(osc, view, index, ris_m, seed=0, pixels=None, threads=None, margins=True, reuse=(0, 0)):
    """Demodulated lighting of the monochrome light regulariser (Appendix A, L_light) per
    pixel: dict(c [n,3] = mean over samples of c_d + c_s at the primary vertex, cov [n] =
    fraction of samples that hit a surface, margin [n] as render's)."""
    L = lib()
    n = view.width * view.height if pixels is None else len(pixels)
    pix = None if pixels is None else np.ascontiguousarray(pixels, dtype=np.int32)
    out = np.zeros((n, 4))
    mg = np.zeros((n, 2)) if margins else None
    cnt = np.zeros(8, dtype=np.int64)
    v = make_view(view, index)
    p = make_params(ris_m, seed, threads, 0, int(margins), reuse=reuse)
    if L.orc_light_demod(osc.h, C.byref(v), C.byref(p), _p(pix), n, _p(out), _p(mg), _p(cnt)):
        raise ValueError("orc_light_demod rejected its arguments")
    return dict(c=out[:, :3].copy(), cov=out[:, 3].copy(), margin=None if mg is None else mg[:, 0], counts=cnt)


def light_backward(osc, view, index, ris_m, d_c, seed=0, pixels=None, threads=None, want_abs=True, reuse=(0, 0)):
    """Adjoint of light_demod's c for the upstream gradient d_c [n,3]; dict of FP64 gradients."""
    L = lib()
    n = view.width * view.height if pixels is None else len(pixels)
    pix = None if pixels is None else np.ascontiguousarray(pixels, dtype=np.int32)
    d = _f64(d_c).reshape(n, 3)
    out = _grad_out(osc.scene, want_abs)
    g = Grads(*[_p(out.get(k)) for k in GRAD_FIELDS])
    cnt = np.zeros(8, dtype=np.int64)
    v = make_view(view, index)
    p = make_params(ris_m, seed, threads, 0, 0, 0, reuse)
    if L.orc_light_backward(osc.h, C.byref(v), C.byref(p), _p(pix), n, _p(d), C.byref(g), _p(cnt)):
        raise ValueError("orc_light_backward rejected its arguments")
    out["counts"] = cnt
    return out


def light_demod_detached(frozen, evaled, view, index, ris_m, seed=0, pixels=None, threads=None, reuse=(0, 0)):
    """light_demod's c re-evaluated with `evaled`'s parameters, every sampled quantity from `frozen`."""
    L = lib()
    n = view.width * view.height if pixels is None else len(pixels)
    pix = None if pixels is None else np.ascontiguousarray(pixels, dtype=np.int32)
    out = np.zeros((n, 3))
    v = make_view(view, index)
    p = make_params(ris_m, seed, threads, 0, 0, 0, reuse)
    if L.orc_light_demod_detached(frozen.h, evaled.h, C.byref(v), C.byref(p), _p(pix), n, _p(out)):
        raise ValueError("orc_light_demod_detached rejected its arguments")
    return out


def trace(osc, origins, dirs, mode=0, skip=None, margins=False):
    """mode 0 closest (BVH), 1 any (BVH), 2 closest (brute force), 3 any (brute force)."""
    L = lib()
    rays = _f64(np.concatenate([np.asarray(origins, float), np.asarray(dirs, float)], axis=1))
    n = rays.shape[0]
    sk = None if skip is None else np.ascontiguousarray(skip, dtype=np.int32)
    tri = np.zeros(n, dtype=np.int32)
    tuv = np.zeros((n, 3))
    mg = np.zeros(n) if margins else None
    L.orc_trace(osc.h, _p(rays), _p(sk), n, mode, _p(tri), _p(tuv), _p(mg))
    return tri, tuv, mg


def lbvh(verts, tris):
    L = lib()
    v = np.ascontiguousarray(verts, dtype=np.float32)
    t = np.ascontiguousarray(tris, dtype=np.int32)
    n = t.shape[0]
    keys = np.zeros(n, dtype=np.uint64)
    left = np.zeros(max(n - 1, 0), dtype=np.int32)
    right = np.zeros(max(n - 1, 0), dtype=np.int32)
    parent = np.zeros(max(2 * n - 1, 0), dtype=np.int32)
    lo = np.zeros((max(2 * n - 1, 0), 3), dtype=np.float32)
    hi = np.zeros((max(2 * n - 1, 0), 3), dtype=np.float32)
    L.orc_lbvh(_p(v), _p(t), n, _p(keys), _p(left), _p(right), _p(parent), _p(lo), _p(hi))
    return dict(keys=keys, left=left, right=right, parent=parent, lo=lo, hi=hi)


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(o))
    return o


def brdf_cos(n, wo, wi, albedo, rough, metal, kind=0):
    out = np.zeros(3)
    lib().orc_brdf_cos(_p(_f64(n)), _p(_f64(wo)), _p(_f64(wi)), _p(_f64(albedo)), float(rough), float(metal),
                       int(kind), _p(out))
    return out


def brdf_cos_grad(n, wo, wi, albedo, rough, metal, g, kind=0):
    out = np.zeros(8)
    lib().orc_brdf_cos_grad(_p(_f64(n)), _p(_f64(wo)), _p(_f64(wi)), _p(_f64(albedo)), float(rough), float(metal),
                            int(kind), _p(_f64(g)), _p(out))
    return out


def vndf_sample(n, wo, alpha, u1, u2):
    out = np.zeros(3)
    lib().orc_vndf_sample(_p(_f64(n)), _p(_f64(wo)), float(alpha), float(u1), float(u2), _p(out))
    return out


def vndf_pdf(n, wo, wi, alpha):
    return lib().orc_vndf_pdf(_p(_f64(n)), _p(_f64(wo)), _p(_f64(wi)), float(alpha))


def sample_continuation(osc, n, wo, albedo, rough, metal, words):
    out = np.zeros(3)
    w = np.ascontiguousarray(words, dtype=np.uint32)
    p = lib().orc_sample_continuation(osc.h, _p(_f64(n)), _p(_f64(wo)), _p(_f64(albedo)), float(rough),
                                      float(metal), 0, _p(w), _p(out))
    return out, p


def pdf_continuation(osc, n, wo, albedo, rough, metal, wi):
    return lib().orc_pdf_continuation(osc.h, _p(_f64(n)), _p(_f64(wo)), _p(_f64(albedo)), float(rough),
                                      float(metal), 0, _p(_f64(wi)))


def env_sample(osc, words):
    out = np.zeros(3)
    tex = C.c_int32(0)
    w = np.ascontiguousarray(words, dtype=np.uint32)
    p = lib().orc_env_sample(osc.h, _p(w), _p(out), C.byref(tex))
    return out, tex.value, p


def env_pdf(osc, d):
    return lib().orc_env_pdf(osc.h, _p(_f64(d)))


def env_texel(osc, d):
    return lib().orc_env_texel(osc.h, _p(_f64(d)))


def taps_reach(w, h, su, sv, dfx, dfy):
    """texels whose bilinear weight an FP32 lookup at (su, sv) within (dfx, dfy) texels of its
    fractional position may change (the texel-gradient sensitivity's support), as a sorted list"""
    out = np.zeros(16, dtype=np.int32)
    n = lib().orc_taps_reach(int(w), int(h), float(su), float(sv), float(dfx), float(dfy), _p(out))
    return sorted(int(x) for x in out[:n])


def wrs(gamma, u):
    g = _f64(gamma)
    uu = _f64(u)
    ws = np.zeros(1)
    sel = lib().orc_wrs(_p(g), _p(uu), len(g), _p(ws))
    return sel, float(ws[0])


def ggx_d(alpha, cnh):
    return lib().orc_ggx_d(float(alpha), float(cnh))


def smith_g1(alpha, c):
    return lib().orc_smith_g1(float(alpha), float(c))


def uniform(x):
    return lib().orc_uniform(int(x) & 0xFFFFFFFF)
