"""Seeded synthetic inputs: meshes, textures, environment maps and cameras.

This module only *generates inputs*. It holds none of the rendering arithmetic (no ray
generation, no sampling, no shading), so both the CUDA path and the CPU oracle can take
their inputs from it without sharing any of the method's code.

The workloads are stand-ins for the paper's evaluation scenes (TensoIR synthetic and OWL
objects: single objects under an HDR environment map, rendered from many calibrated views;
Sec. 5.1 of the paper). Those datasets are not used; the shapes below only mimic their
structure: a closed object with self-shadowing, multi-view cameras on a ring or hemisphere,
spatially varying albedo/roughness/metallic textures and an HDR environment map with a sun.

Conventions (also followed by the library):
  * verts   float32 [V][3], world space, y up.
  * tris    int32   [F][3] vertex indices, outward counter-clockwise winding.
  * tri_uv  float32 [F][3][2] per-corner texture coordinates in [0, 1]^2.
  * textures: albedo float32 [th][tw][3], roughness / metallic float32 [th][tw]; row = v * th.
  * env     float32 [eh][ew][3], latitude-longitude, row 0 = +y (zenith).
  * camera  K = (fx, fy, cx, cy) in pixels; c2w = row-major 3x4 [R | t]; the columns of R
            are the camera x (right), y (down) and z (forward) axes in world space.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ----------------------------------------------------------------------------------------
# hashing and value noise (input generation only)
# ----------------------------------------------------------------------------------------

_M32 = np.uint64(0xFFFFFFFF)


def _u32(a):
    return (np.asarray(a).astype(np.int64) & 0xFFFFFFFF).astype(np.uint64)


def _fmix32(h):
    """MurmurHash3 32-bit finaliser on uint64 arrays holding 32-bit values."""
    h = h & _M32
    h ^= h >> np.uint64(16)
    h = (h * np.uint64(0x85EBCA6B)) & _M32
    h ^= h >> np.uint64(13)
    h = (h * np.uint64(0xC2B2AE35)) & _M32
    h ^= h >> np.uint64(16)
    return h


def _lattice(ix, iy, iz, seed):
    """Pseudo-random lattice value in [-1, 1] hashed from integer coordinates and a seed."""
    h = (_u32(ix) * np.uint64(0x8DA6B343)) ^ (_u32(iy) * np.uint64(0xD8163841))
    h ^= _u32(iz) * np.uint64(0xCB1AB31F)
    h ^= np.uint64((seed * 0x9E3779B1) & 0xFFFFFFFF)
    h = _fmix32(_fmix32(h) ^ np.uint64(seed & 0xFFFFFFFF))
    return h.astype(np.float64) * (2.0 / 4294967296.0) - 1.0


def _smooth(t):
    return t * t * (3.0 - 2.0 * t)


def value_noise3(p, seed):
    """Trilinear value noise at points p [..., 3] with a unit lattice."""
    p = np.asarray(p, dtype=np.float64)
    f = np.floor(p)
    i = f.astype(np.int64)
    t = _smooth(p - f)
    # hash only the lattice box that the points touch, then gather
    lo = i.reshape(-1, 3).min(axis=0)
    ext = i.reshape(-1, 3).max(axis=0) - lo + 2
    gx, gy, gz = np.meshgrid(*(lo[k] + np.arange(ext[k]) for k in range(3)), indexing="ij")
    table = _lattice(gx, gy, gz, seed)
    r = i - lo
    out = np.zeros(p.shape[:-1])
    for dx in (0, 1):
        wx = t[..., 0] if dx else 1.0 - t[..., 0]
        for dy in (0, 1):
            wy = t[..., 1] if dy else 1.0 - t[..., 1]
            for dz in (0, 1):
                wz = t[..., 2] if dz else 1.0 - t[..., 2]
                out += wx * wy * wz * table[r[..., 0] + dx, r[..., 1] + dy, r[..., 2] + dz]
    return out


def fbm3(p, seed, lattice=4.0, octaves=3, lacunarity=2.0, gain=0.5):
    """Fractal sum of value noise, normalised to [-1, 1]."""
    p = np.asarray(p, dtype=np.float64)
    total, amp, norm, freq = np.zeros(p.shape[:-1]), 1.0, 0.0, lattice
    for o in range(octaves):
        total += amp * value_noise3(p * freq, seed + 1013 * o)
        norm += amp
        amp *= gain
        freq *= lacunarity
    return total / norm


def noise_texture(h, w, channels, seed, lattice=8.0, lo=0.05, hi=0.95):
    """Smooth seeded value-noise texture mapped to [lo, hi], float32 [h][w][channels]."""
    v, u = np.meshgrid((np.arange(h) + 0.5) / h, (np.arange(w) + 0.5) / w, indexing="ij")
    out = np.empty((h, w, channels), dtype=np.float32)
    for c in range(channels):
        p = np.stack([u, v, np.full_like(u, 0.37 * c + 0.11)], axis=-1)
        n = fbm3(p, seed + 7919 * c, lattice=lattice)
        out[..., c] = (lo + (hi - lo) * (0.5 + 0.5 * n)).astype(np.float32)
    return out


# ----------------------------------------------------------------------------------------
# meshes
# ----------------------------------------------------------------------------------------

def icosphere(subdiv: int):
    """Unit icosphere: 20 * 4**subdiv triangles (subdiv 3 -> 1280)."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t),
         (0, 1, -t), (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    verts = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in v]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
             (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
             (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(subdiv):
        cache = {}

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    return np.array(verts), np.array(faces, dtype=np.int64)


def spherical_corner_uv(verts, tris):
    """Per-corner latitude-longitude UVs of a sphere-like mesh (used for 1x1 textures)."""
    p = verts[tris]  # [F][3][3]
    u = np.arctan2(p[..., 0], -p[..., 2]) / (2 * np.pi) + 0.5
    r = np.linalg.norm(p, axis=-1)
    v = np.arccos(np.clip(p[..., 1] / np.maximum(r, 1e-30), -1, 1)) / np.pi
    return np.clip(np.stack([u, v], axis=-1), 0.0, 1.0)


def uv_sphere(n_lon: int, n_lat: int):
    """Unit UV sphere: 2*n_lon cap triangles + 2*n_lon*(n_lat-2) band triangles.

    Returns unit directions [V][3], triangles [F][3] and per-corner UVs [F][3][2]
    (u = longitude / 2pi, v = colatitude / pi; the seam column uses u = 1).
    """
    th = np.pi * np.arange(1, n_lat) / n_lat
    ph = 2 * np.pi * np.arange(n_lon) / n_lon
    T, P = np.meshgrid(th, ph, indexing="ij")
    ring = np.stack([np.sin(T) * np.sin(P), np.cos(T), -np.sin(T) * np.cos(P)], -1).reshape(-1, 3)
    verts = np.concatenate([[[0.0, 1.0, 0.0]], ring, [[0.0, -1.0, 0.0]]])
    north, south = 0, len(verts) - 1
    j = np.arange(n_lon)
    u0, u1 = j / n_lon, (j + 1) / n_lon
    um = 0.5 * (u0 + u1)

    def rv(i, jj):  # ring i in [0, n_lat-2], column jj (mod n_lon)
        return 1 + i * n_lon + (jj % n_lon)

    # north cap
    t_n = np.stack([np.full(n_lon, north), rv(0, j), rv(0, j + 1)], -1)
    uv_n = np.stack([np.stack([um, np.zeros(n_lon)], -1),
                     np.stack([u0, np.full(n_lon, 1 / n_lat)], -1),
                     np.stack([u1, np.full(n_lon, 1 / n_lat)], -1)], 1)
    # bands: ring i, column j -> two triangles
    I, J = np.meshgrid(np.arange(n_lat - 2), j, indexing="ij")
    a, b, c, d = rv(I, J), rv(I + 1, J), rv(I + 1, J + 1), rv(I, J + 1)
    va, vb = (I + 1) / n_lat, (I + 2) / n_lat
    U0, U1 = J / n_lon, (J + 1) / n_lon
    t1 = np.stack([a, b, c], -1)
    t2 = np.stack([a, c, d], -1)
    uv1 = np.stack([np.stack([U0, va], -1), np.stack([U0, vb], -1), np.stack([U1, vb], -1)], -2)
    uv2 = np.stack([np.stack([U0, va], -1), np.stack([U1, vb], -1), np.stack([U1, va], -1)], -2)
    t_b = np.stack([t1, t2], 2).reshape(-1, 3)
    uv_b = np.stack([uv1, uv2], 2).reshape(-1, 3, 2)
    # south cap
    i = n_lat - 2
    vs = (n_lat - 1) / n_lat
    t_s = np.stack([rv(i, j), np.full(n_lon, south), rv(i, j + 1)], -1)
    uv_s = np.stack([np.stack([u0, np.full(n_lon, vs)], -1),
                     np.stack([um, np.ones(n_lon)], -1),
                     np.stack([u1, np.full(n_lon, vs)], -1)], 1)
    # reverse the corner order so that the winding is outward (counter-clockwise from outside)
    tris = np.concatenate([t_n, t_b, t_s])[:, ::-1].astype(np.int64)
    uvs = np.concatenate([uv_n, uv_b, uv_s])[:, ::-1, :].astype(np.float64)
    return verts, np.ascontiguousarray(tris), np.ascontiguousarray(uvs)


def box(lo, hi):
    """Axis-aligned box, 8 vertices and 12 outward triangles with simple per-corner UVs."""
    lo, hi = np.asarray(lo, float), np.asarray(hi, float)
    c = np.array([[x, y, z] for x in (0, 1) for y in (0, 1) for z in (0, 1)], dtype=float)
    verts = lo + c * (hi - lo)
    quads = [(0, 1, 3, 2), (4, 6, 7, 5), (0, 4, 5, 1), (2, 3, 7, 6), (0, 2, 6, 4), (1, 5, 7, 3)]
    tris, uvs = [], []
    for a, b, cc, d in quads:
        tris += [(a, b, cc), (a, cc, d)]
        uvs += [((0, 0), (1, 0), (1, 1)), ((0, 0), (1, 1), (0, 1))]
    return verts, np.array(tris, dtype=np.int64), np.array(uvs, dtype=np.float64)


def merge(parts):
    vs, ts, us, off = [], [], [], 0
    for v, t, u in parts:
        vs.append(v)
        ts.append(t + off)
        us.append(u)
        off += len(v)
    return np.concatenate(vs), np.concatenate(ts), np.concatenate(us)


def displaced_sphere(n_lon, n_lat, seed, amp=0.15, folds=0.0):
    """Noise-displaced UV sphere: radius 1 + amp * fbm (+ folds * (1 - |fbm'|)^2)."""
    d, t, uv = uv_sphere(n_lon, n_lat)
    r = 1.0 + amp * fbm3(d, seed, lattice=4.0)
    if folds:
        r += folds * (1.0 - np.abs(fbm3(d, seed + 77, lattice=4.0))) ** 2
    return d * r[:, None], t, uv


def occluder_boxes(seed, count=3):
    rng = np.random.Generator(np.random.PCG64(seed + 4242))
    parts = []
    for k in range(count):
        ang = 2 * np.pi * (k + rng.uniform(0.1, 0.9)) / count
        rad = rng.uniform(1.35, 1.7)
        c = np.array([rad * math.cos(ang), rng.uniform(-0.5, 0.6), rad * math.sin(ang)])
        h = rng.uniform(0.12, 0.3, size=3)
        parts.append(box(c - h, c + h))
    return parts


# ----------------------------------------------------------------------------------------
# environment maps
# ----------------------------------------------------------------------------------------

def env_constant(ew, eh, value):
    return np.full((eh, ew, 3), value, dtype=np.float32)


def env_lognormal_sun(ew, eh, seed, sigma=1.5, sun=1e3, sun_size=2):
    rng = np.random.Generator(np.random.PCG64(seed + 99))
    env = np.exp(rng.normal(0.0, sigma, size=(eh, ew, 3))).astype(np.float32)
    r = int(rng.integers(eh // 8, eh // 3))
    c = int(rng.integers(0, ew - sun_size))
    env[r:r + sun_size, c:c + sun_size, :] = sun
    return env


# ----------------------------------------------------------------------------------------
# cameras
# ----------------------------------------------------------------------------------------

def look_at(eye, target, width, height, fov_deg=40.0, up=(0.0, 1.0, 0.0)):
    """Pinhole camera (OpenCV axes: x right, y down, z forward) with a vertical field of view."""
    eye, target, up = (np.asarray(a, float) for a in (eye, target, up))
    z = target - eye
    z /= np.linalg.norm(z)
    x = np.cross(z, up)
    if np.linalg.norm(x) < 1e-9:
        x = np.cross(z, np.array([0.0, 0.0, 1.0]))
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z], axis=1)
    c2w = np.concatenate([R, eye[:, None]], axis=1).astype(np.float32).reshape(12)
    f = 0.5 * height / math.tan(math.radians(fov_deg) / 2)
    K = np.array([f, f, 0.5 * width, 0.5 * height], dtype=np.float32)
    return K, c2w


# ----------------------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------------------

@dataclass
class Scene:
    verts: np.ndarray
    tris: np.ndarray
    tri_uv: np.ndarray
    albedo: np.ndarray
    roughness: np.ndarray
    metallic: np.ndarray
    env: np.ndarray

    @property
    def n_tris(self):
        return int(self.tris.shape[0])


@dataclass
class View:
    K: np.ndarray
    c2w: np.ndarray
    width: int
    height: int
    spp: int
    bounces: int
    scene: int = 0


@dataclass
class Workload:
    name: str
    scenes: list
    views: list
    ris_m: int
    seed: int = 0
    notes: dict = field(default_factory=dict)

    @property
    def samples(self):
        return sum(v.width * v.height * v.spp for v in self.views)


def _scene(verts, tris, uv, albedo, rough, metal, env):
    return Scene(np.ascontiguousarray(verts, dtype=np.float32),
                 np.ascontiguousarray(tris, dtype=np.int32),
                 np.ascontiguousarray(uv, dtype=np.float32),
                 np.ascontiguousarray(albedo, dtype=np.float32),
                 np.ascontiguousarray(rough, dtype=np.float32),
                 np.ascontiguousarray(metal, dtype=np.float32),
                 np.ascontiguousarray(env, dtype=np.float32))


def tiny_scene(albedo=0.5, roughness=0.5, metallic=0.0, env_value=0.2, sun=500.0,
               ground=True, subdiv=3, env_w=32, env_h=16, sun_texel=(3, 8)):
    """Icosphere (r=1, centre (0,1,0)) above a 2-triangle ground quad, uniform 1x1 material."""
    v, t = icosphere(subdiv)
    uv = spherical_corner_uv(v, t)
    v = v + np.array([0.0, 1.0, 0.0])
    parts = [(v, t, uv)]
    if ground:
        gv = np.array([[-5, 0, -5], [5, 0, -5], [5, 0, 5], [-5, 0, 5]], dtype=float)
        gt = np.array([[0, 2, 1], [0, 3, 2]])
        guv = np.array([((0, 0), (1, 1), (1, 0)), ((0, 0), (0, 1), (1, 1))], dtype=float)
        parts.append((gv, gt, guv))
    verts, tris, uvs = merge(parts)
    env = env_constant(env_w, env_h, env_value)
    if sun is not None:
        env[sun_texel[0], sun_texel[1], :] = sun
    return _scene(verts, tris, uvs,
                  np.full((1, 1, 3), albedo, np.float32), np.full((1, 1), roughness, np.float32),
                  np.full((1, 1), metallic, np.float32), env)


def config1(albedo=0.5, width=64, height=64):
    """Tiny forward+backward: icosphere (1280 tris) + ground, 64x64, 4 spp, 2 bounces, M=8."""
    sc = tiny_scene(albedo=albedo)
    K, c2w = look_at((0.0, 1.5, 4.0), (0.0, 1.0, 0.0), width, height, 40.0)
    return Workload("config1-icosphere-64", [sc], [View(K, c2w, width, height, 4, 2)], ris_m=8, seed=0)


def object_scene(n_seg_lon, n_seg_lat, seed, tex, env_w, env_h, folds=0.0, boxes=True):
    parts = [displaced_sphere(n_seg_lon, n_seg_lat, seed, 0.15, folds)]
    if boxes:
        parts += occluder_boxes(seed)
    verts, tris, uvs = merge(parts)
    albedo = noise_texture(tex, tex, 3, seed + 1)
    rough = noise_texture(tex, tex, 1, seed + 2)[..., 0]
    metal = noise_texture(tex, tex, 1, seed + 3)[..., 0]
    env = env_lognormal_sun(env_w, env_h, seed)
    return _scene(verts, tris, uvs, albedo, rough, metal, env)


def ring_views(n, res, spp, bounces, radius=3.5, height=1.0, scene=0):
    views = []
    for k in range(n):
        a = 2 * np.pi * k / n + 0.3
        K, c2w = look_at((radius * math.cos(a), height, radius * math.sin(a)), (0, 0, 0), res, res)
        views.append(View(K, c2w, res, res, spp, bounces, scene))
    return views


def hemisphere_views(n, res, spp, bounces, seed, radius=3.5, scene=0):
    rng = np.random.Generator(np.random.PCG64(seed + 555))
    views = []
    for _ in range(n):
        a = rng.uniform(0, 2 * np.pi)
        el = np.arcsin(rng.uniform(math.sin(math.radians(8)), math.sin(math.radians(75))))
        eye = radius * np.array([math.cos(el) * math.cos(a), math.sin(el), math.cos(el) * math.sin(a)])
        K, c2w = look_at(eye, (0, 0, 0), res, res)
        views.append(View(K, c2w, res, res, spp, bounces, scene))
    return views


def config2(seed=0, res=256, n_views=4, tex=512, spp=8, bounces=3):
    """Self-shadowing object: displaced UV sphere (160x157) + 3 boxes (49,956 tris)."""
    sc = object_scene(160, 157, seed, tex, 256, 128)
    return Workload("config2-object-50k", [sc], ring_views(n_views, res, spp, bounces), ris_m=32, seed=seed)


def config3(seed=0, res=800, n_views=100, tex=1024, spp=16, bounces=4, segments=500):
    """Paper-shaped batch: 500x500-segment displaced sphere with folds + boxes (499,036 tris)."""
    sc = object_scene(segments, segments, seed, tex, 1024, 512, folds=0.1)
    return Workload("config3-multiview-500k", [sc],
                    hemisphere_views(n_views, res, spp, bounces, seed), ris_m=32, seed=seed)


def config5(seed=0, n_scenes=64, max_tris=1_000_000, res_choices=(128, 256, 512, 1024),
            spp_choices=(4, 8, 16, 32), tex=256):
    """Uneven serving batch: scenes with log-uniform triangle counts, mixed resolution/spp/bounces."""
    rng = np.random.Generator(np.random.PCG64(seed + 2024))
    scenes, views = [], []
    for s in range(n_scenes):
        f = math.exp(rng.uniform(math.log(1000), math.log(max_tris)))
        n = max(4, int(round(math.sqrt(f / 2.0))))
        scenes.append(object_scene(n, n, seed + 31 * s, tex, 256, 128))
        res = int(rng.choice(res_choices))
        spp = int(rng.choice(spp_choices))
        b = int(rng.integers(2, 6))
        a = rng.uniform(0, 2 * np.pi)
        K, c2w = look_at((3.5 * math.cos(a), 1.0, 3.5 * math.sin(a)), (0, 0, 0), res, res)
        views.append(View(K, c2w, res, res, spp, b, s))
    return Workload("config5-uneven-64", scenes, views, ris_m=32, seed=seed)
