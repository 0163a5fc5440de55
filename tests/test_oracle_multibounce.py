"""Pin of the oracle's multi-bounce transport (Eq. sec_bouce, Eq. mc_indir) against an
independent estimator: a plain numpy path tracer over every triangle (brute force), Lambert
surfaces, cosine-sampled continuations and the environment added when a ray escapes -- no
RIS, no shadow rays, no MIS. Both estimate the same sum over paths camera -> x_1 .. x_k ->
env (k <= bounces), so their pixel means must agree within their combined standard errors.
The scene (sphere over a ground plane, constant env) has real interreflection."""
import math

import numpy as np

from oracle import oracle as O
from paper_2406_16360_gb300 import synth


def _intersect(o, d, v0, e1, e2, skip):
    """closest hit of each ray over all triangles (Moller-Trumbore, float64), -1 = miss"""
    n = o.shape[0]
    best_t = np.full(n, np.inf)
    best = np.full(n, -1)
    for t0 in range(0, v0.shape[0], 256):
        a, b, c = v0[t0:t0 + 256], e1[t0:t0 + 256], e2[t0:t0 + 256]
        p = np.cross(d[:, None, :], c[None, :, :])
        det = (b[None] * p).sum(-1)
        inv = np.where(det != 0, 1.0 / np.where(det != 0, det, 1.0), 0.0)
        s = o[:, None, :] - a[None]
        u = (s * p).sum(-1) * inv
        q = np.cross(s, b[None])
        v = (d[:, None, :] * q).sum(-1) * inv
        t = (c[None] * q).sum(-1) * inv
        ok = (det != 0) & (u >= 0) & (v >= 0) & (u + v <= 1) & (t > 1e-6)
        ids = np.arange(t0, t0 + a.shape[0])[None]
        ok &= ids != skip[:, None]
        t = np.where(ok, t, np.inf)
        j = np.argmin(t, axis=1)
        tj = t[np.arange(n), j]
        better = tj < best_t
        best_t = np.where(better, tj, best_t)
        best = np.where(better, t0 + j, best)
    return best, best_t


def _path_trace(sc, view, pixels, spp, bounces, rho, L, rng):
    V = sc.verts.astype(np.float64)
    F = sc.tris
    v0, e1, e2 = V[F[:, 0]], V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]]
    nrm = np.cross(e1, e2)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    K = np.asarray(view.K, float)
    c2w = np.asarray(view.c2w, float).reshape(3, 4)
    px = np.repeat(pixels % view.width, spp)
    py = np.repeat(pixels // view.width, spp)
    dc = np.stack([(px + rng.random(px.size) - K[2]) / K[0], (py + rng.random(px.size) - K[3]) / K[1],
                   np.ones(px.size)], 1)
    d = dc @ c2w[:, :3].T
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o = np.tile(c2w[:, 3], (px.size, 1))
    rad = np.zeros(px.size)
    beta = np.ones(px.size)
    alive = np.ones(px.size, bool)
    skip = np.full(px.size, -1)
    for b in range(bounces + 1):
        idx = np.flatnonzero(alive)
        if idx.size == 0:
            break
        tri, t = _intersect(o[idx], d[idx], v0, e1, e2, skip[idx])
        miss = tri < 0
        rad[idx[miss]] += beta[idx[miss]] * L  # escaped: the environment, weighted by the path
        alive[idx[miss]] = False
        hit = idx[~miss]
        if b == bounces or hit.size == 0:
            alive[hit] = False
            break
        th = tri[~miss]
        x = o[hit] + t[~miss, None] * d[hit]
        n = nrm[th]
        n = np.where(((n * d[hit]).sum(1) > 0)[:, None], -n, n)
        # cosine-weighted direction; Lambert f cos / pdf = rho
        u1, u2 = rng.random(hit.size), rng.random(hit.size)
        r, ph = np.sqrt(u1), 2 * np.pi * u2
        a = np.where(np.abs(n[:, 0:1]) > 0.9, np.array([[0.0, 1.0, 0.0]]), np.array([[1.0, 0.0, 0.0]]))
        tt = np.cross(n, a)
        tt /= np.linalg.norm(tt, axis=1, keepdims=True)
        bb = np.cross(n, tt)
        wi = (r * np.cos(ph))[:, None] * tt + (r * np.sin(ph))[:, None] * bb + np.sqrt(1 - u1)[:, None] * n
        beta[hit] *= rho
        o[hit] = x
        d[hit] = wi
        skip[hit] = th
    return rad.reshape(len(pixels), spp)


def test_multibounce_matches_independent_path_tracer():
    rho, L = 0.8, 1.0
    sc = synth.tiny_scene(albedo=rho, env_value=L, sun=None, subdiv=2)
    K, c2w = synth.look_at((0.0, 0.9, 3.0), (0.0, 0.55, 0.0), 12, 12, 50.0)
    view = synth.View(K, c2w, 12, 12, 1024, 3)
    pixels = np.arange(144, dtype=np.int32)
    osc = O.OracleScene(sc)
    # oracle: eight independent seeds give its per-pixel standard error (seven degrees of
    # freedom: with four seeds the estimate's heavy t tails alone push some |z| past 5)
    runs = np.stack([O.render(osc, view, 0, 4, seed=s, brdf_kind=1, margins=False)["rgb"][:, 0] for s in range(8)])
    o_mean = runs.mean(0)
    o_se = runs.std(0, ddof=1) / math.sqrt(runs.shape[0])
    rng = np.random.Generator(np.random.PCG64(123))
    pt = _path_trace(sc, view, pixels, 1024, 3, rho, L, rng)
    p_mean = pt.mean(1)
    p_se = pt.std(1, ddof=1) / math.sqrt(pt.shape[1])
    z = (o_mean - p_mean) / np.sqrt(o_se ** 2 + p_se ** 2 + 1e-30)
    lit = p_mean < L * 0.999  # pixels on geometry (the others see the env directly)
    assert lit.sum() > 40
    assert np.abs(z).max() < 5.0, np.abs(z).max()
    assert abs(z[lit].mean()) < 4.0 / math.sqrt(lit.sum()) * 1.5
    # the indirect light is really there: one bounce alone is biased low somewhere
    one = O.render(osc, synth.View(K, c2w, 12, 12, 2048, 1), 0, 4, seed=9, brdf_kind=1, margins=False)["rgb"][:, 0]
    assert (p_mean - one)[lit].max() > 10 * p_se[lit].max()
