"""FP64 oracle of the material smoothness regulariser L_k (Appendix A, "Training details"):

  L_k = (1 / |X|) sum_{x in X} |k(x) - k(x + eps)|,   k in {albedo, roughness}

TEST INFRASTRUCTURE ONLY: imported by the tests; the CUDA library never imports it.

Readings of what the paper leaves open (its materials are a field over space; here they are
textures):
  * X is the set of surface points seen through the pixel centres of one view (the same rays
    as the denoiser's G-buffer); |X| is their number, escaped pixels are not in X;
  * k(x) is the material lookup at the point's texture coordinates (bilinear, texel centres at
    (i + 1/2) / size, clamp to edge) and the small random offset is taken in texture space:
    k(x + eps) is the lookup at (s + eps_s, t + eps_t), eps uniform in [-sigma, sigma]^2;
  * eps comes from Philox4x32-10 with counter (pixel, 0, view << 16 | 4, 0) and key = seed:
    eps = sigma (2 u - 1) with u = (x >> 8) 2^-24 of the first two output words;
  * |.| of the three-channel albedo is the mean of its channels' absolute differences;
  * the normal term is left out: the normals come from the mesh (face normals, or the
    interpolated vertex normals), with no texture of their own that a texture-space offset
    could move along (the mesh regularisers act on the geometry);
  * the gradient takes sign(0) = 0.
L = w_albedo L_albedo + w_roughness L_roughness; its gradient with respect to the texels is
(w / |X|) sign(k(x) - k(x + eps)) (bilinear weights at x - bilinear weights at x + eps), with a
further 1/3 per albedo channel.
"""
from __future__ import annotations

import numpy as np

PURPOSE_SMOOTH = 4
M32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32-10 (Salmon et al., SC'11) on arrays of counters: ten rounds of two 32 x 32 -> 64
    multiplications (constants 0xD2511F53, 0xCD9E8D57), the key bumped by the Weyl constants
    (0x9E3779B9, 0xBB67AE85) after every round."""
    c = [np.asarray(x, dtype=np.uint64) & M32 for x in (c0, c1, c2, c3)]
    k0 = np.uint64(int(k0) & 0xFFFFFFFF)
    k1 = np.uint64(int(k1) & 0xFFFFFFFF)
    for _ in range(10):
        p0 = np.uint64(0xD2511F53) * c[0]
        p1 = np.uint64(0xCD9E8D57) * c[2]
        c = [((p1 >> np.uint64(32)) ^ c[1] ^ k0) & M32, p1 & M32,
             ((p0 >> np.uint64(32)) ^ c[3] ^ k1) & M32, p0 & M32]
        k0 = (k0 + np.uint64(0x9E3779B9)) & M32
        k1 = (k1 + np.uint64(0xBB67AE85)) & M32
    return [x.astype(np.uint32) for x in c]


def offsets(n_pixels, view_index, sigma, seed):
    """eps [n_pixels][2] of every pixel of a view"""
    pix = np.arange(n_pixels, dtype=np.uint64)
    z = np.zeros_like(pix)
    w = philox4x32_10(pix, z, z + np.uint64((view_index << 16) | PURPOSE_SMOOTH), z, seed & 0xFFFFFFFF, seed >> 32)
    u = np.stack([(w[0] >> 8).astype(np.float64), (w[1] >> 8).astype(np.float64)], -1) * 2.0 ** -24
    return sigma * (2.0 * u - 1.0)


def taps(w, h, s, t):
    """bilinear lookup of [h][w] texels at texture coordinates (s, t): flat texel indices [n][4]
    and weights [n][4]"""
    x = np.asarray(s, dtype=np.float64) * w - 0.5
    y = np.asarray(t, dtype=np.float64) * h - 0.5
    x0, y0 = np.floor(x), np.floor(y)
    fx, fy = x - x0, y - y0
    ix0 = np.clip(x0.astype(np.int64), 0, w - 1)
    ix1 = np.clip(x0.astype(np.int64) + 1, 0, w - 1)
    iy0 = np.clip(y0.astype(np.int64), 0, h - 1)
    iy1 = np.clip(y0.astype(np.int64) + 1, 0, h - 1)
    idx = np.stack([iy0 * w + ix0, iy0 * w + ix1, iy1 * w + ix0, iy1 * w + ix1], -1)
    wt = np.stack([(1 - fx) * (1 - fy), fx * (1 - fy), (1 - fx) * fy, fx * fy], -1)
    return idx, wt


def pixel_centre_hits(osc, view):
    """closest hit through every pixel centre: triangle (-1 on escape), texture coordinates
    [n][2] and the hit decision's margin (the oracle tracer's normalised distance to a tie)"""
    from oracle import oracle as O
    H, W = view.height, view.width
    K = np.asarray(view.K, dtype=np.float64)
    c2w = np.asarray(view.c2w, dtype=np.float64).reshape(3, 4)
    py, px = np.mgrid[0:H, 0:W]
    dc = np.stack([(px + 0.5 - K[2]) / K[0], (py + 0.5 - K[3]) / K[1], np.ones((H, W))], -1).reshape(-1, 3)
    d = dc @ c2w[:, :3].T
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o = np.repeat(c2w[:, 3][None], d.shape[0], 0)
    tri, tuv, mg = O.trace(osc, o, d, mode=0, margins=True)
    st = np.zeros((tri.size, 2))
    hit = tri >= 0
    uv = np.asarray(osc.scene.tri_uv, dtype=np.float64).reshape(-1, 3, 2)[tri[hit]]
    u, v = tuv[hit, 1], tuv[hit, 2]
    st[hit] = (1 - u - v)[:, None] * uv[:, 0] + u[:, None] * uv[:, 1] + v[:, None] * uv[:, 2]
    return tri, st, mg


def material_smoothness(osc, view, view_index, sigma, w_albedo, w_rough, seed=0, tau=None):
    """Returns (loss, d loss / d albedo [th][tw][3], d loss / d roughness [th][tw], info) with info
    = {n_points, flagged (pixels whose hit or sign decision lies within the FP32 error of its
    threshold: trace margin < 1 or some |k(x) - k(x + eps)| < tau), abs_albedo, abs_rough (per
    texel, the sum of |gradient terms| of the flagged pixels)}. tau defaults to about ten times
    the FP32 error of a lookup difference: a texture coordinate is good to ~1e-7, i.e. 1e-7 x size
    texels, and texel values lie in [0, 1]."""
    sc = osc.scene
    alb = np.asarray(sc.albedo, dtype=np.float64)
    rough = np.asarray(sc.roughness, dtype=np.float64)
    th, tw = rough.shape
    if tau is None:
        tau = 1e-6 * max(th, tw) + 1e-6
    tri, st, mg = pixel_centre_hits(osc, view)
    eps = offsets(tri.size, view_index, sigma, seed)
    hit = tri >= 0
    n = int(hit.sum())
    ga = np.zeros((th * tw, 3))
    gr = np.zeros(th * tw)
    aa = np.zeros((th * tw, 3))
    ar = np.zeros(th * tw)
    flagged = np.zeros(tri.size, dtype=bool)
    if n == 0:
        return 0.0, ga.reshape(th, tw, 3), gr.reshape(th, tw), dict(n_points=0, flagged=flagged, abs_albedo=aa,
                                                                     abs_rough=ar)
    s0, t0 = st[hit, 0], st[hit, 1]
    i0, w0 = taps(tw, th, s0, t0)
    i1, w1 = taps(tw, th, s0 + eps[hit, 0], t0 + eps[hit, 1])
    a_flat = alb.reshape(-1, 3)
    r_flat = rough.reshape(-1)
    ka = (w0[..., None] * a_flat[i0]).sum(1) - (w1[..., None] * a_flat[i1]).sum(1)  # [n][3]
    kr = (w0 * r_flat[i0]).sum(1) - (w1 * r_flat[i1]).sum(1)
    loss = w_albedo * np.abs(ka).mean(1).sum() / n + w_rough * np.abs(kr).sum() / n
    fl = (mg[hit] < 1.0) | (np.abs(ka).min(1) < tau) | (np.abs(kr) < tau)
    flagged[np.flatnonzero(hit)[fl]] = True
    sa = np.sign(ka) * (w_albedo / (3.0 * n))
    sr = np.sign(kr) * (w_rough / n)
    for j in range(4):
        for c in range(3):
            np.add.at(ga[:, c], i0[:, j], sa[:, c] * w0[:, j])
            np.add.at(ga[:, c], i1[:, j], -sa[:, c] * w1[:, j])
            np.add.at(aa[:, c], i0[fl, j], w_albedo / (3.0 * n) * w0[fl, j])
            np.add.at(aa[:, c], i1[fl, j], w_albedo / (3.0 * n) * w1[fl, j])
        np.add.at(gr, i0[:, j], sr * w0[:, j])
        np.add.at(gr, i1[:, j], -sr * w1[:, j])
        np.add.at(ar, i0[fl, j], w_rough / n * w0[fl, j])
        np.add.at(ar, i1[fl, j], w_rough / n * w1[fl, j])
    info = dict(n_points=n, flagged=flagged, abs_albedo=aa.reshape(th, tw, 3), abs_rough=ar.reshape(th, tw))
    return float(loss), ga.reshape(th, tw, 3), gr.reshape(th, tw), info
