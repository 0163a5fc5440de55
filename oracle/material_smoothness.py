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
  * |.| of the three-channel albedo (and of the normal) is the mean of its channels' absolute
    differences;
  * the normal n(x) is the shading normal of interpolated vertex normals, S / |S| with
    S = w0 VN_a + u VN_b + v VN_c (VN_i the normalised sum of the incident faces' e1 x e2), so
    it varies over the surface; the same texture-space offset moves the point within the hit
    triangle: the barycentric offset is (du, dv) = J^-1 eps, J = [uv_b - uv_a | uv_c - uv_a] the
    triangle's texture-coordinate map, and n(x + eps) = S' / |S'| with the same blend at
    (u + du, v + dv) (the triangle's linear blend continued where the offset leaves it). With
    face normals the normal is constant on a triangle and the term vanishes; a triangle whose
    texture map is singular adds no normal term. The hit point itself is held fixed (as for the
    albedo and roughness terms), so the normal term's gradient reaches the vertices through the
    vertex normals only;
  * the gradient takes sign(0) = 0.
L = w_albedo L_albedo + w_roughness L_roughness + w_normal L_normal; its gradient with respect
to the texels is (w / |X|) sign(k(x) - k(x + eps)) (bilinear weights at x - bilinear weights at
x + eps), with a further 1/3 per albedo channel; with respect to the vertices see normal_term.
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


def pixel_centre_hits(osc, view, with_bary=False):
    """closest hit through every pixel centre: triangle (-1 on escape), texture coordinates
    [n][2] and the hit decision's margin (the oracle tracer's normalised distance to a tie);
    with_bary also returns the barycentrics (u, v) [n][2] of the hits"""
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
    if with_bary:
        return tri, st, mg, tuv[:, 1:3].copy()
    return tri, st, mg


def vertex_normals(verts, tris):
    """area-weighted vertex normals: VA_i = sum of e1 x e2 of the faces around i, VN = VA / |VA|
    (0 where |VA| = 0); returns (VN, VA)"""
    v = np.asarray(verts, dtype=np.float64)
    t = np.asarray(tris, dtype=np.int64)
    N = np.cross(v[t[:, 1]] - v[t[:, 0]], v[t[:, 2]] - v[t[:, 0]])
    VA = np.zeros_like(v)
    for c in range(3):
        np.add.at(VA, t[:, c], N)
    ln = np.linalg.norm(VA, axis=1)
    VN = np.where(ln[:, None] > 0, VA / np.where(ln > 0, ln, 1.0)[:, None], 0.0)
    return VN, VA


def normal_term(verts, tris, tri_uv, tri, u, v, eps, n_points, w_normal):
    """The normal part of L_k for given hits: points with tri >= 0, barycentrics (u, v), texture
    offsets eps [n][2], mean over n_points (|X|). Returns (w_normal L_normal, d / d verts [V][3],
    number of points with a normal term, abs [V][3] = per vertex the sum of |gradient terms|).

    n0 = S0 / |S0|, n1 = S1 / |S1|, S1 = S0 + du (VN_b - VN_a) + dv (VN_c - VN_a), (du, dv) =
    J^-1 eps; L = (w / (3 |X|)) sum_x sum_c |n0_c - n1_c|. Gradient: through n -> S (the
    projection (I - n n^T) / |S|), S -> the three vertex normals (blend weights), VN -> VA (the
    normalisation), VA -> the vertices of every face around (d(e1 x e2))."""
    V = np.asarray(verts, dtype=np.float64)
    T = np.asarray(tris, dtype=np.int64)
    UV = np.asarray(tri_uv, dtype=np.float64).reshape(-1, 3, 2)
    VN, VA = vertex_normals(V, T)
    g_vn = np.zeros_like(V)
    a_vn = np.zeros_like(V)
    loss = 0.0
    counted = 0
    if n_points == 0:
        return 0.0, np.zeros_like(V), 0, np.zeros_like(V)
    cw = w_normal / (3.0 * n_points)
    for k in np.flatnonzero(np.asarray(tri) >= 0):
        f = T[tri[k]]
        J = np.stack([UV[tri[k], 1] - UV[tri[k], 0], UV[tri[k], 2] - UV[tri[k], 0]], axis=1)  # columns
        det = J[0, 0] * J[1, 1] - J[0, 1] * J[1, 0]
        if det == 0.0:
            continue
        du, dv = np.linalg.solve(J, eps[k])
        w0 = 1.0 - u[k] - v[k]
        b0 = np.array([w0, u[k], v[k]])
        b1 = np.array([w0 - du - dv, u[k] + du, v[k] + dv])
        S0 = b0 @ VN[f]
        S1 = b1 @ VN[f]
        l0, l1 = np.linalg.norm(S0), np.linalg.norm(S1)
        if l0 == 0.0 or l1 == 0.0:
            continue
        n0, n1 = S0 / l0, S1 / l1
        diff = n0 - n1
        loss += cw * np.abs(diff).sum()
        counted += 1
        g = cw * np.sign(diff)
        gS0 = (g - n0 * (n0 @ g)) / l0
        gS1 = (-g - n1 * (n1 @ -g)) / l1
        for j in range(3):
            g_vn[f[j]] += b0[j] * gS0 + b1[j] * gS1
            a_vn[f[j]] += np.abs(b0[j] * gS0) + np.abs(b1[j] * gS1)
    # VN -> VA -> vertices
    lva = np.linalg.norm(VA, axis=1)
    ok = lva > 0
    gVA = np.zeros_like(V)
    aVA = np.zeros_like(V)
    gVA[ok] = (g_vn[ok] - VN[ok] * (VN[ok] * g_vn[ok]).sum(1, keepdims=True)) / lva[ok, None]
    aVA[ok] = a_vn[ok] / lva[ok, None]
    gV = np.zeros_like(V)
    aV = np.zeros_like(V)
    e1 = V[T[:, 1]] - V[T[:, 0]]
    e2 = V[T[:, 2]] - V[T[:, 0]]
    gN = gVA[T[:, 0]] + gVA[T[:, 1]] + gVA[T[:, 2]]  # every face adds its N to its three vertices
    aN = aVA[T[:, 0]] + aVA[T[:, 1]] + aVA[T[:, 2]]
    ge1 = np.cross(e2, gN)
    ge2 = np.cross(gN, e1)
    np.add.at(gV, T[:, 0], -(ge1 + ge2))
    np.add.at(gV, T[:, 1], ge1)
    np.add.at(gV, T[:, 2], ge2)
    ae = np.linalg.norm(aN, axis=1, keepdims=True) * (np.linalg.norm(e1, axis=1, keepdims=True) +
                                                       np.linalg.norm(e2, axis=1, keepdims=True))
    for c in range(3):
        np.add.at(aV, T[:, c], np.repeat(ae, 3, axis=1))
    return float(loss), gV, counted, aV


def material_smoothness_normal(osc, view, view_index, sigma, w_normal, seed=0):
    """The normal term of L_k over one view (X, |X| and eps as material_smoothness's): returns
    (w_normal L_normal, d / d verts [V][3], info) with info = {n_points, n_normal (points with a
    normal term), flagged (hit decision within the tracer's margin), abs_verts}."""
    sc = osc.scene
    tri, st, mg, bary = pixel_centre_hits(osc, view, with_bary=True)
    eps = offsets(tri.size, view_index, sigma, seed)
    n = int((tri >= 0).sum())
    loss, gV, counted, aV = normal_term(sc.verts, sc.tris, sc.tri_uv, tri, bary[:, 0], bary[:, 1], eps, n, w_normal)
    flagged = (tri >= 0) & (mg < 1.0)
    return loss, gV, dict(n_points=n, n_normal=counted, flagged=flagged, abs_verts=aV)


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
