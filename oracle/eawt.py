"""FP64 oracle of the edge-avoiding a-trous wavelet denoiser (EAWT) that sits between the
rendered image and the loss (Appendix A, "Denoiser"), and of its G-buffer.

TEST INFRASTRUCTURE ONLY: imported by the tests and by the benchmark's CPU-baseline leg; the
CUDA library never imports it.

What the paper fixes (Appendix A): the image is smoothed level by level with a B3-spline
kernel whose taps spread apart at every level (a-trous), each tap weighted by
w(p, q) = w_rt w_n w_x and normalised by k = sum_q h_i(q) w(p, q); w_rt = exp(-|I_p - I_q|^2 /
sigma_rt^2) on colour differences; three levels. Readings of what it leaves open:
  * B3 taps (1, 4, 6, 4, 1) / 16 per axis, 5 x 5 support; level i (i = 0, 1, 2) places its taps
    2^i pixels apart (2^i - 1 zeros between coefficients);
  * I in w_rt is the image entering the level (c_i); sigma_rt is halved at every level;
  * w_n = exp(-|n_p - n_q|^2 / sigma_n^2) and w_x = exp(-|x_p - x_q|^2 / sigma_x^2) on the
    G-buffer's normals and positions, the forms of the cited wavelet denoiser;
  * taps outside the image are left out (k renormalises);
  * the G-buffer is the primary hit through each pixel centre: face normal turned towards the
    camera and hit position; a pixel whose ray escapes has normal 0 and position 0;
  * the adjoint holds the weights fixed (they are computed from the forward's images and
    treated as constants), so it is the transpose of the linear filter the forward applied.
Every function here is plain numpy over the whole image, one shifted copy per tap.
"""
from __future__ import annotations

import numpy as np

B3 = np.array([1.0, 4.0, 6.0, 4.0, 1.0]) / 16.0


def _shift(a, dy, dx):
    """a[y + dy, x + dx] at every (y, x), zero outside, and the mask of taps inside"""
    H, W = a.shape[:2]
    out = np.zeros_like(a)
    m = np.zeros((H, W), dtype=bool)
    ys, ye = max(0, -dy), min(H, H - dy)
    xs, xe = max(0, -dx), min(W, W - dx)
    if ys < ye and xs < xe:
        out[ys:ye, xs:xe] = a[ys + dy:ye + dy, xs + dx:xe + dx]
        m[ys:ye, xs:xe] = True
    return out, m


def _weights(c, n, x, step, s_rt, s_n, s_x):
    """for each of the 25 taps: (dy, dx, h * w(p, p + tap), inside mask)"""
    taps = []
    for a in range(5):
        for b in range(5):
            dy, dx = (a - 2) * step, (b - 2) * step
            cq, m = _shift(c, dy, dx)
            nq, _ = _shift(n, dy, dx)
            xq, _ = _shift(x, dy, dx)
            e = ((c - cq) ** 2).sum(-1) / s_rt ** 2 + ((n - nq) ** 2).sum(-1) / s_n ** 2 + \
                ((x - xq) ** 2).sum(-1) / s_x ** 2
            w = B3[a] * B3[b] * np.exp(-e) * m
            taps.append((dy, dx, w, m))
    return taps


def eawt(image, normal, position, sigma_rt, sigma_n, sigma_x, levels=3):
    """Returns (denoised image, record) with record = [(c_i, k_i, taps_i)] per level."""
    c = np.asarray(image, dtype=np.float64)
    n = np.asarray(normal, dtype=np.float64)
    x = np.asarray(position, dtype=np.float64)
    record = []
    for i in range(levels):
        step = 1 << i
        taps = _weights(c, n, x, step, sigma_rt / step, sigma_n, sigma_x)
        num = np.zeros_like(c)
        k = np.zeros(c.shape[:2])
        for dy, dx, w, m in taps:
            cq, _ = _shift(c, dy, dx)
            num += w[..., None] * cq
            k += w
        record.append((c, k, taps))
        c = num / k[..., None]
    return c, record


def eawt_apply_frozen(image, record):
    """The linear filter of a recorded forward (weights held fixed) applied to another image:
    the operator whose transpose eawt_backward applies."""
    c = np.asarray(image, dtype=np.float64)
    for _, k, taps in record:
        num = np.zeros_like(c)
        for dy, dx, w, m in taps:
            cq, _ = _shift(c, dy, dx)
            num += w[..., None] * cq
        c = num / k[..., None]
    return c


def eawt_backward(d_out, record):
    """Adjoint with the weights held fixed: the transpose of each level's filter, last level
    first. Level i maps c_i to c_{i+1}(p) = sum_q a(p, q) c_i(q) / k(p) with a(p, q) = h w(p, q)
    symmetric in p and q, so its transpose is g_i(q) = sum_p a(q, p) g_{i+1}(p) / k(p)."""
    g = np.asarray(d_out, dtype=np.float64)
    for c, k, taps in reversed(record):
        s = g / k[..., None]
        out = np.zeros_like(g)
        for dy, dx, w, m in taps:
            sq, _ = _shift(s, dy, dx)
            out += w[..., None] * sq  # a(q, q + tap) s(q + tap), a symmetric
        g = out
    return g


def gbuffer(osc, view):
    """Pixel-centre primary hits of one view through the oracle's own tracer: normal [H][W][3]
    (face normal turned towards the camera, 0 on a miss) and position [H][W][3] (0 on a miss)."""
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
    s = osc.scene
    normal = np.zeros((H * W, 3))
    pos = np.zeros((H * W, 3))
    hit = tri >= 0
    v = s.verts.astype(np.float64)
    f = s.tris[tri[hit]]
    a, b, c = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    nn = np.cross(b - a, c - a)
    nn /= np.linalg.norm(nn, axis=1, keepdims=True)
    nn[(nn * d[hit]).sum(1) > 0] *= -1.0
    normal[hit] = nn
    pos[hit] = o[hit] + d[hit] * tuv[hit, :1]
    return normal.reshape(H, W, 3), pos.reshape(H, W, 3), tri.reshape(H, W), mg.reshape(H, W)
