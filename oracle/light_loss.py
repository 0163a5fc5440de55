"""FP64 oracle of the monochrome light regulariser's loss (Appendix A, "Training details",
L_light, after NVdiffrec-MC): the luminance of the demodulated lighting against the value
channel of the reference image.

TEST INFRASTRUCTURE ONLY: imported by the tests; the CUDA library never imports it.

  L_light = (1 / |P|) sum_{p in P} | Y(c_d + c_s)(p) - V(I_ref)(p) |
  Y(x) = (x_r + x_g + x_b) / 3,   V(x) = max(x_r, x_g, x_b)

c_d + c_s per pixel comes from oracle.light_demod (the mean over the pixel's samples). Readings:
the paper writes |.| without a sum; the loss is the mean over P, the pixels of all views of the
call whose primary rays hit a surface at least once (coverage > 0: an escaping pixel has no
lighting term); the gradient takes sign(0) = 0 and reaches each channel of c through Y's 1/3.
"""
from __future__ import annotations

import numpy as np


def luminance(x):
    x = np.asarray(x, dtype=np.float64)
    return (x[..., 0] + x[..., 1] + x[..., 2]) / 3.0


def value(x):
    return np.asarray(x, dtype=np.float64).max(axis=-1)


def light_loss(c_list, cov_list, ref_list, weight=1.0):
    """c_list[v] [n,3], cov_list[v] [n], ref_list[v] [n,3] per view. Returns (weight * L_light,
    list of d(weight * L_light) / dc [n,3] per view)."""
    n_p = sum(int((np.asarray(cv) > 0).sum()) for cv in cov_list)
    loss = 0.0
    grads = []
    for c, cv, ref in zip(c_list, cov_list, ref_list):
        c = np.asarray(c, dtype=np.float64).reshape(-1, 3)
        ref = np.asarray(ref, dtype=np.float64).reshape(-1, 3)
        inside = np.asarray(cv).reshape(-1) > 0
        diff = luminance(c) - value(ref)
        g = np.zeros_like(c)
        if n_p > 0:
            loss += weight * np.abs(diff[inside]).sum() / n_p
            g[inside] = (weight * np.sign(diff[inside]) / (3.0 * n_p))[:, None]
        grads.append(g)
    return loss, grads
