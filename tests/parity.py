"""Shared helpers of the GPU parity tests: comparison rules against the FP64 oracle.

Forward: a pixel is compared when none of its samples took a discrete decision within the
oracle's margin of its threshold (ray grazing an edge, RIS accept near the boundary, env
texel boundary, lobe threshold, ...). Compared pixels must agree to 1e-4 of the pixel's
largest channel; flagged pixels are counted and reported.

Adjoint: the seed gradient dL/dI is zeroed at flagged pixels on both sides, so both compute
the same sum; each parameter must agree to 1e-3 relative, with a floor of 1e-5 times the
sum of absolute scattered terms (the FP32 accumulation-order bound) and of 1e-6 times the
largest gradient of the tensor (FP32 rounding of terms that cancel exactly in FP64), plus
2x the oracle's FP32 sensitivity bound of the field:
  - texels: a single-precision camera ray moves the hit point by ~1e-7 of the distance, which
    shifts bilinear weight between neighbouring texels; a texel touched with a small weight
    then differs by more than 1e-3 of itself while the image does not;
  - vertices: the sum over samples and over the primary vertex's inputs (camera direction,
    barycentrics, light and continuation directions, shading normal) of the change of each
    vertex term when that input moves by its FP32 rounding scale. A vertex gradient runs
    through derivatives of the GGX lobe with respect to the normal (conditioned like 1 / alpha^2
    near the specular peak, alpha down to 2.5e-3 here), through the bilinear derivative (which
    jumps at texel centres) and, with interpolated normals, through differences of vertex
    normals; where the per-sample terms cancel, FP32 rounding of these inputs is legitimately
    visible at 1e-3 of the sum.
"""
import numpy as np

FWD_RTOL = 1e-4
GRAD_RTOL = 1e-3
GRAD_ABS_FLOOR = 1e-5
GRAD_TENSOR_FLOOR = 1e-6


def compare_pixels(gpu_rgb, or_rgb, or_margin, rtol=FWD_RTOL):
    gpu_rgb = np.asarray(gpu_rgb, dtype=np.float64).reshape(-1, 3)
    or_rgb = np.asarray(or_rgb, dtype=np.float64).reshape(-1, 3)
    scale = np.maximum(np.abs(or_rgb).max(axis=1), 1e-30)
    err = np.abs(gpu_rgb - or_rgb).max(axis=1) / scale
    flagged = or_margin < 1.0
    ok = ~flagged
    bad = ok & (err > rtol)
    return dict(n=len(err), flagged=int(flagged.sum()), failures=int(bad.sum()),
                max_err_unflagged=float(err[ok].max()) if ok.any() else 0.0,
                median_err=float(np.median(err[ok])) if ok.any() else 0.0,
                bad_idx=np.flatnonzero(bad), err=err)


def grad_tolerance(field):
    """extra keyword arguments of compare_grads for a gradient field (none: every field, vertices
    included, is compared at GRAD_RTOL plus the oracle's FP32 sensitivity bound of that field)"""
    return {}


def compare_grads(gpu, ora, ora_abs, ora_sens=None, rtol=GRAD_RTOL, floor=GRAD_ABS_FLOOR, tfloor=GRAD_TENSOR_FLOOR):
    gpu = np.asarray(gpu, dtype=np.float64).reshape(-1)
    ora = np.asarray(ora, dtype=np.float64).reshape(-1)
    ab = np.asarray(ora_abs, dtype=np.float64).reshape(-1)
    tol = rtol * np.abs(ora) + floor * ab + tfloor * (np.abs(ora).max() if len(ora) else 0.0)
    if ora_sens is not None:
        tol = tol + 2.0 * np.asarray(ora_sens, dtype=np.float64).reshape(-1)
    diff = np.abs(gpu - ora)
    bad = diff > tol
    nz = np.abs(ora) > 0
    rel = diff[nz] / np.abs(ora[nz]) if nz.any() else np.zeros(1)
    bi = np.flatnonzero(bad)
    detail = [(int(i), float(gpu[i]), float(ora[i]), float(ab[i])) for i in bi[:6]]
    return dict(n=len(ora), nonzero=int(nz.sum()), failures=int(bad.sum()), bad_idx=bi, detail=detail,
                median_rel=float(np.median(rel)) if len(rel) else 0.0, max_rel=float(rel.max()) if len(rel) else 0.0)


def compare_tapes(a, b, rtol=2e-6):
    """Two tapes of the same views (uint32 words, shape [TAPE_WORDS, n]) took the same discrete
    decisions (hit triangle, selected candidate and its texel) and hold the same floats up to
    rtol, word by word, wherever the word is defined (words 9-12 where a candidate was
    selected, 13-16 where L_ind != 0)."""
    import numpy as np
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    sel = a[1].view(np.int32) >= 0
    assert np.array_equal(a[9][sel], b[9][sel])
    fa, fb = a.view(np.float32), b.view(np.float32)
    ind = np.any(fa[3:6] != 0.0, axis=0) | np.any(fb[3:6] != 0.0, axis=0)

    def close(x, y, floor=1e-30):
        return np.all(np.abs(x - y) <= rtol * np.maximum(np.abs(x), floor))

    assert close(fa[2:9], fb[2:9])
    assert close(fa[10:13][:, sel], fb[10:13][:, sel], floor=1.0)  # unit vectors
    assert close(fa[13:16][:, ind], fb[13:16][:, ind], floor=1.0)
    assert close(fa[16][ind], fb[16][ind])
