"""Pins of the oracle's spatial reuse at the primary vertex (Appendix A, "Spatial-temporal
Reuse": reservoirs of neighbouring pixels merged into each pixel's own).

* reuse off reproduces the plain renderer exactly;
* on a flat Lambertian plane under a non-constant environment every pixel has the same target
  p_hat, so a neighbour's reservoir is a valid RIS sample here and the merged reservoir is an
  unbiased RIS estimate over sum m_i candidates: the image mean must match the exact
  irradiance (closed-form integral of L_env cos over the env texels of the upper hemisphere,
  times albedo / pi) within the statistical error, and the per-pixel variance must drop below
  that of the plain RIS estimate. A wrong normalisation of the merged weight (the candidate
  count m or the neighbour weight p_hat_here w_sum / p_hat_there) biases this mean.
"""
import math

import numpy as np

from oracle import oracle as O
from paper_2406_16360_gb300 import synth


def test_reuse_off_is_the_plain_render():
    w = synth.config1(width=20, height=16)
    osc = O.OracleScene(w.scenes[0])
    a = O.render(osc, w.views[0], 0, w.ris_m, seed=2)["rgb"]
    b = O.render(osc, w.views[0], 0, w.ris_m, seed=2, reuse=(0, 0))["rgb"]
    np.testing.assert_array_equal(a, b)
    c = O.render(osc, w.views[0], 0, w.ris_m, seed=2, reuse=(4, 3))["rgb"]
    assert np.abs(c - a).max() > 0  # reuse changes the estimate


def _plane_scene(rho, env):
    v = np.array([[-20, 0, -20], [20, 0, -20], [20, 0, 20], [-20, 0, 20]], dtype=float)
    t = np.array([[0, 2, 1], [0, 3, 2]])
    uv = np.array([((0, 0), (1, 1), (1, 0)), ((0, 0), (0, 1), (1, 1))], dtype=float)
    return synth._scene(v, t, uv, np.full((1, 1, 3), rho, np.float32), np.full((1, 1), 0.5, np.float32),
                        np.zeros((1, 1), np.float32), env)


def _exact_irradiance(env):
    """int over the upper hemisphere (y up) of L_env cos theta, texel by texel"""
    H, W = env.shape[:2]
    E = np.zeros(3)
    for r in range(H):
        t0, t1 = math.pi * r / H, min(math.pi * (r + 1) / H, math.pi / 2)
        if t0 >= math.pi / 2:
            break
        ring = 0.5 * (math.sin(t1) ** 2 - math.sin(t0) ** 2) * (2 * math.pi / W)
        E += ring * env[r].astype(np.float64).sum(0)
    return E


def test_reuse_is_unbiased_where_targets_agree_and_reduces_variance():
    env = synth.env_lognormal_sun(32, 16, seed=4, sigma=1.0, sun=60.0)
    rho = 0.6
    sc = _plane_scene(rho, env)
    K, c2w = synth.look_at((0.0, 6.0, 0.01), (0.0, 0.0, 0.0), 48, 48, 50.0)
    view = synth.View(K, c2w, 48, 48, 4, 1)
    osc = O.OracleScene(sc)
    exact = rho / math.pi * _exact_irradiance(env)
    plain = O.render(osc, view, 0, 4, seed=11, brdf_kind=1)["rgb"]
    reuse = O.render(osc, view, 0, 4, seed=11, brdf_kind=1, reuse=(6, 4))["rgb"]
    n = plain.shape[0]
    for img in (plain, reuse):
        se = img.std(0) / math.sqrt(n)
        assert np.all(np.abs(img.mean(0) - exact) <= 6 * se + 1e-9), (img.mean(0), exact, se)
    assert plain.var(0).sum() > 1.5 * reuse.var(0).sum()


def test_temporal_record_only_is_the_plain_estimate_and_history_is_consistent():
    w = synth.config1(width=20, height=16)
    v = w.views[0]
    osc = O.OracleScene(w.scenes[0])
    a = O.render(osc, v, 0, w.ris_m, seed=2)
    b = O.render(osc, v, 0, w.ris_m, seed=2, temporal=1)
    np.testing.assert_allclose(b["rgb"], a["rgb"], rtol=1e-12, atol=1e-14)
    h = b["history"]
    prim = O.render(osc, v, 0, w.ris_m, seed=2, prim=True)["prim"].reshape(-1)
    assert np.all(h[prim < 0, 0] == -1)            # escaped primary rays leave no reservoir
    hit = prim >= 0
    assert np.all(h[hit, 0] >= -2) and np.all(h[hit, 4] == w.ris_m)  # one fresh reservoir of M candidates
    sel = h[:, 0] >= 0
    assert sel.any() and np.all(h[sel, 2] > 0) and np.all(h[sel, 3] > 0)


def test_temporal_and_spatial_reuse_unbiased_where_targets_agree():
    env = synth.env_lognormal_sun(32, 16, seed=4, sigma=1.0, sun=60.0)
    rho = 0.6
    sc = _plane_scene(rho, env)
    K, c2w = synth.look_at((0.0, 6.0, 0.01), (0.0, 0.0, 0.0), 48, 48, 50.0)
    view = synth.View(K, c2w, 48, 48, 4, 1)
    osc = O.OracleScene(sc)
    exact = rho / math.pi * _exact_irradiance(env)
    plain = O.render(osc, view, 0, 4, seed=12, brdf_kind=1)["rgb"]
    for reuse in ((0, 0), (4, 4)):
        f1 = O.render(osc, view, 0, 4, seed=11, brdf_kind=1, reuse=reuse, temporal=1)
        f2 = O.render(osc, view, 0, 4, seed=12, brdf_kind=1, reuse=reuse, temporal=2, temporal_cap=8,
                      history=f1["history"])
        img = f2["rgb"]
        se = img.std(0) / math.sqrt(img.shape[0])
        assert np.all(np.abs(img.mean(0) - exact) <= 6 * se + 1e-9), (reuse, img.mean(0), exact, se)
        assert plain.var(0).sum() > 1.3 * img.var(0).sum(), reuse
        hit = f2["history"][:, 4] > 0
        assert np.all(f2["history"][hit, 4] >= 4 + 1)  # the history's candidates were counted too
