"""Pins of the oracle's FULL-mode adjoint (the gradients of the indirect rays that Sec. 4.2
detaches and Appendix C lists as the method's missing part).

FULL mode differentiates the detached estimator over the whole path: every vertex's direct
term and every vertex's BRDF factor on the light from the rest of the path, with sampling
decisions, RIS weights, visibility and p_ind held fixed and the hit points after the primary
vertex held fixed on their triangles.

Pinned by
* the detached forward at eval == frozen reproducing the forward render (the recorded path);
* Euler's theorem for homogeneous functions, checked against forward renders only: with a
  Lambert BRDF (f = albedo cos / pi) the radiance a path collects at vertex b is a product of
  b + 1 albedo factors and one env factor, so sum_i theta_i dL/dtheta_i over all albedo texels
  is sum_b (b + 1) L_b in FULL mode and L in PRIMARY mode (the sky seen directly excluded),
  and over all env texels it is L in FULL mode and L_0 in PRIMARY mode. L_b = render(bounces b + 1) - render(bounces b), because
  the random counters of the first vertices do not depend on the bounce count;
* central differences of the detached FULL forward for every material field and the env.
"""
import copy

import numpy as np
import pytest

from oracle import oracle as O
from paper_2406_16360_gb300 import synth


def _scene(tex=6, seed=31):
    rng = np.random.Generator(np.random.PCG64(seed))
    sc = synth.tiny_scene(subdiv=2, env_w=16, env_h=8)
    sc.albedo = rng.uniform(0.3, 0.95, size=(tex, tex, 3)).astype(np.float32)
    sc.roughness = rng.uniform(0.2, 0.9, size=(tex, tex)).astype(np.float32)
    sc.metallic = rng.uniform(0.0, 0.6, size=(tex, tex)).astype(np.float32)
    sc.env = np.exp(rng.normal(0, 1.0, size=(8, 16, 3))).astype(np.float32)
    sc.env[2, 5] = 40.0
    K, c2w = synth.look_at((0.3, 1.6, 3.5), (0, 0.9, 0), 12, 12, 40.0)
    return sc, K, c2w, rng


def _view(K, c2w, bounces, spp=2):
    return synth.View(K, c2w, 12, 12, spp, bounces)


@pytest.mark.parametrize("mode", [0, 1])
def test_detached_forward_at_frozen_is_the_forward(mode):
    sc, K, c2w, rng = _scene()
    view = _view(K, c2w, 4)
    osc = O.OracleScene(sc)
    fwd = O.render(osc, view, 0, 4, seed=3, margins=False)["rgb"]
    det = O.render_detached(osc, osc, view, 0, 4, seed=3, grad_mode=mode)
    np.testing.assert_allclose(det, fwd, rtol=1e-12, atol=1e-14)


def test_full_mode_rejects_too_many_bounces():
    sc, K, c2w, rng = _scene()
    osc = O.OracleScene(sc)
    view = _view(K, c2w, 17)
    with pytest.raises(ValueError):
        O.backward(osc, view, 0, 4, np.ones((144, 3)), seed=3, grad_mode=1)


def test_euler_homogeneity_against_forward_renders():
    sc, K, c2w, rng = _scene()
    sc.metallic[:] = 0.0
    B = 4
    osc = O.OracleScene(sc)
    n = 144
    g = rng.normal(size=(n, 3))
    # per-bounce radiance from forward renders alone (Lambert BRDF)
    Lb = [np.zeros((n, 3))]
    for b in range(1, B + 1):
        Lb.append(O.render(osc, _view(K, c2w, b), 0, 4, seed=5, brdf_kind=1, margins=False)["rgb"])
    per = [Lb[b + 1] - Lb[b] for b in range(B)]  # radiance collected at vertex b (b = 0: and the sky)
    L = Lb[B]
    # the sky seen by primary rays that escape carries no albedo factor: a render with black
    # albedo keeps exactly that part
    dark = copy.deepcopy(sc)
    dark.albedo[:] = 0.0
    BG = O.render(O.OracleScene(dark), _view(K, c2w, B), 0, 4, seed=5, brdf_kind=1, margins=False)["rgb"]
    assert float(BG.sum()) > 0
    assert all(float(np.abs(p).sum()) > 0 for p in per[:3]), "every vertex must contribute"
    view = _view(K, c2w, B)
    for mode in (0, 1):
        gr = O.backward(osc, view, 0, 4, g, seed=5, brdf_kind=1, grad_mode=mode, want_abs=False)
        alb_side = float((sc.albedo.astype(np.float64) * gr["albedo"]).sum())
        env_side = float((sc.env.astype(np.float64) * gr["env"]).sum())
        if mode == 1:
            alb_ref = float(sum((b + 1) * (g * per[b]).sum() for b in range(B)) - (g * BG).sum())
            env_ref = float((g * L).sum())
        else:
            alb_ref = float((g * (L - BG)).sum())
            env_ref = float((g * per[0]).sum())
        assert abs(alb_side - alb_ref) <= 1e-9 * max(abs(alb_ref), 1.0), (mode, alb_side, alb_ref)
        assert abs(env_side - env_ref) <= 1e-9 * max(abs(env_ref), 1.0), (mode, env_side, env_ref)
    # FULL adds the later vertices' terms: it must differ from PRIMARY where the path bounces
    p0 = O.backward(osc, view, 0, 4, g, seed=5, brdf_kind=1, grad_mode=0, want_abs=False)
    p1 = O.backward(osc, view, 0, 4, g, seed=5, brdf_kind=1, grad_mode=1, want_abs=False)
    assert np.abs(p1["albedo"] - p0["albedo"]).max() > 1e-6 * np.abs(p0["albedo"]).max()
    np.testing.assert_array_equal(p1["verts"], p0["verts"])  # geometry: primary vertex only


def _fd(sc0, view, g, field, idx, h, mode):
    def F(delta):
        sc1 = copy.deepcopy(sc0)
        x = getattr(sc1, field).reshape(-1)
        x[idx] = np.float32(x[idx] + delta)
        actual = float(x[idx]) - float(getattr(sc0, field).reshape(-1)[idx])
        rgb = O.render_detached(O.OracleScene(sc0), O.OracleScene(sc1), view, 0, 4, seed=2, grad_mode=mode)
        return float((g * rgb).sum()), actual

    fp, hp = F(h)
    fm, hm = F(-h)
    return (fp - fm) / (hp - hm)


@pytest.mark.parametrize("field,h", [("albedo", 1e-3), ("roughness", 1e-3), ("metallic", 1e-3), ("env", 1e-2),
                                     ("verts", 1e-4)])
def test_full_adjoint_matches_central_differences(field, h):
    sc, K, c2w, rng = _scene(tex=4, seed=21)
    view = _view(K, c2w, 3)
    osc = O.OracleScene(sc)
    g = rng.normal(size=(144, 3))
    gr = O.backward(osc, view, 0, 4, g, seed=2, grad_mode=1, want_abs=False)
    gp = O.backward(osc, view, 0, 4, g, seed=2, grad_mode=0, want_abs=False)
    an = gr[field].reshape(-1)
    # prefer texels where the later vertices change the gradient
    diff = np.abs(an - gp[field].reshape(-1))
    cand = np.flatnonzero(diff > 1e-6 * np.abs(an).max()) if field != "verts" else np.array([], int)
    if len(cand) < 4:
        cand = np.flatnonzero(np.abs(an) > 1e-6 * np.abs(an).max())
    assert len(cand) > 0
    pick = rng.choice(cand, size=min(8, len(cand)), replace=False)
    checked = 0
    for idx in pick:
        fd = _fd(sc, view, g, field, int(idx), h, 1)
        fd2 = _fd(sc, view, g, field, int(idx), h / 4, 1)
        if abs(fd - fd2) > 1e-3 * max(abs(fd), 1e-9):
            continue  # a kink (bilinear cell edge, horizon) inside the step
        assert abs(an[idx] - fd2) <= 2e-5 * max(abs(fd2), 1e-3 * np.abs(an).max()), (field, idx, an[idx], fd2)
        checked += 1
    assert checked >= min(5, len(pick))
