"""Pins of the oracle's monochrome light regulariser (Appendix A, L_light): the demodulated
lighting c_d + c_s of each pixel's primary vertex (oracle.light_demod), its adjoint
(oracle.light_backward) and the loss (oracle/light_loss.py).

* the loss on a small example worked out by hand;
* the demodulated lobes differ from the BRDF by exactly the diffuse reflectance:
  Q_demod - f_r cos = (1 - (1 - m) albedo) cos / pi, and Q_demod no longer depends on the
  albedo when metallic = 0;
* with metallic = 0 the demodulated lighting is the detached render with a white diffuse
  albedo (same samples, same arithmetic up to the bilinear lookup of the all-ones texture,
  whose weights need not sum to exactly 1), and an escaping pixel has none;
* a flat surface under a uniform white sky: the mean of c_d + c_s is 1 (cosine-weighted
  irradiance / pi) plus the directional albedo of the specular lobe, that one integrated by
  quadrature of the oracle's BRDF;
* the adjoint equals central differences of the detached evaluation, for every parameter.
"""
import copy

import numpy as np
import pytest

from oracle import oracle as O
from oracle.light_loss import light_loss
from paper_2406_16360_gb300 import synth


def test_loss_worked_example():
    # view 0: Y(c) = 0.6, (uncovered), 1.0 against V(ref) = 0.8, 5, 2; view 1: Y = 2 against V = 1
    c = [np.array([[0.3, 0.6, 0.9], [0.0, 0.0, 0.0], [1.0, 1.0, 1.0]]), np.array([[2.0, 2.0, 2.0]])]
    cov = [np.array([1.0, 0.0, 0.5]), np.array([1.0])]
    ref = [np.array([[0.1, 0.8, 0.2], [5.0, 5.0, 5.0], [2.0, 0.0, 0.0]]), np.array([[0.5, 1.0, 0.25]])]
    loss, g = light_loss(c, cov, ref, weight=1.5)
    # |P| = 3: (0.2 + 1 + 1) / 3, times the weight
    assert loss == pytest.approx(1.5 * 2.2 / 3.0, rel=1e-15)
    w = 1.5 / 9.0
    np.testing.assert_array_equal(g[0], [[-w] * 3, [0.0] * 3, [-w] * 3])
    np.testing.assert_array_equal(g[1], [[w] * 3])
    # nothing covered: no loss, no gradient
    loss0, g0 = light_loss([c[0]], [np.zeros(3)], [ref[0]])
    assert loss0 == 0.0 and not g0[0].any()


def test_demodulated_lobes():
    rng = np.random.Generator(np.random.PCG64(11))
    for _ in range(200):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        wo, wi = rng.normal(size=3), rng.normal(size=3)
        wo = wo / np.linalg.norm(wo) * np.sign(wo @ n)
        wi = wi / np.linalg.norm(wi) * np.sign(wi @ n)
        alb, r, m = rng.uniform(0.05, 0.95, 3), rng.uniform(0.1, 1.0), rng.uniform(0.0, 1.0)
        q0 = O.brdf_cos(n, wo, wi, alb, r, m, kind=0)
        q2 = O.brdf_cos(n, wo, wi, alb, r, m, kind=2)
        np.testing.assert_allclose(q2 - q0, (1.0 - (1.0 - m) * alb) * (n @ wi) / np.pi, rtol=1e-12, atol=1e-15)
        # metallic 0: no albedo left in the demodulated lobes
        np.testing.assert_array_equal(O.brdf_cos(n, wo, wi, alb, r, 0.0, kind=2),
                                      O.brdf_cos(n, wo, wi, rng.uniform(0, 1, 3), r, 0.0, kind=2))
        # the kind-2 gradient against central differences of its value
        g = rng.normal(size=3)
        an = O.brdf_cos_grad(n, wo, wi, alb, r, m, g, kind=2)
        h = 1e-6
        for k, (which, idx) in enumerate([("a", 0), ("a", 1), ("a", 2), ("r", 0), ("m", 0)]):
            def f(s):
                a2, r2, m2 = alb.copy(), r, m
                if which == "a":
                    a2[idx] += s
                elif which == "r":
                    r2 += s
                else:
                    m2 += s
                return g @ O.brdf_cos(n, wo, wi, a2, r2, m2, kind=2)
            fd = (f(h) - f(-h)) / (2 * h)
            assert abs(an[k] - fd) <= 1e-6 * max(1.0, abs(fd)), (k, an[k], fd)


def _scene(metallic=None):
    rng = np.random.Generator(np.random.PCG64(5))
    sc = synth.tiny_scene(subdiv=2, env_w=32, env_h=16)
    sc.albedo = rng.uniform(0.1, 0.9, size=(8, 8, 3)).astype(np.float32)
    sc.roughness = rng.uniform(0.2, 0.9, size=(8, 8)).astype(np.float32)
    sc.metallic = (rng.uniform(0.0, 0.8, size=(8, 8)) if metallic is None else np.full((8, 8), metallic)).astype(
        np.float32)
    sc.env = np.exp(rng.normal(0, 1.0, size=(16, 32, 3))).astype(np.float32)
    sc.env[3, 8] = 200.0
    return sc


@pytest.mark.parametrize("normals", [0, 1])
def test_demod_is_the_detached_render_with_white_diffuse(normals):
    sc = _scene(metallic=0.0)
    K, c2w = synth.look_at((0.4, 1.8, 3.2), (0.0, 0.8, 0.0), 20, 16, 50.0)
    view = synth.View(K, c2w, 20, 16, 4, 3)
    osc = O.OracleScene(sc, normals=normals)
    d = O.light_demod(osc, view, 0, 8, seed=4, margins=False)
    white = copy.deepcopy(sc)
    white.albedo = np.ones_like(sc.albedo)
    ref = O.render_detached(osc, O.OracleScene(white, normals=normals), view, 0, 8, seed=4)
    full, none = d["cov"] == 1.0, d["cov"] == 0.0
    assert full.sum() > 100 and none.sum() > 20
    np.testing.assert_allclose(d["c"][full], ref[full], rtol=1e-14, atol=0.0)
    assert not d["c"][none].any()
    # the demodulated lighting is not the render: the albedo is gone from it
    rgb = O.render(osc, view, 0, 8, seed=4, margins=False)["rgb"]
    assert np.abs(rgb[full] - d["c"][full]).max() > 0.1 * np.abs(d["c"][full]).max()


def test_furnace_expectation():
    # a flat quad seen through a narrow lens under a uniform white sky, direct light only
    v = np.array([[-5.0, 0, -5], [5, 0, -5], [5, 0, 5], [-5, 0, 5]])
    t = np.array([[0, 2, 1], [0, 3, 2]])
    rough = 0.5
    sc = synth._scene(v, t, np.zeros((2, 3, 2)), np.full((1, 1, 3), 0.6), np.full((1, 1), rough),
                      np.zeros((1, 1)), np.ones((16, 32, 3)))
    eye = np.array([0.0, 3.0, 3.0])
    K, c2w = synth.look_at(tuple(eye), (0.0, 0.0, 0.0), 48, 48, 4.0)
    view = synth.View(K, c2w, 48, 48, 8, 1)
    d = O.light_demod(O.OracleScene(sc), view, 0, 8, seed=9, margins=False)
    assert np.all(d["cov"] == 1.0)

    # directional albedo of the specular lobe by midpoint quadrature (albedo 0: no diffuse)
    n = np.array([0.0, 1.0, 0.0])

    def e_spec(wo):
        nt, nphi = 96, 192
        th = (np.arange(nt) + 0.5) * (0.5 * np.pi / nt)
        ph = (np.arange(nphi) + 0.5) * (2 * np.pi / nphi)
        acc = 0.0
        for a in th:
            for b in ph:
                wi = np.array([np.sin(a) * np.cos(b), np.cos(a), np.sin(a) * np.sin(b)])
                acc += O.brdf_cos(n, wo, wi, np.zeros(3), rough, 0.0)[0] * np.sin(a)
        return acc * (0.5 * np.pi / nt) * (2 * np.pi / nphi)

    wo_c = eye / np.linalg.norm(eye)
    tilt = np.radians(2.9)  # the lens's half-diagonal
    wo_lo = np.array([0.0, np.cos(np.pi / 4 + tilt), np.sin(np.pi / 4 + tilt)])
    wo_hi = np.array([0.0, np.cos(np.pi / 4 - tilt), np.sin(np.pi / 4 - tilt)])
    es = [e_spec(w) for w in (wo_c, wo_lo, wo_hi)]
    spread = max(es) - min(es)
    expect = 1.0 + es[0]
    y = d["c"].mean(axis=1)
    se = y.std(ddof=1) / np.sqrt(len(y))
    assert abs(y.mean() - expect) <= 4.0 * se + spread, (y.mean(), expect, se, spread)
    assert se < 0.01 * expect
    # grey: every channel the same
    np.testing.assert_allclose(d["c"][:, 0], d["c"][:, 2], rtol=1e-12)


@pytest.mark.parametrize("normals", [0, 1])
def test_adjoint_matches_central_differences(normals):
    sc = _scene()
    K, c2w = synth.look_at((0.3, 1.6, 3.5), (0, 0.9, 0), 14, 14, 40.0)
    view = synth.View(K, c2w, 14, 14, 2, 3)
    osc = O.OracleScene(sc, normals=normals)
    rng = np.random.Generator(np.random.PCG64(21))
    g = rng.normal(size=(14 * 14, 3))
    base = O.light_demod(osc, view, 0, 4, seed=2, margins=False)
    np.testing.assert_allclose(O.light_demod_detached(osc, osc, view, 0, 4, seed=2), base["c"], rtol=1e-14,
                               atol=1e-14)
    an = O.light_backward(osc, view, 0, 4, g, seed=2)

    def F(field, idx, delta):
        sc1 = copy.deepcopy(sc)
        x = getattr(sc1, field).reshape(-1)
        x[idx] = np.float32(x[idx] + delta)
        actual = float(x[idx]) - float(getattr(sc, field).reshape(-1)[idx])
        c = O.light_demod_detached(osc, O.OracleScene(sc1, normals=normals), view, 0, 4, seed=2)
        return float((g * c).sum()), actual

    def fd(field, idx, h):
        fp, hp = F(field, idx, h)
        fm, hm = F(field, idx, -h)
        return (fp - fm) / (hp - hm)

    for field, h in (("albedo", 1e-3), ("roughness", 1e-3), ("metallic", 1e-3), ("env", 1e-2), ("verts", 1e-4)):
        a = an[field].reshape(-1)
        cand = np.flatnonzero(np.abs(a) > 1e-3 * np.abs(a).max())
        assert len(cand) > 0, field
        pick = rng.choice(cand, size=min(6, len(cand)), replace=False)
        checked = 0
        for idx in pick:
            f1, f2 = fd(field, int(idx), h), fd(field, int(idx), h / 4)
            if abs(f1 - f2) > 1e-3 * max(abs(f1), 1e-9):
                continue  # a kink inside the step
            assert abs(a[idx] - f2) <= 2e-5 * max(abs(f2), 1e-3 * np.abs(a).max()), (field, idx, a[idx], f2)
            checked += 1
        assert checked >= 3, field
    # metallic 0 leaves the albedo untouched
    osc0 = O.OracleScene(_scene(metallic=0.0), normals=normals)
    an0 = O.light_backward(osc0, view, 0, 4, g, seed=2)
    assert not an0["albedo"].any() and an0["roughness"].any()


def test_sky_only_view_has_no_lighting_and_no_gradient():
    sc = _scene()
    K, c2w = synth.look_at((0.0, 3.0, 0.0), (0.0, 10.0, 0.5), 8, 6, 30.0)
    view = synth.View(K, c2w, 8, 6, 2, 2)
    osc = O.OracleScene(sc)
    d = O.light_demod(osc, view, 0, 4, seed=1, margins=False)
    assert not d["c"].any() and not d["cov"].any()
    an = O.light_backward(osc, view, 0, 4, np.ones((48, 3)), seed=1)
    for k in ("albedo", "roughness", "metallic", "env", "verts"):
        assert not an[k].any(), k
    # while the render's adjoint puts the sky's gradient on the env
    assert O.backward(osc, view, 0, 4, np.ones((48, 3)), seed=1)["env"].any()
