"""Pins of the oracle's estimators (Sec. 4.1 RIS / Appendix A WRS, Eq. pbr_render, Eq. incident).

  * WRS accept rule and exact unbiasedness of the RIS estimator on a tiny discrete domain,
    by enumeration of every candidate tuple and of every selection outcome.
  * RIS selection distribution tends to p_hat / sum(p_hat) as M grows.
  * White furnace: a convex Lambertian object of albedo 1 under a constant environment returns
    the environment radiance (the expectation; the estimator is noisy), albedo rho gives rho L,
    a ground plane alone gives rho L.
  * Full GGX + Lambert BRDF, coloured albedo and coloured constant env, one pixel with a
    needle camera: the mean equals L * int f_r cos (quadrature of the pinned BRDF). Here
    f / p_hat varies with direction, so the selection and the RIS weight are exercised.
  * Variance: RIS with M candidates beats plain env importance sampling (M = 1) at equal spp
    (the synthetic analogue of the paper's Fig. 3 / Table 3 reservoir ablation).
"""
import itertools
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import oracle as O
from paper_2406_16360_gb300 import synth


def test_wrs_accept_rule():
    assert O.wrs([1.0, 3.0], [0.0, 0.7499999])[0] == 1   # 0.7499999 * 4 < 3
    assert O.wrs([1.0, 3.0], [0.0, 0.75])[0] == 0        # 0.75 * 4 == 3: strict, not accepted
    assert O.wrs([2.0, 1.0], [0.999999, 0.999999])[0] == 0  # the first positive weight is always kept
    sel, ws = O.wrs([0.0, 0.0, 0.0], [0.0, 0.0, 0.0])
    assert sel == -1 and ws == 0.0                           # a zero weight is never accepted
    assert O.wrs([0.0, 5.0, 0.0], [0.3, 0.9, 0.0]) == (1, 5.0)


def _accept_threshold(gammas, k):
    """measure of {u_k : step k accepts}, found by bisection on the oracle's own WRS"""
    lo, hi = 0.0, 1.0
    g = list(gammas[:k + 1])
    u = [0.5] * (k + 1)
    u[k] = 0.0
    if O.wrs(g, u)[0] != k:
        return 0.0
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        u[k] = mid
        if O.wrs(g, u)[0] == k:
            lo = mid
        else:
            hi = mid
    return lo


def test_ris_unbiased_by_exact_enumeration():
    # discrete domain of K items; target f, unnormalised p_hat > 0 where f != 0, proposal q
    f = np.array([0.3, 0.0, 1.7, 0.9])
    phat = np.array([0.5, 0.2, 1.0, 1.1])
    q = np.array([0.4, 0.3, 0.2, 0.1])
    K = len(f)
    for M in (1, 2, 3):
        expect = 0.0
        sel_prob = np.zeros(K)
        for tup in itertools.product(range(K), repeat=M):
            w_tup = float(np.prod(q[list(tup)]))
            gam = [phat[x] / q[x] for x in tup]
            t = [_accept_threshold(gam, k) for k in range(M)]
            _, wsum = O.wrs(gam, [0.0] * M)
            for j in range(M):
                pj = t[j] * np.prod([1.0 - t[k] for k in range(j + 1, M)])
                if pj == 0.0:
                    continue
                x = tup[j]
                W = wsum / (M * phat[x])  # Eq. restir with N = 1
                expect += w_tup * pj * f[x] * W
                sel_prob[x] += w_tup * pj
        assert abs(expect - f.sum()) < 1e-12, (M, expect, f.sum())
        assert abs(sel_prob.sum() - 1.0) < 1e-12


def test_ris_selection_tends_to_target():
    rng = np.random.Generator(np.random.PCG64(9))
    phat = np.array([0.5, 0.2, 1.0, 1.1, 3.0])
    q = np.full(5, 0.2)
    M, trials = 64, 20000
    counts = np.zeros(5)
    for _ in range(trials):
        xs = rng.integers(0, 5, size=M)
        sel, _ = O.wrs(phat[xs] / q[xs], rng.uniform(size=M))
        counts[xs[sel]] += 1
    np.testing.assert_allclose(counts / trials, phat / phat.sum(), atol=0.015)


def _sphere_only(albedo, env_value, roughness=0.5, metallic=0.0, subdiv=3):
    sc = synth.tiny_scene(albedo=albedo, roughness=roughness, metallic=metallic, env_value=env_value, sun=None,
                          ground=False, subdiv=subdiv)
    return sc


def _stats(img, mask):
    v = img[mask]
    return v.mean(axis=0), v.std(axis=0) / math.sqrt(len(v))


@pytest.mark.parametrize("rho", [1.0, 0.3])
def test_white_furnace_lambert(rho):
    L = 0.7
    sc = _sphere_only(rho, L)
    osc = O.OracleScene(sc)
    K, c2w = synth.look_at((0, 1.0, 3.2), (0, 1.0, 0), 48, 48, 45.0)
    view = synth.View(K, c2w, 48, 48, 16, 2)
    r = O.render(osc, view, 0, 8, seed=3, brdf_kind=1, prim=True, margins=False)
    img = r["rgb"]
    hit = (r["prim"] >= 0).all(axis=1)
    miss = (r["prim"] < 0).all(axis=1)
    assert hit.sum() > 300 and miss.sum() > 300
    np.testing.assert_array_equal(img[miss], np.full((miss.sum(), 3), np.float32(L)))
    mean, se = _stats(img, hit)
    assert np.all(np.abs(mean - rho * np.float32(L)) < 4 * se + 1e-12), (mean, se)
    assert np.all(se < 0.01 * L)


def test_ground_plane_alone():
    rho, L = 0.4, 1.3
    v = np.array([[-5, 0, -5], [5, 0, -5], [5, 0, 5], [-5, 0, 5]], dtype=np.float32)
    t = np.array([[0, 2, 1], [0, 3, 2]])
    sc = synth._scene(v, t, np.zeros((2, 3, 2)), np.full((1, 1, 3), rho), np.full((1, 1), 0.5),
                      np.zeros((1, 1)), np.full((16, 32, 3), L))
    osc = O.OracleScene(sc)
    K, c2w = synth.look_at((0, 2.0, 2.0), (0, 0.0, 0), 32, 32, 40.0)
    r = O.render(osc, synth.View(K, c2w, 32, 32, 16, 3), 0, 8, seed=1, brdf_kind=1, prim=True, margins=False)
    hit = (r["prim"] >= 0).all(axis=1)
    assert hit.all()
    mean, se = _stats(r["rgb"], hit)
    assert np.all(np.abs(mean - np.float32(rho) * np.float32(L)) < 4 * se + 1e-12)


def test_full_brdf_coloured_furnace_single_pixel():
    alb = np.array([0.2, 0.5, 0.9], dtype=np.float32)
    Lc = np.array([0.3, 0.7, 1.2], dtype=np.float32)
    sc = synth.tiny_scene(albedo=0.5, roughness=0.5, metallic=0.0, env_value=1.0, sun=None, ground=False)
    sc.albedo[:] = alb
    sc.env[:] = Lc
    osc = O.OracleScene(sc)
    eye = np.array([0.4, 1.5, 3.0])
    target = np.array([0.1, 1.2, 0.5])
    K, c2w = synth.look_at(eye, target, 1, 1, 1e-4)
    view = synth.View(K, c2w, 1, 1, 40000, 2)
    # the hit triangle and its face normal
    d0 = (target - eye) / np.linalg.norm(target - eye)
    tri, tuv, _ = O.trace(osc, [eye], [d0], mode=0)
    assert tri[0] >= 0
    p = sc.verts[sc.tris[tri[0]]].astype(np.float64)
    n = np.cross(p[1] - p[0], p[2] - p[0])
    n /= np.linalg.norm(n)
    if n @ d0 > 0:
        n = -n
    wo = -d0
    # quadrature of int f_r cos over the hemisphere of n
    t1 = np.cross(n, [0.0, 0.0, 1.0])
    t1 /= np.linalg.norm(t1)
    t2 = np.cross(n, t1)

    def comp(ch):
        def fn(phi, mu):
            s = math.sqrt(max(0.0, 1 - mu * mu))
            wi = s * math.cos(phi) * t1 + s * math.sin(phi) * t2 + mu * n
            return O.brdf_cos(n, wo, wi, alb, 0.5, 0.0)[ch]  # f_r cos; d omega = d mu d phi
        return integrate.dblquad(fn, 0, 1, 0, 2 * np.pi, epsabs=1e-8, epsrel=1e-7)[0]

    A = np.array([comp(c) for c in range(3)])
    expect = Lc.astype(np.float64) * A
    r = O.render(osc, view, 0, 8, seed=5, margins=False, threads=8)
    # standard error of the 40000-sample mean from four independent 10000-sample renders
    halves = []
    for seed in (11, 12, 13, 14):
        v2 = synth.View(K, c2w, 1, 1, 10000, 2)
        halves.append(O.render(osc, v2, 0, 8, seed=seed, margins=False, threads=8)["rgb"][0])
    se = np.std(halves, axis=0, ddof=1) / 2.0
    got = r["rgb"][0]
    assert np.all(np.abs(got - expect) < 5 * se + 1e-12), (got, expect, se)
    assert np.all(np.abs(got - expect) / expect < 0.01)


def test_ris_variance_below_plain_importance_sampling():
    w = synth.config1(width=24, height=24)
    osc = O.OracleScene(w.scenes[0])
    view = w.views[0]
    imgs = {1: [], 8: []}
    for m in imgs:
        for seed in range(8):
            imgs[m].append(O.render(osc, view, 0, m, seed=seed, margins=False)["rgb"])
    var = {m: np.var(np.stack(imgs[m]), axis=0).mean() for m in imgs}
    assert var[8] < 0.8 * var[1], var
