"""Pins of the oracle's environment sampling, BRDF and continuation sampling.

  * Env proposal (Sec. 4.1, q_dir proportional to L_env): closed-form texel probabilities for a
    constant map (proportional to sin(theta_row)), pdf integrates to 1 over the sphere, samples
    land in their texel, sample frequencies follow the table, black rows are never drawn.
  * BRDF (Sec. 3.2, GGX + Lambert): GGX D normalisation, visible-normal normalisation (G1),
    closed-form value at normal incidence, reciprocity, Fresnel endpoints, analytic gradient
    against central differences.
  * Sampling (Sec. 4.2, MIS of light and GGX sampling): E[phi / pdf] equals the exact integral
    of phi for the VNDF sampler and for the full one-sample mixture.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import oracle as O
from paper_2406_16360_gb300 import synth


def _scene_with_env(env):
    return synth._scene(np.zeros((3, 3), np.float32), np.zeros((0, 3), np.int32), np.zeros((0, 3, 2)),
                        np.full((1, 1, 3), 0.5), np.full((1, 1), 0.5), np.zeros((1, 1)), env)


def _sphere_grid(nt, nphi):
    th = (np.arange(nt) + 0.5) * np.pi / nt
    ph = (np.arange(nphi) + 0.5) * 2 * np.pi / nphi - np.pi
    T, P = np.meshgrid(th, ph, indexing="ij")
    d = np.stack([np.sin(T) * np.sin(P), np.cos(T), -np.sin(T) * np.cos(P)], -1).reshape(-1, 3)
    w = (np.sin(T) * (np.pi / nt) * (2 * np.pi / nphi)).reshape(-1)
    return d, w


def test_env_constant_map_closed_form():
    W, H = 16, 8
    osc = O.OracleScene(_scene_with_env(np.full((H, W, 3), 2.0, np.float32)))
    cond, marg, prob, total = osc.env_tables()
    st = np.sin(np.pi * (np.arange(H) + 0.5) / H)
    np.testing.assert_allclose(prob, np.repeat((st / (W * st.sum()))[:, None], W, 1), rtol=1e-14)
    np.testing.assert_allclose(total, 2.0 * W * st.sum(), rtol=1e-14)
    np.testing.assert_allclose(cond, np.tile(np.arange(W + 1) / W, (H, 1)), rtol=0, atol=1e-15)
    assert marg[0] == 0.0 and marg[-1] == 1.0 and np.all(np.diff(marg) > 0)


def test_env_pdf_integrates_to_one_and_samples_follow_table():
    rng = np.random.Generator(np.random.PCG64(1))
    W, H = 8, 4
    env = np.exp(rng.normal(0, 1.5, size=(H, W, 3))).astype(np.float32)
    env[1] = 0.0  # a black row
    osc = O.OracleScene(_scene_with_env(env))
    cond, marg, prob, total = osc.env_tables()
    assert np.all(prob[1] == 0) and abs(prob.sum() - 1) < 1e-14
    d, w = _sphere_grid(H * 24, W * 24)
    pdf = np.array([O.env_pdf(osc, x) for x in d])
    assert abs((pdf * w).sum() - 1.0) < 2e-3
    # sampling: frequencies vs table, samples inside their texel
    n = 40000
    words = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    counts = np.zeros(W * H)
    for k in range(n):
        dirv, tex, p = O.env_sample(osc, words[k])
        counts[tex] += 1
        if k < 2000:
            assert O.env_texel(osc, dirv) == tex
            np.testing.assert_allclose(p, O.env_pdf(osc, dirv), rtol=1e-9)
    exp = prob.reshape(-1) * n
    assert counts[exp == 0].sum() == 0
    m = exp > 0
    chi2 = (((counts[m] - exp[m]) ** 2) / exp[m]).sum()
    dof = m.sum() - 1
    assert chi2 < dof + 6 * math.sqrt(2 * dof)


def test_env_draw_inverts_the_texel_cdf_with_a_53_bit_uniform():
    """the draw takes u = (w0 2^21 + (w1 >> 11)) / 2^53 and the texel t with flat[t] <= u <
    flat[t + 1]; flat is the marginal-times-conditional factorisation written out per texel"""
    rng = np.random.Generator(np.random.PCG64(2))
    W, H = 8, 4
    env = np.exp(rng.normal(0, 1.5, size=(H, W, 3))).astype(np.float32)
    env[2, 3] = 0.0  # a black texel
    osc = O.OracleScene(_scene_with_env(env))
    cond, marg, prob, total = osc.env_tables()
    flat = osc.env_flat()
    fact = (marg[:-1, None] + (marg[1:] - marg[:-1])[:, None] * cond[:, :-1]).reshape(-1)
    np.testing.assert_allclose(flat[:-1], fact, rtol=0, atol=1e-15)
    assert flat[-1] == 1.0 and np.all(np.diff(flat) >= 0)
    np.testing.assert_allclose(np.diff(flat), prob.reshape(-1), rtol=0, atol=1e-15)
    words = rng.integers(0, 2 ** 32, size=(3000, 4), dtype=np.uint64).astype(np.uint32)
    words[0, :2] = 0  # u = 0: the first texel with weight
    words[1, :2] = 0xFFFFFFFF  # u just below 1: the last texel with weight
    for k in range(len(words)):
        _, tex, _ = O.env_sample(osc, words[k])
        u = ((int(words[k, 0]) << 21) | (int(words[k, 1]) >> 11)) / 2.0 ** 53
        assert flat[tex] <= u < flat[tex + 1], (k, tex, u)
        assert tex != 2 * W + 3


@pytest.mark.parametrize("alpha", [0.05, 0.3, 1.0])
def test_ggx_d_normalised(alpha):
    val, _ = integrate.quad(lambda mu: 2 * np.pi * O.ggx_d(alpha, mu) * mu, 0, 1, limit=200, points=[1 - alpha])
    assert abs(val - 1.0) < 1e-8


def test_ggx_and_smith_closed_forms():
    for a in (0.1, 0.5, 1.0):
        assert O.ggx_d(a, 1.0) == pytest.approx(1 / (np.pi * a * a), rel=1e-14)
        assert O.ggx_d(a, 0.0) == pytest.approx(a * a / np.pi, rel=1e-14)
        assert O.smith_g1(a, 1.0) == pytest.approx(1.0, rel=1e-14)
    for c in (0.1, 0.5, 0.9):
        assert O.smith_g1(1.0, c) == pytest.approx(2 * c / (c + 1), rel=1e-14)


@pytest.mark.parametrize("alpha,theta_o", [(0.3, 0.2), (0.6, 1.0), (0.9, 1.3)])
def test_visible_normals_normalised(alpha, theta_o):
    # int G1(wo) max(0, wo.m) D(m) / cos_o dm = 1 over the hemisphere of m
    wo = np.array([math.sin(theta_o), 0.0, math.cos(theta_o)])

    def f(phi, mu):
        s = math.sqrt(max(0.0, 1 - mu * mu))
        m = np.array([s * math.cos(phi), s * math.sin(phi), mu])
        return O.smith_g1(alpha, wo[2]) * max(0.0, float(wo @ m)) * O.ggx_d(alpha, mu) / wo[2]

    val, _ = integrate.dblquad(f, 0, 1, 0, 2 * np.pi, epsabs=1e-7, epsrel=1e-7)
    assert abs(val - 1.0) < 1e-5


def test_brdf_normal_incidence_reciprocity_fresnel():
    n = np.array([0, 0, 1.0])
    alb = np.array([0.2, 0.5, 0.8])
    for r, m in [(0.5, 0.0), (0.7, 0.3), (0.2, 1.0)]:
        a = max(r * r, 1e-3)
        val = O.brdf_cos(n, n, n, alb, r, m)
        f0 = 0.04 * (1 - m) + m * alb
        np.testing.assert_allclose(val, (1 - m) * alb / np.pi + f0 / (4 * np.pi * a * a), rtol=1e-13)
    rng = np.random.Generator(np.random.PCG64(5))
    for _ in range(50):
        wo, wi = rng.normal(size=3), rng.normal(size=3)
        wo[2], wi[2] = abs(wo[2]) + 0.05, abs(wi[2]) + 0.05
        wo, wi = wo / np.linalg.norm(wo), wi / np.linalg.norm(wi)
        r, m = rng.uniform(0.05, 1), rng.uniform(0, 1)
        f1 = O.brdf_cos(n, wo, wi, alb, r, m) / wi[2]
        f2 = O.brdf_cos(n, wi, wo, alb, r, m) / wo[2]
        np.testing.assert_allclose(f1, f2, rtol=1e-12)
    # below either horizon the product is zero
    assert np.all(O.brdf_cos(n, np.array([0, 0, 1.0]), np.array([0, 0.6, -0.8]), alb, 0.5, 0) == 0)
    # Schlick: with metallic 1 the ratio F(F0 = 0) / F(F0 = 1) is (1 - wo.h)^5 exactly
    for th in (0.3, 1.0, 1.5):
        wo = np.array([math.sin(th), 0, math.cos(th)])
        wi = np.array([-math.sin(th) * 0.8, 0.6 * math.sin(th), math.cos(th)])
        wi /= np.linalg.norm(wi)
        h = (wo + wi) / np.linalg.norm(wo + wi)
        s0 = O.brdf_cos(n, wo, wi, np.zeros(3), 0.5, 1.0)
        s1 = O.brdf_cos(n, wo, wi, np.ones(3), 0.5, 1.0)
        np.testing.assert_allclose(s0 / s1, (1 - wo @ h) ** 5, rtol=1e-12)


def test_brdf_gradient_central_differences():
    rng = np.random.Generator(np.random.PCG64(11))
    for _ in range(40):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        wo, wi = rng.normal(size=3), rng.normal(size=3)
        wo += 2 * n
        wi += 2 * n
        wo /= np.linalg.norm(wo)
        wi /= np.linalg.norm(wi)
        if wo @ n < 0.05 or wi @ n < 0.05:
            continue
        alb = rng.uniform(0.05, 0.95, 3)
        r, m = rng.uniform(0.1, 0.95), rng.uniform(0.05, 0.95)
        g = rng.normal(size=3)
        an = O.brdf_cos_grad(n, wo, wi, alb, r, m, g)
        x0 = np.concatenate([alb, [r, m], n])

        def F(x):
            return g @ O.brdf_cos(x[5:8], wo, wi, x[0:3], x[3], x[4])

        h = 1e-6
        fd = np.array([(F(x0 + h * e) - F(x0 - h * e)) / (2 * h) for e in np.eye(8)])
        np.testing.assert_allclose(an, fd, rtol=2e-6, atol=2e-7 * np.abs(fd).max())


def _mc_check(samples_pdf_fn, phi, exact, n):
    vals = np.empty(n)
    for i in range(n):
        d, p = samples_pdf_fn(i)
        vals[i] = phi(d) / p if p > 0 else 0.0
    mean, se = vals.mean(), vals.std() / math.sqrt(n)
    assert abs(mean - exact) < 4.5 * se + 1e-12, (mean, exact, se)


def test_vndf_sampling_matches_its_pdf():
    rng = np.random.Generator(np.random.PCG64(2))
    n_ = np.array([0.3, 0.8, 0.52])
    n_ /= np.linalg.norm(n_)
    wo = np.array([0.9, 0.1, 0.2]) + n_
    wo /= np.linalg.norm(wo)
    for alpha in (0.15, 0.6):
        u = rng.uniform(size=(20000, 2))

        def sp(i):
            d = O.vndf_sample(n_, wo, alpha, u[i, 0], u[i, 1])
            return d, O.vndf_pdf(n_, wo, d, alpha)

        # E[phi / p] over the upper hemisphere of n: int cos^2 = 2 pi / 3
        _mc_check(sp, lambda d: max(0.0, d @ n_) ** 2, 2 * np.pi / 3, 20000)


def test_continuation_mixture_matches_its_pdf():
    rng = np.random.Generator(np.random.PCG64(4))
    env = np.exp(rng.normal(0, 1.0, size=(16, 32, 3))).astype(np.float32)
    osc = O.OracleScene(_scene_with_env(env))
    n_ = np.array([0.0, 1.0, 0.0])
    wo = np.array([0.5, 0.8, 0.1])
    wo /= np.linalg.norm(wo)
    alb = np.array([0.6, 0.4, 0.2])
    words = rng.integers(0, 2 ** 32, size=(30000, 4), dtype=np.uint64).astype(np.uint32)

    def sp(i):
        d, p = O.sample_continuation(osc, n_, wo, alb, 0.4, 0.3, words[i])
        assert p == pytest.approx(O.pdf_continuation(osc, n_, wo, alb, 0.4, 0.3, d), rel=1e-12)
        return d, p

    # the env lobe covers the whole sphere: E[1 / p] = 4 pi
    _mc_check(sp, lambda d: 1.0, 4 * np.pi, 30000)
    # quadrature: the mixture pdf integrates to one
    d, w = _sphere_grid(128, 256)
    pdf = np.array([O.pdf_continuation(osc, n_, wo, alb, 0.4, 0.3, x) for x in d])
    assert abs((pdf * w).sum() - 1.0) < 5e-3
