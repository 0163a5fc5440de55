"""Pins of the material smoothness oracle L_k (Appendix A, "Training details"; readings in
oracle/material_smoothness.py).

* its vectorised Philox4x32-10 against the published known-answer vectors;
* texture coordinates of the pixel-centre hits on a quad equal the analytic ray/plane
  intersection mapped through the quad's linear UV chart;
* linear ramp textures: bilinear lookups reproduce a linear function exactly away from the
  edges, so |k(x) - k(x + eps)| = |beta eps| and L = |beta| mean |eps| over the HIT pixels only;
  the mean of |eps| tends to sigma / 2 (eps uniform in [-sigma, sigma]);
* a constant texture has L = 0; a texel no lookup touches has zero gradient;
* central differences of L with respect to texels of a noise texture on a real mesh (L is
  piecewise linear in the texels, so away from sign changes the difference is exact).
"""
import os

import numpy as np
import pytest

from oracle import material_smoothness as S
from oracle import oracle as O
from paper_2406_16360_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def test_vectorised_philox_known_answers():
    rows = [[int(x, 16) for x in l.split()] for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    for w in rows:
        out = S.philox4x32_10(*(np.array([x], dtype=np.uint64) for x in w[0:4]), w[4], w[5])
        assert [int(o[0]) for o in out] == w[6:10]


def _quad_scene(half, rough_tex, albedo_tex):
    v = np.array([[-half, -half, 0.0], [half, -half, 0.0], [half, half, 0.0], [-half, half, 0.0]])
    t = np.array([[0, 1, 2], [0, 2, 3]])
    st = 0.25 + 0.5 * (v[:, :2] + half) / (2 * half)  # the quad maps to [1/4, 3/4]^2 in texture space
    uv = st[t]
    return synth._scene(v, t, uv, albedo_tex, rough_tex, np.zeros_like(rough_tex), np.ones((4, 8, 3)))


def _view(res=64):
    K, c2w = synth.look_at((0.0, 0.0, 3.0), (0.0, 0.0, 0.0), res, res, 40.0)
    return synth.View(K, c2w, res, res, 1, 1)


def _ramps(n=64, beta_r=0.5, beta_a=0.25):
    # dyadic texel values: the FP32 textures hold the ramps exactly
    c = (np.arange(n) + 0.5) / n
    rough = np.tile(0.25 + beta_r * c[None, :], (n, 1))  # ramp in s (columns)
    alb = np.full((n, n, 3), 0.5)
    alb[..., 0] = 0.125 + beta_a * c[:, None]  # ramp in t (rows), channel 0 only
    return rough.astype(np.float32), alb.astype(np.float32)


def test_texture_coordinates_on_a_quad():
    rough, alb = _ramps()
    sc = _quad_scene(2.0, rough, alb)
    v = _view(32)
    tri, st, _ = S.pixel_centre_hits(O.OracleScene(sc), v)
    assert np.all(tri >= 0)
    K = np.asarray(v.K, float)
    c2w = np.asarray(v.c2w, float).reshape(3, 4)
    py, px = np.mgrid[0:32, 0:32]
    d = np.stack([(px + 0.5 - K[2]) / K[0], (py + 0.5 - K[3]) / K[1], np.ones((32, 32))], -1).reshape(-1, 3) @ c2w[:, :3].T
    o = c2w[:, 3]
    x = o + d * (-o[2] / d[:, 2])[:, None]  # the plane z = 0
    assert np.abs(st - (0.25 + 0.5 * (x[:, :2] + 2.0) / 4.0)).max() < 1e-6


@pytest.mark.parametrize("half", [2.0, 0.6])  # the quad fills the view / leaves most pixels escaping
def test_linear_ramps_give_mean_abs_offset(half):
    rough, alb = _ramps()
    sc = _quad_scene(half, rough, alb)
    v = _view(64)
    sigma = 0.01
    osc = O.OracleScene(sc)
    tri, st, _ = S.pixel_centre_hits(osc, v)
    hit = tri >= 0
    assert (half == 2.0) == bool(hit.all())
    eps = S.offsets(64 * 64, 0, sigma, 123)
    # every lookup stays inside the exact-interpolation region
    for sh in (st[hit], st[hit] + eps[hit]):
        assert sh.min() > 0.5 / 64 and sh.max() < 1 - 0.5 / 64
    L, ga, gr, info = S.material_smoothness(osc, v, 0, sigma, 0.0, 1.0, seed=123)
    assert info["n_points"] == hit.sum()
    assert abs(L - 0.5 * np.abs(eps[hit, 0]).mean()) < 1e-12
    L, _, _, _ = S.material_smoothness(osc, v, 0, sigma, 1.0, 0.0, seed=123)
    assert abs(L - 0.25 * np.abs(eps[hit, 1]).mean() / 3.0) < 1e-12  # one channel of three
    # |eps| uniform on [0, sigma]: mean sigma / 2, standard deviation sigma / sqrt(12)
    e = np.abs(eps[hit]).ravel()
    assert abs(e.mean() - sigma / 2) < 5 * sigma / np.sqrt(12 * e.size)
    assert eps.min() >= -sigma and eps.max() < sigma


def test_constant_texture_and_untouched_texels():
    n = 16
    sc = _quad_scene(0.6, np.full((n, n), 0.4, np.float32), np.full((n, n, 3), 0.25, np.float32))
    L, ga, gr, _ = S.material_smoothness(O.OracleScene(sc), _view(32), 0, 0.02, 1.0, 1.0, seed=5)
    assert abs(L) < 1e-12
    # a quad covering s, t in [0, 1] seen through a narrow view touches only central texels
    rough, alb = _ramps(n)
    sc = _quad_scene(2.0, rough, alb)
    K, c2w = synth.look_at((0.0, 0.0, 3.0), (0.0, 0.0, 0.0), 16, 16, 10.0)
    L, ga, gr, _ = S.material_smoothness(O.OracleScene(sc), synth.View(K, c2w, 16, 16, 1, 1), 0, 0.01, 1.0, 1.0)
    assert L > 0
    assert np.all(gr[0] == 0) and np.all(gr[:, 0] == 0) and np.all(ga[-1] == 0)
    assert np.abs(gr).sum() > 0


def test_central_differences_on_a_mesh():
    sc = synth.object_scene(40, 20, 2, 16, 16, 8)
    K, c2w = synth.look_at((0.0, 1.0, 3.5), (0.0, 1.0, 0.0), 48, 48, 40.0)
    v = synth.View(K, c2w, 48, 48, 1, 1)
    osc = O.OracleScene(sc)
    sigma, wa, wr = 0.05, 0.7, 1.3
    L, ga, gr, info = S.material_smoothness(osc, v, 3, sigma, wa, wr, seed=11)
    assert info["n_points"] > 500
    rng = np.random.Generator(np.random.PCG64(4))
    th, tw = sc.roughness.shape

    def loss_with(field, idx, delta):
        a = np.asarray(sc.albedo, np.float64).copy()
        r = np.asarray(sc.roughness, np.float64).copy()
        (a if field == "a" else r).reshape(-1)[idx] += delta
        osc.scene = synth.Scene(sc.verts, sc.tris, sc.tri_uv, a, r, sc.metallic, sc.env)  # FP64 texels
        try:
            return S.material_smoothness(osc, v, 3, sigma, wa, wr, seed=11)[0]
        finally:
            osc.scene = sc

    checked = 0
    for field, g, absg in (("r", gr, info["abs_rough"]), ("a", ga, info["abs_albedo"])):
        flat = g.reshape(-1)
        cand = np.flatnonzero((np.abs(flat) > 0) & (absg.reshape(-1) == 0))
        for idx in rng.choice(cand, size=min(6, cand.size), replace=False):
            h = 1e-6
            fd = (loss_with(field, idx, h) - loss_with(field, idx, -h)) / (2 * h)
            assert abs(fd - flat[idx]) <= 1e-6 * max(1.0, abs(fd)), (field, idx, fd, flat[idx])
            checked += 1
    assert checked >= 10


# ---------------------------------------------------------------------------------------
# the normal term of L_k (interpolated vertex normals)
# ---------------------------------------------------------------------------------------
def _tetra():
    v = np.array([[1.0, 1.0, 1.0], [1.0, -1.0, -1.0], [-1.0, 1.0, -1.0], [-1.0, -1.0, 1.0]])
    t = np.array([[0, 1, 2], [0, 3, 1], [0, 2, 3], [1, 3, 2]])  # outward
    uv = np.tile(np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]]), (4, 1, 1))
    return v, t, uv


def test_vertex_normals_of_a_regular_tetrahedron_point_from_the_centre():
    from oracle.material_smoothness import vertex_normals
    v, t, _ = _tetra()
    VN, _ = vertex_normals(v, t)
    np.testing.assert_allclose(VN, v / np.linalg.norm(v, axis=1, keepdims=True), atol=1e-14)


def test_normal_term_worked_example_at_a_vertex():
    """a hit at vertex a (u = v = 0) of a face whose texture map is the identity, offset (1, 0):
    the offset point is vertex b, so the term is w / 3 sum_c |VN_a - VN_b|_c with the
    tetrahedron's radial normals"""
    from oracle.material_smoothness import normal_term
    v, t, uv = _tetra()
    loss, g, counted, _ = normal_term(v, t, uv, np.array([0]), np.array([0.0]), np.array([0.0]),
                                      np.array([[1.0, 0.0]]), 1, 0.6)
    na, nb = v[0] / np.sqrt(3.0), v[1] / np.sqrt(3.0)
    assert counted == 1
    assert abs(loss - 0.6 / 3.0 * np.abs(na - nb).sum()) < 1e-14
    # an offset of (0, 1) reaches vertex c; a half offset lands between a and b
    loss_c, _, _, _ = normal_term(v, t, uv, np.array([0]), np.array([0.0]), np.array([0.0]),
                                  np.array([[0.0, 1.0]]), 1, 0.6)
    assert abs(loss_c - 0.2 * np.abs(na - v[2] / np.sqrt(3.0)).sum()) < 1e-14
    loss_h, _, _, _ = normal_term(v, t, uv, np.array([0]), np.array([0.0]), np.array([0.0]),
                                  np.array([[0.5, 0.0]]), 1, 0.6)
    mid = (na + nb) / np.linalg.norm(na + nb)
    assert abs(loss_h - 0.2 * np.abs(na - mid).sum()) < 1e-14


def test_normal_term_vanishes_on_a_flat_mesh_and_for_a_singular_texture_map():
    from oracle.material_smoothness import normal_term
    rng = np.random.Generator(np.random.PCG64(3))
    v = np.array([[0.0, 0, 0], [1, 0, 0], [0, 0, 1], [1, 0, 1]])
    t = np.array([[0, 2, 1], [1, 2, 3]])
    uv = rng.uniform(size=(2, 3, 2))
    loss, g, counted, _ = normal_term(v, t, uv, np.array([0, 1, 1]), rng.uniform(0, 0.5, 3), rng.uniform(0, 0.5, 3),
                                      rng.uniform(-0.1, 0.1, (3, 2)), 3, 1.0)
    assert counted == 3 and loss == 0.0 and np.all(g == 0.0)
    vt, tt, uvt = _tetra()
    uvt[1] = [[0.0, 0.0], [1.0, 1.0], [2.0, 2.0]]  # collinear texture coordinates
    loss, g, counted, _ = normal_term(vt, tt, uvt, np.array([1]), np.array([0.2]), np.array([0.3]),
                                      np.array([[0.05, 0.0]]), 1, 1.0)
    assert counted == 0 and loss == 0.0 and np.all(g == 0.0)


def test_normal_term_gradient_matches_central_differences():
    """the hit (triangle, barycentrics) and the offsets held fixed, L_normal is a smooth function
    of the vertex positions away from sign changes: d L / d vertex against central differences"""
    from oracle.material_smoothness import normal_term
    from paper_2406_16360_gb300 import synth
    sc = synth.config1().scenes[0]
    v = sc.verts.astype(np.float64)[:642]  # the icosphere (the ground quad's vertices follow)
    t = sc.tris[:1280].astype(np.int64)
    uv = sc.tri_uv[:1280].astype(np.float64)
    rng = np.random.Generator(np.random.PCG64(11))
    v = v + rng.normal(scale=0.02, size=v.shape)  # away from the symmetric sphere
    n = 200
    tri = rng.integers(0, t.shape[0], n)
    u = rng.uniform(0.05, 0.45, n)
    w = rng.uniform(0.05, 0.45, n)
    eps = rng.uniform(-0.01, 0.01, (n, 2))
    loss, g, counted, _ = normal_term(v, t, uv, tri, u, w, eps, n, 0.7)
    assert counted > 0.9 * n and loss > 0
    touched = np.flatnonzero(np.abs(g).sum(1) > 0)
    for k in rng.choice(touched, size=12, replace=False):
        for c in range(3):
            h = 1e-6
            vp, vm = v.copy(), v.copy()
            vp[k, c] += h
            vm[k, c] -= h
            fd = (normal_term(vp, t, uv, tri, u, w, eps, n, 0.7)[0] - normal_term(vm, t, uv, tri, u, w, eps, n, 0.7)[0]) / (2 * h)
            assert abs(fd - g[k, c]) <= 1e-5 * abs(fd) + 1e-8, (k, c, fd, g[k, c])
