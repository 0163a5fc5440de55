"""Pins of the oracle's interpolated shading normals (OracleScene(..., normals=1)).

The paper shades with "the surface normal" without saying how it is formed; the face normal
is the default reading, and the interpolated one -- the barycentric blend of area-weighted
vertex normals, turned to the viewer's side of the face, with light and continuation
directions below the face dropped -- is the option pinned here:

* a regular tetrahedron's vertex normal points from its centre to the vertex (symmetry), and
  an icosphere's vertex normals are radial to within a degree;
* on a flat mesh the interpolated normal is the face normal: the renders agree;
* the leak rule: a roof whose left face does not see the only light stays black even where
  its interpolated normal leans towards the light, while the right face is lit;
* the adjoint through the interpolated normal (to the barycentrics and, through the vertex
  normals, to every face around the hit triangle's vertices) equals central differences of the
  detached forward.
"""
import copy

import numpy as np
import pytest

from oracle import oracle as O
from paper_2406_16360_gb300 import synth


def test_vertex_normals_tetrahedron_and_icosphere():
    tet = 0.8 * np.array([[1.0, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]])
    tris = np.array([[0, 1, 2], [0, 3, 1], [0, 2, 3], [1, 3, 2]])
    sc = synth._scene(tet, tris, np.zeros((4, 3, 2)), np.full((1, 1, 3), 0.5), np.full((1, 1), 0.5),
                      np.zeros((1, 1)), np.ones((4, 8, 3)))
    vn = O.OracleScene(sc, normals=1).vertex_normals()
    ref = tet.astype(np.float32).astype(np.float64)
    ref /= np.linalg.norm(ref, axis=1, keepdims=True)
    # outward or inward depending on the winding; the direction is the pin
    assert np.abs(np.abs((vn * ref).sum(1)) - 1.0).max() < 1e-12
    ico = synth.tiny_scene(subdiv=3, ground=False)
    vn = O.OracleScene(ico, normals=1).vertex_normals()
    r = ico.verts.astype(np.float64) - np.array([0.0, 1.0, 0.0])
    r /= np.linalg.norm(r, axis=1, keepdims=True)
    ang = np.degrees(np.arccos(np.clip(np.abs((vn * r).sum(1)), -1, 1)))
    assert ang.max() < 1.0


def test_flat_mesh_interpolated_equals_face_normals():
    # a ground quad of several coplanar triangles, seen from above
    x = np.linspace(-2, 2, 4)
    gx, gz = np.meshgrid(x, x)
    v = np.c_[gx.ravel(), np.zeros(16), gz.ravel()]
    t = []
    for i in range(3):
        for j in range(3):
            a = i * 4 + j
            t += [[a, a + 4, a + 1], [a + 1, a + 4, a + 5]]
    t = np.array(t)
    base = synth.tiny_scene()
    sc = synth._scene(v, t, np.zeros((len(t), 3, 2)), base.albedo, base.roughness, base.metallic, base.env)
    K, c2w = synth.look_at((0.3, 2.0, 1.5), (0.0, 0.0, 0.0), 12, 10)
    view = synth.View(K, c2w, 12, 10, 2, 2)
    a = O.render(O.OracleScene(sc, normals=0), view, 0, 4, seed=3, margins=False)["rgb"]
    b = O.render(O.OracleScene(sc, normals=1), view, 0, 4, seed=3, margins=False)["rgb"]
    assert np.abs(a - b).max() <= 1e-12 * max(1.0, np.abs(a).max())


def _roof():
    # two faces meeting at a ridge along z (x = 0, y = 1), sloping down to y = 0 at x = -1 / +1;
    # near the ridge the interpolated normal leans from each face towards the other
    v = np.array([[-1.0, 0, -1], [-1, 0, 1], [0, 1, -1], [0, 1, 1], [1, 0, -1], [1, 0, 1]])
    t = np.array([[0, 1, 3], [0, 3, 2], [2, 3, 5], [2, 5, 4]])
    # the only light: env texel (row 6, column 24) of a 16 x 32 map, 11-22 degrees above the
    # horizon towards +x: below the left face's plane (d.y < d.x), above the right face's
    env = np.zeros((16, 32, 3), np.float32)
    env[6, 24] = 500.0
    sc = synth._scene(v, t, np.zeros((4, 3, 2)), np.full((1, 1, 3), 0.7), np.full((1, 1), 0.6),
                      np.zeros((1, 1)), env)
    K, c2w = synth.look_at((0.0, 2.5, 2.5), (0.0, 0.5, 0.0), 24, 18, 50.0)
    return sc, synth.View(K, c2w, 24, 18, 4, 1)


def test_leak_rule_keeps_an_unlit_face_dark():
    sc, view = _roof()
    r0 = O.render(O.OracleScene(sc, normals=0), view, 0, 8, seed=1, margins=False, prim=True)
    r1 = O.render(O.OracleScene(sc, normals=1), view, 0, 8, seed=1, margins=False, prim=True)
    assert np.array_equal(r0["prim"], r1["prim"])
    prim = r1["prim"][:, 0]
    left, right = np.isin(prim, [0, 1]), np.isin(prim, [2, 3])
    assert left.sum() > 20 and right.sum() > 20
    # every sample of a left-face pixel hit the left face
    left &= np.isin(r1["prim"], [0, 1]).all(1)
    assert np.all(r1["rgb"][left] == 0.0) and np.all(r0["rgb"][left] == 0.0)
    assert r1["rgb"][right].mean() > 0.0 and r0["rgb"][right].mean() > 0.0
    # and without the rule the left face would be lit: its interpolated normals face the light
    osc = O.OracleScene(sc, normals=1)
    light = np.array([np.cos(np.radians(17)), np.sin(np.radians(17)), 0.0])
    vn = osc.vertex_normals()
    assert (vn[[2, 3]] @ light).max() > 0.0


def _fd_scene():
    rng = np.random.Generator(np.random.PCG64(5))
    sc = synth.tiny_scene(subdiv=1, env_w=16, env_h=8)
    sc.verts = (sc.verts + rng.normal(scale=0.03, size=sc.verts.shape)).astype(np.float32)
    sc.albedo = rng.uniform(0.1, 0.9, size=(4, 4, 3)).astype(np.float32)
    sc.roughness = rng.uniform(0.2, 0.9, size=(4, 4)).astype(np.float32)
    sc.metallic = rng.uniform(0.0, 0.8, size=(4, 4)).astype(np.float32)
    sc.env = np.exp(rng.normal(0, 1.0, size=(8, 16, 3))).astype(np.float32)
    sc.env[2, 5] = 40.0
    K, c2w = synth.look_at((0.3, 1.6, 3.5), (0, 0.9, 0), 14, 14, 40.0)
    return sc, synth.View(K, c2w, 14, 14, 2, 3), rng


def test_vertex_gradient_through_interpolated_normals_matches_central_differences():
    sc, view, rng = _fd_scene()
    osc = O.OracleScene(sc, normals=1)
    n = view.width * view.height
    g = rng.normal(size=(n, 3))
    fwd = O.render(osc, view, 0, 4, seed=2, margins=False)["rgb"]
    np.testing.assert_allclose(O.render_detached(osc, osc, view, 0, 4, seed=2), fwd, rtol=1e-14, atol=1e-14)
    an = O.backward(osc, view, 0, 4, g, seed=2)["verts"].reshape(-1)
    # the face-normal adjoint differs: the interpolated chain is what is being checked
    an_face = O.backward(O.OracleScene(sc, normals=0), view, 0, 4, g, seed=2)["verts"].reshape(-1)
    assert np.abs(an - an_face).max() > 1e-3 * np.abs(an).max()

    def F(idx, delta):
        sc1 = copy.deepcopy(sc)
        x = sc1.verts.reshape(-1)
        x[idx] = np.float32(x[idx] + delta)
        actual = float(x[idx]) - float(sc.verts.reshape(-1)[idx])
        rgb = O.render_detached(osc, O.OracleScene(sc1, normals=1), view, 0, 4, seed=2)
        return float((g * rgb).sum()), actual

    def fd(idx, h):
        fp, hp = F(idx, h)
        fm, hm = F(idx, -h)
        return (fp - fm) / (hp - hm)

    cand = np.flatnonzero(np.abs(an) > 1e-3 * np.abs(an).max())
    pick = rng.choice(cand, size=min(10, len(cand)), replace=False)
    checked = 0
    for idx in pick:
        f1, f2 = fd(int(idx), 1e-4), fd(int(idx), 2.5e-5)
        if abs(f1 - f2) > 1e-3 * max(abs(f1), 1e-9):
            continue  # a kink inside the step
        assert abs(an[idx] - f2) <= 2e-5 * max(abs(f2), 1e-3 * np.abs(an).max()), (idx, an[idx], f2)
        checked += 1
    assert checked >= 6
