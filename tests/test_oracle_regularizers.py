"""Pins of the mesh regulariser oracle (Appendix A, "Training details": Laplacian smoothness of
the refined vertices, offset penalty).

* a single triangle: every vertex has two neighbours, so L_smooth = sum over the three edges of
  |e|^2 (each edge seen from both ends with weight 1/2);
* a regular tetrahedron of edge length s: 4 vertices x 3 neighbours x s^2 / 3 = 4 s^2;
* translation invariance, and the gradient of L_smooth sums to zero;
* central differences of both terms on a real mesh; L_offset's closed form.
"""
import numpy as np

from oracle import regularizers as R
from paper_2406_16360_gb300 import synth


def test_single_triangle_and_tetrahedron():
    v = np.array([[0.0, 0, 0], [1.0, 0, 0], [0.3, 2.0, 0]])
    L, _ = R.l_smooth(v, [[0, 1, 2]])
    ref = sum(float(((v[a] - v[b]) ** 2).sum()) for a, b in ((0, 1), (1, 2), (2, 0)))
    assert abs(L - ref) < 1e-12
    tet = 0.7 * np.array([[1.0, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]])  # regular, edge 0.7 * 2 sqrt 2
    el = 0.7 * 2 * np.sqrt(2)
    L, _ = R.l_smooth(tet, [[0, 1, 2], [0, 3, 1], [0, 2, 3], [1, 3, 2]])
    assert abs(L - 4 * el ** 2) < 1e-10


def test_invariance_and_gradients():
    sc = synth.tiny_scene(subdiv=2)
    rng = np.random.Generator(np.random.PCG64(3))
    v = sc.verts.astype(np.float64) + rng.normal(scale=0.01, size=sc.verts.shape)
    L, g = R.l_smooth(v, sc.tris)
    L2, _ = R.l_smooth(v + np.array([3.0, -1.0, 0.5]), sc.tris)
    assert abs(L - L2) <= 1e-10 * L
    assert np.abs(g.sum(0)).max() <= 1e-10 * np.abs(g).max()
    for idx in rng.choice(v.size, size=8, replace=False):
        h = 1e-6
        vp, vm = v.copy().reshape(-1), v.copy().reshape(-1)
        vp[idx] += h
        vm[idx] -= h
        fd = (R.l_smooth(vp.reshape(v.shape), sc.tris)[0] - R.l_smooth(vm.reshape(v.shape), sc.tris)[0]) / (2 * h)
        assert abs(fd - g.reshape(-1)[idx]) <= 1e-6 * max(1.0, abs(fd))
    rest = sc.verts.astype(np.float64)
    Lo, go = R.l_offset(v, rest)
    assert abs(Lo - float(((v - rest) ** 2).sum())) < 1e-14
    np.testing.assert_allclose(go, 2 * (v - rest))


def test_degenerate_edges_and_isolated_vertices():
    v = np.array([[0.0, 0, 0], [1.0, 0, 0], [0, 1.0, 0], [5.0, 5, 5]])  # vertex 3 unused
    L, g = R.l_smooth(v, [[0, 1, 2], [0, 1, 1]])  # a degenerate triangle adds no new edge
    L1, _ = R.l_smooth(v, [[0, 1, 2]])
    assert abs(L - L1) < 1e-14 and np.all(g[3] == 0)
