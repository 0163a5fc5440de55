"""Pins of the oracle's random numbers, ray-triangle intersection and median-split BVH.

Pins (things other than the oracle itself):
  * Philox4x32-10 against the published known-answer vectors (tests/golden).
  * Moller-Trumbore against hand-computed hits on one triangle (t, barycentrics by inspection).
  * BVH closest / any hit against brute force over every triangle (FP64), and the tie rule.
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2406_16360_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def test_philox_known_answers():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        w = [int(x, 16) for x in r]
        out = O.philox(w[0:4], w[4:6])
        assert [int(x) for x in out] == w[6:10]


def test_uniform_is_exact_24_bit():
    assert O.uniform(0) == 0.0
    assert O.uniform(0xFFFFFFFF) == (2 ** 24 - 1) / 2 ** 24
    assert O.uniform(0x80000000) == 0.5
    assert O.uniform(0x000000FF) == 0.0  # low 8 bits dropped


def _one_triangle(v):
    v = np.asarray(v, dtype=np.float32)
    return synth._scene(v, np.array([[0, 1, 2]]), np.zeros((1, 3, 2)), np.full((1, 1, 3), 0.5),
                        np.full((1, 1), 0.5), np.zeros((1, 1)), np.ones((2, 4, 3)))


def test_single_triangle_hand_computed():
    sc = _one_triangle([[0, 0, 0], [1, 0, 0], [0, 1, 0]])
    osc = O.OracleScene(sc)
    # straight down onto the point 0.25 e1 + 0.25 e2, one unit above the plane
    tri, tuv, _ = O.trace(osc, [[0.25, 0.25, 1.0]], [[0, 0, -1.0]], mode=0)
    assert tri[0] == 0
    np.testing.assert_allclose(tuv[0], [1.0, 0.25, 0.25], rtol=0, atol=1e-15)
    # slanted ray through the same point: o = p + 2 (0.6, 0, 0.8), d = -(0.6, 0, 0.8) -> t = 2
    o = np.array([0.25 + 1.2, 0.25, 1.6])
    tri, tuv, _ = O.trace(osc, [o], [[-0.6, 0, -0.8]], mode=0)
    np.testing.assert_allclose(tuv[0], [2.0, 0.25, 0.25], rtol=0, atol=1e-14)
    # outside the edge u + v = 1, pointing away, parallel
    for o, d in [([0.6, 0.6, 1.0], [0, 0, -1.0]), ([0.2, 0.2, 1.0], [0, 0, 1.0]), ([0.2, 0.2, 1.0], [1.0, 0, 0])]:
        tri, _, _ = O.trace(osc, [o], [d], mode=0)
        assert tri[0] == -1
    # the hit is ignored when it is the skipped triangle, and below t_min
    tri, _, _ = O.trace(osc, [[0.25, 0.25, 1.0]], [[0, 0, -1.0]], mode=0, skip=[0])
    assert tri[0] == -1
    tri, _, _ = O.trace(osc, [[0.25, 0.25, 0.5 * osc.tmin]], [[0, 0, -1.0]], mode=0)
    assert tri[0] == -1
    tri, _, _ = O.trace(osc, [[0.25, 0.25, 2.0 * osc.tmin]], [[0, 0, -1.0]], mode=0)
    assert tri[0] == 0


def test_tie_goes_to_smaller_triangle_id():
    # a unit quad split along its diagonal; a ray through the diagonal hits both at the same t
    v = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0]], dtype=np.float32)
    t = np.array([[0, 1, 2], [0, 2, 3]])
    sc = synth._scene(v, t, np.zeros((2, 3, 2)), np.full((1, 1, 3), 0.5), np.full((1, 1), 0.5),
                      np.zeros((1, 1)), np.ones((2, 4, 3)))
    osc = O.OracleScene(sc)
    tri, tuv, mg = O.trace(osc, [[0.5, 0.5, 1.0]], [[0, 0, -1.0]], mode=0, margins=True)
    assert tri[0] == 0 and tuv[0, 0] == 1.0
    assert mg[0] < 1.0  # flagged as a grazing tie
    # reversed triangle order: still the smaller id
    sc2 = synth._scene(v, t[::-1].copy(), np.zeros((2, 3, 2)), np.full((1, 1, 3), 0.5), np.full((1, 1), 0.5),
                       np.zeros((1, 1)), np.ones((2, 4, 3)))
    tri, _, _ = O.trace(O.OracleScene(sc2), [[0.5, 0.5, 1.0]], [[0, 0, -1.0]], mode=0)
    assert tri[0] == 0


def _random_rays(rng, n, centre, radius):
    o = centre + rng.normal(size=(n, 3)) * radius
    tgt = centre + rng.normal(size=(n, 3)) * 0.7 * radius
    d = tgt - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return o, d


@pytest.mark.parametrize("which", ["config1", "object2k"])
def test_bvh_matches_brute_force(which):
    if which == "config1":
        sc = synth.config1().scenes[0]
        centre, radius = np.array([0, 1.0, 0]), 2.5
    else:
        parts = [synth.displaced_sphere(32, 32, 3)] + synth.occluder_boxes(3)
        v, t, uv = synth.merge(parts)
        sc = synth._scene(v, t, uv, np.full((1, 1, 3), 0.5), np.full((1, 1), 0.5), np.zeros((1, 1)),
                          np.ones((4, 8, 3)))
        centre, radius = np.zeros(3), 2.0
    assert sc.n_tris <= 2100
    osc = O.OracleScene(sc)
    rng = np.random.Generator(np.random.PCG64(7))
    o, d = _random_rays(rng, 20000, centre, radius)
    a_tri, a_tuv, mg = O.trace(osc, o, d, mode=0, margins=True)
    b_tri, b_tuv, _ = O.trace(osc, o, d, mode=2)
    assert np.array_equal(a_tri, b_tri)
    hit = a_tri >= 0
    assert hit.mean() > 0.3
    np.testing.assert_array_equal(a_tuv[hit], b_tuv[hit])
    a_any, _, _ = O.trace(osc, o, d, mode=1)
    b_any, _, _ = O.trace(osc, o, d, mode=3)
    assert np.array_equal(a_any, b_any)
    assert np.array_equal(a_any >= 0, hit)
    # grazing decisions are rare on random rays
    assert (mg < 1).mean() < 0.01
