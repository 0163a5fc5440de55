"""Pins of the EAWT denoiser oracle (Appendix A, "Denoiser") and of its G-buffer.

* the weights are normalised: a constant image with constant buffers comes out unchanged;
* with every sigma infinite the filter is plain a-trous B3 smoothing: an impulse far from the
  border comes out as the separable product of the three dilated B3 kernels, convolved by
  numpy (a library routine, not the oracle's shifting);
* edge stopping: a sharp normal edge (sigma_n small) or colour edge (sigma_rt small) between two
  constant halves lets nothing across;
* the adjoint is the transpose of the recorded linear filter: <A x, y> = <x, A^T y>, and the
  recorded filter applied to the input reproduces the output;
* the G-buffer's normals face the camera, its positions lie on the camera rays and on the hit
  triangles' planes.
"""
import numpy as np

from oracle import eawt as E
from oracle import oracle as O
from paper_2406_16360_gb300 import synth


def test_constant_image_is_a_fixed_point():
    img = np.full((9, 13, 3), 0.7)
    n = np.zeros((9, 13, 3))
    n[..., 2] = 1.0
    x = np.zeros((9, 13, 3))
    out, _ = E.eawt(img, n, x, 0.5, 0.3, 0.2)
    np.testing.assert_allclose(out, img, rtol=1e-15)


def test_infinite_sigmas_give_the_atrous_b3_kernel():
    H = W = 64
    img = np.zeros((H, W, 3))
    img[32, 32, :] = 1.0
    z = np.zeros((H, W, 3))
    out, _ = E.eawt(img, z, z, 1e30, 1e30, 1e30)
    k1 = np.array([1.0])
    for i in range(3):
        h = np.zeros(4 * (1 << i) + 1)
        h[:: 1 << i] = [1, 4, 6, 4, 1]
        k1 = np.convolve(k1, h / 16.0)
    r = (len(k1) - 1) // 2
    ref = np.outer(k1, k1)
    np.testing.assert_allclose(out[32 - r:32 + r + 1, 32 - r:32 + r + 1, 0], ref, rtol=1e-12, atol=1e-17)
    assert abs(out[..., 0].sum() - 1.0) < 1e-12


def test_edges_stop_the_filter():
    H, W = 12, 16
    img = np.zeros((H, W, 3))
    img[:, :8] = 0.2
    img[:, 8:] = 0.9
    n = np.zeros((H, W, 3))
    n[:, :8, 2] = 1.0
    n[:, 8:, 0] = 1.0
    x = np.zeros((H, W, 3))
    out, _ = E.eawt(img, n, x, 1e30, 0.01, 1e30)  # a normal edge
    np.testing.assert_allclose(out, img, rtol=1e-14)
    n2 = np.zeros((H, W, 3))
    n2[..., 2] = 1.0
    out2, _ = E.eawt(img, n2, x, 0.01, 1e30, 1e30)  # a colour edge
    np.testing.assert_allclose(out2, img, rtol=1e-14)
    out3, _ = E.eawt(img, n2, x, 1e30, 1e30, 1e30)  # no edge: the halves mix
    assert abs(out3[5, 7, 0] - 0.2) > 1e-3


def test_adjoint_is_the_transpose_of_the_recorded_filter():
    rng = np.random.Generator(np.random.PCG64(3))
    H, W = 11, 14
    img = rng.uniform(0, 1, (H, W, 3))
    n = rng.normal(size=(H, W, 3))
    n /= np.linalg.norm(n, axis=-1, keepdims=True)
    x = rng.normal(size=(H, W, 3))
    out, rec = E.eawt(img, n, x, 0.4, 0.8, 1.5)
    np.testing.assert_allclose(E.eawt_apply_frozen(img, rec), out, rtol=1e-13)
    a, b = rng.normal(size=(H, W, 3)), rng.normal(size=(H, W, 3))
    lhs = float((E.eawt_apply_frozen(a, rec) * b).sum())
    rhs = float((a * E.eawt_backward(b, rec)).sum())
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)
    # every level's normaliser includes the centre tap, whose weight is exactly (6/16)^2
    for _, k, _ in rec:
        assert k.min() >= (6 / 16) ** 2 * (1 - 1e-15)


def test_gbuffer_normals_and_positions():
    w = synth.config1(width=24, height=20)
    v = w.views[0]
    osc = O.OracleScene(w.scenes[0])
    n, x, tri, mg = E.gbuffer(osc, v)
    hit = tri >= 0
    assert hit.any() and (~hit).any()
    assert np.allclose(np.linalg.norm(n[hit], axis=-1), 1.0)
    assert np.all(n[~hit] == 0) and np.all(x[~hit] == 0)
    o = np.asarray(v.c2w, float).reshape(3, 4)[:, 3]
    d = x[hit] - o
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    assert np.all((n[hit] * d).sum(-1) < 0)  # facing the camera
    s = w.scenes[0]
    f = s.tris[tri[hit]]
    a = s.verts[f[:, 0]].astype(float)
    assert np.allclose((n[hit] * (x[hit] - a)).sum(-1), 0.0, atol=1e-9)  # on the hit plane
