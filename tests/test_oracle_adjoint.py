"""Pin of the oracle's adjoint (PRIMARY mode, Sec. 4.2: gradients of indirect rays detached).

The PRIMARY-mode gradient is the derivative of the detached forward: the primary-vertex terms
evaluated with the parameters being differentiated, every sampling decision and every detached
quantity (RIS weight, visibility, continuation pdf, incident indirect light) held at the values
of the frozen scene. Central finite differences of that function (FP64, the same frozen random
stream) must equal the analytic adjoint for albedo, roughness and metallic texels, env texels
and vertex positions.
"""
import copy

import numpy as np
import pytest

from oracle import oracle as O
from paper_2406_16360_gb300 import synth


def _scene():
    rng = np.random.Generator(np.random.PCG64(21))
    sc = synth.tiny_scene(subdiv=2, env_w=16, env_h=8)
    sc.albedo = rng.uniform(0.1, 0.9, size=(4, 4, 3)).astype(np.float32)
    sc.roughness = rng.uniform(0.2, 0.9, size=(4, 4)).astype(np.float32)
    sc.metallic = rng.uniform(0.0, 0.8, size=(4, 4)).astype(np.float32)
    sc.env = np.exp(rng.normal(0, 1.0, size=(8, 16, 3))).astype(np.float32)
    sc.env[2, 5] = 40.0
    K, c2w = synth.look_at((0.3, 1.6, 3.5), (0, 0.9, 0), 14, 14, 40.0)
    view = synth.View(K, c2w, 14, 14, 2, 3)
    return sc, view, rng


def _loss_fd(sc0, view, g, field, idx, h):
    def F(delta):
        sc1 = copy.deepcopy(sc0)
        arr = getattr(sc1, field)
        x = arr.reshape(-1)
        x[idx] = np.float32(x[idx] + delta)
        actual = float(x[idx]) - float(getattr(sc0, field).reshape(-1)[idx])
        rgb = O.render_detached(O.OracleScene(sc0), O.OracleScene(sc1), view, 0, 4, seed=2)
        return float((g * rgb).sum()), actual

    fp, hp = F(h)
    fm, hm = F(-h)
    return (fp - fm) / (hp - hm)


@pytest.mark.parametrize("field,h", [("albedo", 1e-3), ("roughness", 1e-3), ("metallic", 1e-3),
                                     ("env", 1e-2), ("verts", 1e-4)])
def test_adjoint_matches_central_differences(field, h):
    sc, view, rng = _scene()
    osc = O.OracleScene(sc)
    n = view.width * view.height
    g = rng.normal(size=(n, 3))
    # the detached forward at eval == frozen is the forward itself
    fwd = O.render(osc, view, 0, 4, seed=2, margins=False)["rgb"]
    np.testing.assert_allclose(O.render_detached(osc, osc, view, 0, 4, seed=2), fwd, rtol=1e-14, atol=1e-14)
    gr = O.backward(osc, view, 0, 4, g, seed=2)
    an = gr[field].reshape(-1)
    cand = np.flatnonzero(np.abs(an) > 1e-6 * np.abs(an).max())
    assert len(cand) > 0
    pick = rng.choice(cand, size=min(8, len(cand)), replace=False)
    checked = 0
    for idx in pick:
        fd = _loss_fd(sc, view, g, field, int(idx), h)
        fd2 = _loss_fd(sc, view, g, field, int(idx), h / 4)
        if abs(fd - fd2) > 1e-3 * max(abs(fd), 1e-9):
            continue  # a kink (bilinear cell edge, horizon) inside the step: skip
        assert abs(an[idx] - fd2) <= 2e-5 * max(abs(fd2), 1e-3 * np.abs(an).max()), (field, idx, an[idx], fd2)
        checked += 1
    assert checked >= min(5, len(pick))


def test_adjoint_is_linear_in_seed_gradient_and_local():
    sc, view, rng = _scene()
    osc = O.OracleScene(sc)
    n = view.width * view.height
    g1, g2 = rng.normal(size=(n, 3)), rng.normal(size=(n, 3))
    a = O.backward(osc, view, 0, 4, g1, seed=2)
    b = O.backward(osc, view, 0, 4, g2, seed=2)
    c = O.backward(osc, view, 0, 4, 2 * g1 - g2, seed=2)
    for k in ("albedo", "env", "verts"):
        np.testing.assert_allclose(c[k], 2 * a[k] - b[k], rtol=1e-9, atol=1e-12)
    # a single pixel's gradient equals the full call with a one-hot seed
    pix = [37]
    one = np.zeros((n, 3))
    one[37] = g1[37]
    full = O.backward(osc, view, 0, 4, one, seed=2)
    part = O.backward(osc, view, 0, 4, g1[37:38], seed=2, pixels=pix)
    for k in ("albedo", "roughness", "metallic", "env", "verts"):
        np.testing.assert_allclose(part[k], full[k], rtol=1e-12, atol=1e-15)
