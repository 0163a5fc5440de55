"""GPU parity of the mesh regularisers (Appendix A, "Training details": Laplacian smoothness of
the refined vertices and the offset penalty), through the C ABI, against the FP64 oracle
(oracle/regularizers.py)."""
import numpy as np
import pytest
import torch

from oracle import regularizers as R
from paper_2406_16360_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_16360_gb300 import mirres
    return mirres


@pytest.fixture(scope="module")
def ctx(M):
    c = M.mirres_context_create(0)
    yield c
    c.close()


def _perturbed(sc, seed, scale):
    rng = np.random.Generator(np.random.PCG64(seed))
    return (sc.verts + rng.normal(scale=scale, size=sc.verts.shape)).astype(np.float32)


def _run(M, ctx, sc, verts, ws, wo, loss=True, grad=True, calls=1):
    from paper_2406_16360_gb300.renderer import DeviceScene
    ds = DeviceScene(ctx, sc)
    ds.verts.copy_(torch.as_tensor(verts, device="cuda"))  # the scene reads the borrowed array
    rest = torch.as_tensor(sc.verts, device="cuda").contiguous()
    L = torch.zeros(1, device="cuda") if loss else None
    g = torch.zeros_like(ds.verts) if grad else None
    for _ in range(calls):
        M.mirres_mesh_regularizers(ctx, ds.handle, rest, ws, wo, L, g)
    torch.cuda.synchronize()
    out = (None if L is None else float(L.item()), None if g is None else g.cpu().numpy().astype(np.float64))
    ds.close()
    return out


def _oracle(sc, verts, ws, wo):
    v = verts.astype(np.float64)
    ls, gs = R.l_smooth(v, sc.tris)
    lo, go = R.l_offset(v, sc.verts)
    return ws * ls + wo * lo, ws * gs + wo * go


@pytest.mark.parametrize("which", ["icosphere", "object"])
def test_regularizers_match_oracle(M, ctx, which):
    if which == "icosphere":
        sc = synth.tiny_scene(subdiv=3)
    else:  # displaced sphere plus occluder boxes, about 40k triangles
        sc = synth.object_scene(200, 100, 4, 8, 16, 8)
    verts = _perturbed(sc, 7, 0.01)
    ws, wo = 0.7, 0.3
    L, g = _run(M, ctx, sc, verts, ws, wo)
    Lr, gr = _oracle(sc, verts, ws, wo)
    assert abs(L - Lr) <= 1e-4 * abs(Lr)
    assert np.abs(g - gr).max() <= 2e-5 * max(1e-3, np.abs(gr).max())
    # two calls accumulate
    L2, g2 = _run(M, ctx, sc, verts, ws, wo, calls=2)
    assert abs(L2 - 2 * Lr) <= 2e-4 * abs(Lr)
    assert np.abs(g2 - 2 * gr).max() <= 4e-5 * max(1e-3, np.abs(gr).max())


def test_regularizers_degenerate_mesh(M, ctx):
    """an unused vertex, a degenerate triangle (repeated index) and a duplicated triangle: every
    neighbour counted once, nothing for the isolated vertex"""
    v = np.array([[0.0, 0, 0], [1.0, 0, 0], [0, 1.0, 0], [5.0, 5, 5], [0.2, 0.3, 1.0]], np.float32)
    t = np.array([[0, 1, 2], [0, 1, 1], [1, 2, 0], [2, 1, 4]], np.int32)
    uv = np.zeros((t.shape[0], 3, 2), np.float32)
    base = synth.tiny_scene()
    sc = synth._scene(v, t, uv, base.albedo, base.roughness, base.metallic, base.env)
    verts = _perturbed(sc, 3, 0.05)
    for ws, wo in ((1.0, 0.0), (0.0, 2.0), (0.5, 0.25)):
        L, g = _run(M, ctx, sc, verts, ws, wo)
        Lr, gr = _oracle(sc, verts, ws, wo)
        assert abs(L - Lr) <= 1e-5 * max(1e-6, abs(Lr))
        assert np.abs(g - gr).max() <= 1e-5 * max(1e-3, np.abs(gr).max())
    assert np.all(g[3] == (2 * 0.25 * (verts[3] - v[3])).astype(np.float32))  # offset term only
    # loss only, gradient only
    L, g = _run(M, ctx, sc, verts, 0.5, 0.25, grad=False)
    assert g is None and abs(L - _oracle(sc, verts, 0.5, 0.25)[0]) <= 1e-5 * abs(L)
    L, g = _run(M, ctx, sc, verts, 0.5, 0.25, loss=False)
    assert L is None and np.abs(g - _oracle(sc, verts, 0.5, 0.25)[1]).max() <= 1e-5


def test_regularizers_argument_checks(M, ctx):
    from paper_2406_16360_gb300.renderer import DeviceScene
    ds = DeviceScene(ctx, synth.tiny_scene(subdiv=1))
    L = torch.zeros(1, device="cuda")
    with pytest.raises(M.MirresError):
        M.mirres_mesh_regularizers(ctx, ds.handle, ds.verts, -1.0, 0.0, L, None)
    with pytest.raises(M.MirresError):
        M.mirres_mesh_regularizers(ctx, ds.handle, None, 0.0, 1.0, L, None)
    M.mirres_mesh_regularizers(ctx, ds.handle, None, 0.0, 0.0, L, None)  # nothing to add
    torch.cuda.synchronize()
    assert float(L.item()) == 0.0
    ds.close()
