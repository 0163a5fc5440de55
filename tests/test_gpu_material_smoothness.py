"""GPU parity of the material smoothness regulariser L_k (Appendix A, "Training details") through
the C ABI against the FP64 oracle (oracle/material_smoothness.py), on the same seeded inputs."""
import numpy as np
import pytest
import torch

from oracle import material_smoothness as S
from oracle import oracle as O
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


def _gpu(M, ctx, sc, view, vi, sigma, wa, wr, seed, calls=1):
    from paper_2406_16360_gb300.renderer import DeviceScene
    ds = DeviceScene(ctx, sc)
    L = torch.zeros(1, device="cuda")
    ga = torch.zeros_like(ds.albedo)
    gr = torch.zeros_like(ds.roughness)
    p = M.LkParams(sigma, wa, wr, seed & 0xFFFFFFFF, seed >> 32)
    for _ in range(calls):
        M.mirres_material_smoothness(ctx, ds.handle, view, vi, p, L, ga, gr)
    torch.cuda.synchronize()
    out = float(L.item()), ga.cpu().numpy().astype(np.float64), gr.cpu().numpy().astype(np.float64)
    ds.close()
    return out


def _compare(M, ctx, sc, view, vi, sigma, wa, wr, seed):
    L, ga, gr = _gpu(M, ctx, sc, view, vi, sigma, wa, wr, seed)
    Lr, gar, grr, info = S.material_smoothness(O.OracleScene(sc), view, vi, sigma, wa, wr, seed=seed)
    n = max(info["n_points"], 1)
    # pixels whose hit decision is within FP32 error may change triangle (and |X| by one)
    _, _, mg = S.pixel_centre_hits(O.OracleScene(sc), view)
    n_hit_flag = int((mg < 1.0).sum())
    assert abs(L - Lr) <= 2e-4 * abs(Lr) + (wa + wr) * n_hit_flag / n + 1e-6 * (wa + wr)
    for g, r, ab in ((ga, gar, info["abs_albedo"]), (gr, grr, info["abs_rough"])):
        tol = 1e-3 * max(np.abs(r).max(), 1e-9) + 2.0 * ab
        bad = np.abs(g - r) > tol
        assert not bad.any(), (np.abs(g - r)[bad].max(), bad.sum())
    return L, Lr, info


def _quad(half=2.0, n=64):
    v = np.array([[-half, -half, 0.0], [half, -half, 0.0], [half, half, 0.0], [-half, half, 0.0]])
    t = np.array([[0, 1, 2], [0, 2, 3]])
    uv = (0.25 + 0.5 * (v[:, :2] + half) / (2 * half))[t]
    return v, t, uv


def test_ramp_quad_matches_oracle(M, ctx):
    n = 64
    c = (np.arange(n) + 0.5) / n
    rough = np.tile(0.25 + 0.5 * c[None, :], (n, 1)).astype(np.float32)
    alb = np.full((n, n, 3), 0.5, np.float32)
    alb[..., 0] = 0.125 + 0.25 * c[:, None]
    v, t, uv = _quad(0.6)
    sc = synth._scene(v, t, uv, alb, rough, np.zeros_like(rough), np.ones((4, 8, 3)))
    K, c2w = synth.look_at((0.0, 0.0, 3.0), (0.0, 0.0, 0.0), 64, 64, 40.0)
    view = synth.View(K, c2w, 64, 64, 1, 1)
    L, Lr, info = _compare(M, ctx, sc, view, 0, 0.01, 1.0, 1.0, 123)
    assert 0 < info["n_points"] < 64 * 64  # escaped pixels are not in X


@pytest.mark.parametrize("res,vi,seed", [((96, 96), 0, 7), ((37, 23), 5, 2 ** 40 + 3)])
def test_noise_textures_match_oracle(M, ctx, res, vi, seed):
    sc = synth.object_scene(60, 30, 3, 48, 16, 8)
    K, c2w = synth.look_at((0.3, 1.2, 3.2), (0.0, 1.0, 0.0), res[0], res[1], 45.0)
    view = synth.View(K, c2w, res[0], res[1], 1, 1)
    L, Lr, info = _compare(M, ctx, sc, view, vi, 0.03, 0.8, 1.5, seed)
    assert info["n_points"] > 100 and L > 0


def test_accumulates_and_no_hits(M, ctx):
    sc = synth.object_scene(30, 15, 1, 16, 16, 8)
    K, c2w = synth.look_at((0.0, 1.0, 3.5), (0.0, 1.0, 0.0), 32, 32, 40.0)
    view = synth.View(K, c2w, 32, 32, 1, 1)
    L1, ga1, gr1 = _gpu(M, ctx, sc, view, 0, 0.05, 1.0, 1.0, 9)
    L2, ga2, gr2 = _gpu(M, ctx, sc, view, 0, 0.05, 1.0, 1.0, 9, calls=2)
    assert abs(L2 - 2 * L1) <= 1e-5 * L1
    assert np.abs(gr2 - 2 * gr1).max() <= 1e-5 * np.abs(gr1).max()
    # a camera looking away from everything: X is empty, nothing is added
    K, c2w = synth.look_at((0.0, 1.0, 3.5), (0.0, 1.0, 10.0), 16, 16, 20.0)
    L, ga, gr = _gpu(M, ctx, sc, synth.View(K, c2w, 16, 16, 1, 1), 0, 0.05, 1.0, 1.0, 9)
    assert L == 0.0 and not ga.any() and not gr.any()


def test_argument_checks(M, ctx):
    from paper_2406_16360_gb300.renderer import DeviceScene
    sc = synth.tiny_scene(subdiv=1)
    ds = DeviceScene(ctx, sc)
    K, c2w = synth.look_at((0.0, 1.0, 3.5), (0.0, 1.0, 0.0), 8, 8, 40.0)
    view = synth.View(K, c2w, 8, 8, 1, 1)
    L = torch.zeros(1, device="cuda")
    for bad in (M.LkParams(0.0, 1.0, 1.0, 0, 0), M.LkParams(0.1, -1.0, 1.0, 0, 0), M.LkParams(0.1, 1.0, -1.0, 0, 0)):
        with pytest.raises(M.MirresError):
            M.mirres_material_smoothness(ctx, ds.handle, view, 0, bad, L)
    with pytest.raises(M.MirresError):
        M.mirres_material_smoothness(ctx, ds.handle, view, 70000, M.LkParams(0.1, 1.0, 1.0, 0, 0), L)
    ds.close()


@pytest.mark.parametrize("res,vi,seed,sigma", [((64, 64), 0, 3, 0.01), ((41, 27), 9, 2 ** 33 + 5, 0.05)])
def test_normal_term_matches_oracle(M, ctx, res, vi, seed, sigma):
    """the normal term of L_k (interpolated vertex normals, the texture-space offset carried into
    the hit triangle by its texture map): loss and vertex gradient against the oracle, alone and
    added to the albedo / roughness terms of the same call"""
    from paper_2406_16360_gb300.renderer import DeviceScene
    w = synth.config2(res=res[0], n_views=1, tex=32, spp=1)
    sc = w.scenes[0]
    K, c2w = synth.look_at((0.3, 1.2, 3.2), (0.0, 0.0, 0.0), res[0], res[1], 40.0)
    view = synth.View(K, c2w, res[0], res[1], 1, 1)
    ds = DeviceScene(ctx, sc, normals=M.MIRRES_NORMALS_INTERPOLATED)
    wn = 0.7
    L = torch.zeros(1, device="cuda")
    gv = torch.zeros_like(ds.verts)
    M.mirres_material_smoothness(ctx, ds.handle, view, vi, M.LkParams(sigma, 0.0, 0.0, seed & 0xFFFFFFFF,
                                                                          seed >> 32, wn), L, None, None, gv)
    torch.cuda.synchronize()
    osc = O.OracleScene(sc, normals=1)
    Lr, gvr, info = S.material_smoothness_normal(osc, view, vi, sigma, wn, seed=seed)
    assert info["n_normal"] > 0.5 * info["n_points"] > 100
    # a pixel whose hit is a grazing decision may take another triangle: its term (at most
    # 2 w / |X| for unit normals) and its gradient are left out of the bar
    n_flag = int(info["flagged"].sum())
    n = info["n_points"]
    assert abs(float(L) - Lr) <= 1e-3 * abs(Lr) + 2.0 * wn * n_flag / n + 1e-7, (float(L), Lr, n_flag)
    # vertex gradients away from the flagged pixels: a grazing hit may land on the neighbouring
    # triangle, whose normal terms reach the vertices two rings around it (the vertex normals'
    # normalisation spreads them over the faces around each vertex)
    g = gv.cpu().numpy().astype(np.float64)
    keep = np.ones(sc.verts.shape[0], dtype=bool)
    if n_flag:
        tri_of, _, _ = S.pixel_centre_hits(osc, view)
        ring = np.unique(sc.tris[tri_of[info["flagged"]]])
        for _ in range(2):
            ring = np.unique(sc.tris[np.isin(sc.tris, ring).any(axis=1)])
        keep[ring] = False
    tol = 1e-3 * np.abs(gvr) + 1e-4 * np.abs(gvr).max() + 1e-5 * info["abs_verts"]
    bad = (np.abs(g - gvr) > tol).any(axis=1) & keep
    assert not bad.any(), (int(bad.sum()), np.abs(g - gvr)[bad].max(), np.abs(gvr).max())
    assert keep.sum() > 0.9 * keep.size
    # the normal term adds to the texture terms of the same call; face normals give no normal term
    L2 = torch.zeros(1, device="cuda")
    M.mirres_material_smoothness(ctx, ds.handle, view, vi, M.LkParams(sigma, 1.0, 1.0, seed & 0xFFFFFFFF,
                                                                          seed >> 32, wn), L2)
    L3 = torch.zeros(1, device="cuda")
    M.mirres_material_smoothness(ctx, ds.handle, view, vi, M.LkParams(sigma, 1.0, 1.0, seed & 0xFFFFFFFF,
                                                                          seed >> 32, 0.0), L3)
    torch.cuda.synchronize()
    assert abs(float(L2) - float(L3) - float(L)) <= 1e-5 * float(L2) + 1e-7
    ds.close()
    df = DeviceScene(ctx, sc)
    L4 = torch.zeros(1, device="cuda")
    gv4 = torch.zeros_like(df.verts)
    M.mirres_material_smoothness(ctx, df.handle, view, vi, M.LkParams(sigma, 0.0, 0.0, 0, 0, wn), L4, None, None, gv4)
    torch.cuda.synchronize()
    assert float(L4) == 0.0 and float(gv4.abs().max()) == 0.0
    df.close()
