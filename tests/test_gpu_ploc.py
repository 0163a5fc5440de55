"""GPU checks of the PLOC hierarchy builder (mirres_bvh_set_builder(MIRRES_BVH_PLOC)): the tree
is a valid binary BVH in the LBVH's layout with exact nested boxes, its surface-area cost is
below the LBVH's, refit after a move equals a rebuild, and closest hits and renders are the
LBVH's bit for bit (closest hit = smallest t, then smallest triangle id, whatever the tree)."""
import numpy as np
import pytest
import torch

from paper_2406_16360_gb300 import synth
from tests.parity import compare_tapes

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


def _mesh_scene(v, t):
    n = len(t)
    return synth._scene(v, t, np.zeros((n, 3, 2)), np.full((1, 1, 3), 0.5), np.full((1, 1), 0.5), np.zeros((1, 1)),
                        np.ones((4, 8, 3)))


def _cases():
    rng = np.random.Generator(np.random.PCG64(3))
    cases = {}
    for n in (2, 3, 17, 1000, 4097):
        v = rng.normal(size=(3 * n, 3)).astype(np.float32)
        cases[f"random{n}"] = _mesh_scene(v, np.arange(3 * n).reshape(-1, 3))
    pts = np.concatenate([np.tile([[0.3, 0.2, 0.0]], (40, 1)), np.c_[rng.uniform(size=(60, 2)), np.zeros(60)]])
    cases["duplicates_flat"] = _mesh_scene(np.repeat(pts, 3, 0).astype(np.float32), np.arange(300).reshape(-1, 3))
    cases["object40k"] = synth.object_scene(200, 100, 4, 8, 16, 8)
    return cases


def _export(M, ds, F):
    dev = torch.device("cuda")
    keys = torch.zeros(F, dtype=torch.int64, device=dev)
    left = torch.zeros(max(F - 1, 1), dtype=torch.int32, device=dev)
    right = torch.zeros(max(F - 1, 1), dtype=torch.int32, device=dev)
    parent = torch.zeros(2 * F - 1, dtype=torch.int32, device=dev)
    lo = torch.zeros((2 * F - 1, 3), dtype=torch.float32, device=dev)
    hi = torch.zeros((2 * F - 1, 3), dtype=torch.float32, device=dev)
    M.mirres_bvh_export(ds.handle, keys, left, right, parent, lo, hi)
    torch.cuda.synchronize()
    return dict(keys=keys.cpu().numpy().view(np.uint64), left=left.cpu().numpy()[:F - 1],
                right=right.cpu().numpy()[:F - 1], parent=parent.cpu().numpy(), lo=lo.cpu().numpy(),
                hi=hi.cpu().numpy())


def _scene(ctx, M, sc, builder, traversal=0):
    from paper_2406_16360_gb300.renderer import DeviceScene
    return DeviceScene(ctx, sc, builder=builder, traversal=traversal)


def _check_tree(g, sc):
    F = sc.n_tris
    idx = lambda c: np.where(c >= 0, c, (F - 1) + ~c)
    kids = np.concatenate([idx(g["left"]), idx(g["right"])])
    # every node but the root (0) is the child of exactly one node, and its parent says so
    assert np.array_equal(np.sort(kids), np.arange(1, 2 * F - 1))
    assert g["parent"][0] == -1
    assert np.array_equal(g["parent"][idx(g["left"])], np.arange(F - 1))
    assert np.array_equal(g["parent"][idx(g["right"])], np.arange(F - 1))
    # leaves hold the Morton-sorted triangles' exact boxes, internal boxes the exact unions
    perm = (g["keys"] & np.uint64(0xFFFFFFFF)).astype(np.int64)
    tv = sc.verts[sc.tris[perm]]
    assert np.array_equal(g["lo"][F - 1:], tv.min(1)) and np.array_equal(g["hi"][F - 1:], tv.max(1))
    l, r = idx(g["left"]), idx(g["right"])
    assert np.array_equal(g["lo"][:F - 1], np.minimum(g["lo"][l], g["lo"][r]))
    assert np.array_equal(g["hi"][:F - 1], np.maximum(g["hi"][l], g["hi"][r]))


def _sah(g, F):
    d = (g["hi"][:F - 1] - g["lo"][:F - 1]).astype(np.float64)
    a = d[:, 0] * d[:, 1] + d[:, 1] * d[:, 2] + d[:, 2] * d[:, 0]
    return a.sum() / max(a[0], 1e-300)


@pytest.mark.parametrize("name", list(_cases().keys()))
def test_ploc_tree_is_valid_and_cheaper(M, ctx, name):
    sc = _cases()[name]
    F = sc.n_tris
    dp = _scene(ctx, M, sc, M.MIRRES_BVH_PLOC)
    gp = _export(M, dp, F)
    _check_tree(gp, sc)
    dl = _scene(ctx, M, sc, M.MIRRES_BVH_LBVH)
    gl = _export(M, dl, F)
    assert np.array_equal(gp["keys"], gl["keys"])  # the same Morton order underneath
    if F >= 1000:
        assert _sah(gp, F) < 0.95 * _sah(gl, F), (_sah(gp, F), _sah(gl, F))
    dp.close()
    dl.close()


def test_ploc_refit_equals_rebuild(M, ctx):
    sc = synth.config2(res=32, n_views=1, tex=8).scenes[0]
    F = sc.n_tris
    ds = _scene(ctx, M, sc, M.MIRRES_BVH_PLOC)
    with torch.no_grad():
        ds.verts.mul_(4.0)  # exact: every Morton code and every area comparison is kept
    M.mirres_bvh_refit(ds.handle)
    g = _export(M, ds, F)
    _check_tree(g, synth.Scene(ds.verts.cpu().numpy(), sc.tris, sc.tri_uv, sc.albedo, sc.roughness, sc.metallic,
                               sc.env))
    M.mirres_bvh_build(ds.handle)
    g2 = _export(M, ds, F)
    for k in g:
        assert np.array_equal(g[k], g2[k]), k
    ds.close()


@pytest.mark.parametrize("traversal", [0, 1])
def test_ploc_hits_equal_lbvh_hits(M, ctx, traversal):
    """hits do not depend on the hierarchy: the clustering tree and the Karras tree give the
    same closest and any hits, through the binary trees and through the 8-wide BVHs collapsed
    from them (a clustering tree's small subtrees need not cover consecutive leaves)"""
    sc = synth.object_scene(200, 100, 4, 8, 16, 8)
    rng = np.random.Generator(np.random.PCG64(5))
    n = 200000
    o = rng.normal(size=(n, 3)) * 2.5 + np.array([0.0, 1.0, 0.0])
    d = rng.normal(size=(n, 3)) * 0.8 + np.array([0.0, 1.0, 0.0]) - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    dev = torch.device("cuda")
    rays = torch.as_tensor(np.concatenate([o, d], 1).astype(np.float32), device=dev).contiguous()
    out = {}
    for b in (M.MIRRES_BVH_LBVH, M.MIRRES_BVH_PLOC):
        ds = _scene(ctx, M, sc, b, traversal)
        tri = torch.zeros(n, dtype=torch.int32, device=dev)
        tuv = torch.zeros((n, 3), dtype=torch.float32, device=dev)
        anyh = torch.zeros(n, dtype=torch.int32, device=dev)
        M.mirres_trace(ctx, ds.handle, rays, tri, tuv)
        M.mirres_trace(ctx, ds.handle, rays, anyh, any_hit=True)
        torch.cuda.synchronize()
        out[b] = (tri.cpu().numpy(), tuv.cpu().numpy(), anyh.cpu().numpy() >= 0)
        ds.close()
    a, b = out[M.MIRRES_BVH_LBVH], out[M.MIRRES_BVH_PLOC]
    assert (a[0] >= 0).mean() > 0.3
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_ploc_render_equals_lbvh_render(M, ctx):
    from paper_2406_16360_gb300.renderer import GpuWorkload
    w = synth.config2(res=48, n_views=2, tex=16, spp=2)
    res = {}
    for b in (M.MIRRES_BVH_LBVH, M.MIRRES_BVH_PLOC):
        gw = GpuWorkload(w, 0, ctx=ctx, builder=b)
        images, tape = gw.render(launch=1)
        torch.cuda.synchronize()
        res[b] = ([im.cpu().numpy() for im in images], tape.cpu().numpy())
        for s in gw.scenes:
            s.close()
    (ia, ta), (ib, tb) = res[M.MIRRES_BVH_LBVH], res[M.MIRRES_BVH_PLOC]
    # every defined tape word equal (words without a defined value are left unwritten)
    compare_tapes(ta.view(np.uint32).reshape(M.TAPE_WORDS, -1), tb.view(np.uint32).reshape(M.TAPE_WORDS, -1), rtol=0)
    for x, y in zip(ia, ib):
        assert np.array_equal(x, y)


def test_too_deep_clustering_falls_back_to_karras(M, ctx):
    """triangles at x = 3^k: every cluster's nearest neighbour is the previous one, so the
    clustering degenerates into a chain 79 deep, deeper than the 64-entry traversal stack; the
    build then keeps the Karras tree, bit for bit the oracle's LBVH"""
    from oracle import oracle as O
    n = 80
    x = 3.0 ** np.arange(n)
    v = np.stack([np.c_[x, np.zeros(n), np.zeros(n)], np.c_[x, np.ones(n), np.zeros(n)],
                  np.c_[x, np.zeros(n), np.ones(n)]], 1).reshape(-1, 3).astype(np.float32)
    sc = _mesh_scene(v, np.arange(3 * n).reshape(-1, 3))
    ds = _scene(ctx, M, sc, M.MIRRES_BVH_PLOC)
    g = _export(M, ds, n)
    o = O.lbvh(sc.verts, sc.tris)
    for k in ("keys", "left", "right", "parent", "lo", "hi"):
        assert np.array_equal(g[k], o[k]), k
    ds.close()


def test_set_builder_rejects_unknown(M, ctx):
    from paper_2406_16360_gb300.renderer import DeviceScene
    ds = DeviceScene(ctx, synth.tiny_scene(subdiv=1))
    with pytest.raises(M.MirresError):
        M.mirres_bvh_set_builder(ds.handle, 7)
    ds.close()
