"""GPU parity against the FP64 oracle, through the C ABI (libmirres.so)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2406_16360_gb300 import synth
from paper_2406_16360_gb300.mirres import TAPE_WORDS

pytestmark = pytest.mark.gpu

from tests.parity import compare_grads, grad_tolerance, compare_pixels, compare_tapes  # noqa: E402


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


def _gw(ctx, workload):
    from paper_2406_16360_gb300.renderer import GpuWorkload
    return GpuWorkload(workload, 0, ctx=ctx)


def _export_bvh(M, ds, F):
    dev = torch.device("cuda")
    keys = torch.zeros(F, dtype=torch.int64, device=dev)
    left = torch.zeros(max(F - 1, 1), dtype=torch.int32, device=dev)
    right = torch.zeros(max(F - 1, 1), dtype=torch.int32, device=dev)
    parent = torch.zeros(2 * F - 1, dtype=torch.int32, device=dev)
    lo = torch.zeros((2 * F - 1, 3), dtype=torch.float32, device=dev)
    hi = torch.zeros((2 * F - 1, 3), dtype=torch.float32, device=dev)
    M.mirres_bvh_export(ds.handle, keys, left, right, parent, lo, hi)
    torch.cuda.synchronize()
    return dict(keys=keys.cpu().numpy().view(np.uint64), left=left.cpu().numpy()[:max(F - 1, 0)],
                right=right.cpu().numpy()[:max(F - 1, 0)], parent=parent.cpu().numpy(), lo=lo.cpu().numpy(),
                hi=hi.cpu().numpy())


def _mesh_scene(v, t):
    n = len(t)
    return synth._scene(v, t, np.zeros((n, 3, 2)), np.full((1, 1, 3), 0.5), np.full((1, 1), 0.5), np.zeros((1, 1)),
                        np.ones((4, 8, 3)))


def _lbvh_cases():
    rng = np.random.Generator(np.random.PCG64(3))
    cases = {"config1": synth.config1().scenes[0]}
    for n in (1, 2, 3, 1000, 4097):
        v = rng.normal(size=(3 * n, 3)).astype(np.float32)
        cases[f"random{n}"] = _mesh_scene(v, np.arange(3 * n).reshape(-1, 3))
    pts = np.concatenate([np.tile([[0.3, 0.2, 0.0]], (40, 1)), np.c_[rng.uniform(size=(60, 2)), np.zeros(60)]])
    cases["duplicates_flat"] = _mesh_scene(np.repeat(pts, 3, 0).astype(np.float32), np.arange(300).reshape(-1, 3))
    cases["config2"] = synth.config2(res=32, n_views=1, tex=8).scenes[0]
    return cases


@pytest.mark.parametrize("name", list(_lbvh_cases().keys()))
def test_lbvh_bit_exact(M, ctx, name):
    from paper_2406_16360_gb300.renderer import DeviceScene
    sc = _lbvh_cases()[name]
    ds = DeviceScene(ctx, sc)
    F = sc.n_tris
    g = _export_bvh(M, ds, F)
    o = O.lbvh(sc.verts, sc.tris)
    assert np.array_equal(g["keys"], o["keys"])
    assert np.array_equal(g["left"], o["left"]) and np.array_equal(g["right"], o["right"])
    assert np.array_equal(g["parent"], o["parent"])
    assert np.array_equal(g["lo"], o["lo"]) and np.array_equal(g["hi"], o["hi"])
    ds.close()


def test_refit_equals_rebuild(M, ctx):
    from paper_2406_16360_gb300.renderer import DeviceScene
    sc = synth.config2(res=32, n_views=1, tex=8).scenes[0]
    ds = DeviceScene(ctx, sc)
    F = sc.n_tris
    # an exact power-of-two scale keeps every centroid ratio, hence every Morton code
    with torch.no_grad():
        ds.verts.mul_(4.0)
    M.mirres_bvh_refit(ds.handle)
    g = _export_bvh(M, ds, F)
    o = O.lbvh(ds.verts.cpu().numpy(), sc.tris)
    assert np.array_equal(g["keys"], o["keys"])
    assert np.array_equal(g["lo"], o["lo"]) and np.array_equal(g["hi"], o["hi"])
    # and a rebuild from the moved vertices gives the same arrays
    M.mirres_bvh_build(ds.handle)
    g2 = _export_bvh(M, ds, F)
    for k in g:
        assert np.array_equal(g[k], g2[k])
    ds.close()


def test_bad_index_rejected(M, ctx):
    """indices are checked when the scene is created and on request, not by every build (which
    then needs no host synchronisation)"""
    sc = synth.config1().scenes[0]
    dev = torch.device("cuda")
    t = torch.as_tensor(sc.tris, device=dev).contiguous()
    t[5, 1] = 10 ** 6
    args = [torch.as_tensor(a, device=dev).contiguous() for a in (sc.verts, t, sc.tri_uv, sc.albedo, sc.roughness,
                                                                 sc.metallic, sc.env)]
    with pytest.raises(M.MirresError) as e:
        M.mirres_scene_create(ctx, *args)
    assert e.value.status == 1 and "n_verts" in str(e.value)
    # a valid scene whose caller-owned indices go bad later: mirres_scene_validate finds it
    t[5, 1] = 0
    s = M.mirres_scene_create(ctx, *args)
    M.mirres_bvh_build(s)
    M.mirres_scene_validate(s)
    t[7, 2] = -3
    with pytest.raises(M.MirresError) as e:
        M.mirres_scene_validate(s)
    assert e.value.status == 1
    s.close()


def test_traversal_cap_reports_timeout(M, ctx):
    """failure detection: a traversal that reaches its iteration cap ends as a miss and raises the
    context's error counter, which mirres_get_counters reports as MIRRES_ERR_TIMEOUT; the context
    stays usable (no fault, no hang) and a reset clears the error"""
    from paper_2406_16360_gb300.renderer import GpuWorkload
    w = synth.config1(width=24, height=16)
    gw = GpuWorkload(w, 0, ctx=ctx)
    M.mirres_reset_counters(ctx)
    for launch in (0, 1, 2):
        gw.render(launch=launch, max_visits=3)
        torch.cuda.synchronize()
        with pytest.raises(M.MirresError) as e:
            M.mirres_get_counters(ctx)
        assert e.value.status == 4 and "iteration cap" in str(e.value)
        M.mirres_reset_counters(ctx)
    images, _ = gw.render(launch=1)
    torch.cuda.synchronize()
    c = M.mirres_get_counters(ctx)
    assert c[7] == 0 and c[0] == w.samples
    assert torch.isfinite(images[0]).all()
    for s in gw.scenes:
        s.close()


@pytest.mark.parametrize("which", ["config1", "config2"])
def test_env_tables(M, ctx, which):
    from paper_2406_16360_gb300.renderer import DeviceScene
    sc = synth.config1().scenes[0] if which == "config1" else synth.config2(res=32, n_views=1, tex=8).scenes[0]
    ds = DeviceScene(ctx, sc)
    eh, ew = sc.env.shape[:2]
    dev = torch.device("cuda")
    marg = torch.zeros(eh + 1, dtype=torch.int32, device=dev)
    cond = torch.zeros((eh, ew + 1), dtype=torch.int32, device=dev)
    texel = torch.zeros((eh, ew, 4), dtype=torch.float32, device=dev)
    total = torch.zeros(1, dtype=torch.float64, device=dev)
    M.mirres_env_export(ds.handle, marg, cond, texel, total)
    torch.cuda.synchronize()
    ocond, omarg, oprob, ototal = O.OracleScene(sc).env_tables()
    thr = lambda c: np.ceil(c * 2.0 ** 24).astype(np.int64)
    gm = marg.cpu().numpy().view(np.uint32).astype(np.int64)
    gc = cond.cpu().numpy().view(np.uint32).astype(np.int64)
    # FP64 sums in the same order on both sides; FP64 sin may differ by an ulp between CUDA and
    # the host libm, which can only move a threshold by one where the CDF sits on the 2^-24 grid
    for gpu_thr, cdf in ((gm, omarg), (gc, ocond)):
        diff = gpu_thr - thr(cdf)
        assert np.abs(diff).max() <= 1
        x = cdf[diff != 0] * 2.0 ** 24
        assert np.all(np.abs(x - np.round(x)) < 1e-6), "threshold differs away from a grid tie"
    assert abs(total.item() - ototal) <= 1e-12 * ototal
    np.testing.assert_allclose(texel.cpu().numpy()[..., 3], oprob * ew * eh, rtol=1e-6)
    np.testing.assert_array_equal(texel.cpu().numpy()[..., :3], sc.env)
    # the CDF over all texels the draw inverts: 53-bit thresholds, the same ordered sums; an
    # ulp of difference in a weight's sin moves a threshold by a few units of 2^-53 at most
    flat = torch.zeros(eh * ew + 1, dtype=torch.int64, device=dev)
    M.mirres_env_export_flat(ds.handle, flat)
    torch.cuda.synchronize()
    oflat = O.OracleScene(sc).env_flat()
    ref = np.array([int(np.ceil(x * 2.0 ** 53)) for x in oflat], dtype=object)
    got = flat.cpu().numpy().view(np.uint64).astype(object)
    diff = np.array([int(a) - int(b) for a, b in zip(got, ref)])
    assert np.abs(diff).max() <= 64, np.abs(diff).max()
    ds.close()


def test_trace_vs_oracle(M, ctx):
    from paper_2406_16360_gb300.renderer import DeviceScene
    sc = synth.config2(res=32, n_views=1, tex=8).scenes[0]
    ds = DeviceScene(ctx, sc)
    rng = np.random.Generator(np.random.PCG64(5))
    n = 100000
    o = rng.normal(size=(n, 3)) * 2.5
    d = rng.normal(size=(n, 3)) * 0.8 - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o32, d32 = o.astype(np.float32), d.astype(np.float32)
    dev = torch.device("cuda")
    rays = torch.as_tensor(np.concatenate([o32, d32], 1), device=dev).contiguous()
    tri = torch.zeros(n, dtype=torch.int32, device=dev)
    tuv = torch.zeros((n, 3), dtype=torch.float32, device=dev)
    M.mirres_trace(ctx, ds.handle, rays, tri, tuv)
    anyh = torch.zeros(n, dtype=torch.int32, device=dev)
    M.mirres_trace(ctx, ds.handle, rays, anyh, any_hit=True)
    torch.cuda.synchronize()
    osc = O.OracleScene(sc)
    otri, otuv, omg = O.trace(osc, o32.astype(np.float64), d32.astype(np.float64), mode=0, margins=True)
    gtri = tri.cpu().numpy()
    mism = gtri != otri
    assert (gtri >= 0).mean() > 0.3
    # every mismatch is a grazing decision the oracle flagged
    assert np.all(omg[mism] < 1.0), (mism.sum(), omg[mism].max() if mism.any() else None)
    assert mism.mean() < 1e-3
    same = ~mism & (gtri >= 0)
    np.testing.assert_allclose(tuv.cpu().numpy()[same, 0], otuv[same, 0], rtol=2e-5, atol=1e-6)
    # barycentrics: FP32 error ~ eps (|o - v0| + |o|) / (size * |cos|), the conditioning of the solve
    v = sc.verts.astype(np.float64)[sc.tris[otri[same]]]
    e1, e2 = v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]
    N = np.cross(e1, e2)
    area2 = np.linalg.norm(N, axis=1)
    cosang = np.abs((N * d32[same]).sum(1)) / area2
    ell = np.sqrt(area2)
    os_ = o32[same].astype(np.float64)
    bound = 64 * 2.0 ** -24 * (np.linalg.norm(os_ - v[:, 0], axis=1) + np.linalg.norm(os_, axis=1) + ell) / (
        ell * cosang)
    err = np.abs(tuv.cpu().numpy()[same, 1:] - otuv[same, 1:]).max(axis=1)
    assert np.all(err <= bound), (err / bound).max()
    assert np.median(err) < 1e-5
    ga = anyh.cpu().numpy() >= 0
    assert np.all((ga == (otri >= 0)) | (omg < 1.0))
    ds.close()


def _oracle_view(osc, w, vi, pixels=None, margins=True):
    v = w.views[vi]
    return O.render(osc, v, vi, w.ris_m, seed=w.seed, pixels=pixels, margins=margins)


def _check_forward(gw, w, launch):
    images, tape = gw.render(launch=launch)
    torch.cuda.synchronize()
    stats = []
    for vi, v in enumerate(w.views):
        osc = O.OracleScene(w.scenes[v.scene])
        r = _oracle_view(osc, w, vi)
        st = compare_pixels(images[vi].cpu().numpy(), r["rgb"], r["margin"])
        assert st["failures"] == 0, (vi, st["failures"], st["max_err_unflagged"], st["bad_idx"][:10])
        assert st["flagged"] <= 0.05 * st["n"], st["flagged"]
        stats.append(st)
    return images, tape, stats


def test_config1_forward_plain_and_batched_identical(M, ctx):
    w = synth.config1()
    gw = _gw(ctx, w)
    imgs0, tape0, st = _check_forward(gw, w, 0)
    # the launch paths take every discrete decision identically (hit triangle, selected
    # candidate); their values differ only by FP32 contraction choices of the kernels
    N = w.samples
    a = tape0.cpu().numpy().view(np.uint32).reshape(TAPE_WORDS, N)
    for launch in (1, 2):
        imgs1, tape1 = gw.render(launch=launch)
        torch.cuda.synchronize()
        b = tape1.cpu().numpy().view(np.uint32).reshape(TAPE_WORDS, N)
        compare_tapes(a, b, rtol=2e-6)
        torch.testing.assert_close(imgs0[0], imgs1[0], rtol=2e-6, atol=0)
    print("config1 forward:", {k: st[0][k] for k in ("n", "flagged", "max_err_unflagged", "median_err")})


def _grad_check(gw, w, images, tape, seed=123):
    rng = np.random.Generator(np.random.PCG64(seed))
    d_imgs, d_np = [], []
    for vi, v in enumerate(w.views):
        osc = O.OracleScene(w.scenes[v.scene])
        r = _oracle_view(osc, w, vi)
        g = rng.normal(size=(v.height * v.width, 3))
        g[r["margin"] < 1.0] = 0.0
        d_np.append(g)
        d_imgs.append(torch.as_tensor(g.reshape(v.height, v.width, 3), dtype=torch.float32, device="cuda"))
    grads = gw.backward(d_imgs, tape)
    torch.cuda.synchronize()
    for si, sc in enumerate(w.scenes):
        osc = O.OracleScene(sc)
        acc = None
        for vi, v in enumerate(w.views):
            if v.scene != si:
                continue
            gi = O.backward(osc, v, vi, w.ris_m, d_imgs[vi].double().cpu().numpy().reshape(-1, 3), seed=w.seed)
            if acc is None:
                acc = gi
            else:
                for k in gi:
                    if k != "counts":
                        acc[k] = acc[k] + gi[k]
        for k in ("albedo", "roughness", "metallic", "env", "verts"):
            st = compare_grads(grads[si][k].cpu().numpy(), acc[k], acc[k + "_abs"], acc.get(k + "_sens"),
                               **grad_tolerance(k))
            print(f"grad {k}: failures={st['failures']} {st['detail'][:3]}")
            assert st["failures"] == 0, (k, st["failures"], st["max_rel"], st["detail"])
            print(f"grad {k}: nonzero={st['nonzero']} median_rel={st['median_rel']:.2e} max_rel={st['max_rel']:.2e}")


def test_config1_backward(M, ctx):
    w = synth.config1()
    gw = _gw(ctx, w)
    images, tape = gw.render(launch=0)
    _grad_check(gw, w, images, tape)


def test_config2_reduced_forward_backward(M, ctx):
    w = synth.config2(res=48, n_views=2, tex=64, spp=4)
    gw = _gw(ctx, w)
    images, tape, st = _check_forward(gw, w, 1)
    _grad_check(gw, w, images, tape)


def _wide_workloads():
    return {"config1": synth.config1(),
            "config2_reduced": synth.config2(res=40, n_views=2, tex=64, spp=4),
            "scenes3": synth.config5(seed=3, n_scenes=3, max_tris=6000, res_choices=(16, 24), spp_choices=(2, 3),
                                     tex=16)}


def _defined_words_differ(a, b, rtol=0.0):
    """per sample: any tape word that both renders define differs (words 9-12 are defined where a
    candidate was selected, 13-16 where L_ind != 0; the rest always). The integer words (hit
    triangle, selected candidate, env texel) must be equal; with rtol > 0 the float words may
    differ by that relative amount (kernels compiled apart may contract multiply-adds
    differently), else they must be equal too."""
    fa, fb = a.view(np.float32).astype(np.float64), b.view(np.float32).astype(np.float64)

    def fdiff(rows):
        if rtol == 0.0:
            return np.any(a[rows] != b[rows], axis=0)
        return np.any(np.abs(fa[rows] - fb[rows]) > rtol * np.maximum(np.abs(fa[rows]), np.abs(fb[rows])), axis=0)

    differ = np.any(a[:2] != b[:2], axis=0) | fdiff(slice(2, 9))
    sel = (a[1].view(np.int32) >= 0) | (b[1].view(np.int32) >= 0)
    differ |= sel & ((a[9] != b[9]) | fdiff(slice(10, 13)))
    ind = np.any(fa[3:6] != 0.0, axis=0) | np.any(fb[3:6] != 0.0, axis=0)
    differ |= ind & fdiff(slice(13, 17))
    return differ


@pytest.mark.parametrize("name", list(_wide_workloads().keys()))
@pytest.mark.parametrize("launch", [0, 1, 2])
def test_wide_bvh_takes_the_binary_trees_hits(M, ctx, name, launch):
    """the 8-wide BVH (quantised child boxes rounded outwards) and the binary tree it was
    collapsed from find the same closest hits: renders through either agree word for word on
    every sample, except samples with a grazing decision the oracle flags (a ray that touches a
    binary box within rounding may be culled by the binary tree's exact box, not by the wide
    tree's wider one); also after the vertices moved and both trees were refitted. (The
    persistent launch compiles its wide-BVH variant as a kernel of its own, whose shading may
    round differently: there the float words agree to 1e-5, the decisions exactly.)"""
    from paper_2406_16360_gb300.renderer import GpuWorkload
    w = _wide_workloads()[name]
    gb = GpuWorkload(w, 0, ctx=ctx)
    gw = GpuWorkload(w, 0, ctx=ctx, traversal=M.MIRRES_TRAVERSAL_WIDE)
    n = w.samples
    for moved in (False, True):
        scenes = w.scenes
        if moved:
            rng = np.random.Generator(np.random.PCG64(8))
            scenes = []
            for sb, sw, sc in zip(gb.scenes, gw.scenes, w.scenes):
                v = (sc.verts + rng.normal(scale=0.003, size=sc.verts.shape)).astype(np.float32)
                for ds in (sb, sw):
                    with torch.no_grad():
                        ds.verts.copy_(torch.as_tensor(v, device="cuda"))
                    M.mirres_bvh_refit(ds.handle)
                scenes.append(synth.Scene(v, sc.tris, sc.tri_uv, sc.albedo, sc.roughness, sc.metallic, sc.env))
        _, tape_w = gw.render(launch=launch)
        _, tape_b = gb.render(launch=launch)
        torch.cuda.synchronize()
        a = tape_w.cpu().numpy().view(np.uint32).reshape(-1, n)[:17]
        b = tape_b.cpu().numpy().view(np.uint32).reshape(-1, n)[:17]
        differ = _defined_words_differ(a, b, rtol=1e-5 if launch == 2 else 0.0)
        if differ.any():
            margins = np.concatenate([O.render_samples(O.OracleScene(scenes[v.scene]), v, vi, w.ris_m, seed=w.seed)
                                      ["sample_margin"].reshape(-1) for vi, v in enumerate(w.views)])
            assert np.all(margins[differ] < 1.0), (name, launch, moved, int(differ.sum()),
                                                   margins[differ].max())
        assert differ.mean() < 1e-3, (name, launch, moved, int(differ.sum()))
    c = M.mirres_get_counters(ctx)  # no traversal reached a cap or overflowed
    assert c[7] == 0
    for s in gb.scenes + gw.scenes:
        s.close()
