"""GPU parity on edge cases, multi-scene batches, the full-size config-3 workload (sampled
pixels, in the launch mode the benchmark times), finite differences, and the config-4
optimisation loop -- all through the C ABI, all against the FP64 oracle."""
import copy
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2406_16360_gb300 import synth
from paper_2406_16360_gb300.mirres import TAPE_WORDS
from tests.parity import compare_grads, grad_tolerance, compare_pixels, compare_tapes

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


def _gw(ctx, w):
    from paper_2406_16360_gb300.renderer import GpuWorkload
    return GpuWorkload(w, 0, ctx=ctx)


def _forward_parity(gw, w, launch, pixels=None, max_flag_frac=0.08):
    images, tape = gw.render(launch=launch)
    torch.cuda.synchronize()
    for vi, v in enumerate(w.views):
        osc = O.OracleScene(w.scenes[v.scene])
        r = O.render(osc, v, vi, w.ris_m, seed=w.seed, pixels=pixels)
        got = images[vi].cpu().numpy().reshape(-1, 3)
        if pixels is not None:
            got = got[pixels]
        st = compare_pixels(got, r["rgb"], r["margin"])
        assert st["failures"] == 0, (vi, st["failures"], st["max_err_unflagged"])
        assert st["flagged"] <= max_flag_frac * st["n"] + 1, (vi, st["flagged"], st["n"])
    return images, tape


def _grad_parity(gw, w, tape, pixels_per_view=None, seed=7, grad_mode=0):
    rng = np.random.Generator(np.random.PCG64(seed))
    d_imgs, plist = [], []
    for vi, v in enumerate(w.views):
        osc = O.OracleScene(w.scenes[v.scene])
        npx = v.width * v.height
        pix = None if pixels_per_view is None else np.sort(rng.choice(npx, size=min(npx, pixels_per_view),
                                                                      replace=False)).astype(np.int32)
        r = O.render(osc, v, vi, w.ris_m, seed=w.seed, pixels=pix)
        g = rng.normal(size=(npx if pix is None else len(pix), 3))
        g[r["margin"] < 1.0] = 0.0
        full = np.zeros((npx, 3))
        if pix is None:
            full[:] = g
        else:
            full[pix] = g
        d_imgs.append(torch.as_tensor(full.reshape(v.height, v.width, 3), dtype=torch.float32, device="cuda"))
        plist.append((pix, full if pix is None else full[pix]))
    grads = gw.backward(d_imgs, tape, grad_mode=grad_mode)
    torch.cuda.synchronize()
    for si, sc in enumerate(w.scenes):
        osc = O.OracleScene(sc)
        acc = None
        for vi, v in enumerate(w.views):
            if v.scene != si:
                continue
            pix, g = plist[vi]
            gi = O.backward(osc, v, vi, w.ris_m, d_imgs[vi].double().cpu().numpy().reshape(-1, 3)[pix]
                            if pix is not None else d_imgs[vi].double().cpu().numpy().reshape(-1, 3),
                            seed=w.seed, pixels=pix, grad_mode=grad_mode)
            if acc is None:
                acc = gi
            else:
                for k in gi:
                    if k != "counts":
                        acc[k] = acc[k] + gi[k]
        if acc is None:
            continue
        for k in ("albedo", "roughness", "metallic", "env", "verts"):
            st = compare_grads(grads[si][k].cpu().numpy(), acc[k], acc[k + "_abs"], acc.get(k + "_sens"),
                               **grad_tolerance(k))
            assert st["failures"] == 0, (si, k, st["failures"], st["detail"])


# ---------------------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------------------
def _edge_workloads():
    out = {}
    # no triangles at all: every ray escapes, the image is the environment
    sc = synth.tiny_scene()
    empty = synth._scene(np.zeros((1, 3)), np.zeros((0, 3), np.int32), np.zeros((0, 3, 2)), sc.albedo,
                         sc.roughness, sc.metallic, sc.env)
    K, c2w = synth.look_at((0.0, 1.5, 4.0), (0.0, 1.0, 0.0), 13, 7)
    out["empty_scene"] = synth.Workload("empty", [empty], [synth.View(K, c2w, 13, 7, 3, 2)], ris_m=4)
    # a single triangle (LBVH without internal nodes)
    one = synth._scene(np.array([[-1, 0, -1], [1, 0, -1], [0, 2, -1.2]]), np.array([[0, 1, 2]]),
                       np.array([[[0, 0], [1, 0], [0.5, 1]]]), np.full((2, 2, 3), 0.6), np.full((2, 2), 0.4),
                       np.full((2, 2), 0.2), sc.env)
    K, c2w = synth.look_at((0.0, 0.8, 2.5), (0.0, 0.8, -1.0), 17, 11)
    out["single_triangle"] = synth.Workload("one", [one], [synth.View(K, c2w, 17, 11, 5, 3)], ris_m=3)
    # black environment: no RIS candidate has weight, the image is black
    black = copy.deepcopy(sc)
    black.env[:] = 0.0
    K, c2w = synth.look_at((0.0, 1.5, 4.0), (0.0, 1.0, 0.0), 9, 9)
    out["black_env"] = synth.Workload("black", [black], [synth.View(K, c2w, 9, 9, 2, 3)], ris_m=8)
    # one bounce, one candidate, one sample, a 1x1 image and a ragged 31x3 image
    K, c2w = synth.look_at((0.0, 1.5, 4.0), (0.0, 1.0, 0.0), 1, 1)
    K2, c2w2 = synth.look_at((0.3, 1.2, 3.5), (0.0, 0.9, 0.0), 31, 3)
    out["tiny_views"] = synth.Workload("tiny", [sc], [synth.View(K, c2w, 1, 1, 1, 1),
                                                      synth.View(K2, c2w2, 31, 3, 7, 2)], ris_m=1, seed=5)
    return out


@pytest.mark.parametrize("name", list(_edge_workloads().keys()))
@pytest.mark.parametrize("launch", [0, 1, 2])
def test_edge_cases_forward(M, ctx, name, launch):
    w = _edge_workloads()[name]
    gw = _gw(ctx, w)
    images, tape = _forward_parity(gw, w, launch, max_flag_frac=0.2)
    if name == "black_env":
        assert float(images[0].abs().max()) == 0.0
    if name == "empty_scene":
        t = tape.cpu().numpy().view(np.int32).reshape(TAPE_WORDS, -1)
        assert np.all(t[0] == -1)
    for s in gw.scenes:
        s.close()


@pytest.mark.parametrize("name", ["single_triangle", "tiny_views"])
def test_edge_cases_backward(M, ctx, name):
    w = _edge_workloads()[name]
    gw = _gw(ctx, w)
    images, tape = gw.render(launch=1)
    _grad_parity(gw, w, tape)
    for s in gw.scenes:
        s.close()


def test_multi_scene_batch_mixed_bounces(M, ctx):
    """several scenes of different sizes and views of different resolution / spp / bounces in
    one call: the batched and persistent launches against the oracle and the plain launch"""
    w = synth.config5(seed=3, n_scenes=4, max_tris=6000, res_choices=(16, 24, 40), spp_choices=(2, 3, 5), tex=16)
    for s in w.scenes:
        s.env[:] = np.minimum(s.env, 50.0)  # keep the per-pixel check well conditioned
    gw = _gw(ctx, w)
    img0, tape0 = gw.render(launch=0)
    for launch in (1, 2):
        img, tape = _forward_parity(gw, w, launch, max_flag_frac=0.15)
        n = w.samples
        a = tape0.cpu().numpy().view(np.uint32).reshape(TAPE_WORDS, n)
        b = tape.cpu().numpy().view(np.uint32).reshape(TAPE_WORDS, n)
        assert np.array_equal(a[:2], b[:2])
    _grad_parity(gw, w, tape0)
    for s in gw.scenes:
        s.close()


# ---------------------------------------------------------------------------------------
# full-size workloads in the benchmark's launch (batched): every sample of sampled pixels
# against the oracle's own samples, read from the tape (words 6-8 hold each sample's radiance)
# ---------------------------------------------------------------------------------------
MAX_FLAGGED_SAMPLES = 0.05  # samples with a decision within the oracle's margin (config 1: 0.1%)


def _tape_sample_rgb(tape, n_total, gids):
    """the radiance words of the listed samples, gathered on the device (the tape can be tens of GB)"""
    t = tape.view(-1)
    idx = torch.as_tensor(gids.astype(np.int64), device=t.device)
    out = np.stack([t[(6 + k) * n_total + idx].cpu().numpy().view(np.float32) for k in range(3)], axis=-1)
    return out.astype(np.float64)


def _sample_parity(images, tape, w, osc_of, views, pixels_of, reuse=(0, 0), max_flagged=MAX_FLAGGED_SAMPLES):
    """per view: every sample of the chosen pixels against the oracle (unflagged samples within
    1e-4 of the sample's largest channel), the unflagged pixels' means within 1e-4; returns the
    oracle renders and the flagged counts"""
    n_total = w.samples
    out, flagged, n_smp = {}, 0, 0
    for vi in views:
        v = w.views[vi]
        pix = pixels_of(vi)
        q = O.render_samples(osc_of(v.scene), v, vi, w.ris_m, seed=w.seed, pixels=pix, reuse=reuse)
        npx = len(pix) if pix is not None else v.width * v.height
        pid = np.arange(npx) if pix is None else pix.astype(np.int64)
        first = sum(u.width * u.height * u.spp for u in w.views[:vi])  # the view's first sample
        gids = (first + pid[:, None] * v.spp + np.arange(v.spp)[None, :]).reshape(-1)
        got = _tape_sample_rgb(tape, n_total, gids)
        ref = q["sample_rgb"].reshape(-1, 3)
        ok = q["sample_margin"].reshape(-1) >= 1.0
        # a sample is held to 1e-4 of the larger of its own and its pixel's largest channel (its
        # share of the pixel's 1e-4 bar: a dim sample of a bright pixel carries the same absolute
        # FP32 error as its neighbours), plus twice the oracle's FP32 sensitivity of the sample
        # (the rounding of RIS weights and throughput on glossy lobes, conditioned like 1 / alpha)
        pix_scale = np.repeat(np.abs(q["rgb"]).max(axis=1), v.spp)
        scale = np.maximum(np.maximum(np.abs(ref).max(axis=1), pix_scale), 1e-30)
        sens = q["sample_sens"].reshape(-1)
        err = np.abs(got - ref).max(axis=1) / scale
        bad = ok & (np.abs(got - ref).max(axis=1) > 1e-4 * scale + 2.0 * sens)
        if bad.any():
            for b in np.flatnonzero(bad)[:8]:
                print("view", vi, "pixel", int(pid[b // v.spp]), "sample", int(b % v.spp), "margin",
                      float(q["sample_margin"].reshape(-1)[b]), "pixel margin", float(q["margin"][b // v.spp]),
                      "gpu", got[b], "oracle", ref[b], "pixel", q["rgb"][b // v.spp], "err", float(err[b]))
        assert not bad.any(), (vi, int(bad.sum()), float(err[ok].max()), np.flatnonzero(bad)[:5])
        flagged += int((~ok).sum())
        n_smp += len(ok)
        img = images[vi].view(-1, 3)
        gimg = img[torch.as_tensor(pid, device=img.device)].cpu().numpy() if pix is not None else img.cpu().numpy()
        # the pixels: 1e-4 of the largest channel plus twice the mean of their samples' bounds
        perr = np.abs(gimg.astype(np.float64) - q["rgb"]).max(axis=1)
        pscale = np.maximum(np.abs(q["rgb"]).max(axis=1), 1e-30)
        pbad = (q["margin"] >= 1.0) & (perr > 1e-4 * pscale + 2.0 * q["sens"])
        assert not pbad.any(), (vi, int(pbad.sum()), float((perr / pscale)[pbad].max()))
        out[vi] = q
    frac = flagged / max(n_smp, 1)
    print(f"samples compared {n_smp}, flagged {flagged} ({100 * frac:.2f}%)")
    assert frac <= max_flagged, (flagged, n_smp)
    return out


def _seeded_adjoint(gw, w, tape, osc, vi, pix, seed, field_list=("albedo", "roughness", "metallic", "env", "verts")):
    """the adjoint of one view's listed pixels (flagged pixels zeroed on both sides) against the
    oracle, every field at GRAD_RTOL plus the oracle's FP32 sensitivity bounds; returns the
    number of seeded pixels"""
    v = w.views[vi]
    rng = np.random.Generator(np.random.PCG64(seed))
    r = O.render(osc, v, vi, w.ris_m, seed=w.seed, pixels=pix)
    g = rng.normal(size=(len(pix), 3))
    g[r["margin"] < 1.0] = 0.0
    d = [torch.zeros((vv.height, vv.width, 3), device="cuda") for vv in w.views]
    d[vi].view(-1, 3)[torch.as_tensor(pix.astype(np.int64), device="cuda")] = torch.as_tensor(
        g, dtype=torch.float32, device="cuda")
    grads = gw.backward(d, tape)
    torch.cuda.synchronize()
    og = O.backward(osc, v, vi, w.ris_m, d[vi].double().cpu().numpy().reshape(-1, 3)[pix], seed=w.seed, pixels=pix)
    for k in field_list:
        st = compare_grads(grads[v.scene][k].cpu().numpy(), og[k], og[k + "_abs"], og.get(k + "_sens"))
        assert st["failures"] == 0, (k, st["failures"], st["detail"])
    return int((r["margin"] >= 1.0).sum())


def test_config3_full_size_sampled(M, ctx):
    """config 3 at full size (499,036 triangles, 100 views at 800x800, 16 spp, 4 bounces, M = 32):
    2048 pixels on each of five views sample by sample, and the adjoint of 1536 pixels"""
    w = synth.config3(n_views=100)
    gw = _gw(ctx, w)
    images, tape = gw.render(launch=1)
    torch.cuda.synchronize()
    osc = O.OracleScene(w.scenes[0])
    rng = np.random.Generator(np.random.PCG64(11))
    picks = {vi: np.sort(rng.choice(640000, size=2048, replace=False)).astype(np.int32) for vi in (0, 25, 37, 75, 99)}
    _sample_parity(images, tape, w, lambda si: osc, sorted(picks), picks.get)
    seeded = _seeded_adjoint(gw, w, tape, osc, 37,
                             np.sort(rng.choice(640000, size=1536, replace=False)).astype(np.int32), seed=12)
    print("adjoint pixels seeded (unflagged):", seeded)
    assert seeded >= 512
    for s in gw.scenes:
        s.close()


def test_config3_full_adjoint_at_full_view_size(M, ctx):
    """the FULL-mode adjoint (every vertex of every path) at config 3's per-view size (499,036
    triangles, 800x800, 16 spp, 4 bounces, M = 32; four of its views, a 7.2 GB tape): 384 seeded
    pixels per view against the oracle's FULL adjoint"""
    w = synth.config3(n_views=4)
    gw = _gw(ctx, w)
    images, tape = gw.render(launch=1, grad_mode=1)
    torch.cuda.synchronize()
    _grad_parity(gw, w, tape, pixels_per_view=384, grad_mode=1)
    for s in gw.scenes:
        s.close()


def test_config3_spatial_reuse_at_full_view_size(M, ctx):
    """spatial reuse as the benchmark runs it (4 neighbours within radius 8) at config 3's
    per-view size (499,036 triangles, 800x800, 16 spp, 4 bounces; two views): 1024 pixels per
    view sample by sample against the oracle's reuse. A reused sample carries the decisions of
    five reservoirs (its own and four neighbours', each with its candidates' accepts and the
    neighbour's primary hit), so up to 15% of samples may sit within a margin, as in the
    smaller reuse tests; every other sample is held to the usual bound."""
    w = synth.config3(n_views=2)
    gw = _gw(ctx, w)
    images, tape = gw.render(launch=1, reuse=(4, 8))
    torch.cuda.synchronize()
    osc = O.OracleScene(w.scenes[0])
    rng = np.random.Generator(np.random.PCG64(15))
    picks = {vi: np.sort(rng.choice(640000, size=1024, replace=False)).astype(np.int32) for vi in (0, 1)}
    _sample_parity(images, tape, w, lambda si: osc, (0, 1), picks.get, reuse=(4, 8), max_flagged=0.15)
    for s in gw.scenes:
        s.close()


def test_config5_full_size_sampled(M, ctx):
    """config 5 at full size (64 scenes, 1k-1M triangles each, 9.5 M in all, views of 128-1024
    squared pixels with 4-32 spp and 2-5 bounces, one batched launch): 1024 pixels (all of
    smaller views) on six views sample by sample -- the scene with the most triangles, the
    largest view and four drawn at random -- and the adjoint of 768 pixels of one of them"""
    w = synth.config5()
    gw = _gw(ctx, w)
    images, tape = gw.render(launch=1)
    torch.cuda.synchronize()
    osc_cache = {}

    def osc_of(si):
        if si not in osc_cache:
            osc_cache[si] = O.OracleScene(w.scenes[si])
        return osc_cache[si]

    rng = np.random.Generator(np.random.PCG64(13))
    biggest = int(np.argmax([s.n_tris for s in w.scenes]))
    largest = int(np.argmax([v.width * v.height * v.spp for v in w.views]))
    chosen = {biggest, largest}
    while len(chosen) < 6:
        chosen.add(int(rng.integers(0, len(w.views))))
    picks = {}
    for vi in sorted(chosen):
        npx = w.views[vi].width * w.views[vi].height
        picks[vi] = np.sort(rng.choice(npx, size=min(1024, npx), replace=False)).astype(np.int32)
    _sample_parity(images, tape, w, osc_of, sorted(picks), picks.get)
    vi = largest
    npx = w.views[vi].width * w.views[vi].height
    seeded = _seeded_adjoint(gw, w, tape, osc_of(w.views[vi].scene), vi,
                             np.sort(rng.choice(npx, size=768, replace=False)).astype(np.int32), seed=14)
    print("adjoint pixels seeded (unflagged):", seeded)
    assert seeded >= 256
    for s in gw.scenes:
        s.close()


def test_config2_full_size(M, ctx):
    """config 2 at its stated size (49,956 triangles, 4 views at 256x256, 512x512 textures, 8 spp,
    3 bounces, M = 32): every sample of every pixel, and the adjoint of all pixels of two views"""
    w = synth.config2()
    gw = _gw(ctx, w)
    images, tape = gw.render(launch=1)
    torch.cuda.synchronize()
    osc = O.OracleScene(w.scenes[0])
    _sample_parity(images, tape, w, lambda si: osc, range(len(w.views)), lambda vi: None)
    for vi in (0, 2):
        npx = w.views[vi].width * w.views[vi].height
        _seeded_adjoint(gw, w, tape, osc, vi, np.arange(npx, dtype=np.int32), seed=20 + vi)
    for s in gw.scenes:
        s.close()


# ---------------------------------------------------------------------------------------
# gradients against central finite differences (config 2 scene, 64 random texels)
# ---------------------------------------------------------------------------------------
def test_config2_gradients_vs_finite_differences(M, ctx):
    w = synth.config2(res=48, n_views=1, tex=512, spp=8)
    gw = _gw(ctx, w)
    images, tape = gw.render(launch=1)
    v = w.views[0]
    osc = O.OracleScene(w.scenes[0])
    r = O.render(osc, v, 0, w.ris_m, seed=w.seed)
    rng = np.random.Generator(np.random.PCG64(17))
    g = rng.normal(size=(v.width * v.height, 3))
    g[r["margin"] < 1.0] = 0.0
    d = [torch.as_tensor(g.reshape(v.height, v.width, 3), dtype=torch.float32, device="cuda")]
    grads = gw.backward(d, tape)
    torch.cuda.synchronize()
    ga = grads[0]["albedo"].cpu().numpy().reshape(-1)
    oa = O.backward(osc, v, 0, w.ris_m, d[0].double().cpu().numpy().reshape(-1, 3), seed=w.seed)
    touched = np.flatnonzero(np.abs(oa["albedo"].reshape(-1)) > 1e-3 * np.abs(oa["albedo"]).max())
    pick = rng.choice(touched, size=min(64, len(touched)), replace=False)
    sc0 = w.scenes[0]
    gf = d[0].double().cpu().numpy().reshape(-1, 3)
    checked = 0
    for idx in pick:
        h = 2e-3
        vals = []
        for sgn in (+1, -1):
            sc1 = copy.deepcopy(sc0)
            flat = sc1.albedo.reshape(-1)
            flat[idx] = np.float32(flat[idx] + sgn * h)
            dh = float(flat[idx]) - float(sc0.albedo.reshape(-1)[idx])
            rgb = O.render_detached(osc, O.OracleScene(sc1), v, 0, w.ris_m, seed=w.seed)
            vals.append(((gf * rgb).sum(), dh))
        fd = (vals[0][0] - vals[1][0]) / (vals[0][1] - vals[1][1])
        sens = oa["albedo_sens"].reshape(-1)[idx]
        assert abs(ga[idx] - fd) <= 1e-3 * abs(fd) + 2.0 * sens + 1e-6 * np.abs(oa["albedo"]).max(), (
            idx, ga[idx], fd, sens)
        checked += 1
    assert checked == len(pick)
    for s in gw.scenes:
        s.close()


# ---------------------------------------------------------------------------------------
# config 4: optimisation loop through the autograd Function vs the same loop driven by
# the oracle's gradients
# ---------------------------------------------------------------------------------------
def test_config4_loop_tracks_oracle_gradients(M, ctx):
    from paper_2406_16360_gb300.renderer import GpuWorkload, MirresRender
    res, steps = 24, 16
    target_w = synth.config2(res=res, n_views=2, tex=16, spp=4, bounces=2)
    gt = target_w.scenes[0]
    tgw = GpuWorkload(target_w, 0, ctx=ctx)
    targets, _ = tgw.render(launch=1, seed=99)
    targets = torch.stack([t.clone() for t in targets])
    init = copy.deepcopy(gt)
    init.albedo[:] = 0.5
    init.roughness[:] = 0.5
    init.env[:] = 1.0
    losses = {}
    for mode in ("gpu", "oracle"):
        w = synth.Workload(target_w.name, [copy.deepcopy(init)], target_w.views, target_w.ris_m, seed=1)
        gw = GpuWorkload(w, 0, ctx=ctx)
        ds = gw.scenes[0]
        params = [ds.albedo, ds.env]
        for p in params:
            p.requires_grad_(True)
        opt = torch.optim.Adam(params, lr=5e-2)
        curve = []
        for it in range(steps):
            opt.zero_grad()
            if mode == "gpu":
                img = MirresRender.apply(gw, 1, 1 + it, ds.albedo, ds.roughness, ds.metallic, ds.env, ds.verts)
                loss = ((img - targets) ** 2).sum()
                loss.backward()
            else:
                with torch.no_grad():
                    sc = synth.Workload(w.name, [synth._scene(gt.verts, gt.tris, gt.tri_uv, ds.albedo.cpu().numpy(),
                                                              ds.roughness.cpu().numpy(), ds.metallic.cpu().numpy(),
                                                              ds.env.cpu().numpy())], w.views, w.ris_m, seed=1 + it)
                    osc = O.OracleScene(sc.scenes[0])
                    tot = 0.0
                    ga = np.zeros(ds.albedo.shape)
                    ge = np.zeros(ds.env.shape)
                    for vi, v in enumerate(w.views):
                        rr = O.render(osc, v, vi, w.ris_m, seed=1 + it, margins=False)["rgb"]
                        diff = rr - targets[vi].double().cpu().numpy().reshape(-1, 3)
                        tot += float((diff ** 2).sum())
                        gg = O.backward(osc, v, vi, w.ris_m, 2 * diff, seed=1 + it, want_abs=False)
                        ga += gg["albedo"]
                        ge += gg["env"]
                    loss = torch.tensor(tot)
                    ds.albedo.grad = torch.as_tensor(ga, dtype=torch.float32, device="cuda")
                    ds.env.grad = torch.as_tensor(ge, dtype=torch.float32, device="cuda")
            curve.append(float(loss))
            opt.step()
        losses[mode] = curve
        for p in params:
            p.requires_grad_(False)
        gw.scenes[0].close()
    a, b = np.array(losses["gpu"]), np.array(losses["oracle"])
    assert a[-1] < 0.95 * a[0], a
    # same seeds, same gradients up to FP32: the two loops follow the same curve
    np.testing.assert_allclose(a, b, rtol=1e-2)
    for s in tgw.scenes:
        s.close()


def test_autotune_and_set_launch(M, ctx):
    w = synth.config2(res=32, n_views=2, tex=16, spp=4)
    gw = _gw(ctx, w)
    tape = gw.new_tape()
    res = M.mirres_autotune(ctx, [s.handle for s in gw.scenes], gw.views, gw.params(2), tape, 0)
    assert res["block"] in (64, 128, 256) and res["blocks_per_sm"] >= 1 and res["chunk"] in (64, 256, 1024)
    assert res["ms"] > 0
    ref, reft = gw.render(launch=0)
    for blk, per in ((128, 3), (256, 2), (64, 8)):
        M.mirres_set_launch(ctx, blk, per, 64)
        img, t = gw.render(launch=2)
        torch.cuda.synchronize()
        n = w.samples
        assert np.array_equal(t.cpu().numpy().view(np.uint32).reshape(TAPE_WORDS, n)[:2],
                              reft.cpu().numpy().view(np.uint32).reshape(TAPE_WORDS, n)[:2])
    M.mirres_set_launch(ctx, 0, 0, 0)
    for s in gw.scenes:
        s.close()


def test_wavefront_autotune_and_shapes(M, ctx):
    """the batched wavefront's launch shape (wave size = queue capacity, per-stage block and grid)
    is tuned on the first views of a batch, becomes the context's shape, and changes nothing but
    the time: renders under the tuned, the default and small odd shapes (waves that split views,
    64-thread blocks, one block per SM, waves spread over 2 and 3 concurrent chains) write the
    same tape word for word and count the same rays"""
    w = synth.config5(seed=5, n_scenes=3, max_tris=6000, res_choices=(96, 128), spp_choices=(3, 4), tex=16)
    assert w.samples > 1 << 16  # several waves of 2^16 samples below
    gw = _gw(ctx, w)
    M.mirres_set_wave_shape(ctx, None)
    M.mirres_reset_counters(ctx)
    ref, reft = gw.render(launch=1)
    torch.cuda.synchronize()
    ref_t = reft.cpu().numpy().copy()
    ref_rays = M.mirres_get_counters(ctx)[:3]
    tape = gw.new_tape()
    res = M.mirres_autotune_wave(ctx, [s.handle for s in gw.scenes], gw.views, gw.params(1), tape, 0)
    assert res["ms"] > 0 and 16 <= res["wave_log2"] <= 25
    assert all(b in (64, 128, 256) for b in res["block"]) and all(1 <= g <= 64 for g in res["blocks_per_sm"])
    assert M.mirres_get_wave_shape(ctx) == {k: res[k] for k in ("wave_log2", "block", "blocks_per_sm", "branches")}
    shapes = [None, dict(wave_log2=16, block=[64, 128, 256, 64], blocks_per_sm=[1, 2, 3, 64]),
              dict(wave_log2=16, block=[256] * 4, blocks_per_sm=[8] * 4, branches=2),
              dict(wave_log2=17, block=[128, 256, 64, 256], blocks_per_sm=[16, 8, 32, 8], branches=3),
              M.mirres_get_wave_shape(ctx)]
    for sh in shapes:
        if sh is not None:
            M.mirres_set_wave_shape(ctx, sh)
        M.mirres_reset_counters(ctx)
        img, t = gw.render(launch=1)
        torch.cuda.synchronize()
        assert M.mirres_get_counters(ctx)[:3] == ref_rays, sh
        # every defined tape word equal (words without a defined value are left unwritten)
        compare_tapes(t.cpu().numpy().view(np.uint32).reshape(TAPE_WORDS, -1),
                      ref_t.view(np.uint32).reshape(TAPE_WORDS, -1), rtol=0)
        for a, b in zip(img, ref):
            assert torch.equal(a, b)
    with pytest.raises(M.MirresError):
        M.mirres_set_wave_shape(ctx, dict(wave_log2=12, block=[256] * 4, blocks_per_sm=[8] * 4))
    with pytest.raises(M.MirresError):
        M.mirres_set_wave_shape(ctx, dict(wave_log2=20, block=[96, 256, 256, 256], blocks_per_sm=[8] * 4))
    with pytest.raises(M.MirresError):
        M.mirres_set_wave_shape(ctx, dict(wave_log2=20, block=[256] * 4, blocks_per_sm=[8] * 4, branches=5))
    M.mirres_set_wave_shape(ctx, None)
    for s in gw.scenes:
        s.close()


@pytest.mark.parametrize("branches", [1, 2])
def test_binned_continuation_rays_change_nothing_but_order(M, ctx, branches):
    """flags bit 3 reorders each bounce's continuation rays by origin cell and direction octant
    before tracing them: the tape, the images and the ray counts are those of the unbinned
    render (multi-scene batch, mixed bounces, waves that split views)"""
    w = synth.config5(seed=8, n_scenes=3, max_tris=6000, res_choices=(64, 96), spp_choices=(3, 4), tex=16)
    gw = _gw(ctx, w)
    M.mirres_set_wave_shape(ctx, dict(wave_log2=16, block=[256] * 4, blocks_per_sm=[8] * 4, branches=branches))
    out = []
    for flags in (0, M.MIRRES_FLAG_BIN):
        M.mirres_reset_counters(ctx)
        img, t = gw.render(launch=1, flags=flags)
        torch.cuda.synchronize()
        out.append(([i.clone() for i in img], t.cpu().numpy().copy(), M.mirres_get_counters(ctx)[:3]))
    (ia, ta, ca), (ib, tb, cb) = out
    assert ca == cb
    compare_tapes(tb.view(np.uint32).reshape(TAPE_WORDS, -1), ta.view(np.uint32).reshape(TAPE_WORDS, -1), rtol=0)
    for a, b in zip(ia, ib):
        assert torch.equal(a, b)
    M.mirres_set_wave_shape(ctx, None)
    for s in gw.scenes:
        s.close()


def test_stage_trace_lists_every_stage_launch(M, ctx):
    """the stage events of a batched render one by one: ray generation then (closest, shade,
    shadow) per bounce for every wave, summing per stage to mirres_stage_times"""
    w = synth.config5(seed=6, n_scenes=2, max_tris=4000, res_choices=(96,), spp_choices=(4,), tex=16)
    gw = _gw(ctx, w)
    M.mirres_set_wave_shape(ctx, dict(wave_log2=16, block=[256] * 4, blocks_per_sm=[8] * 4, branches=2))
    gw.render(launch=1, flags=1)
    torch.cuda.synchronize()
    tr = M.mirres_stage_trace(ctx)
    sums = M.mirres_stage_times(ctx)
    B = max(v.bounces for v in w.views)
    n_waves = -(-w.samples // (1 << 16))
    assert len(tr) == n_waves * (1 + 3 * B)
    for k in range(n_waves):
        chunk = tr[k * (1 + 3 * B):(k + 1) * (1 + 3 * B)]
        assert chunk[0][:2] == ("raygen", -1)
        assert [c[:2] for c in chunk[1:]] == [(s, b) for b in range(B) for s in ("closest", "shade", "shadow")]
    for name, (ms, n) in sums.items():
        part = [c[2] for c in tr if c[0] == name]
        assert len(part) == n and abs(sum(part) - ms) <= 1e-6 * max(ms, 1.0) + 1e-9
        assert all(t >= 0.0 for t in part)
    M.mirres_set_wave_shape(ctx, None)
    for s in gw.scenes:
        s.close()


def test_stage_times_need_an_event_recording_render(M):
    """a context that has not rendered with flags bit 0 has no stage events to report"""
    c = M.mirres_context_create(0)
    with pytest.raises(M.MirresError):
        M.mirres_stage_times(c)
    with pytest.raises(M.MirresError):
        M.mirres_stage_trace(c)
    c.close()


# ---------------------------------------------------------------------------------------
# FULL-mode adjoint (the gradients of the indirect rays at every vertex)
# ---------------------------------------------------------------------------------------
def _full_workload():
    w = synth.config2(res=40, n_views=2, tex=32, spp=4, bounces=4)
    for s in w.scenes:
        s.env[:] = np.minimum(s.env, 80.0)  # keep the per-pixel check well conditioned
    return w


@pytest.mark.parametrize("launch", [0, 1, 2])
def test_full_mode_gradients_match_oracle(M, ctx, launch):
    """FULL-mode gradients from the tape of each launch mode against the oracle's FULL adjoint"""
    w = _full_workload()
    gw = _gw(ctx, w)
    images, tape = gw.render(launch=launch, grad_mode=1)
    torch.cuda.synchronize()
    _grad_parity(gw, w, tape, grad_mode=1)
    for s in gw.scenes:
        s.close()


def test_full_mode_records_identical_across_launches(M, ctx):
    w = _full_workload()
    gw = _gw(ctx, w)
    n = w.samples
    nvx = max(v.bounces for v in w.views) - 1
    words = TAPE_WORDS + 9 * nvx
    tapes = []
    for launch in (0, 1, 2):
        _, t = gw.render(launch=launch, grad_mode=1)
        torch.cuda.synchronize()
        tapes.append(t.cpu().numpy().view(np.uint32).reshape(words, n))
    a = tapes[0]
    for b in tapes[1:]:
        assert np.array_equal(a[:2], b[:2])
        for k in range(nvx):
            r0, r1 = a[TAPE_WORDS + 9 * k:TAPE_WORDS + 9 * (k + 1)], b[TAPE_WORDS + 9 * k:TAPE_WORDS + 9 * (k + 1)]
            assert np.array_equal(r0[0], r1[0])  # the vertex reached, by the same triangle
            live = r0[0].view(np.int32) >= 0
            assert np.array_equal(r0[3][live], r1[3][live])  # the same RIS candidate
            f0, f1 = r0.view(np.float32), r1.view(np.float32)
            for wd in (1, 2, 5, 6, 7, 8):
                assert np.all(np.abs(f0[wd][live] - f1[wd][live]) <= 2e-6 * np.maximum(np.abs(f0[wd][live]), 1.0))
    # reached vertices thin out along the path, and every FULL record sits behind a hit
    reach = [(a[TAPE_WORDS + 9 * k].view(np.int32) >= 0).sum() for k in range(nvx)]
    assert reach[0] > 0 and all(x >= y for x, y in zip(reach, reach[1:]))
    assert np.all(a[0].view(np.int32)[a[TAPE_WORDS].view(np.int32) >= 0] >= 0)
    for s in gw.scenes:
        s.close()


def test_full_mode_edge_cases(M, ctx):
    for name in ("single_triangle", "tiny_views", "empty_scene"):
        w = _edge_workloads()[name]
        gw = _gw(ctx, w)
        images, tape = gw.render(launch=1, grad_mode=1)
        _grad_parity(gw, w, tape, grad_mode=1)
        for s in gw.scenes:
            s.close()


def test_full_mode_argument_checks(M, ctx):
    w = synth.config1()
    gw = _gw(ctx, w)
    assert M.mirres_tape_bytes_mode(gw.views, 1) == M.mirres_tape_bytes(gw.views) + 36 * w.samples * (
        w.views[0].bounces - 1)
    images, tape = gw.render(launch=1)  # a PRIMARY-size tape is too small for FULL mode
    with pytest.raises(M.MirresError):
        gw.render(launch=1, tape=tape, grad_mode=1)
    with pytest.raises(M.MirresError):
        M.mirres_render_noalloc([s.handle for s in gw.scenes], gw.views, gw.params(1, grad_mode=1), images,
                                gw.new_tape(1))
    deep = synth.Workload("deep", w.scenes, [synth.View(w.views[0].K, w.views[0].c2w, 4, 4, 1, 17)], ris_m=2)
    gd = _gw(ctx, deep)
    with pytest.raises(M.MirresError):
        gd.render(launch=1, grad_mode=1)
    for s in gw.scenes + gd.scenes:
        s.close()


def test_work_counters_are_deterministic_and_change_nothing(M, ctx):
    """the counting variant of the traversal stages renders the same image and counts the
    same work every time (the roofline uses one counted render for the timed ones)"""
    w = synth.config2(res=48, n_views=2, tex=32, spp=4)
    gw = _gw(ctx, w)
    ref, tape = gw.render(launch=1)
    counts = []
    for _ in range(2):
        w0 = M.mirres_get_work_counters(ctx)
        img, _ = gw.render(launch=1, tape=tape, flags=2)
        torch.cuda.synchronize()
        counts.append([b - a for a, b in zip(w0, M.mirres_get_work_counters(ctx))])
        for x, y in zip(img, ref):
            assert torch.equal(x, y)
    assert counts[0] == counts[1]
    c = counts[0]
    assert c[0] > 0 and c[1] > 0 and c[2] > 0  # box and triangle tests of both ray kinds
    # at least one box test per primary ray; at most two per node of the tree per ray
    assert c[0] >= w.samples and c[0] <= 2 * w.scenes[0].n_tris * 2 * w.samples
    for s in gw.scenes:
        s.close()
