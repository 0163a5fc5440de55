"""GPU parity of the spatial reservoir reuse at the primary vertex (Appendix A, "Spatial-temporal
Reuse") through the C ABI, against the FP64 oracle's restatement (same random streams, same
neighbours, same merge rule), forward and PRIMARY-mode adjoint."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2406_16360_gb300 import synth
from tests.parity import compare_grads, grad_tolerance, compare_pixels

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


@pytest.mark.parametrize("which,reuse", [("config1", (4, 3)), ("config2", (6, 5)), ("config1", (1, 1))])
def test_reuse_forward_and_adjoint_match_oracle(M, ctx, which, reuse):
    if which == "config1":
        w = synth.config1(width=40, height=36)
    else:
        w = synth.config2(res=40, n_views=2, tex=32, spp=4)
        for s in w.scenes:
            s.env[:] = np.minimum(s.env, 80.0)
    gw = _gw(ctx, w)
    images, tape = gw.render(launch=1, reuse=reuse)
    torch.cuda.synchronize()
    rng = np.random.Generator(np.random.PCG64(4))
    d_imgs, dlist = [], []
    for vi, v in enumerate(w.views):
        osc = O.OracleScene(w.scenes[v.scene])
        r = O.render(osc, v, vi, w.ris_m, seed=w.seed, reuse=reuse)
        st = compare_pixels(images[vi].cpu().numpy().reshape(-1, 3), r["rgb"], r["margin"])
        assert st["failures"] == 0, (vi, st["failures"], st["max_err_unflagged"])
        assert st["flagged"] <= 0.15 * st["n"] + 1, (vi, st["flagged"], st["n"])
        g = rng.normal(size=(v.width * v.height, 3))
        g[r["margin"] < 1.0] = 0.0
        d_imgs.append(torch.as_tensor(g.reshape(v.height, v.width, 3), dtype=torch.float32, device="cuda"))
        dlist.append(g)
    grads = gw.backward(d_imgs, tape)
    torch.cuda.synchronize()
    acc = None
    for vi, v in enumerate(w.views):
        gi = O.backward(O.OracleScene(w.scenes[v.scene]), v, vi, w.ris_m, dlist[vi], seed=w.seed, reuse=reuse)
        acc = gi if acc is None else {k: acc[k] + gi[k] for k in gi if k != "counts"}
    for k in ("albedo", "roughness", "metallic", "env", "verts"):
        st = compare_grads(grads[0][k].cpu().numpy(), acc[k], acc[k + "_abs"], acc.get(k + "_sens"),
                               **grad_tolerance(k))
        assert st["failures"] == 0, (k, st["failures"], st["detail"])
    for s in gw.scenes:
        s.close()


def test_reuse_changes_the_estimate_and_off_changes_nothing(M, ctx):
    w = synth.config1(width=32, height=32)
    gw = _gw(ctx, w)
    a, _ = gw.render(launch=1)
    b, _ = gw.render(launch=1, reuse=(0, 0))
    c, _ = gw.render(launch=1, reuse=(4, 3))
    torch.cuda.synchronize()
    assert torch.equal(a[0], b[0])
    assert not torch.equal(a[0], c[0])
    for s in gw.scenes:
        s.close()


def test_reuse_argument_checks(M, ctx):
    w = synth.config1(width=8, height=8)
    gw = _gw(ctx, w)
    for launch in (0, 2):
        with pytest.raises(M.MirresError):
            gw.render(launch=launch, reuse=(4, 3))
    for bad in ((65, 3), (4, 0), (-1, 3)):
        with pytest.raises(M.MirresError):
            gw.render(launch=1, reuse=bad)
    for s in gw.scenes:
        s.close()


def _history_np(h, n):
    """GPU history (5 word arrays over the samples) -> the oracle's [samples][5] doubles"""
    a = h.cpu().numpy().view(np.uint32).reshape(5, n)
    return np.stack([a[0].view(np.int32).astype(np.float64), a[1].astype(np.float64),
                     a[2].view(np.float32).astype(np.float64), a[3].view(np.float32).astype(np.float64),
                     a[4].view(np.float32).astype(np.float64)], axis=1)


@pytest.mark.parametrize("reuse", [(0, 0), (4, 3)])
def test_temporal_reuse_two_frames_match_oracle(M, ctx, reuse):
    """frame 1 records the reservoir history, frame 2 (another seed) merges it: images, the
    recorded histories and the adjoint against the oracle, frame 2 fed the GPU's own history"""
    w = synth.config1(width=40, height=36)
    gw = _gw(ctx, w)
    v = w.views[0]
    n = w.samples
    osc = O.OracleScene(w.scenes[0])
    hist = gw.new_history()
    img1, _ = gw.render(launch=1, reuse=reuse, temporal=1, history=hist)
    torch.cuda.synchronize()
    h1 = _history_np(hist, n)
    r1 = O.render(osc, v, 0, w.ris_m, seed=w.seed, reuse=reuse, temporal=1)
    st = compare_pixels(img1[0].cpu().numpy().reshape(-1, 3), r1["rgb"], r1["margin"])
    assert st["failures"] == 0, st["max_err_unflagged"]
    sure = np.repeat(r1["margin"] >= 1.0, v.spp)  # samples of unflagged pixels
    oh = r1["history"]
    assert np.array_equal(h1[sure, 0], oh[sure, 0]) and np.array_equal(h1[sure, 4], oh[sure, 4])
    sel = sure & (oh[:, 0] >= 0)
    for k in (2, 3):
        assert np.all(np.abs(h1[sel, k] - oh[sel, k]) <= 1e-4 * np.abs(oh[sel, k]))
    # frame 2: another seed, the history merged first
    img2, tape2 = gw.render(launch=1, seed=w.seed + 7, reuse=reuse, temporal=2, temporal_cap=8, history=hist)
    torch.cuda.synchronize()
    r2 = O.render(osc, v, 0, w.ris_m, seed=w.seed + 7, reuse=reuse, temporal=2, temporal_cap=8, history=h1)
    st = compare_pixels(img2[0].cpu().numpy().reshape(-1, 3), r2["rgb"], r2["margin"])
    assert st["failures"] == 0, st["max_err_unflagged"]
    assert st["flagged"] <= 0.15 * st["n"] + 1
    g = np.random.Generator(np.random.PCG64(8)).normal(size=(v.width * v.height, 3))
    g[r2["margin"] < 1.0] = 0.0
    grads = gw.backward([torch.as_tensor(g.reshape(v.height, v.width, 3), dtype=torch.float32, device="cuda")],
                        tape2, seed=w.seed + 7)
    torch.cuda.synchronize()
    og = O.backward(osc, v, 0, w.ris_m, g, seed=w.seed + 7, reuse=reuse, temporal=2, temporal_cap=8, history=h1)
    for k in ("albedo", "roughness", "metallic", "env", "verts"):
        st = compare_grads(grads[0][k].cpu().numpy(), og[k], og[k + "_abs"], og.get(k + "_sens"),
                               **grad_tolerance(k))
        assert st["failures"] == 0, (k, st["detail"])
    for s in gw.scenes:
        s.close()


def test_temporal_reuse_argument_checks(M, ctx):
    w = synth.config1(width=8, height=8)
    gw = _gw(ctx, w)
    with pytest.raises(M.MirresError):
        gw.render(launch=1, temporal=1)  # no history buffer
    small = torch.zeros(16, device="cuda", dtype=torch.int32)
    with pytest.raises(M.MirresError):
        gw.render(launch=1, temporal=1, history=small)
    with pytest.raises(M.MirresError):
        gw.render(launch=0, temporal=1, history=gw.new_history())
    with pytest.raises(M.MirresError):
        gw.render(launch=1, temporal=2, temporal_cap=0, history=gw.new_history())
    assert M.mirres_reuse_history_bytes(gw.views) == 20 * w.samples
    for s in gw.scenes:
        s.close()


def test_reuse_under_wave_chains_and_views_larger_than_a_wave(M, ctx):
    """spatial + temporal reuse with the waves dealt to two concurrent chains and a wave size
    below the largest view (the wave grows to hold it): the same images, tape and history as the
    default launch shape"""
    from tests.parity import compare_tapes
    w = synth.config5(seed=9, n_scenes=3, max_tris=5000, res_choices=(96, 160), spp_choices=(3, 4), tex=16)
    assert max(v.width * v.height * v.spp for v in w.views) > 1 << 16
    gw = _gw(ctx, w)
    out = []
    for shape in (None, dict(wave_log2=16, block=[128] * 4, blocks_per_sm=[16] * 4, branches=2)):
        M.mirres_set_wave_shape(ctx, shape)
        hist = gw.new_history()
        gw.render(launch=1, reuse=(4, 3), temporal=1, history=hist)
        img, tape = gw.render(launch=1, seed=w.seed + 3, reuse=(4, 3), temporal=2, history=hist)
        torch.cuda.synchronize()
        out.append(([i.clone() for i in img], tape.cpu().numpy().copy(), hist.cpu().numpy().copy()))
    M.mirres_set_wave_shape(ctx, None)
    (ia, ta, ha), (ib, tb, hb) = out
    compare_tapes(tb.view(np.uint32).reshape(M.TAPE_WORDS, -1), ta.view(np.uint32).reshape(M.TAPE_WORDS, -1), rtol=0)
    assert np.array_equal(ha, hb)
    for a, b in zip(ia, ib):
        assert torch.equal(a, b)
    for s in gw.scenes:
        s.close()
