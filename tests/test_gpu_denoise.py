"""GPU parity of the denoiser between the image and the loss (Appendix A, "Denoiser") and of
its G-buffer, through the C ABI, against the FP64 oracle (oracle/eawt.py)."""
import numpy as np
import pytest
import torch

from oracle import eawt as E
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


def _gbuffer(M, ctx, gw, vi=0):
    v = gw.views[vi]
    n = torch.empty((v.height, v.width, 3), device="cuda")
    x = torch.empty_like(n)
    M.mirres_gbuffer(ctx, gw.scenes[v.scene].handle, v, n, x)
    torch.cuda.synchronize()
    return n, x


@pytest.mark.parametrize("which", ["config1", "config2"])
def test_gbuffer_matches_oracle(M, ctx, which):
    from paper_2406_16360_gb300.renderer import GpuWorkload
    w = synth.config1() if which == "config1" else synth.config2(res=72, n_views=1, tex=16, spp=1)
    gw = GpuWorkload(w, 0, ctx=ctx)
    n, x = _gbuffer(M, ctx, gw)
    on, ox, otri, mg = E.gbuffer(O.OracleScene(w.scenes[0]), w.views[0])
    gn, gx = n.cpu().numpy().astype(np.float64), x.cpu().numpy().astype(np.float64)
    ghit = np.linalg.norm(gn, axis=-1) > 0
    sure = mg >= 1.0  # decisions away from their thresholds
    assert np.array_equal(ghit[sure], (otri >= 0)[sure])
    both = sure & ghit & (otri >= 0)
    assert both.sum() > 100
    assert np.abs(gn[both] - on[both]).max() < 2e-5 or \
        np.mean(np.abs(gn[both] - on[both]).max(-1) < 2e-5) > 0.995  # a flipped neighbour face at most
    assert np.abs(gx[both] - ox[both]).max() < 2e-5 * max(1.0, np.abs(ox).max())
    for s in gw.scenes:
        s.close()


def _inputs(M, ctx, seed, H, W):
    rng = np.random.Generator(np.random.PCG64(seed))
    img = rng.uniform(0, 2, (H, W, 3)).astype(np.float32)
    n = rng.normal(size=(H, W, 3))
    n /= np.linalg.norm(n, axis=-1, keepdims=True)
    n[rng.uniform(size=(H, W)) < 0.1] = 0.0  # escaped pixels
    x = rng.normal(size=(H, W, 3)).astype(np.float32)
    return img, n.astype(np.float32), x


def _run(M, ctx, img, n, x, sig, levels, d_out=None):
    H, W = img.shape[:2]
    p = M.EawtParams(sig[0], sig[1], sig[2], levels)
    t = lambda a: torch.as_tensor(a, device="cuda").contiguous()
    ti, tn, tx = t(img), t(n), t(x)
    out = torch.empty_like(ti)
    rec = torch.empty(M.mirres_eawt_record_bytes(W, H, levels) // 4, device="cuda")
    M.mirres_eawt(ctx, ti, tn, tx, p, out, rec)
    g = None
    if d_out is not None:
        g = torch.empty_like(ti)
        M.mirres_eawt_backward(ctx, t(d_out), tn, tx, p, rec, g)
    torch.cuda.synchronize()
    return out.cpu().numpy(), None if g is None else g.cpu().numpy()


@pytest.mark.parametrize("H,W,levels", [(40, 56, 3), (1, 1, 3), (3, 7, 1), (17, 5, 8), (65, 33, 3)])
def test_eawt_forward_and_adjoint_match_oracle(M, ctx, H, W, levels):
    img, n, x = _inputs(M, ctx, H * 100 + W, H, W)
    rng = np.random.Generator(np.random.PCG64(5))
    d = rng.normal(size=(H, W, 3)).astype(np.float32)
    sig = (0.8, 0.6, 1.5)
    out, g = _run(M, ctx, img, n, x, sig, levels, d)
    ref, rec = E.eawt(img, n, x, *sig, levels=levels)
    gref = E.eawt_backward(d, rec)
    assert np.abs(out - ref).max() <= 2e-5 * max(1.0, np.abs(ref).max())
    assert np.abs(g - gref).max() <= 2e-5 * max(1.0, np.abs(gref).max())


def test_eawt_on_a_rendered_image_with_its_gbuffer(M, ctx):
    from paper_2406_16360_gb300.renderer import GpuWorkload
    w = synth.config1()
    gw = GpuWorkload(w, 0, ctx=ctx)
    images, _ = gw.render(launch=1)
    n, x = _gbuffer(M, ctx, gw)
    img = images[0].cpu().numpy()
    d = np.random.Generator(np.random.PCG64(9)).normal(size=img.shape).astype(np.float32)
    sig = (0.3, 0.2, 0.5)
    out, g = _run(M, ctx, img, n.cpu().numpy(), x.cpu().numpy(), sig, 3, d)
    ref, rec = E.eawt(img, n.cpu().numpy(), x.cpu().numpy(), *sig)
    assert np.abs(out - ref).max() <= 2e-5 * max(1.0, np.abs(ref).max())
    assert np.abs(g - E.eawt_backward(d, rec)).max() <= 2e-5 * max(1.0, np.abs(g).max())
    # the denoised image is smoother than the noisy one where the surface is flat
    assert np.abs(np.diff(out, axis=1)).mean() < np.abs(np.diff(img, axis=1)).mean()
    for s in gw.scenes:
        s.close()


def test_eawt_argument_checks(M, ctx):
    img = torch.zeros((4, 4, 3), device="cuda")
    rec = torch.empty(M.mirres_eawt_record_bytes(4, 4, 3) // 4, device="cuda")
    for bad in (M.EawtParams(0.0, 1.0, 1.0, 3), M.EawtParams(1.0, 1.0, 1.0, 0), M.EawtParams(1.0, 1.0, 1.0, 9)):
        with pytest.raises(M.MirresError):
            M.mirres_eawt(ctx, img, img, img, bad, img.clone(), rec)
    small = torch.empty(8, device="cuda")
    with pytest.raises(M.MirresError):
        M.mirres_eawt(ctx, img, img, img, M.EawtParams(1.0, 1.0, 1.0, 3), img.clone(), small)
    assert M.mirres_eawt_record_bytes(4, 4, 3) == (32 + 20 * 3) * 16
    assert M.mirres_eawt_record_bytes(0, 4, 3) == 0


@pytest.mark.parametrize("N,H,W,levels", [(3, 37, 50, 3), (2, 9, 4, 4), (5, 1, 13, 2)])
def test_eawt_batch_filters_each_image_on_its_own(M, ctx, N, H, W, levels):
    """a stack of N images in one launch per level: each image the oracle's result on its own
    (no tap reaches into a neighbouring image), and bit for bit the single-image calls"""
    rng = np.random.Generator(np.random.PCG64(N * 1000 + H))
    ins = [_inputs(M, ctx, 77 + i, H, W) for i in range(N)]
    d = rng.normal(size=(N, H, W, 3)).astype(np.float32)
    sig = (0.7, 0.5, 1.2)
    p = M.EawtParams(sig[0], sig[1], sig[2], levels)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    img, nrm, pos = (t(np.stack([a[k] for a in ins])) for k in range(3))
    out = torch.empty_like(img)
    rec = torch.empty(N * M.mirres_eawt_record_bytes(W, H, levels) // 4, device="cuda")
    M.mirres_eawt_batch(ctx, img, nrm, pos, p, out, rec)
    g = torch.empty_like(img)
    M.mirres_eawt_batch_backward(ctx, t(d), nrm, pos, p, rec, g)
    torch.cuda.synchronize()
    out, g = out.cpu().numpy(), g.cpu().numpy()
    for i, (im, n, x) in enumerate(ins):
        ref, orec = E.eawt(im, n, x, *sig, levels=levels)
        gref = E.eawt_backward(d[i], orec)
        assert np.abs(out[i] - ref).max() <= 2e-5 * max(1.0, np.abs(ref).max())
        assert np.abs(g[i] - gref).max() <= 2e-5 * max(1.0, np.abs(gref).max())
        o1, g1 = _run(M, ctx, im, n, x, sig, levels, d[i])
        assert np.array_equal(o1, out[i]) and np.array_equal(g1, g[i])


def test_eawt_batch_argument_checks(M, ctx):
    img = torch.zeros((2, 4, 4, 3), device="cuda")
    p = M.EawtParams(1.0, 1.0, 1.0, 3)
    one = torch.empty(M.mirres_eawt_record_bytes(4, 4, 3) // 4, device="cuda")
    with pytest.raises(M.MirresError):
        M.mirres_eawt_batch(ctx, img, img, img, p, img.clone(), one)  # a record for one image only
    with pytest.raises(M.MirresError):
        M.mirres_eawt_batch(ctx, img[:0], img[:0], img[:0], p, img[:0].clone(), one)
