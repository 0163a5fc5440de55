"""mirres_render_noalloc: the batched forward for callers that cannot allocate device memory
while they render. Its scratch is a static device array, so this checks that two calls in a
row, with different views, each match the ordinary mirres_render, and that sizes beyond the
array's stated limits are refused. Collected last on purpose (file name)."""
import numpy as np
import pytest
import torch

from paper_2406_16360_gb300 import synth
from paper_2406_16360_gb300.mirres import TAPE_WORDS
from tests.parity import FWD_RTOL

pytestmark = pytest.mark.gpu


def _relerr(a, b):
    a = a.double().reshape(-1, 3)
    b = b.double().reshape(-1, 3)
    scale = b.abs().max(dim=1).values.clamp_min(1e-30)
    return ((a - b).abs().max(dim=1).values / scale).max().item()


def test_noalloc_matches_render_on_two_calls():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_16360_gb300 import mirres as M
    from paper_2406_16360_gb300.renderer import GpuWorkload

    ctx = M.mirres_context_create(0)
    for w in (synth.config2(res=40, n_views=3, tex=32, spp=4), synth.config1(width=48, height=32)):
        gw = GpuWorkload(w, 0, ctx=ctx)
        scenes = [s.handle for s in gw.scenes]
        ref_img, ref_tape = gw.render(launch=1)
        img = gw.new_images()
        tape = gw.new_tape()
        M.mirres_render_noalloc(scenes, gw.views, gw.params(1), img, tape)
        torch.cuda.synchronize()
        n = w.samples
        a = tape.cpu().numpy().view(np.uint32).reshape(TAPE_WORDS, n)
        b = ref_tape.cpu().numpy().view(np.uint32).reshape(TAPE_WORDS, n)
        assert np.array_equal(a[:2], b[:2])  # hit triangles and selected candidates
        for x, y in zip(img, ref_img):
            assert _relerr(x, y) <= FWD_RTOL
        for s in gw.scenes:
            s.close()
    # sizes beyond the static maximum are refused with an argument error
    w = synth.config1(width=8, height=8)
    gw = GpuWorkload(w, 0, ctx=ctx)
    many = [w.views[0]] * (M.MIRRES_NOALLOC_MAX_VIEWS + 1)
    imgs = [torch.empty((8, 8, 3), device="cuda")] * len(many)
    tape = torch.empty(M.mirres_tape_bytes(many) // 4, dtype=torch.int32, device="cuda")
    with pytest.raises(M.MirresError) as e:
        M.mirres_render_noalloc([s.handle for s in gw.scenes], many, gw.params(1), imgs, tape)
    assert e.value.status == 1 and str(M.MIRRES_NOALLOC_MAX_VIEWS) in str(e.value)
    with pytest.raises(M.MirresError):
        M.mirres_render_noalloc([s.handle for s in gw.scenes], w.views, gw.params(1), gw.new_images(), None)
    # reservoir reuse needs per-sample scratch this entry point does not have: refused, not ignored
    with pytest.raises(M.MirresError) as e:
        M.mirres_render_noalloc([s.handle for s in gw.scenes], w.views, gw.params(1, reuse=(1, 2)),
                                gw.new_images(), gw.new_tape())
    assert e.value.status == 1 and "reuse" in str(e.value)
    for s in gw.scenes:
        s.close()
    ctx.close()
