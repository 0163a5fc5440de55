"""GPU checks of primary visibility by rasterisation (params.flags bit 2 of the batched launch):
against the FP64 oracle on the parity workloads and edge cases, and against the traced
primary rays of the same launch (the rasteriser runs the traversal's FP32 ray/triangle solve
and closest rule, so hits agree except where two solves are within rounding of each other)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2406_16360_gb300 import synth
from paper_2406_16360_gb300.mirres import TAPE_WORDS
from tests.parity import compare_pixels

pytestmark = pytest.mark.gpu

RASTER = 4


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


def _close(gw):
    for s in gw.scenes:
        s.close()


def _oracle_check(w, images, max_flag_frac=0.08):
    for vi, v in enumerate(w.views):
        r = O.render(O.OracleScene(w.scenes[v.scene]), v, vi, w.ris_m, seed=w.seed)
        st = compare_pixels(images[vi].cpu().numpy().reshape(-1, 3), r["rgb"], r["margin"])
        assert st["failures"] == 0, (vi, st["failures"], st["max_err_unflagged"])
        assert st["flagged"] <= max_flag_frac * st["n"] + 1, (vi, st["flagged"], st["n"])


def _tri_ids(tape, n):
    return tape.cpu().numpy().view(np.int32).reshape(TAPE_WORDS, -1)[0][:n]


def _workloads():
    out = {"config1": synth.config1(), "config2_small": synth.config2(res=40, n_views=3, tex=16, spp=2)}
    sc = synth.tiny_scene()
    # a ragged 31x3 view and a 1x1 view
    K, c2w = synth.look_at((0.0, 1.5, 4.0), (0.0, 1.0, 0.0), 1, 1)
    K2, c2w2 = synth.look_at((0.3, 1.2, 3.5), (0.0, 0.9, 0.0), 31, 3)
    out["tiny_views"] = synth.Workload("tiny", [sc], [synth.View(K, c2w, 1, 1, 1, 1),
                                                      synth.View(K2, c2w2, 31, 3, 7, 2)], ris_m=1, seed=5)
    # the camera between the sphere and the ground, looking along it: ground triangles cross
    # the camera plane (the whole-screen path) and the sphere is seen up close
    K, c2w = synth.look_at((0.0, 0.3, 2.2), (0.0, 0.9, 0.0), 24, 20, 70.0)
    out["inside"] = synth.Workload("inside", [sc], [synth.View(K, c2w, 24, 20, 3, 2)], ris_m=4, seed=2)
    # no triangles: every sample misses
    empty = synth._scene(np.zeros((1, 3)), np.zeros((0, 3), np.int32), np.zeros((0, 3, 2)), sc.albedo,
                         sc.roughness, sc.metallic, sc.env)
    K, c2w = synth.look_at((0.0, 1.5, 4.0), (0.0, 1.0, 0.0), 13, 7)
    out["empty_scene"] = synth.Workload("empty", [empty], [synth.View(K, c2w, 13, 7, 3, 2)], ris_m=4)
    return out


@pytest.mark.parametrize("name", list(_workloads().keys()))
def test_raster_matches_oracle_and_tracing(M, ctx, name):
    w = _workloads()[name]
    gw = _gw(ctx, w)
    img_r, tape_r = gw.render(launch=1, flags=RASTER)
    torch.cuda.synchronize()
    _oracle_check(w, img_r, max_flag_frac=0.2 if name in ("tiny_views", "inside") else 0.08)
    img_t, tape_t = gw.render(launch=1)
    torch.cuda.synchronize()
    a, b = _tri_ids(tape_r, w.samples), _tri_ids(tape_t, w.samples)
    assert np.mean(a != b) <= 1e-4 + 1.0 / w.samples, np.mean(a != b)
    if name == "empty_scene":
        assert np.all(a == -1)
    _close(gw)


def test_raster_views_straddling_waves(M, ctx):
    """four 800x800 views at 16 spp (41M samples): waves of 2^25 samples cut views in two, so
    each wave rasterises the part of a view it holds"""
    w = synth.config3(n_views=4)
    gw = _gw(ctx, w)
    _, tape_r = gw.render(launch=1, flags=RASTER)
    _, tape_t = gw.render(launch=1)
    torch.cuda.synchronize()
    a, b = _tri_ids(tape_r, w.samples), _tri_ids(tape_t, w.samples)
    assert (a >= 0).mean() > 0.2
    assert np.mean(a != b) <= 1e-5, np.mean(a != b)
    _close(gw)


def test_raster_backward_equals_tracing_backward(M, ctx):
    """the adjoint replays the primary vertex from the tape: with the same hits it is the same"""
    w = synth.config1()
    gw = _gw(ctx, w)
    grads = []
    for flags in (RASTER, 0):
        images, tape = gw.render(launch=1, flags=flags)
        d = [torch.ones_like(im) for im in images]
        g = gw.backward(d, tape, launch=1)
        torch.cuda.synchronize()
        grads.append({k: v.cpu().numpy() for k, v in g[0].items()})
    # identical hits give identical gradients up to the order of the FP32 atomics; a hit that
    # differs (a near-tie) moves one sample's terms
    for k in grads[0]:
        a, b = grads[0][k], grads[1][k]
        assert np.abs(a - b).max() <= 1e-3 * max(np.abs(b).max(), 1e-12), k
    _close(gw)
