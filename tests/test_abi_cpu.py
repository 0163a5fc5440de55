"""The C ABI without a GPU: the library builds for sm_103a, loads, exports every entry point
declared in include/mirres.h, and rejects bad arguments on the host before touching CUDA."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in sorted(os.listdir(os.path.join(ROOT, "include")))
           if h.endswith(".h")]


@pytest.fixture(scope="module")
def lib():
    from paper_2406_16360_gb300 import build
    path = build.build()
    return C.CDLL(path)


def declared():
    """every entry point declared in include/*.h"""
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names.update(re.findall(r"\b(mirres_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared()
    for n in ("mirres_context_create", "mirres_scene_create", "mirres_bvh_build", "mirres_bvh_refit",
              "mirres_render", "mirres_backward", "mirres_last_error", "mirres_scene_validate",
              "mirres_peak_fp32", "mirres_peak_l2"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_side_argument_checks(lib):
    lib.mirres_last_error.restype = C.c_char_p
    vp = C.c_void_p
    # NULL context / descriptors are rejected with MIRRES_ERR_ARG and a message
    lib.mirres_scene_create.argtypes = [vp, vp, vp]
    assert lib.mirres_scene_create(None, None, None) == 1
    assert lib.mirres_last_error()
    lib.mirres_render.argtypes = [vp, vp, C.c_int32, vp, C.c_int32, vp, vp, vp, C.c_size_t, vp]
    assert lib.mirres_render(None, None, 0, None, 0, None, None, None, 0, None) == 1
    lib.mirres_backward.argtypes = [vp, vp, C.c_int32, vp, C.c_int32, vp, vp, vp, C.c_size_t, vp, vp]
    assert lib.mirres_backward(None, None, 0, None, 0, None, None, None, 0, None, None) == 1
    lib.mirres_l2_loss.argtypes = [vp, vp, C.c_int64, vp, vp, vp]
    assert lib.mirres_l2_loss(None, None, 4, None, None, None) == 1
    lib.mirres_bvh_build.argtypes = [vp, vp]
    assert lib.mirres_bvh_build(None, None) == 1
    lib.mirres_get_counters.argtypes = [vp, vp]
    assert lib.mirres_get_counters(None, None) == 1
    out = vp()
    lib.mirres_context_create.argtypes = [C.c_int32, C.POINTER(vp)]
    assert lib.mirres_context_create(0, None) == 1


def test_tape_bytes_per_sample(lib):
    from paper_2406_16360_gb300 import mirres as M
    hdr = open(os.path.join(ROOT, "include", "mirres.h")).read()
    assert re.search(r"#define MIRRES_TAPE_BYTES_PER_SAMPLE (\d+)", hdr).group(1) == str(M.MIRRES_TAPE_BYTES_PER_SAMPLE)
    views = (M.View * 2)(M.make_view([1, 1, 0, 0], [0] * 12, 64, 32, 4, 2), M.make_view([1, 1, 0, 0], [0] * 12, 5, 3, 7, 3))
    lib.mirres_tape_bytes.restype = C.c_size_t
    lib.mirres_tape_bytes.argtypes = [C.POINTER(M.View), C.c_int32]
    assert lib.mirres_tape_bytes(views, 2) == M.MIRRES_TAPE_BYTES_PER_SAMPLE * (64 * 32 * 4 + 5 * 3 * 7)
    assert lib.mirres_tape_bytes(views, 0) == 0


def test_context_without_gpu_reports_cuda_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib.mirres_context_create.argtypes = [C.c_int32, C.POINTER(C.c_void_p)]
    h = C.c_void_p()
    st = lib.mirres_context_create(0, C.byref(h))
    assert st in (1, 2) and not h.value
