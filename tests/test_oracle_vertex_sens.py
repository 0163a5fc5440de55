"""The oracle's FP32 sensitivity bound of the vertex gradients (test tolerance only).

The bound sums, over samples and over the primary vertex's inputs (camera direction,
barycentrics, selected light and continuation directions, shading normal), the change of each
vertex term when that input moves by its FP32 rounding scale. These tests check that it is a
bound of the right size: non-negative, present exactly where vertex terms are, tight for rough
materials, and growing where the method is ill-conditioned (a glossy GGX lobe, whose derivative
with respect to the normal is conditioned like 1 / alpha^2).
"""
import copy

import numpy as np
import pytest

from oracle import oracle as O
from paper_2406_16360_gb300 import synth


@pytest.fixture(scope="module", autouse=True)
def _build():
    O.build()


def _grads(w, normals=0, rough=None):
    sc = copy.deepcopy(w.scenes[0])
    if rough is not None:
        sc.roughness[:] = rough
    osc = O.OracleScene(sc, normals=normals)
    v = w.views[0]
    r = O.render(osc, v, 0, w.ris_m, seed=w.seed)
    g = np.random.Generator(np.random.PCG64(3)).normal(size=(v.width * v.height, 3))
    g[r["margin"] < 1.0] = 0.0
    return O.backward(osc, v, 0, w.ris_m, g, seed=w.seed)


def test_sensitivity_is_a_nonnegative_bound_where_vertex_terms_are():
    out = _grads(synth.config1(width=32, height=32))
    sens, ab = out["verts_sens"], out["verts_abs"]
    assert np.all(np.isfinite(sens)) and np.all(sens >= 0.0)
    assert np.all(sens[ab == 0.0] == 0.0)
    touched = ab > 0.0
    assert touched.sum() > 100 and np.mean(sens[touched] > 0.0) > 0.9


def test_sensitivity_is_small_for_a_rough_material_and_grows_for_a_glossy_one():
    w = synth.config1(width=32, height=32)
    rough = _grads(w, rough=0.8)
    glossy = _grads(w, rough=0.1)
    nz_r, nz_g = rough["verts_abs"] > 0, glossy["verts_abs"] > 0
    q_r = rough["verts_sens"][nz_r] / rough["verts_abs"][nz_r]
    q_g = glossy["verts_sens"][nz_g] / glossy["verts_abs"][nz_g]
    # FP32 rounding of a well-conditioned term is a few 1e-7 to 1e-6 of it
    assert np.median(q_r) < 1e-5 and np.quantile(q_r, 0.9) < 1e-5, np.quantile(q_r, [0.5, 0.9])
    # alpha = r^2: 1e-2 against 0.64, so near the specular peak the lobe's normal derivative is
    # far worse conditioned: the vertices that see it carry a much larger bound
    assert np.quantile(q_g, 0.9) > 20.0 * np.quantile(q_r, 0.9), (np.quantile(q_g, 0.9), np.quantile(q_r, 0.9))
