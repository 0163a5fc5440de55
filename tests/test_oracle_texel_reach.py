"""Pins of the oracle's texel-gradient sensitivity support (the texels whose bilinear weight a
single-precision lookup may change): against brute force over the window of fractional
positions the FP32 error allows, with the bilinear lookup written out from its definition
(texel centres at (i + 1/2) / w, clamped to the edge)."""
import numpy as np
import pytest

from oracle import oracle as O


def _touched(w, h, su, sv):
    """texels with a nonzero bilinear weight at (su, sv)"""
    x, y = su * w - 0.5, sv * h - 0.5
    x0, y0 = np.floor(x), np.floor(y)
    fx, fy = x - x0, y - y0
    out = set()
    for dy, wy in ((0, 1 - fy), (1, fy)):
        for dx, wx in ((0, 1 - fx), (1, fx)):
            if wx * wy > 0.0:
                xi = int(min(max(x0 + dx, 0), w - 1))
                yi = int(min(max(y0 + dy, 0), h - 1))
                out.add(yi * w + xi)
    return out


def _window(w, h, su, sv, dfx, dfy, n=41):
    got = set()
    for ex in np.linspace(-dfx, dfx, n):
        for ey in np.linspace(-dfy, dfy, n):
            got |= _touched(w, h, su + ex / w, sv + ey / h)
    return got


@pytest.mark.parametrize("seed", range(6))
def test_reach_covers_every_texel_a_perturbed_lookup_touches(seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    for _ in range(200):
        w, h = int(rng.integers(1, 9)), int(rng.integers(1, 9))
        # positions near texel centres (the case that moves the footprint) and anywhere
        if rng.uniform() < 0.5:
            su = (rng.integers(0, w) + 0.5 + rng.normal(scale=1e-3)) / w
            sv = (rng.integers(0, h) + 0.5 + rng.normal(scale=1e-3)) / h
        else:
            su, sv = rng.uniform(-0.2, 1.2), rng.uniform(-0.2, 1.2)
        dfx, dfy = float(rng.uniform(0, 4e-3)), float(rng.uniform(0, 4e-3))
        reach = set(O.taps_reach(w, h, su, sv, dfx, dfy))
        need = _window(w, h, su, sv, dfx, dfy)
        assert need <= reach, (w, h, su, sv, dfx, dfy, sorted(need - reach))
        # and no more than the window plus the unperturbed footprint's four taps
        base = set()
        x0, y0 = int(np.floor(su * w - 0.5)), int(np.floor(sv * h - 0.5))
        for dy in (0, 1):
            for dx in (0, 1):
                base.add(min(max(y0 + dy, 0), h - 1) * w + min(max(x0 + dx, 0), w - 1))
        assert reach <= need | base, (w, h, su, sv, dfx, dfy, sorted(reach - need - base))


def test_reach_at_an_exact_texel_centre_spans_three_columns():
    # su on the centre of texel column 2 of 5: fx = 0 exactly, so a lookup a hair to the left
    # takes columns 1 and 2, one to the right columns 2 and 3
    r = O.taps_reach(5, 1, 2.5 / 5, 0.5, 1e-4, 0.0)
    assert r == [1, 2, 3]
    # away from any centre the four (here two) taps of the footprint only
    assert O.taps_reach(5, 1, 2.25 / 5, 0.5, 1e-4, 0.0) == [1, 2]
    # clamped at the edges
    assert O.taps_reach(4, 1, 0.5 / 4, 0.5, 1e-4, 0.0) == [0, 1]
