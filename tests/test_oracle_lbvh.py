"""Pins of the oracle's LBVH restatement (Appendix A, LBVH of Karras 2012).

  * Morton keys of hand-placed centroids, with the expected bit patterns written out by hand.
  * Radix-tree invariants that hold for the Karras hierarchy whatever the input: keys sorted,
    every leaf reached exactly once, each internal node's index is one end of its key range,
    the split sits at the highest differing bit, parents consistent, boxes exact and nested.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2406_16360_gb300 import synth


def _points_as_triangles(pts):
    """degenerate triangles whose centroid is exactly the given point"""
    pts = np.asarray(pts, dtype=np.float32)
    verts = np.repeat(pts, 3, axis=0)
    tris = np.arange(3 * len(pts), dtype=np.int32).reshape(-1, 3)
    return verts, tris


def test_morton_keys_hand_computed():
    pts = [(0, 0, 0), (1, 1, 1), (0.5, 0, 0), (0, 0.5, 0), (0, 0, 0.5), (0.25, 0.75, 0.5)]
    v, t = _points_as_triangles(pts)
    out = O.lbvh(v, t)
    # q = min(floor(c * 1024), 1023) per axis; x bits at positions 3b+2, y at 3b+1, z at 3b
    expected = {
        0: 0,
        1: (1 << 30) - 1,            # q = (1023, 1023, 1023): all 30 bits set
        2: 1 << 29,                  # qx = 512 = bit 9 -> position 3*9+2
        3: 1 << 28,                  # qy = 512 -> 3*9+1
        4: 1 << 27,                  # qz = 512 -> 3*9
        5: (1 << 26) | (1 << 28) | (1 << 25) | (1 << 27),  # qx=256 (bit 8), qy=768 (bits 9,8), qz=512
    }
    keys = sorted((code << 32) | tri for tri, code in expected.items())
    assert [int(k) for k in out["keys"]] == keys


def _reach(left, right, n):
    """leaves reached from the root, with the key range of every internal node"""
    seen = np.zeros(n, dtype=int)
    ranges = {}

    def rec(node):
        lo_hi = []
        for c in (left[node], right[node]):
            if c < 0:
                seen[~c] += 1
                lo_hi.append((~c, ~c))
            else:
                lo_hi.append(rec(c))
        r = (min(lo_hi[0][0], lo_hi[1][0]), max(lo_hi[0][1], lo_hi[1][1]))
        assert lo_hi[0][1] + 1 == lo_hi[1][0], "children must cover adjacent key ranges"
        ranges[node] = r
        return r

    if n >= 2:
        rec(0)
    else:
        seen[0] = 1
    return seen, ranges


def _clz64(x):
    return 64 - int(x).bit_length()


def check_lbvh(verts, tris):
    out = O.lbvh(verts, tris)
    n = len(tris)
    keys, left, right, parent, lo, hi = (out[k] for k in ("keys", "left", "right", "parent", "lo", "hi"))
    assert np.all(keys[1:] > keys[:-1])
    assert sorted(int(k) & 0xFFFFFFFF for k in keys) == list(range(n))
    seen, ranges = _reach(left, right, n)
    assert np.all(seen == 1)
    for node, (a, b) in ranges.items():
        assert node in (a, b), "Karras numbering: an internal node sits at one end of its range"
        dn = _clz64(int(keys[a]) ^ int(keys[b]))
        l = left[node]
        la, lb = (~l, ~l) if l < 0 else ranges[l]
        # the split is at the highest differing bit: both halves share more than dn bits
        assert _clz64(int(keys[la]) ^ int(keys[lb])) > dn
        r = right[node]
        ra, rb = (~r, ~r) if r < 0 else ranges[r]
        assert _clz64(int(keys[ra]) ^ int(keys[rb])) > dn
        for c in (l, r):
            ci = c if c >= 0 else (n - 1) + ~c
            assert parent[ci] == node
    if n >= 1:
        assert parent[0 if n >= 2 else 0] == -1
    # leaf boxes: exact vertex min / max; internal: exact union of the children
    for i in range(n):
        t = int(keys[i]) & 0xFFFFFFFF
        p = verts[tris[t]]
        assert np.array_equal(lo[n - 1 + i], p.min(axis=0)) and np.array_equal(hi[n - 1 + i], p.max(axis=0))
    for node in range(n - 1):
        cs = [left[node], right[node]]
        ids = [c if c >= 0 else (n - 1) + ~c for c in cs]
        assert np.array_equal(lo[node], np.minimum(lo[ids[0]], lo[ids[1]]))
        assert np.array_equal(hi[node], np.maximum(hi[ids[0]], hi[ids[1]]))
    return out


def test_lbvh_invariants_config1():
    sc = synth.config1().scenes[0]
    check_lbvh(sc.verts, sc.tris)


@pytest.mark.parametrize("n", [1, 2, 3, 7, 64, 1000])
def test_lbvh_invariants_random_and_edge_sizes(n):
    rng = np.random.Generator(np.random.PCG64(n))
    v = rng.normal(size=(3 * n, 3)).astype(np.float32)
    t = np.arange(3 * n, dtype=np.int32).reshape(-1, 3)
    check_lbvh(v, t)


def test_lbvh_duplicate_centroids_and_flat_axis():
    # many triangles with the same centroid (identical codes, ordered by id) and a flat z extent
    rng = np.random.Generator(np.random.PCG64(3))
    same = np.tile([[0.3, 0.2, 0.0]], (20, 1))
    spread = np.c_[rng.uniform(size=(30, 2)), np.zeros(30)]
    pts = np.concatenate([same, spread])
    v, t = _points_as_triangles(pts)
    out = check_lbvh(v, t)
    codes = out["keys"] >> np.uint64(32)
    assert len(np.unique(codes)) < len(codes)
