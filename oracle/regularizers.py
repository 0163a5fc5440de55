"""FP64 oracle of the mesh regularisers added to the rendering loss (Appendix A, "Training
details"): the Laplacian smoothness of the refined vertices and the vertex-offset penalty.

TEST INFRASTRUCTURE ONLY: imported by the tests; the CUDA library never imports it.

  L_smooth = sum_i sum_{j in X_i} |v_i - v_j|^2 / |X_i|,  X_i = the vertices sharing an edge with i
  L_offset = sum_i |v_i - v0_i|^2                          (v = v0 + offset)

with v the current (refined) positions and v0 the positions before refinement. Readings: X_i
is taken from the triangles' edges, each neighbour once; a vertex without edges adds nothing.
"""
from __future__ import annotations

import numpy as np


def edges(tris):
    """unique undirected edges (a < b) of a triangle list, and every vertex's neighbour count"""
    t = np.asarray(tris, dtype=np.int64).reshape(-1, 3)
    e = np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]], axis=0)
    e = np.sort(e, axis=1)
    e = e[e[:, 0] != e[:, 1]]
    e = np.unique(e, axis=0)
    return e


def degrees(e, n_verts):
    deg = np.zeros(n_verts)
    np.add.at(deg, e[:, 0], 1.0)
    np.add.at(deg, e[:, 1], 1.0)
    return deg


def l_smooth(verts, tris):
    """(loss, d loss / d verts) of the Laplacian smoothness term"""
    v = np.asarray(verts, dtype=np.float64)
    e = edges(tris)
    deg = degrees(e, v.shape[0])
    g = np.zeros_like(v)
    loss = 0.0
    # X_i as explicit neighbour lists, summed term by term as the formula reads
    nb = [[] for _ in range(v.shape[0])]
    for a, b in e:
        nb[a].append(b)
        nb[b].append(a)
    for i in range(v.shape[0]):
        for j in nb[i]:
            d = v[i] - v[j]
            loss += float(d @ d) / deg[i]
            g[i] += 2.0 * d / deg[i]
            g[j] -= 2.0 * d / deg[i]
    return loss, g


def l_offset(verts, rest):
    d = np.asarray(verts, dtype=np.float64) - np.asarray(rest, dtype=np.float64)
    return float((d * d).sum()), 2.0 * d
