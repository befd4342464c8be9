"""Oracle of one Loop subdivision step (Section 5.2).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper applies its reuse methods to Loop subdivision (Loop, "Smooth
Subdivision Surfaces Based on Triangles", 1987): every input triangle adds a
vertex on each edge and moves its three vertices, both by convex
combinations of neighbouring vertices, and is replaced by four triangles.
Written out from the subdivision rules, in float64:

* vertex rule (interior, valence n): (1 - n beta) v + beta * sum of the ring,
  beta = (5/8 - (3/8 + cos(2 pi / n) / 4)^2) / n;
* vertex rule on a boundary (a vertex on an edge used by one triangle, with
  exactly two such boundary neighbours): 3/4 v + 1/8 (b0 + b1);
* edge rule: 3/8 (a + b) + 1/8 (c + d) with c, d the vertices opposite the
  edge in its two triangles; on a boundary edge: (a + b) / 2.

Readings: triangle t = (v0, v1, v2) yields (E0, M0, M2), (E1, M1, M0),
(E2, M2, M1), (M0, M1, M2), with E the moved vertices and M_k the new vertex
of edge (v_k, v_k+1), so the output keeps the input's orientation.  A vertex
with more than two boundary neighbours (non-manifold) takes the interior rule
over all its neighbours.
"""
import math

import numpy as np


def adjacency(index_buffer, num_vertices: int):
    """Rings (lists), boundary flags and, per triangle edge, the opposite vertex (or -1)."""
    tris = np.asarray(index_buffer, np.int64).reshape(-1, 3)
    third = {}
    for t in range(len(tris)):
        for k in range(3):
            third[(int(tris[t, k]), int(tris[t, (k + 1) % 3]))] = int(tris[t, (k + 2) % 3])
    nbrs = [set() for _ in range(num_vertices)]
    bnb = [[] for _ in range(num_vertices)]
    opposite = np.full(3 * len(tris), -1, np.int64)
    for t in range(len(tris)):
        for k in range(3):
            a, b = int(tris[t, k]), int(tris[t, (k + 1) % 3])
            nbrs[a].add(b)
            nbrs[b].add(a)
            twin = third.get((b, a))
            if twin is None:
                bnb[a].append(b)
                bnb[b].append(a)
            else:
                opposite[3 * t + k] = twin
    boundary = np.array([len(b) == 2 for b in bnb])
    rings = [sorted(bnb[v]) if boundary[v] else sorted(nbrs[v]) for v in range(num_vertices)]
    return rings, boundary, opposite


def loop_beta(n: int) -> float:
    """Loop's vertex weight for valence n."""
    c = 3.0 / 8.0 + 0.25 * math.cos(2.0 * math.pi / n)
    return (5.0 / 8.0 - c * c) / n


def subdivide(positions, index_buffer):
    """One step: float64 [T, 4, 3, 3] (output triangle, corner, xyz)."""
    P = np.asarray(positions, np.float64)
    tris = np.asarray(index_buffer, np.int64).reshape(-1, 3)
    rings, boundary, opposite = adjacency(index_buffer, len(P))
    E = np.empty_like(P)
    for v in range(len(P)):
        r = rings[v]
        if boundary[v]:
            E[v] = 0.75 * P[v] + 0.125 * (P[r[0]] + P[r[1]])
        elif len(r) == 0:
            E[v] = P[v]
        else:
            b = loop_beta(len(r))
            E[v] = (1.0 - len(r) * b) * P[v] + b * P[r].sum(axis=0)
    out = np.empty((len(tris), 4, 3, 3))
    for t in range(len(tris)):
        v = tris[t]
        M = []
        for k in range(3):
            a, bb, c, d = v[k], v[(k + 1) % 3], v[(k + 2) % 3], opposite[3 * t + k]
            M.append(0.5 * (P[a] + P[bb]) if d < 0 else 0.375 * (P[a] + P[bb]) + 0.125 * (P[c] + P[d]))
        out[t] = [[E[v[0]], M[0], M[2]], [E[v[1]], M[1], M[0]], [E[v[2]], M[2], M[1]], [M[0], M[1], M[2]]]
    return out
