"""Pins of the Loop subdivision oracle (Section 5.2): Loop's weights in closed
form, planes reproduced exactly (affine invariance of convex combinations on
a regular planar lattice), translation invariance, the tetrahedron worked by
hand, straight boundaries staying straight, and adjacency by brute force."""
import math

import numpy as np
import pytest

import meshgen as mg
from oracle import loop as L


def test_loop_beta_closed_forms():
    assert L.loop_beta(6) == pytest.approx(1.0 / 16.0, abs=1e-15)
    assert L.loop_beta(3) == pytest.approx(3.0 / 16.0, abs=1e-15)
    # n beta -> 5/8 - (5/8)^2 = 15/64 for large valence
    assert L.loop_beta(100000) * 100000 == pytest.approx(15.0 / 64.0, rel=1e-6)


def _flat_lattice(n):
    # regular triangulated lattice in the plane z = 0.3 x - 0.2 y + 1 (every interior vertex has valence 6)
    xs, ys = np.meshgrid(np.arange(n, dtype=np.float64), np.arange(n, dtype=np.float64))
    P = np.stack([xs.ravel(), ys.ravel(), 0.3 * xs.ravel() - 0.2 * ys.ravel() + 1.0], axis=1)
    tris = []
    for j in range(n - 1):
        for i in range(n - 1):
            a, b, c, d = j * n + i, j * n + i + 1, (j + 1) * n + i, (j + 1) * n + i + 1
            tris += [a, b, d, a, d, c]
    return P, np.array(tris, np.uint32)


def test_plane_and_lattice_are_reproduced():
    P, idx = _flat_lattice(8)
    out = L.subdivide(P, idx)
    # every new point stays on the plane
    pts = out.reshape(-1, 3)
    assert np.allclose(pts[:, 2], 0.3 * pts[:, 0] - 0.2 * pts[:, 1] + 1.0, atol=1e-12)
    # interior vertices of a regular lattice do not move; interior edge points are edge midpoints
    tris = idx.reshape(-1, 3)
    rings, boundary, opp = L.adjacency(idx, len(P))
    for t in range(len(tris)):
        for k in range(3):
            v = tris[t, k]
            if not boundary[v] and len(rings[v]) == 6:
                assert np.allclose(out[t, k, 0], P[v], atol=1e-12)
            if opp[3 * t + k] >= 0:
                a, b = tris[t, k], tris[t, (k + 1) % 3]
                assert np.allclose(out[t, 3, k], 0.5 * (P[a] + P[b]), atol=1e-12)


def test_translation_invariance():
    m = mg.geodesic_sphere(3, 1)
    P = m.vertices[:, :3].astype(np.float64)
    shift = np.array([0.25, -1.5, 3.0])
    a = L.subdivide(P, m.indices)
    b = L.subdivide(P + shift, m.indices)
    assert np.allclose(b, a + shift, atol=1e-12)


def test_tetrahedron_by_hand():
    P = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], np.float64)
    idx = np.array([0, 1, 2, 0, 3, 1, 0, 2, 3, 1, 3, 2], np.uint32)
    out = L.subdivide(P, idx)
    # valence 3: v' = (1 - 9/16) v + 3/16 (sum of the other three) = 7/16 v - 3/16 v = v / 4 here (sum of all = 0)
    for t, tri in enumerate(idx.reshape(-1, 3)):
        for k in range(3):
            assert np.allclose(out[t, k, 0], P[tri[k]] / 4.0, atol=1e-15)
    # edge (0, 1): 3/8 (P0 + P1) + 1/8 (P2 + P3)
    assert np.allclose(out[0, 3, 0], 0.375 * (P[0] + P[1]) + 0.125 * (P[2] + P[3]), atol=1e-15)


def test_straight_boundary_stays_straight():
    P, idx = _flat_lattice(6)
    out = L.subdivide(P, idx)
    rings, boundary, opp = L.adjacency(idx, len(P))
    tris = idx.reshape(-1, 3)
    for t in range(len(tris)):
        for k in range(3):
            v = tris[t, k]
            if boundary[v] and P[v][1] == 0 and 0 < P[v][0] < 5:  # interior points of the bottom edge
                assert np.allclose(out[t, k, 0], P[v], atol=1e-12)  # 3/4 v + 1/8 (v - e + v + e) = v


def test_adjacency_brute_force():
    m = mg.grid_patch(7, 5, 3)
    rings, boundary, opp = L.adjacency(m.indices, m.num_vertices)
    tris = m.indices.reshape(-1, 3).tolist()
    for t, tri in enumerate(tris):
        for k in range(3):
            a, b = tri[k], tri[(k + 1) % 3]
            others = [x for s, x2 in enumerate(tris) if s != t and a in x2 and b in x2 for x in x2 if x not in (a, b)]
            assert opp[3 * t + k] == (others[0] if others else -1)


# --- the native adjacency builder (host code of the library; no GPU) against the oracle

@pytest.mark.parametrize("which", ["sphere", "patch"])
def test_native_adjacency_matches_oracle(which):
    import paper_1805_08893_gb300 as gp
    m = mg.geodesic_sphere(6, 2) if which == "sphere" else mg.grid_patch(9, 6, 4)
    off, ring, opp, flags = gp.gp_loop_adjacency(m.indices, m.num_vertices)
    rings, boundary, opposite = L.adjacency(m.indices, m.num_vertices)
    assert np.array_equal(flags.astype(bool), boundary)
    for v in range(m.num_vertices):
        assert sorted(ring[off[v]:off[v + 1]].tolist()) == rings[v]
    assert np.array_equal(opp.astype(np.int64), np.where(opposite < 0, 0xFFFFFFFF, opposite))


def test_native_adjacency_rejects_bad_indices():
    import paper_1805_08893_gb300 as gp
    with pytest.raises(gp.GpError) as e:
        gp.gp_loop_adjacency(np.array([0, 1, 5], np.uint32), 3)
    assert e.value.status == gp.GP_ERR_INDEX_RANGE
