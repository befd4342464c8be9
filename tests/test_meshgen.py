"""Checks of the seeded input generators (CPU only)."""
import numpy as np
import pytest

import meshgen as mg


@pytest.mark.parametrize("f", [1, 2, 5, 12])
def test_geodesic_counts_and_closed_manifold(f):
    s = mg.geodesic_sphere(f, 7)
    V, T = s.num_vertices, s.num_tris
    assert V == 10 * f * f + 2 and T == 20 * f * f
    tris = s.indices.reshape(-1, 3).astype(np.int64)
    assert np.unique(s.indices).size == V  # every vertex referenced
    # each directed edge appears once and its reverse once: closed, oriented
    e = np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]])
    key = e[:, 0] * V + e[:, 1]
    rev = e[:, 1] * V + e[:, 0]
    assert np.unique(key).size == key.size
    assert np.array_equal(np.sort(key), np.sort(rev))
    E = key.size // 2
    assert V - E + T == 2  # Euler characteristic of a sphere
    p = s.vertices[:, 0:3].astype(np.float64)
    n = s.vertices[:, 3:6].astype(np.float64)
    assert np.all(np.sum(p * n, axis=1) > 0)  # outward normals
    r = np.linalg.norm(p, axis=1)
    assert r.min() >= 0.98 - 1e-6 and r.max() <= 1.02 + 1e-6
    fn = np.cross(p[tris[:, 1]] - p[tris[:, 0]], p[tris[:, 2]] - p[tris[:, 0]])
    assert np.all(np.sum(fn * p[tris].mean(axis=1), axis=1) > 0)  # CCW outward


def test_geodesic_deterministic_and_seeded():
    a = mg.geodesic_sphere(6, 3)
    b = mg.geodesic_sphere(6, 3)
    c = mg.geodesic_sphere(6, 4)
    assert np.array_equal(a.indices, b.indices) and np.array_equal(a.vertices, b.vertices)
    assert not np.array_equal(a.indices, c.indices)


def test_grid_layout():
    g = mg.grid_mesh(64)
    assert g.num_vertices == 4096 and g.num_tris == 7938
    assert g.indices[:6].tolist() == [0, 1, 65, 0, 65, 64]
    assert g.stride_bytes == 32 and g.vertices.dtype == np.float32
    z = g.vertices[:, 2]
    x, y = g.vertices[:, 0].astype(np.float64), g.vertices[:, 1].astype(np.float64)
    assert np.allclose(z, 0.1 * np.sin(np.pi * x) * np.sin(np.pi * y), atol=1e-7)


def test_skin_layout():
    g = mg.grid_mesh(8)
    s, pal = mg.skin_mesh(g, 2)
    assert s.stride_bytes == 64 and pal.shape == (64, 3, 4)
    bones, w = mg.skin_attributes(s)
    assert bones.max() < 64 and np.all(w > 0)
    R = pal[:, :, :3].astype(np.float64)
    assert np.allclose(np.einsum("bij,bkj->bik", R, R), np.eye(3), atol=1e-6)


def test_skin_nearest_bones():
    # "nearest": each vertex's 4 bones are the 4 closest of 64 centres placed
    # at seeded vertex positions, nearest first; weights and palette are those
    # of the uniform assignment
    g = mg.geodesic_sphere(12, 3)
    u, pal_u = mg.skin_mesh(g, 5)
    s, pal = mg.skin_mesh(g, 5, bones="nearest")
    assert np.array_equal(pal, pal_u)
    assert np.array_equal(s.vertices[:, 9:13], u.vertices[:, 9:13])
    bones, _ = mg.skin_attributes(s)
    assert bones.max() < 64
    assert all(len(set(b)) == 4 for b in bones.tolist())
    pos = g.vertices[:, 0:3].astype(np.float64)
    centres = pos[np.random.default_rng(30_000 + 5).integers(0, g.num_vertices, size=64)]
    d = ((pos[:, None, :] - centres[None, :, :]) ** 2).sum(axis=2)
    picked = np.take_along_axis(d, bones.astype(np.int64), axis=1)
    assert np.all(np.diff(picked, axis=1) >= 0)  # nearest first
    fourth = np.sort(d, axis=1)[:, 3]
    assert np.all(picked[:, 3] <= fourth)  # no closer centre left out
    # neighbouring vertices mostly share their nearest bone
    a, b = g.indices.reshape(-1, 3)[:, 0], g.indices.reshape(-1, 3)[:, 1]
    assert np.mean(bones[a, 0] == bones[b, 0]) > 0.5
    with pytest.raises(ValueError):
        mg.skin_mesh(g, 5, bones="random")


def test_frame_sizes_range():
    sz = mg.frame_sizes()
    assert sz.size == 2000 and sz.min() >= 100 and sz.max() <= 50_000
    assert 6_000 < sz.mean() < 10_000
    m = mg.frame_mesh(1, 500)
    assert abs(m.num_tris - 500) / 500 < 0.3
    m = mg.frame_mesh(0, 500)
    assert abs(m.num_tris - 500) / 500 < 0.3


def test_mvp_uniforms_shape():
    M, N = mg.mvp_uniforms(1)
    assert M.shape == (4, 4) and N.shape == (3, 3) and M.dtype == np.float32
    assert np.allclose(N.astype(np.float64) @ N.T.astype(np.float64), np.eye(3), atol=1e-6)
