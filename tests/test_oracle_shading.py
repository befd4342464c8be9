"""Pins for the oracle's float64 shaders and plain-definition draw (CPU only)."""
import json
import math
import os

import numpy as np
import pytest

import meshgen as mg
from oracle import shading as S

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_mvp_hand_worked():
    g = json.load(open(os.path.join(GOLD, "mvp_worked.json")))
    out = S.mvp(np.array([g["p"]], float), np.array([g["n"]], float), g["M"], g["N"])[0]
    assert out[:4].tolist() == g["clip"]
    assert out[4:].tolist() == g["normal"]


def test_mvp_identity_and_translation():
    rng = np.random.default_rng(0)
    p = rng.uniform(-1, 1, size=(20, 3))
    n = rng.normal(size=(20, 3))
    out = S.mvp(p, n, np.eye(4), np.eye(3))
    assert np.array_equal(out[:, :3], p) and np.all(out[:, 3] == 1.0) and np.array_equal(out[:, 4:], n)
    M = np.eye(4)
    M[:3, 3] = (0.5, -2.0, 3.0)
    out = S.mvp(p, n, M, np.eye(3))
    assert np.allclose(out[:, :3], p + M[:3, 3], atol=0, rtol=0)


def test_mvp_is_linear_in_homogeneous_position():
    rng = np.random.default_rng(1)
    M = rng.normal(size=(4, 4))
    a, b = rng.normal(size=(1, 3)), rng.normal(size=(1, 3))
    z = np.zeros((1, 3))
    fa = S.mvp(a, z, M, np.eye(3))[:, :4] - M[:, 3]
    fb = S.mvp(b, z, M, np.eye(3))[:, :4] - M[:, 3]
    fab = S.mvp(a + b, z, M, np.eye(3))[:, :4] - M[:, 3]
    assert np.allclose(fab, fa + fb, rtol=1e-14, atol=1e-14)


def test_skin_special_cases():
    rng = np.random.default_rng(2)
    n = 16
    p = rng.uniform(-1, 1, size=(n, 3))
    nr = rng.normal(size=(n, 3))
    M = rng.normal(size=(4, 4))
    N = rng.normal(size=(3, 3))
    ident = np.zeros((64, 3, 4))
    ident[:, :, :3] = np.eye(3)
    bones = rng.integers(0, 64, size=(n, 4))
    w = rng.uniform(0.1, 1, size=(n, 4))
    w /= w.sum(axis=1, keepdims=True)
    # identity palette: skinning is a no-op
    assert np.allclose(S.skin(p, nr, bones, w, ident, M, N), S.mvp(p, nr, M, N), rtol=1e-13, atol=1e-13)
    # one bone with weight 1 applies exactly that bone: rotation about z by 90
    # degrees plus a translation (not symmetric, so a transposed bone fails)
    pal = ident.copy()
    pal[5, :, :3] = [[0, -1, 0], [1, 0, 0], [0, 0, 1]]
    pal[5, :, 3] = [1.0, 2.0, 3.0]
    one = np.zeros((1, 4)); one[0, 0] = 1.0
    out = S.skin(np.array([[1.0, 0.0, 0.0]]), np.array([[1.0, 0.0, 0.0]]),
                 np.array([[5, 0, 0, 0]]), one, pal, np.eye(4), np.eye(3))[0]
    assert out.tolist() == [1.0, 3.0, 3.0, 1.0, 0.0, 1.0, 0.0]
    # two opposite translations with equal weight cancel
    pal2 = ident.copy()
    pal2[1, :, 3] = [0.3, 0.0, 0.0]
    pal2[2, :, 3] = [-0.3, 0.0, 0.0]
    half = np.array([[0.5, 0.5, 0.0, 0.0]])
    out = S.skin(np.array([[0.2, 0.4, 0.6]]), np.array([[0.0, 0.0, 1.0]]),
                 np.array([[1, 2, 0, 0]]), half, pal2, np.eye(4), np.eye(3))[0]
    assert np.allclose(out[:3], [0.2, 0.4, 0.6], atol=1e-15)


def test_exp_taylor_matches_library_exp():
    s = np.linspace(-1.0, 1.0, 101)
    assert np.max(np.abs(S.exp_taylor_horner(s) - np.exp(s))) < 1e-15
    # truncation is visible far out (drops the s^32 term and beyond)
    assert S.exp_taylor_horner(np.array([40.0]))[0] < math.exp(40.0)


def test_envelope_special_cases():
    rng = np.random.default_rng(3)
    dirs = mg.envelope_directions()
    p = rng.uniform(-1, 1, size=(10, 3))
    n = rng.normal(size=(10, 3))
    out = S.envelope(p, n, 0.0, dirs)
    assert np.array_equal(out[:, 0:3], p) and np.array_equal(out[:, 4:7], p)
    assert np.all(out[:, 3] == 1) and np.all(out[:, 7] == 1)
    # at the origin every direction gives s = 0 and h = 1: offset is exactly d*n
    o = S.envelope(np.zeros((1, 3)), np.array([[0.0, 0.0, 1.0]]), 0.25, dirs)[0]
    assert o.tolist() == [0.0, 0.0, -0.25, 1.0, 0.0, 0.0, 0.25, 1.0]
    # inner and outer are symmetric about p and the offset equals d * mean exp(s_j)
    d = 0.1
    out = S.envelope(p, n, d, dirs)
    assert np.allclose(out[:, 0:3] + out[:, 4:7], 2 * p, atol=1e-14)
    h = np.exp(0.5 * p @ dirs.astype(np.float64).T).mean(axis=1)
    assert np.allclose(out[:, 4:7] - p, d * h[:, None] * n, rtol=1e-13, atol=1e-15)


def test_load_closed_form():
    rng = np.random.default_rng(4)
    p = rng.uniform(-1, 1, size=(8, 3))
    n = rng.normal(size=(8, 3))
    for steps in (0, 1, 7, 64):
        out = S.load(p, n, np.eye(4), np.eye(3), steps)
        c = 0.5 + 1e-3 * p[:, 0]
        sig = 2 * c + (1 - 2 * c) * 0.5 ** steps  # fixed point 2c of s -> s/2 + c
        assert np.allclose(out[:, 4:7], n * sig[:, None], rtol=1e-14, atol=1e-15)
        assert np.array_equal(out[:, :4], S.mvp(p, n, np.eye(4), np.eye(3))[:, :4])


def test_draw_is_per_corner_shading_in_triangle_order():
    # 2 triangles over 4 vertices; identity shader makes each corner's output
    # the position of the vertex its index names
    verts = np.zeros((4, 8), np.float32)
    verts[:, 0] = [10, 11, 12, 13]
    m = mg.Mesh(verts, np.array([0, 1, 2, 2, 3, 0], np.uint32))
    out = S.draw(m, S.SHADER_MVP, {"M": np.eye(4), "N": np.eye(3)})
    assert out.shape == (2, 3, 7)
    assert out[:, :, 0].tolist() == [[10, 11, 12], [12, 13, 10]]
    sub = S.draw(m, S.SHADER_MVP, {"M": np.eye(4), "N": np.eye(3)}, tris=[1])
    assert sub[0, :, 0].tolist() == [12, 13, 10]


def test_shade_vertices_reads_skin_layout():
    g = mg.grid_mesh(4)
    sm, pal = mg.skin_mesh(g, 1)
    bones, w = mg.skin_attributes(sm)
    M, N = mg.mvp_uniforms(1)
    ids = np.arange(sm.num_vertices)
    got = S.shade_vertices(sm, ids, S.SHADER_SKIN, {"M": M, "N": N, "palette": pal})
    want = S.skin(g.vertices[:, 0:3], g.vertices[:, 3:6], bones, w, pal, M, N)
    assert np.array_equal(got, want)
    assert np.allclose(w.sum(axis=1), 1.0, atol=1e-6)
