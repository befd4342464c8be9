"""Float64 reference shaders and the plain-definition draw.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper fixes the shader only loosely: "a simple matrix multiplication"
and synthetic loads of 256/512/1024 cycles (Section 4.2), plus the skinning
and envelope applications (Section 5).  The concrete shaders below are the
readings used by this project; each is written out from its mathematical
definition, in float64, from the float32 inputs.

Outputs per corner:

* MVP / SKIN / LOAD: 7 values -- clip position (x, y, z, w), normal (x, y, z).
* ENVELOPE: 8 values -- inner offset position (x, y, z, 1), outer (x, y, z, 1).
"""
from __future__ import annotations

import math

import numpy as np

SHADER_MVP = 0
SHADER_SKIN = 1
SHADER_ENVELOPE = 2
SHADER_LOAD = 3

OUT_FLOATS = {SHADER_MVP: 7, SHADER_SKIN: 7, SHADER_ENVELOPE: 8, SHADER_LOAD: 7}

ENVELOPE_TERMS = 32  # degree-31 polynomial, evaluated with 32 Horner steps


def mvp(pos, nrm, M, N):
    """Simple shader (Section 4.2): clip = M (p, 1), n' = N n.

    ``M`` is the 4x4 model-view-projection matrix and ``N`` the 3x3 normal
    matrix, both row-major; the normal is not renormalised.
    """
    pos = np.asarray(pos, np.float64)
    nrm = np.asarray(nrm, np.float64)
    M = np.asarray(M, np.float64)
    N = np.asarray(N, np.float64)
    clip = pos @ M[:, :3].T + M[:, 3]
    n = nrm @ N.T
    return np.concatenate([clip, n], axis=1)


def skin(pos, nrm, bones, weights, palette, M, N):
    """Linear-blend skinning, then the simple shader (Section 5 application).

    p_s = sum_i w_i * B[b_i] (p, 1) and n_s = sum_i w_i * R[b_i] n, where each
    palette entry B = [R | t] is a 3x4 row-major bone matrix.
    """
    pos = np.asarray(pos, np.float64)
    nrm = np.asarray(nrm, np.float64)
    w = np.asarray(weights, np.float64)
    P = np.asarray(palette, np.float64)
    b = np.asarray(bones, np.int64)
    ps = np.zeros_like(pos)
    ns = np.zeros_like(nrm)
    for i in range(4):
        B = P[b[:, i]]  # [n, 3, 4]
        ps += w[:, i:i + 1] * (np.einsum("nij,nj->ni", B[:, :, :3], pos) + B[:, :, 3])
        ns += w[:, i:i + 1] * np.einsum("nij,nj->ni", B[:, :, :3], nrm)
    return mvp(ps, ns, M, N)


def exp_taylor_horner(s, terms: int = ENVELOPE_TERMS):
    """sum_{k<terms} s^k / k!  by Horner's rule (the envelope displacement)."""
    s = np.asarray(s, np.float64)
    h = np.full_like(s, 1.0 / math.factorial(terms - 1))
    for k in range(terms - 2, -1, -1):
        h = h * s + 1.0 / math.factorial(k)
    return h


def envelope(pos, nrm, d, dirs):
    """Envelope-style offset (Section 5.2 application).

    For each fixed unit direction a_j: s_j = 0.5 * dot(p, a_j) and
    h_j = sum_{k<32} s_j^k / k!; h is the mean of the h_j.  The shader writes
    the inner and outer offset surfaces p -/+ d*h*n (w = 1).
    """
    pos = np.asarray(pos, np.float64)
    nrm = np.asarray(nrm, np.float64)
    A = np.asarray(dirs, np.float64)
    s = 0.5 * (pos @ A.T)  # [n, W]
    h = exp_taylor_horner(s).mean(axis=1)
    off = float(d) * h[:, None] * nrm
    one = np.ones((pos.shape[0], 1))
    return np.concatenate([pos - off, one, pos + off, one], axis=1)


def load(pos, nrm, M, N, steps: int):
    """Synthetic load (Section 4.2: the simple shader plus a load of 256, 512 or 1024 cycles).

    The simple shader, with the normal scaled by sigma_L of the contractive
    recurrence sigma_0 = 1, sigma_{k+1} = sigma_k / 2 + c, c = 1/2 + p_x/1000
    -- a chain of ``steps`` dependent multiply-adds.
    """
    out = mvp(pos, nrm, M, N)
    pos = np.asarray(pos, np.float64)
    c = 0.5 + 1e-3 * pos[:, 0]
    sig = np.ones_like(c)
    for _ in range(int(steps)):
        sig = 0.5 * sig + c
    out[:, 4:7] *= sig[:, None]
    return out


def shade_vertices(mesh, ids, shader_id: int, uniforms: dict):
    """shade(vertexBuffer[id]) for every id in ``ids`` (float64 [n, K])."""
    ids = np.asarray(ids, np.int64)
    V = mesh.vertices
    pos = V[ids, 0:3]
    nrm = V[ids, 3:6]
    if shader_id == SHADER_MVP:
        return mvp(pos, nrm, uniforms["M"], uniforms["N"])
    if shader_id == SHADER_SKIN:
        nv = V.shape[0]
        raw = V.view(np.uint8).reshape(nv, V.shape[1] * 4)
        bones = raw[ids, 32:36]
        weights = V[ids, 9:13]
        return skin(pos, nrm, bones, weights, uniforms["palette"], uniforms["M"], uniforms["N"])
    if shader_id == SHADER_ENVELOPE:
        return envelope(pos, nrm, uniforms["d"], uniforms["dirs"])
    if shader_id == SHADER_LOAD:
        return load(pos, nrm, uniforms["M"], uniforms["N"], uniforms["steps"])
    raise ValueError(f"unknown shader {shader_id}")


def draw(mesh, shader_id: int, uniforms: dict, tris=None):
    """The geometry stage's result by its plain definition (Section 3).

    out[t, k] = shade(vertexBuffer[indexBuffer[3t + k]]) for each requested
    triangle t (all by default), in input triangle order.  Returns float64
    [len(tris), 3, K].  Every corner is shaded on its own: this is the result
    that any amount of reuse must reproduce.
    """
    idx = np.asarray(mesh.indices, np.int64)
    if tris is None:
        corner_ids = idx
        nt = idx.size // 3
    else:
        tris = np.asarray(tris, np.int64)
        corner_ids = idx.reshape(-1, 3)[tris].reshape(-1)
        nt = tris.size
    out = shade_vertices(mesh, corner_ids, shader_id, uniforms)
    return out.reshape(nt, 3, out.shape[1])
