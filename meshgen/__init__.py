"""Seeded synthetic inputs for the vertex-reuse geometry stage.

This module builds index buffers, vertex buffers and shader uniforms only.  It
holds none of the method's arithmetic (no batching, no deduplication, no
shading): both the CPU oracle and the CUDA path read its output, and neither
is imported here.

The paper evaluates on scanned models and game captures that are not
available (Section 4, Table 1).  The generators below stand in for them with
the statistics that matter to vertex reuse (Section 4.1, Table 1): a closed
mesh with V/T = 1/2 (ideal reuse 5/6, like the bunny, sphere, buddha and
dragon rows), triangles in a locality order (the paper reorders every model
with a cache optimiser, Section 4), and vertex ids with no relation to
position.

Vertex layouts (little endian, one row per vertex):

* ``PNU32`` -- 8 float32: position xyz, normal xyz, uv (32 bytes).
* ``SKIN64`` -- 16 words: position xyz, normal xyz, uv, 4 x uint8 bone
  indices packed in word 8, 4 float32 weights in words 9..12, 3 words of
  padding (64 bytes).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

FMT_PNU32 = 0
FMT_SKIN64 = 1

PALETTE_BONES = 64
ENVELOPE_DIRS = 16


@dataclass
class Mesh:
    """An indexed triangle list plus its vertex buffer."""

    vertices: np.ndarray  # float32 [V, 8] (PNU32) or [V, 16] (SKIN64)
    indices: np.ndarray  # uint32 [3T]
    fmt: int = FMT_PNU32
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def num_vertices(self) -> int:
        return int(self.vertices.shape[0])

    @property
    def num_tris(self) -> int:
        return int(self.indices.shape[0] // 3)

    @property
    def stride_bytes(self) -> int:
        return int(self.vertices.shape[1] * 4)

    def positions(self) -> np.ndarray:
        return self.vertices[:, 0:3]

    def normals(self) -> np.ndarray:
        return self.vertices[:, 3:6]


# --------------------------------------------------------------------------
# regular grid (the tiny correctness workload)
# --------------------------------------------------------------------------

def grid_mesh(n: int = 64, amplitude: float = 0.1) -> Mesh:
    """n x n vertex grid over [-1,1]^2 with z = amplitude*sin(pi x) sin(pi y).

    Vertex (i, j) (column i, row j) has id j*n + i.  Quad (i, j) is split into
    (v00, v10, v11) and (v00, v11, v01); quads are visited row by row, which
    is the scanline order of the tiny-grid workload.
    """
    if n < 2:
        raise ValueError("grid needs n >= 2")
    lin = np.linspace(-1.0, 1.0, n)
    x, y = np.meshgrid(lin, lin, indexing="xy")  # x varies along columns i
    z = amplitude * np.sin(np.pi * x) * np.sin(np.pi * y)
    dzdx = amplitude * np.pi * np.cos(np.pi * x) * np.sin(np.pi * y)
    dzdy = amplitude * np.pi * np.sin(np.pi * x) * np.cos(np.pi * y)
    nrm = np.stack([-dzdx, -dzdy, np.ones_like(z)], axis=-1)
    nrm /= np.linalg.norm(nrm, axis=-1, keepdims=True)
    verts = np.zeros((n * n, 8), dtype=np.float64)
    verts[:, 0] = x.ravel()
    verts[:, 1] = y.ravel()
    verts[:, 2] = z.ravel()
    verts[:, 3:6] = nrm.reshape(-1, 3)
    verts[:, 6] = (x.ravel() + 1.0) / 2.0
    verts[:, 7] = (y.ravel() + 1.0) / 2.0
    jj, ii = np.meshgrid(np.arange(n - 1), np.arange(n - 1), indexing="ij")
    v00 = (jj * n + ii).ravel()
    v10 = v00 + 1
    v01 = v00 + n
    v11 = v00 + n + 1
    tris = np.empty((v00.size, 2, 3), dtype=np.int64)
    tris[:, 0] = np.stack([v00, v10, v11], axis=-1)
    tris[:, 1] = np.stack([v00, v11, v01], axis=-1)
    return Mesh(verts.astype(np.float32), tris.reshape(-1).astype(np.uint32),
                FMT_PNU32, f"grid{n}x{n}")


def grid_patch(w: int, h: int, seed: int) -> Mesh:
    """w x h quads (2wh triangles) on a gently curved sheet, scanline order."""
    rng = np.random.default_rng(seed)
    xs = np.linspace(-1.0, 1.0, w + 1)
    ys = np.linspace(-1.0, 1.0, h + 1)
    x, y = np.meshgrid(xs, ys, indexing="xy")
    a, b = rng.uniform(0.5, 2.0, size=2)
    z = 0.1 * np.sin(a * np.pi * x) * np.cos(b * np.pi * y)
    dzdx = 0.1 * a * np.pi * np.cos(a * np.pi * x) * np.cos(b * np.pi * y)
    dzdy = -0.1 * b * np.pi * np.sin(a * np.pi * x) * np.sin(b * np.pi * y)
    nrm = np.stack([-dzdx, -dzdy, np.ones_like(z)], axis=-1)
    nrm /= np.linalg.norm(nrm, axis=-1, keepdims=True)
    nv = (w + 1) * (h + 1)
    verts = np.zeros((nv, 8), dtype=np.float64)
    verts[:, 0] = x.ravel()
    verts[:, 1] = y.ravel()
    verts[:, 2] = z.ravel()
    verts[:, 3:6] = nrm.reshape(-1, 3)
    verts[:, 6] = (x.ravel() + 1) / 2
    verts[:, 7] = (y.ravel() + 1) / 2
    jj, ii = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    v00 = (jj * (w + 1) + ii).ravel()
    v10 = v00 + 1
    v01 = v00 + (w + 1)
    v11 = v01 + 1
    tris = np.empty((v00.size, 2, 3), dtype=np.int64)
    tris[:, 0] = np.stack([v00, v10, v11], axis=-1)
    tris[:, 1] = np.stack([v00, v11, v01], axis=-1)
    return Mesh(verts.astype(np.float32), tris.reshape(-1).astype(np.uint32),
                FMT_PNU32, f"grid{w}x{h}")


# --------------------------------------------------------------------------
# class-I geodesic sphere (the scanned-model stand-in)
# --------------------------------------------------------------------------

def _icosahedron():
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    v = []
    for s1 in (-1.0, 1.0):
        for s2 in (-1.0, 1.0):
            v.append((s1, s2 * phi, 0.0))
            v.append((0.0, s1, s2 * phi))
            v.append((s2 * phi, 0.0, s1))
    v = np.array(v, dtype=np.float64)
    n = len(v)
    edges = [(a, b) for a in range(n) for b in range(a + 1, n)
             if abs(np.linalg.norm(v[a] - v[b]) - 2.0) < 1e-9]
    adj = {a: set() for a in range(n)}
    for a, b in edges:
        adj[a].add(b)
        adj[b].add(a)
    faces = []
    for a, b in edges:
        for c in sorted(adj[a] & adj[b]):
            if c > b:
                if np.dot(np.cross(v[b] - v[a], v[c] - v[a]), v[a] + v[b] + v[c]) < 0:
                    faces.append((a, c, b))
                else:
                    faces.append((a, b, c))
    assert len(edges) == 30 and len(faces) == 20
    return v, edges, faces


def _geodesic_topology(f: int):
    """Shared-vertex ids, unit directions and triangles of frequency f.

    Returns (dirs [V,3] float64, tris [20 f^2, 3] int64) with
    V = 10 f^2 + 2: 12 corners, f-1 vertices on each of the 30 edges and
    (f-1)(f-2)/2 inside each of the 20 faces.
    """
    if f < 1:
        raise ValueError("frequency must be >= 1")
    iv, edges, faces = _icosahedron()
    edge_id = {e: k for k, e in enumerate(edges)}
    nint = (f - 1) * (f - 2) // 2
    base_edge = 12
    base_int = 12 + 30 * (f - 1)
    V = 10 * f * f + 2
    dirs = np.zeros((V, 3), dtype=np.float64)
    I, J = np.meshgrid(np.arange(f + 1), np.arange(f + 1), indexing="ij")
    valid = (I + J) <= f
    Iv, Jv = I[valid], J[valid]
    tris_all = []

    def edge_gid(p, q, k):
        # vertex k steps from p toward q on edge (p, q), 0 < k < f
        if p < q:
            e, kk = edge_id[(p, q)], k
        else:
            e, kk = edge_id[(q, p)], f - k
        return base_edge + e * (f - 1) + (kk - 1)

    for F, (A, B, C) in enumerate(faces):
        a = f - Iv - Jv
        gid = np.full(Iv.shape, -1, dtype=np.int64)
        gid[(Iv == 0) & (Jv == 0)] = A
        gid[Iv == f] = B
        gid[Jv == f] = C
        m = (Jv == 0) & (Iv > 0) & (Iv < f)
        gid[m] = edge_gid(A, B, Iv[m])
        m = (Iv == 0) & (Jv > 0) & (Jv < f)
        gid[m] = edge_gid(A, C, Jv[m])
        m = (a == 0) & (Iv > 0) & (Iv < f)
        gid[m] = edge_gid(B, C, Jv[m])
        m = (Iv >= 1) & (Jv >= 1) & (a >= 1)
        ii, jj = Iv[m], Jv[m]
        local = (ii - 1) * (f - 1) - ((ii - 1) * ii) // 2 + (jj - 1)
        gid[m] = base_int + F * nint + local
        assert (gid >= 0).all()
        P = (a[:, None] * iv[A] + Iv[:, None] * iv[B] + Jv[:, None] * iv[C]) / f
        dirs[gid] = P / np.linalg.norm(P, axis=1, keepdims=True)
        G = np.full((f + 1, f + 1), -1, dtype=np.int64)
        G[Iv, Jv] = gid
        ui, uj = np.nonzero(np.add.outer(np.arange(f), np.arange(f)) <= f - 1)
        up = np.stack([G[ui, uj], G[ui + 1, uj], G[ui, uj + 1]], axis=1)
        di, dj = np.nonzero(np.add.outer(np.arange(f), np.arange(f)) <= f - 2)
        dn = np.stack([G[di + 1, dj], G[di + 1, dj + 1], G[di, dj + 1]], axis=1)
        tris_all.append(up)
        tris_all.append(dn)
    tris = np.concatenate(tris_all, axis=0)
    assert tris.shape[0] == 20 * f * f
    return dirs, tris


def _spread21(x: np.ndarray) -> np.ndarray:
    x = x.astype(np.uint64) & np.uint64(0x1FFFFF)
    x = (x | (x << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
    x = (x | (x << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
    x = (x | (x << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
    x = (x | (x << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
    x = (x | (x << np.uint64(2))) & np.uint64(0x1249249249249249)
    return x


def morton_order(points: np.ndarray) -> np.ndarray:
    """Stable argsort of 3D points by their 63-bit Morton code (21 bits/axis)."""
    lo = points.min(axis=0)
    span = np.maximum(points.max(axis=0) - lo, 1e-30)
    q = np.floor((points - lo) / span * (2**21 - 1)).astype(np.int64)
    q = np.clip(q, 0, 2**21 - 1)
    code = _spread21(q[:, 0]) | (_spread21(q[:, 1]) << np.uint64(1)) | (_spread21(q[:, 2]) << np.uint64(2))
    return np.argsort(code, kind="stable")


def vertex_normals(pos: np.ndarray, tris: np.ndarray) -> np.ndarray:
    """Area-weighted vertex normals (float64)."""
    p0, p1, p2 = pos[tris[:, 0]], pos[tris[:, 1]], pos[tris[:, 2]]
    fn = np.cross(p1 - p0, p2 - p0)
    V = pos.shape[0]
    n = np.zeros((V, 3), dtype=np.float64)
    for k in range(3):
        for c in range(3):
            n[:, c] += np.bincount(tris[:, k], weights=fn[:, c], minlength=V)
    ln = np.linalg.norm(n, axis=1, keepdims=True)
    return n / np.maximum(ln, 1e-300)


def geodesic_sphere(f: int, seed: int, noise: float = 0.02, block: int = 256,
                    shuffle_frac: float = 0.05, permute_vertices: bool = True,
                    order: str = "morton") -> Mesh:
    """Noisy class-I geodesic sphere: V = 10 f^2 + 2, T = 20 f^2.

    * radius 1 + noise * u_v, u_v ~ U[-1, 1] per vertex;
    * area-weighted normals in float64, rounded to float32;
    * triangles sorted by the Morton code of their centroid on the noise-free
      sphere, then a fraction ``shuffle_frac`` of the full ``block``-triangle
      blocks permuted among themselves (locality order with local disorder);
    * vertex ids randomly permuted, so an id says nothing about position.
    """
    rng = np.random.default_rng(seed)
    dirs, tris = _geodesic_topology(f)
    V = dirs.shape[0]
    radius = 1.0 + noise * rng.uniform(-1.0, 1.0, size=V)
    pos = dirs * radius[:, None]
    nrm = vertex_normals(pos, tris)
    if order == "morton":
        # the locality order is taken on the noise-free sphere: at high
        # frequency the 2% radial noise is many edge lengths, and ordering the
        # noisy centroids would scatter neighbouring triangles
        cent = (dirs[tris[:, 0]] + dirs[tris[:, 1]] + dirs[tris[:, 2]]) / 3.0
        tris = tris[morton_order(cent)]
        nb = tris.shape[0] // block
        m = int(round(shuffle_frac * nb))
        if m >= 2:
            chosen = np.sort(rng.choice(nb, size=m, replace=False))
            blocks = np.arange(nb)
            blocks[chosen] = rng.permutation(chosen)
            head = tris[: nb * block].reshape(nb, block, 3)[blocks].reshape(-1, 3)
            tris = np.concatenate([head, tris[nb * block:]], axis=0)
    elif order != "none":
        raise ValueError(order)
    verts = np.zeros((V, 8), dtype=np.float64)
    verts[:, 0:3] = pos
    verts[:, 3:6] = nrm
    verts[:, 6] = 0.5 + np.arctan2(dirs[:, 1], dirs[:, 0]) / (2 * np.pi)
    verts[:, 7] = np.arccos(np.clip(dirs[:, 2], -1, 1)) / np.pi
    if permute_vertices:
        perm = rng.permutation(V)
        nverts = np.empty_like(verts)
        nverts[perm] = verts
        verts = nverts
        tris = perm[tris]
    return Mesh(verts.astype(np.float32), tris.reshape(-1).astype(np.uint32), FMT_PNU32,
                f"geosphere_f{f}", {"frequency": f, "seed": seed})


# --------------------------------------------------------------------------
# uniforms
# --------------------------------------------------------------------------

def _look_at(eye, target, up):
    fwd = np.asarray(target, float) - np.asarray(eye, float)
    fwd /= np.linalg.norm(fwd)
    s = np.cross(fwd, up)
    if np.linalg.norm(s) < 1e-6:
        s = np.cross(fwd, (1.0, 0.0, 0.0))
    s /= np.linalg.norm(s)
    u = np.cross(s, fwd)
    R = np.stack([s, u, -fwd])
    view = np.eye(4)
    view[:3, :3] = R
    view[:3, 3] = -R @ np.asarray(eye, float)
    return view


def _perspective(fovy_deg, aspect, near, far):
    t = 1.0 / math.tan(math.radians(fovy_deg) / 2.0)
    P = np.zeros((4, 4))
    P[0, 0] = t / aspect
    P[1, 1] = t
    P[2, 2] = (far + near) / (near - far)
    P[2, 3] = 2 * far * near / (near - far)
    P[3, 2] = -1.0
    return P


def mvp_uniforms(seed: int, distance: float = 3.0):
    """Seeded camera: returns (M [4,4], N [3,3]) as float32, row-major.

    M = P * V (perspective 60 deg, aspect 16:9, near 0.1, far 100) with the
    eye at ``distance`` in a random direction looking at the origin;
    N is the normal matrix (inverse transpose of the view's 3x3 block, which
    for a rigid view is the rotation itself).  Built in float64, rounded once.
    """
    rng = np.random.default_rng(10_000 + seed)
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    view = _look_at(distance * d, (0.0, 0.0, 0.0), (0.0, 0.0, 1.0))
    proj = _perspective(60.0, 16.0 / 9.0, 0.1, 100.0)
    M = proj @ view
    N = np.linalg.inv(view[:3, :3]).T
    return M.astype(np.float32), N.astype(np.float32)


def skin_mesh(mesh: Mesh, seed: int, bones: str = "uniform"):
    """Adds bone indices/weights (64-byte layout) and a 64-bone palette.

    Bones: 4 uint8 ids per vertex.  "uniform": each uniform in [0, 64), so
    neighbouring vertices share no bones (the worst case for palette reads);
    "nearest": 64 bone centres at seeded vertex positions, and each vertex
    takes its 4 nearest centres, nearest first (neighbouring vertices share
    bones, as in an articulated model).  Weights u_i / sum(u), u_i ~ U(0, 1].
    Palette: per bone a 3x4 row-major [R | t] with a small rotation (random
    axis, angle in [-0.2, 0.2] rad) and t in [-0.05, 0.05]^3.
    Returns (Mesh with SKIN64 vertices, palette float32 [64, 3, 4]).
    """
    if bones not in ("uniform", "nearest"):
        raise ValueError(f"unknown bone assignment {bones!r}")
    rng = np.random.default_rng(20_000 + seed)
    V = mesh.num_vertices
    out = np.zeros((V, 16), dtype=np.float32)
    out[:, 0:8] = mesh.vertices[:, 0:8]
    ids = rng.integers(0, PALETTE_BONES, size=(V, 4), dtype=np.uint8)
    if bones == "nearest" and V:
        pos = mesh.vertices[:, 0:3].astype(np.float64)
        centres = pos[np.random.default_rng(30_000 + seed).integers(0, V, size=PALETTE_BONES)]
        ids = np.empty((V, 4), dtype=np.uint8)
        for a in range(0, V, 1 << 16):  # bounded memory: 65,536 vertices x 64 centres at a time
            d = ((pos[a:a + (1 << 16), None, :] - centres[None, :, :]) ** 2).sum(axis=2)
            ids[a:a + (1 << 16)] = np.argsort(d, axis=1, kind="stable")[:, :4]
    out.view(np.uint8).reshape(V, 64)[:, 32:36] = ids
    u = 1.0 - rng.random(size=(V, 4))
    w = (u / u.sum(axis=1, keepdims=True)).astype(np.float32)
    out[:, 9:13] = w
    pal = np.zeros((PALETTE_BONES, 3, 4), dtype=np.float64)
    for b in range(PALETTE_BONES):
        ax = rng.normal(size=3)
        ax /= np.linalg.norm(ax)
        ang = rng.uniform(-0.2, 0.2)
        K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
        R = np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * (K @ K)
        pal[b, :, :3] = R
        pal[b, :, 3] = rng.uniform(-0.05, 0.05, size=3)
    m = Mesh(out, mesh.indices, FMT_SKIN64, mesh.name + "_skin", dict(mesh.meta))
    return m, pal.astype(np.float32)


def skin_attributes(mesh: Mesh):
    """(bones uint8 [V,4], weights float32 [V,4]) of a SKIN64 mesh."""
    V = mesh.num_vertices
    bones = mesh.vertices.view(np.uint8).reshape(V, 64)[:, 32:36].copy()
    return bones, mesh.vertices[:, 9:13].copy()


def envelope_directions(count: int = ENVELOPE_DIRS) -> np.ndarray:
    """``count`` fixed unit directions (Fibonacci sphere), float32 [count, 3]."""
    k = np.arange(count, dtype=np.float64) + 0.5
    z = 1.0 - 2.0 * k / count
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    ang = math.pi * (3.0 - math.sqrt(5.0)) * k
    d = np.stack([r * np.cos(ang), r * np.sin(ang), z], axis=1)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return d.astype(np.float32)


def envelope_offset(mesh: Mesh, frac: float = 0.02) -> np.float32:
    """Offset distance d = frac x bounding-box diagonal (Section 5.2 uses a
    fraction of the model size for the envelope distance)."""
    p = mesh.positions().astype(np.float64)
    return np.float32(frac * np.linalg.norm(p.max(axis=0) - p.min(axis=0)))


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

def frame_sizes(seed: int = 3, count: int = 2000, tmin: int = 100, tmax: int = 50_000) -> np.ndarray:
    """Triangle counts log-uniform in [tmin, tmax] for a frame of draw calls."""
    rng = np.random.default_rng(30_000 + seed)
    return np.rint(np.exp(rng.uniform(math.log(tmin), math.log(tmax), size=count))).astype(np.int64)


def frame_mesh(k: int, tris: int, seed: int = 3) -> Mesh:
    """Mesh k of the frame: even k a grid patch, odd k a small geodesic sphere."""
    if k % 2 == 0:
        w = max(1, int(round(math.sqrt(tris / 2.0))))
        h = max(1, int(round(tris / (2.0 * w))))
        return grid_patch(w, h, seed * 100_003 + k)
    f = max(1, int(round(math.sqrt(tris / 20.0))))
    return geodesic_sphere(f, seed * 100_003 + k, noise=0.02)


def serving_sizes(seed: int, count: int, tmin: int = 50, tmax: int = 200_000) -> np.ndarray:
    rng = np.random.default_rng(50_000 + seed)
    return np.rint(np.exp(rng.uniform(math.log(tmin), math.log(tmax), size=count))).astype(np.int64)


def poisson_arrivals(seed: int, rate_per_s: float, duration_s: float) -> np.ndarray:
    """Arrival times (s) of a Poisson process of the given rate."""
    rng = np.random.default_rng(60_000 + seed)
    n = int(rate_per_s * duration_s * 1.2) + 16
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))
    return t[t < duration_s]


def random_indices(seed: int, num_tris: int, num_vertices: int) -> np.ndarray:
    """Uniform random index buffer (no locality) for edge-case tests."""
    rng = np.random.default_rng(70_000 + seed)
    return rng.integers(0, num_vertices, size=3 * num_tris, dtype=np.uint64).astype(np.uint32)


def random_vertices(seed: int, num_vertices: int) -> np.ndarray:
    """PNU32 vertices with positions in [-1,1]^3 and unit normals."""
    rng = np.random.default_rng(80_000 + seed)
    v = np.zeros((num_vertices, 8), dtype=np.float64)
    v[:, 0:3] = rng.uniform(-1, 1, size=(num_vertices, 3))
    n = rng.normal(size=(num_vertices, 3))
    v[:, 3:6] = n / np.linalg.norm(n, axis=1, keepdims=True)
    v[:, 6:8] = rng.uniform(0, 1, size=(num_vertices, 2))
    return v.astype(np.float32)


# ---------------------------------------------------------------------------
# random-walk inputs (the parallel random walk of Section 5.4)
# ---------------------------------------------------------------------------

def walk_activity(seed: int, width: int = 256, height: int = 256, gaussians: int = 8,
                  scale: int = 4096) -> np.ndarray:
    """Activity field of the random walk: a floor plus several Gaussians
    overlaid on a toroidal width x height grid, quantised to integers
    (uint32 [height, width], values in [scale/20, ~scale * (1/20 + sum of
    amplitudes)]).  Centres, widths (8..40 cells) and amplitudes (0.5..1.5)
    are seeded."""
    rng = np.random.default_rng(90_000 + seed)
    cx = rng.uniform(0, width, size=gaussians)
    cy = rng.uniform(0, height, size=gaussians)
    sig = rng.uniform(8.0, 40.0, size=gaussians)
    amp = rng.uniform(0.5, 1.5, size=gaussians)
    x = np.arange(width, dtype=np.float64)[None, :]
    y = np.arange(height, dtype=np.float64)[:, None]
    a = np.full((height, width), 0.05)
    for g in range(gaussians):
        dx = np.abs(x - cx[g])
        dx = np.minimum(dx, width - dx)
        dy = np.abs(y - cy[g])
        dy = np.minimum(dy, height - dy)
        a += amp[g] * np.exp(-(dx * dx + dy * dy) / (2.0 * sig[g] * sig[g]))
    return np.rint(a * scale).astype(np.uint32)


def walk_agents(seed: int, count: int = 300_000, width: int = 256, height: int = 256) -> np.ndarray:
    """Agents placed uniformly at random; each is the packed key (x << 16) | y."""
    rng = np.random.default_rng(91_000 + seed)
    x = rng.integers(0, width, size=count, dtype=np.uint64)
    y = rng.integers(0, height, size=count, dtype=np.uint64)
    return ((x << np.uint64(16)) | y).astype(np.uint32)
