"""GPU parity of one Loop subdivision step (Section 5.2) through the C ABI:
every output corner within 1e-5 of the float64 oracle (positions of order 1),
reuse outputs bit-identical to the naive kernel's (the same rule code), and
the vertex-rule evaluation counts equal to the oracle's per-batch unique
counts."""
import numpy as np
import pytest

import meshgen as mg
from oracle import batching as B
from oracle import loop as L

pytestmark = pytest.mark.gpu

MESHES = {"sphere": mg.geodesic_sphere(20, 3), "patch": mg.grid_patch(40, 31, 2)}  # closed, and with a boundary


def _subdivide(mesh, variant, **kw):
    import torch
    import paper_1805_08893_gb300 as gp
    adj = [torch.from_numpy(x.view(np.int32).copy()).cuda() for x in gp.gp_loop_adjacency(mesh.indices, mesh.num_vertices)]
    idx = torch.from_numpy(mesh.indices.view(np.int32).copy()).cuda()
    verts = torch.from_numpy(mesh.vertices).cuda()
    out = torch.full((mesh.num_tris * 36,), float("nan"), device="cuda")
    cnt = torch.zeros(3, dtype=torch.int64, device="cuda")
    gp.gp_loop_subdivide(idx, verts, adj, out, cnt, variant, **kw)
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(-1, 4, 3, 3), cnt.cpu().numpy()


@pytest.mark.parametrize("which", ["sphere", "patch"])
@pytest.mark.parametrize("variant,S", [("naive", 0), ("warp", 96), ("warp", 384), ("sort", 768), ("hash", 192),
                                       ("phash", 255), ("hash", 4095)])
def test_static_batches_match_oracle(which, variant, S):
    mesh = MESHES[which]
    threads = 64 if S == 192 or variant == "warp" else 256
    got, cnt = _subdivide(mesh, variant, batch_indices=S, threads=threads)
    ref = L.subdivide(mesh.vertices[:, :3], mesh.indices)
    assert np.allclose(got, ref, rtol=1e-5, atol=1e-5)
    base, _ = _subdivide(mesh, "naive")
    assert np.array_equal(got.view(np.uint32), base.view(np.uint32))
    if variant == "naive":
        assert int(cnt[0]) == 3 * mesh.num_tris
    elif variant == "warp":
        assert int(cnt[0]) == int(B.batch_invocations(mesh.indices, B.static_starts(mesh.num_tris, S), "warp").sum())
    else:
        assert int(cnt[0]) == int(B.batch_invocations(mesh.indices, B.static_starts(mesh.num_tris, S), "hash").sum())
    assert int(cnt[2]) == 0


@pytest.mark.parametrize("variant", ["sort", "hash", "phash"])
def test_dynamic_batches_match_oracle(variant):
    import torch
    import paper_1805_08893_gb300 as gp
    mesh = MESHES["sphere"]
    # the paper's subdivision setting: batches of up to 192 indices and 64 unique vertices
    ctx = gp.gp_create("hash", mode=gp.GP_BATCH_DYNAMIC, max_unique=64, max_tris=64)
    try:
        idx = torch.from_numpy(mesh.indices.view(np.int32).copy()).cuda()
        h, nb = gp.gp_partition(ctx, idx)
        starts = torch.zeros(nb + 1, dtype=torch.int32, device="cuda")
        gp.gp_partition_starts(ctx, h, starts)
        count = torch.tensor([nb], dtype=torch.int32, device="cuda")
        got, cnt = _subdivide(mesh, variant, starts=starts, num_batches=count, max_batches=nb,
                              max_batch_indices=192, max_unique=64, threads=64)
    finally:
        gp.gp_destroy(ctx)
    ref = L.subdivide(mesh.vertices[:, :3], mesh.indices)
    assert np.allclose(got, ref, rtol=1e-5, atol=1e-5)
    want = B.batch_invocations(mesh.indices, B.dynamic_partition(mesh.indices, 64, 64, 4096), "hash")
    assert int(cnt[0]) == int(want.sum())


def test_bad_arguments():
    import torch
    import paper_1805_08893_gb300 as gp
    with pytest.raises(gp.GpError):
        _subdivide(MESHES["sphere"], "warp", batch_indices=387)  # above the warp batch limit
    with pytest.raises(gp.GpError):
        _subdivide(MESHES["sphere"], "hash", batch_indices=100)
