"""GPU parity: every variant, batching mode and shader against the CPU oracle.

Bit-exact: the vertex behind every output corner (connectivity), per-batch
shading-invocation counts, dynamic batch starts, and naive vs reuse outputs.
Within 1e-5 relative (scale floor per attribute): shaded FP32 values vs the
float64 oracle.
"""
import numpy as np
import pytest

import meshgen as mg
from oracle import batching as B
from oracle import shading as S

from helpers_gp import assert_attrs_close, draw_gpu, uniforms_for

pytestmark = pytest.mark.gpu

STATIC_VARIANTS = ["naive", "warp", "sort", "hash", "phash"]
DYNAMIC_VARIANTS = ["sort", "hash", "phash"]


@pytest.fixture(scope="module")
def grid():
    return mg.grid_mesh(64)


@pytest.fixture(scope="module")
def sphere():
    # 6 segments of 4096 triangles plus a ragged tail, T not a multiple of 4
    return mg.geodesic_sphere(35, 5)


def _check(mesh, r, variant, shader_id, uni_o, starts=None):
    assert r.status == 0, r.status
    ref = S.draw(mesh, shader_id, uni_o)
    assert np.array_equal(r.ids, mesh.indices), "connectivity (corner -> vertex) differs"
    assert_attrs_close(r.out, ref, shader_id, mesh)
    st = r.starts if starts is None else starts
    want = B.batch_invocations(mesh.indices, list(st), variant)
    assert np.array_equal(r.inv, want), "per-batch invocation counts differ"
    assert r.stats["invocations"] == int(want.sum())
    assert r.stats["triangles"] == mesh.num_tris


@pytest.mark.parametrize("variant", STATIC_VARIANTS)
def test_tiny_grid_static_mvp(grid, variant):
    uni, uni_o = uniforms_for(grid, S.SHADER_MVP)
    cfg = {"batch_indices": 255} if variant not in ("naive", "warp") else {}
    r = draw_gpu(grid, variant, S.SHADER_MVP, "static", uni, **cfg)
    _check(grid, r, variant, S.SHADER_MVP, uni_o)


@pytest.mark.parametrize("variant", DYNAMIC_VARIANTS)
def test_tiny_grid_dynamic_mvp(grid, variant):
    uni, uni_o = uniforms_for(grid, S.SHADER_MVP)
    r = draw_gpu(grid, variant, S.SHADER_MVP, "dynamic", uni)
    want = B.dynamic_partition(grid.indices, 256, 341, 4096)
    assert r.starts.tolist() == want
    _check(grid, r, variant, S.SHADER_MVP, uni_o)


@pytest.mark.parametrize("variant", DYNAMIC_VARIANTS)
@pytest.mark.parametrize("seg", [4096, 1000, 0xFFFFFFFF])
def test_sphere_dynamic_partition_and_draw(sphere, variant, seg):
    uni, uni_o = uniforms_for(sphere, S.SHADER_MVP)
    r = draw_gpu(sphere, variant, S.SHADER_MVP, "dynamic", uni, segment_tris=seg)
    want = B.dynamic_partition(sphere.indices, 256, 341, 0 if seg == 0xFFFFFFFF else seg)
    assert r.starts.tolist() == want
    _check(sphere, r, variant, S.SHADER_MVP, uni_o)


@pytest.mark.parametrize("variant", STATIC_VARIANTS)
@pytest.mark.parametrize("shader", ["skin", "envelope", "load"])
def test_shaders_static(sphere, variant, shader):
    sid = {"skin": S.SHADER_SKIN, "envelope": S.SHADER_ENVELOPE, "load": S.SHADER_LOAD}[shader]
    mesh = sphere
    pal = None
    if sid == S.SHADER_SKIN:
        mesh, pal = mg.skin_mesh(sphere, 3)
    uni, uni_o = uniforms_for(mesh, sid, palette=pal)
    r = draw_gpu(mesh, variant, sid, "static", uni)
    _check(mesh, r, variant, sid, uni_o)


@pytest.mark.parametrize("shader", ["mvp", "skin", "envelope", "load"])
def test_naive_and_reuse_bit_identical(sphere, shader):
    sid = {"mvp": S.SHADER_MVP, "skin": S.SHADER_SKIN, "envelope": S.SHADER_ENVELOPE, "load": S.SHADER_LOAD}[shader]
    mesh, pal = (mg.skin_mesh(sphere, 3) if sid == S.SHADER_SKIN else (sphere, None))
    uni, _ = uniforms_for(mesh, sid, palette=pal)
    base = draw_gpu(mesh, "naive", sid, "static", uni, debug=False).out
    for variant, mode in [("warp", "static"), ("sort", "static"), ("hash", "dynamic"), ("phash", "dynamic"),
                          ("sort", "dynamic")]:
        out = draw_gpu(mesh, variant, sid, mode, uni, debug=False).out
        assert np.array_equal(out.view(np.uint32), base.view(np.uint32)), (variant, mode)


@pytest.mark.parametrize("variant", ["warp", "sort", "hash", "phash"])
@pytest.mark.parametrize("S_", [3, 6, 96, 99, 192, 384])
def test_static_batch_sizes(sphere, variant, S_):
    if variant != "warp" and S_ > 384:
        pytest.skip()
    uni, uni_o = uniforms_for(sphere, S.SHADER_MVP)
    r = draw_gpu(sphere, variant, S.SHADER_MVP, "static", uni, batch_indices=S_)
    _check(sphere, r, variant, S.SHADER_MVP, uni_o)


@pytest.mark.parametrize("variant", ["sort", "hash", "phash"])
@pytest.mark.parametrize("threads", [32, 128, 512])
def test_threads_per_group(sphere, variant, threads):
    uni, uni_o = uniforms_for(sphere, S.SHADER_MVP)
    r = draw_gpu(sphere, variant, S.SHADER_MVP, "dynamic", uni, threads_per_group=threads)
    _check(sphere, r, variant, S.SHADER_MVP, uni_o)


@pytest.mark.parametrize("variant", ["hash", "phash"])
@pytest.mark.parametrize("slots", [256, 1024])
def test_full_hash_tables(sphere, variant, slots):
    # slots = max_unique (the paper's table size) forces long probe chains
    uni, uni_o = uniforms_for(sphere, S.SHADER_MVP)
    r = draw_gpu(sphere, variant, S.SHADER_MVP, "dynamic", uni, hash_slots=slots, threads_per_group=256)
    _check(sphere, r, variant, S.SHADER_MVP, uni_o)


@pytest.mark.parametrize("variant", ["sort", "hash", "phash"])
@pytest.mark.parametrize("nu,mt", [(3, 1), (16, 5), (64, 100), (512, 682)])
def test_dynamic_limits(sphere, variant, nu, mt):
    uni, uni_o = uniforms_for(sphere, S.SHADER_MVP)
    r = draw_gpu(sphere, variant, S.SHADER_MVP, "dynamic", uni, max_unique=nu, max_tris=mt)
    assert r.starts.tolist() == B.dynamic_partition(sphere.indices, nu, mt, 4096)
    _check(sphere, r, variant, S.SHADER_MVP, uni_o)


# --------------------------------------------------------------------------
# edge cases
# --------------------------------------------------------------------------

def _mesh(indices, nv=None, seed=0):
    indices = np.asarray(indices, dtype=np.uint32)
    nv = int(indices.max()) + 1 if nv is None and indices.size else (nv or 1)
    return mg.Mesh(mg.random_vertices(seed, nv), indices)


EDGE = {
    "one_triangle": [0, 1, 2],
    "degenerate": [5, 5, 5, 1, 1, 2, 0, 3, 0],
    "all_equal": [7] * (3 * 200),
    "all_distinct": list(range(3 * 150)),
    "ragged_tail": list(range(3 * 7)) * 3,  # T = 21: the index buffer ends off a 16-byte boundary
}


@pytest.mark.parametrize("case", sorted(EDGE))
@pytest.mark.parametrize("variant,mode", [("naive", "static"), ("warp", "static"), ("sort", "static"),
                                          ("hash", "static"), ("phash", "static"), ("sort", "dynamic"),
                                          ("hash", "dynamic"), ("phash", "dynamic")])
def test_edge_cases(case, variant, mode):
    mesh = _mesh(EDGE[case], seed=len(EDGE[case]))
    uni, uni_o = uniforms_for(mesh, S.SHADER_MVP)
    r = draw_gpu(mesh, variant, S.SHADER_MVP, mode, uni)
    if mode == "dynamic":
        assert r.starts.tolist() == B.dynamic_partition(mesh.indices, 256, 341, 4096)
    _check(mesh, r, variant, S.SHADER_MVP, uni_o)


@pytest.mark.parametrize("variant,mode", [("naive", "static"), ("warp", "static"), ("hash", "static"),
                                          ("sort", "dynamic"), ("phash", "dynamic")])
def test_empty_draw(variant, mode):
    mesh = mg.Mesh(mg.random_vertices(0, 4), np.zeros(0, np.uint32))
    uni, _ = uniforms_for(mesh, S.SHADER_MVP)
    r = draw_gpu(mesh, variant, S.SHADER_MVP, mode, uni)
    assert r.status == 0 and r.out.shape == (0, 3, 7) and r.stats["invocations"] == 0


@pytest.mark.parametrize("variant,mode", [("naive", "static"), ("warp", "static"), ("sort", "static"),
                                          ("hash", "dynamic"), ("phash", "dynamic")])
def test_index_out_of_range(variant, mode):
    import paper_1805_08893_gb300 as gp
    idx = [0, 1, 2, 2, 1, 9, 3, 0xFFFFFFFF, 1]  # 9 and 0xFFFFFFFF are out of range for 5 vertices
    mesh = _mesh(idx, nv=5)
    uni, uni_o = uniforms_for(mesh, S.SHADER_MVP)
    r = draw_gpu(mesh, variant, S.SHADER_MVP, mode, uni)
    assert r.status == gp.GP_ERR_INDEX_RANGE
    good = mesh.indices < 5
    ref = S.shade_vertices(mesh, np.where(good, mesh.indices, 0), S.SHADER_MVP, uni_o).reshape(-1, 3, 7)
    flat = r.out.reshape(-1, 7)
    assert np.all(flat[~good] == 0.0)
    assert_attrs_close(flat[good], ref.reshape(-1, 7)[good], S.SHADER_MVP, mesh)


def test_invalid_arguments_rejected():
    import torch
    import paper_1805_08893_gb300 as gp
    mesh = mg.grid_mesh(4)
    uni, _ = uniforms_for(mesh, S.SHADER_MVP)
    idx = torch.from_numpy(mesh.indices.view(np.int32)).cuda()
    verts = torch.from_numpy(mesh.vertices).cuda()
    out = torch.zeros(mesh.num_tris * 21, device="cuda")
    with pytest.raises(gp.GpError) as e:
        gp.gp_create("hash", batch_indices=256)  # not a multiple of 3
    assert e.value.status == gp.GP_ERR_INVALID
    with pytest.raises(gp.GpError):
        gp.gp_create("warp", mode=gp.GP_BATCH_DYNAMIC)
    ctx = gp.gp_create("hash")
    try:
        with pytest.raises(gp.GpError) as e:  # output too small
            gp.gp_submit_drawcall(ctx, idx, verts, gp.GP_SHADER_MVP, uni, out[:-1])
        assert e.value.status == gp.GP_ERR_INVALID
        with pytest.raises(gp.GpError) as e:  # index count not a multiple of 3
            gp.gp_submit_drawcall(ctx, idx[:-4], verts, gp.GP_SHADER_MVP, uni, out)
        assert e.value.status == gp.GP_ERR_INVALID
        with pytest.raises(gp.GpError) as e:  # skinning needs the 64-byte layout
            sk, pal = mg.skin_mesh(mesh, 1)
            gp.gp_submit_drawcall(ctx, idx, verts, gp.GP_SHADER_SKIN, gp.uniforms_skin(np.eye(4), np.eye(3), pal), out)
        assert e.value.status == gp.GP_ERR_INVALID
        with pytest.raises(gp.GpError) as e:  # unaligned index pointer
            gp.gp_submit_drawcall(ctx, idx[1:4], verts, gp.GP_SHADER_MVP, uni, out)
        assert e.value.status == gp.GP_ERR_INVALID
        assert gp.gp_sync(ctx) == gp.GP_OK
    finally:
        gp.gp_destroy(ctx)


def test_host_buffer_draw_matches_device_draw(sphere):
    import torch
    import paper_1805_08893_gb300 as gp
    uni, uni_o = uniforms_for(sphere, S.SHADER_MVP)
    for variant, mode in [("hash", gp.GP_BATCH_DYNAMIC), ("warp", gp.GP_BATCH_STATIC)]:
        ctx = gp.gp_create(variant, mode=mode)
        try:
            out = torch.empty(sphere.num_tris * 21, dtype=torch.float32).pin_memory()
            idx = torch.from_numpy(sphere.indices.view(np.int32)).pin_memory()
            verts = torch.from_numpy(sphere.vertices).pin_memory()
            gp.gp_draw_host(ctx, idx, verts, gp.GP_SHADER_MVP, uni, out)
            got = out.numpy().reshape(-1, 3, 7)
        finally:
            gp.gp_destroy(ctx)
        dev = draw_gpu(sphere, variant, S.SHADER_MVP, "dynamic" if mode else "static", uni, debug=False).out
        assert np.array_equal(got.view(np.uint32), dev.view(np.uint32))


@pytest.mark.parametrize("variant,mode,extra", [("hash", 1, {}), ("sort", 0, {"batch_indices": 255}),
                                                ("naive", 0, {}), ("warp", 0, {}), ("multi", 0, {})])
def test_host_buffer_draw_in_chunks(variant, mode, extra):
    # more than 2^20 triangles: the host draw runs in chunks of whole batches,
    # whose output must equal one device draw bit for bit, and the oracle on
    # sampled triangles
    import torch
    import paper_1805_08893_gb300 as gp
    mesh = mg.geodesic_sphere(245, 8)  # 1,200,500 triangles
    uni, uni_o = uniforms_for(mesh, S.SHADER_MVP)
    ctx = gp.gp_create(variant, mode=mode, **extra)
    try:
        out = torch.full((mesh.num_tris * 21,), float("nan"), dtype=torch.float32).pin_memory()
        idx = torch.from_numpy(mesh.indices.view(np.int32)).pin_memory()
        verts = torch.from_numpy(mesh.vertices).pin_memory()
        gp.gp_draw_host(ctx, idx, verts, gp.GP_SHADER_MVP, uni, out)
        got = out.numpy().reshape(-1, 3, 7)
        st = gp.gp_stats(ctx)
        assert st["triangles"] == mesh.num_tris
        if variant != "multi":
            assert st["draws"] >= 2  # chunked
    finally:
        gp.gp_destroy(ctx)
    ref = draw_gpu(mesh, variant, S.SHADER_MVP, "dynamic" if mode else "static", uni, debug=False, **extra)
    assert np.array_equal(got.view(np.uint32), ref.out.view(np.uint32))
    # the chunks' batches are those of the whole draw (chunks hold whole segments or static batches), so the
    # shading invocations match too; dynamic chunks are partitioned on their own stream as their indices arrive
    if variant != "multi":
        assert st["invocations"] == ref.stats["invocations"]
    rng = np.random.default_rng(1)
    tris = np.sort(rng.choice(mesh.num_tris, size=2000, replace=False))
    assert_attrs_close(got[tris], S.draw(mesh, S.SHADER_MVP, uni_o, tris=tris), S.SHADER_MVP, mesh)
