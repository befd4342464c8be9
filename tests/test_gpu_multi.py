"""GPU tests of the multi-kernel comparator (GP_MULTI): shade every vertex of
the buffer once, then assemble (the paper's non-streaming "multi" setup).

Its output must be bit-identical to the naive kernel's (same shader code),
the vertex behind every corner exact, the attributes within 1e-5 of the
float64 oracle, and the invocation count exactly the number of vertices in
the buffer -- referenced or not.
"""
import numpy as np
import pytest

import meshgen as mg
from oracle import shading as S

from helpers_gp import assert_attrs_close, draw_gpu, uniforms_for

pytestmark = pytest.mark.gpu


def _meshes():
    sk, pal = mg.skin_mesh(mg.geodesic_sphere(9, 31), 5)
    return {"grid": mg.grid_mesh(40), "sphere": mg.geodesic_sphere(35, 5), "skin": (sk, pal)}


MESHES = _meshes()


@pytest.mark.parametrize("shader", [S.SHADER_MVP, S.SHADER_SKIN, S.SHADER_ENVELOPE, S.SHADER_LOAD])
def test_multi_matches_naive_and_oracle(shader):
    if shader == S.SHADER_SKIN:
        mesh, pal = MESHES["skin"]
    else:
        mesh, pal = MESHES["sphere"], None
    uni, uni_o = uniforms_for(mesh, shader, palette=pal)
    r = draw_gpu(mesh, "multi", shader, "static", uni)
    assert r.status == 0
    assert np.array_equal(r.ids, mesh.indices)
    assert_attrs_close(r.out, S.draw(mesh, shader, uni_o), shader, mesh)
    base = draw_gpu(mesh, "naive", shader, "static", uni, debug=False)
    assert np.array_equal(r.out.view(np.uint32), base.out.view(np.uint32))
    assert r.stats["invocations"] == mesh.num_vertices
    assert r.inv.tolist() == [mesh.num_vertices]
    assert r.stats["triangles"] == mesh.num_tris


def test_multi_shades_unreferenced_vertices():
    # a vertex buffer with 1000 extra rows no index refers to
    mesh = MESHES["grid"]
    extra = mg.random_vertices(77, 1000)
    big = mg.Mesh(np.concatenate([mesh.vertices, extra]), mesh.indices, mesh.fmt, "grid+extra", {})
    uni, uni_o = uniforms_for(big, S.SHADER_MVP)
    r = draw_gpu(big, "multi", S.SHADER_MVP, "static", uni)
    assert r.status == 0
    assert r.stats["invocations"] == big.num_vertices
    assert_attrs_close(r.out, S.draw(big, S.SHADER_MVP, uni_o), S.SHADER_MVP, big)


def test_multi_index_range_and_empty():
    import paper_1805_08893_gb300 as gp
    mesh = MESHES["grid"]
    bad = mesh.indices.copy()
    bad[5] = mesh.num_vertices + 3
    bad[100] = 0xFFFFFFFF
    m2 = mg.Mesh(mesh.vertices, bad, mesh.fmt, "grid-bad", {})
    uni, uni_o = uniforms_for(m2, S.SHADER_MVP)
    r = draw_gpu(m2, "multi", S.SHADER_MVP, "static", uni)
    assert r.status == gp.GP_ERR_INDEX_RANGE
    assert np.all(r.out[1, 2] == 0) and np.all(r.out[33, 1] == 0)
    ok = np.ones(m2.num_tris, dtype=bool)
    ok[[1, 33]] = False
    ref = S.draw(mesh, S.SHADER_MVP, uni_o)
    assert_attrs_close(r.out[ok], ref[ok], S.SHADER_MVP, mesh)
    empty = mg.Mesh(mesh.vertices, np.zeros(0, np.uint32), mesh.fmt, "empty", {})
    r = draw_gpu(empty, "multi", S.SHADER_MVP, "static", uni)
    assert r.status == 0 and r.stats["triangles"] == 0


def test_multi_buffer_grows_between_draws():
    import torch
    import paper_1805_08893_gb300 as gp
    small, large = MESHES["grid"], MESHES["sphere"]
    ctx = gp.gp_create("multi", stream=torch.cuda.current_stream())
    try:
        for mesh in (small, large, small):
            uni, uni_o = uniforms_for(mesh, S.SHADER_MVP)
            idx = torch.from_numpy(mesh.indices.view(np.int32).copy()).cuda()
            verts = torch.from_numpy(mesh.vertices).cuda()
            out = torch.full((mesh.num_tris * 21,), float("nan"), device="cuda")
            t = gp.gp_submit_drawcall(ctx, idx, verts, S.SHADER_MVP, uni, out)
            assert gp.gp_sync(ctx, t) == gp.GP_OK
            torch.cuda.synchronize()
            assert_attrs_close(out.cpu().numpy().reshape(-1, 3, 7), S.draw(mesh, S.SHADER_MVP, uni_o),
                               S.SHADER_MVP, mesh)
    finally:
        gp.gp_destroy(ctx)
