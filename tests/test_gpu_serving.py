"""GPU tests of the serving loop (continuous batching across requests).

A request's result must be the same whether it runs alone or inside a mix of
requests arriving while others are on the GPU: batches never span requests
and every batch runs the same code, so the outputs are bit-identical.  Each
result also matches the oracle (connectivity bit-exact through the shaded
positions, attributes within 1e-5).
"""
import numpy as np
import pytest

import meshgen as mg
from oracle import shading as S

from helpers_gp import assert_attrs_close, uniforms_for

pytestmark = pytest.mark.gpu


def _pool(seed=0):
    meshes = [mg.grid_mesh(10), mg.geodesic_sphere(4, 21), mg.geodesic_sphere(11, 22), mg.grid_patch(40, 25, 23),
              mg.geodesic_sphere(23, 24)]
    sk, pal = mg.skin_mesh(mg.geodesic_sphere(7, 25), 6)
    return meshes, sk, pal


def _solo(torch, gp, ctx, mesh, sid, uni, **cfg):
    srv = gp.gp_server_create(ctx, **cfg)
    try:
        mid = gp.gp_server_add_mesh(srv, mesh.indices, mesh.vertices)
        out = torch.full((mesh.num_tris * 3 * gp.gp_out_floats(sid),), float("nan"), device="cuda")
        r = gp.gp_server_submit(srv, mid, sid, uni, out)
        assert gp.gp_server_wait(srv, r) == gp.GP_OK
        torch.cuda.synchronize()
        return out.cpu().numpy()
    finally:
        gp.gp_server_destroy(srv)


@pytest.mark.parametrize("variant,mode", [("hash", 1), ("phash", 1), ("sort", 0), ("warp", 0), ("naive", 0)])
def test_mix_invariance(variant, mode):
    import torch
    import paper_1805_08893_gb300 as gp
    meshes, sk, pal = _pool()
    ctx = gp.gp_create("hash")
    cfg = dict(variant=variant, mode=mode, step_max_batches=64, streams=3)
    try:
        srv = gp.gp_server_create(ctx, **cfg)
        try:
            mids = [gp.gp_server_add_mesh(srv, m.indices, m.vertices) for m in meshes]
            skid = gp.gp_server_add_mesh(srv, sk.indices, sk.vertices)
            rng = np.random.default_rng(7)
            n = 120
            arrivals = np.sort(rng.uniform(0.0, 0.03, size=n))
            which = rng.integers(0, len(meshes) + 1, size=n)
            reqs = []
            for i in range(n):
                if which[i] == len(meshes):
                    mesh, mid, sid = sk, skid, S.SHADER_SKIN
                    uni, uni_o = uniforms_for(sk, sid, seed=i % 5, palette=pal)
                else:
                    mesh, mid = meshes[which[i]], mids[which[i]]
                    sid = S.SHADER_MVP if i % 3 else S.SHADER_LOAD
                    uni, uni_o = uniforms_for(mesh, sid, seed=i % 5)
                out = torch.full((mesh.num_tris * 3 * gp.gp_out_floats(sid),), float("nan"), device="cuda")
                reqs.append((mesh, mid, sid, uni, uni_o, out))
            ids = gp.gp_server_replay(srv, arrivals, [r[1] for r in reqs], [r[2] for r in reqs], [r[3] for r in reqs],
                                      [r[5] for r in reqs])
            assert gp.gp_server_wait(srv) == gp.GP_OK
            torch.cuda.synchronize()
            st = gp.gp_server_stats(srv)
            assert st["completed"] == n and st["submitted"] == n
            assert st["p99_ms"] >= st["p50_ms"] > 0 and st["steps"] >= 1
            assert st["triangles"] == sum(r[0].num_tris for r in reqs)
            # device time: the union of the step intervals is at most their sum and the wall time
            # (up to the rounding of float event timestamps, ~0.5 us each)
            assert 0 < st["device_ms"] <= st["busy_ms"] * 1.001 + 1e-3 * st["steps"]
            assert st["device_ms"] <= st["wall_ms"] * 1.001 + 1e-3 * st["steps"]
            for i in (0, 1, 2, 5, n // 2, n - 1):
                mesh, mid, sid, uni, uni_o, out = reqs[i]
                got = out.cpu().numpy()
                solo = _solo(torch, gp, ctx, mesh, sid, uni, **cfg)
                assert np.array_equal(got.view(np.uint32), solo.view(np.uint32)), i
                K = gp.gp_out_floats(sid)
                assert_attrs_close(got.reshape(-1, 3, K), S.draw(mesh, sid, uni_o), sid, mesh)
                assert gp.gp_server_latency(srv, ids[i]) > 0
        finally:
            gp.gp_server_destroy(srv)
    finally:
        gp.gp_destroy(ctx)


def test_eviction_under_a_small_budget():
    import torch
    import paper_1805_08893_gb300 as gp
    meshes, _, _ = _pool()
    ctx = gp.gp_create("hash")
    try:
        biggest = max(m.indices.nbytes + m.vertices.nbytes for m in meshes)
        srv = gp.gp_server_create(ctx, mem_budget_bytes=int(biggest * 1.15), variant="hash", mode=1)
        try:
            mids = [gp.gp_server_add_mesh(srv, m.indices, m.vertices) for m in meshes]
            outs = []
            for rep in range(3):
                for mesh, mid in zip(meshes, mids):
                    uni, uni_o = uniforms_for(mesh, S.SHADER_MVP, seed=rep)
                    out = torch.zeros(mesh.num_tris * 21, device="cuda")
                    gp.gp_server_submit(srv, mid, S.SHADER_MVP, uni, out)
                    outs.append((mesh, uni_o, out))
            assert gp.gp_server_wait(srv) == gp.GP_OK
            torch.cuda.synchronize()
            st = gp.gp_server_stats(srv)
            assert st["evictions"] > 0 and st["uploads"] > len(meshes)
            assert st["resident_bytes"] <= int(biggest * 1.15)
            for mesh, uni_o, out in outs:
                assert_attrs_close(out.cpu().numpy().reshape(-1, 3, 7), S.draw(mesh, S.SHADER_MVP, uni_o),
                                   S.SHADER_MVP, mesh)
        finally:
            gp.gp_server_destroy(srv)
    finally:
        gp.gp_destroy(ctx)


def test_mesh_over_budget_is_refused():
    import torch
    import paper_1805_08893_gb300 as gp
    mesh = mg.geodesic_sphere(10, 3)
    ctx = gp.gp_create("hash")
    try:
        srv = gp.gp_server_create(ctx, mem_budget_bytes=1024)
        try:
            mid = gp.gp_server_add_mesh(srv, mesh.indices, mesh.vertices)
            uni, _ = uniforms_for(mesh, S.SHADER_MVP)
            out = torch.zeros(mesh.num_tris * 21, device="cuda")
            with pytest.raises(gp.GpError) as e:
                gp.gp_server_submit(srv, mid, S.SHADER_MVP, uni, out)
            assert e.value.status == gp.GP_ERR_BUSY
        finally:
            gp.gp_server_destroy(srv)
    finally:
        gp.gp_destroy(ctx)
