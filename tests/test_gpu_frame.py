"""GPU tests of frames: many draws in one persistent, graph-captured launch.

Every draw of a frame must give the same result as on its own: the vertex
behind every corner and the per-batch invocation counts bit-exact against the
oracle, attributes within 1e-5 of the float64 oracle, and the output
bit-identical to the single-draw naive kernel (same shader code).
"""
import numpy as np
import pytest

import meshgen as mg
from oracle import batching as B
from oracle import shading as S

from helpers_gp import assert_attrs_close, draw_gpu, uniforms_for

pytestmark = pytest.mark.gpu


def _meshes():
    g = mg.grid_mesh(24)
    s1 = mg.geodesic_sphere(9, 11)
    s2 = mg.geodesic_sphere(17, 12)
    sk, pal = mg.skin_mesh(mg.geodesic_sphere(6, 13), 4)
    return g, s1, s2, sk, pal


# (mesh key, shader, variant, mode, batch_indices, max_unique, threads_per_group)
FRAME = [
    ("g", "mvp", "naive", 0, 0, 0, 0),
    ("s1", "mvp", "warp", 0, 96, 0, 0),
    ("s2", "mvp", "warp", 0, 192, 0, 0),
    ("g", "mvp", "hash", 0, 255, 0, 256),
    ("s1", "mvp", "hash", 1, 0, 256, 256),
    ("s2", "mvp", "phash", 1, 0, 128, 128),
    ("s2", "mvp", "sort", 1, 0, 64, 64),
    ("s1", "mvp", "sort", 0, 126, 0, 64),
    ("g", "mvp", "phash", 0, 252, 0, 128),
    ("sk", "skin", "hash", 1, 0, 256, 256),
    ("sk", "skin", "warp", 0, 96, 0, 0),
    ("s1", "envelope", "phash", 0, 255, 0, 128),
    ("s2", "load", "sort", 1, 0, 256, 256),
    ("g", "load", "naive", 0, 0, 0, 0),
    # whole-block groups (the pipelined path) for every method, mode and shader
    ("s2", "mvp", "phash", 1, 0, 256, 256),
    ("s2", "mvp", "sort", 0, 510, 0, 256),
    ("s1", "envelope", "sort", 0, 255, 0, 256),
    ("g", "envelope", "phash", 1, 0, 128, 256),
    ("sk", "skin", "phash", 0, 255, 0, 256),
    ("sk", "skin", "sort", 1, 0, 64, 256),
    ("s1", "load", "hash", 0, 96, 0, 256),
]


def _expected_starts(mesh, variant, mode, S_, nu):
    T = mesh.num_tris
    if variant == "naive":
        return list(range(0, T, 256)) + [T]
    if variant == "warp" or mode == 0:
        return B.static_starts(T, S_ or (96 if variant == "warp" else 255))
    return B.dynamic_partition(mesh.indices, nu, (4 * nu - 1) // 3, 4096)


def _build(torch, gp, entries, meshes, variant_override=None):
    g, s1, s2, sk, pal = meshes
    lut = {"g": g, "s1": s1, "s2": s2, "sk": sk}
    descs, bufs = [], []
    for key, shader, variant, mode, S_, nu, G in entries:
        mesh = lut[key]
        sid = {"mvp": S.SHADER_MVP, "skin": S.SHADER_SKIN, "envelope": S.SHADER_ENVELOPE, "load": S.SHADER_LOAD}[shader]
        uni, uni_o = uniforms_for(mesh, sid, palette=pal if sid == S.SHADER_SKIN else None)
        T = mesh.num_tris
        K = gp.gp_out_floats(sid)
        idx = torch.from_numpy(mesh.indices.view(np.int32).copy()).cuda()
        verts = torch.from_numpy(mesh.vertices).cuda()
        out = torch.full((T * 3 * K,), float("nan"), device="cuda")
        ids = torch.full((3 * T,), -1, dtype=torch.int32, device="cuda")
        binv = torch.full((T + 1,), -1, dtype=torch.int32, device="cuda")
        v = variant_override or variant
        descs.append(gp.draw_desc(idx, verts, sid, uni, out, ids, binv, variant=v, mode=mode, batch_indices=S_,
                                  max_unique=nu, threads_per_group=G))
        bufs.append((mesh, sid, uni, uni_o, idx, verts, out, ids, binv, variant, mode, S_, nu))
    return descs, bufs


def test_mixed_frame_matches_oracle_and_single_draws():
    import torch
    import paper_1805_08893_gb300 as gp
    meshes = _meshes()
    ctx = gp.gp_create("hash", stream=torch.cuda.current_stream())
    try:
        descs, bufs = _build(torch, gp, FRAME, meshes)
        frame = gp.gp_frame_create(ctx, descs)
        try:
            for rep in range(2):  # the second launch replays the captured graph
                for _, _, _, _, _, _, out, ids, binv, *_ in bufs:
                    out.fill_(float("nan"))
                    ids.fill_(-1)
                    binv.fill_(-1)
                t = gp.gp_frame_submit(frame, ctx)
                assert gp.gp_sync(ctx, t) == gp.GP_OK
                torch.cuda.synchronize()
                total_inv = 0
                for i, (mesh, sid, uni, uni_o, idx, verts, out, ids, binv, variant, mode, S_, nu) in enumerate(bufs):
                    cfg = gp.gp_frame_draw_config(frame, i)
                    st = _expected_starts(mesh, variant, mode, S_, nu)
                    assert cfg["batches"] == len(st) - 1, (i, cfg)
                    K = gp.gp_out_floats(sid)
                    got = out.cpu().numpy().reshape(mesh.num_tris, 3, K)
                    assert np.array_equal(ids.cpu().numpy().view(np.uint32), mesh.indices), i
                    assert_attrs_close(got, S.draw(mesh, sid, uni_o), sid, mesh)
                    want = B.batch_invocations(mesh.indices, st, variant)
                    assert np.array_equal(binv.cpu().numpy()[: len(st) - 1], want), (i, variant)
                    total_inv += int(want.sum())
                    if rep == 0:
                        base = draw_gpu(mesh, "naive", sid, "static", uni, debug=False).out
                        assert np.array_equal(got.view(np.uint32), base.view(np.uint32)), i
                st_all = gp.gp_stats(ctx, reset=True)
                assert st_all["invocations"] == total_inv
                assert st_all["draws"] == len(FRAME)
                assert st_all["triangles"] == sum(b[0].num_tris for b in bufs)
        finally:
            gp.gp_frame_destroy(frame)
    finally:
        gp.gp_destroy(ctx)


def test_frame_uniform_update():
    import torch
    import paper_1805_08893_gb300 as gp
    meshes = _meshes()
    ctx = gp.gp_create("hash", stream=torch.cuda.current_stream())
    try:
        descs, bufs = _build(torch, gp, FRAME[:5], meshes)
        frame = gp.gp_frame_create(ctx, descs)
        try:
            mesh = bufs[3][0]
            M, N = mg.mvp_uniforms(77)
            gp.gp_frame_set_uniforms(frame, 3, gp.uniforms_mvp(M, N), ctx)
            t = gp.gp_frame_submit(frame, ctx)
            gp.gp_sync(ctx, t)
            torch.cuda.synchronize()
            got = bufs[3][6].cpu().numpy().reshape(mesh.num_tris, 3, 7)
            assert_attrs_close(got, S.draw(mesh, S.SHADER_MVP, {"M": M, "N": N}), S.SHADER_MVP, mesh)
        finally:
            gp.gp_frame_destroy(frame)
    finally:
        gp.gp_destroy(ctx)


def test_autotune_then_auto_frame():
    import torch
    import paper_1805_08893_gb300 as gp
    meshes = _meshes()
    ctx = gp.gp_create("hash", stream=torch.cuda.current_stream())
    try:
        entries = [(k, sh, "hash", 0, 0, 0, 0) for (k, sh, *_rest) in FRAME]
        descs, bufs = _build(torch, gp, entries, meshes)
        gp.gp_autotune(ctx, descs, reps=2)
        table = gp.gp_autotune_table(ctx)
        assert table, "autotune produced no rows"
        for row in table:
            assert row["tris_lo"] < row["tris_hi"] and row["us_per_draw"] > 0
        # GP_AUTO draws take their configuration from the table
        descs, bufs = _build(torch, gp, entries, meshes, variant_override=gp.GP_AUTO)
        frame = gp.gp_frame_create(ctx, descs)
        try:
            t = gp.gp_frame_submit(frame, ctx)
            assert gp.gp_sync(ctx, t) == gp.GP_OK
            torch.cuda.synchronize()
            for i, (mesh, sid, uni, uni_o, idx, verts, out, ids, binv, *_r) in enumerate(bufs):
                cfg = gp.gp_frame_draw_config(frame, i)
                rows = [r for r in table if r["shader_id"] == sid and r["tris_lo"] <= mesh.num_tris < r["tris_hi"]]
                if rows:
                    want = dict(rows[0]["config"])
                    assert {k: cfg[k] for k in want if k != "batches"} == {k: want[k] for k in want if k != "batches"}
                K = gp.gp_out_floats(sid)
                got = out.cpu().numpy().reshape(mesh.num_tris, 3, K)
                assert np.array_equal(ids.cpu().numpy().view(np.uint32), mesh.indices)
                assert_attrs_close(got, S.draw(mesh, sid, uni_o), sid, mesh)
        finally:
            gp.gp_frame_destroy(frame)
        # a saved table can be restored
        gp.gp_autotune_set_table(ctx, table)
        assert gp.gp_autotune_table(ctx) == table
    finally:
        gp.gp_destroy(ctx)


def test_frame_rejects_bad_draws():
    import torch
    import paper_1805_08893_gb300 as gp
    meshes = _meshes()
    ctx = gp.gp_create("hash")
    try:
        descs, _ = _build(torch, gp, [("s1", "mvp", "hash", 0, 256, 0, 256)], meshes)  # 256: not a multiple of 3
        with pytest.raises(gp.GpError) as e:
            gp.gp_frame_create(ctx, descs)
        assert e.value.status == gp.GP_ERR_INVALID and "frame draw 0" in gp.gp_last_error(ctx)
        descs, _ = _build(torch, gp, [("s1", "mvp", "hash", 0, 4095, 0, 64)], meshes)  # too big for 64 threads
        with pytest.raises(gp.GpError) as e:
            gp.gp_frame_create(ctx, descs)
        assert e.value.status == gp.GP_ERR_UNSUPPORTED
    finally:
        gp.gp_destroy(ctx)


def test_bench_frame_2000_skinned_draws_autotuned():
    """The frame bench.py times: 2,000 skinned draws (triangle counts
    log-uniform in [100, 50,000], grids and sphere patches, a 64-bone palette
    each), autotuned, in one graph-replayed launch.  The vertex behind every
    corner of every draw is exact; for a sample of draws the per-batch
    invocation counts (from each draw's chosen configuration) are exact and
    sampled attributes are within 1e-5 of the float64 oracle."""
    import torch
    import paper_1805_08893_gb300 as gp
    sizes = mg.frame_sizes()
    ctx = gp.gp_create("hash", stream=torch.cuda.current_stream())
    try:
        meshes, descs, bufs = [], [], []
        for k, n in enumerate(sizes):
            m, pal = mg.skin_mesh(mg.frame_mesh(k, int(n)), k)
            M, N = mg.mvp_uniforms(1000 + k)
            uni = gp.uniforms_skin(M, N, pal)
            T = m.num_tris
            idx = torch.from_numpy(m.indices.view(np.int32)).cuda()
            verts = torch.from_numpy(m.vertices).cuda()
            out = torch.full((T * 21,), float("nan"), device="cuda")
            ids = torch.full((3 * T,), -1, dtype=torch.int32, device="cuda")
            binv = torch.full((T + 1,), -1, dtype=torch.int32, device="cuda")
            meshes.append((m, pal, M, N))
            bufs.append((idx, verts, out, ids, binv, uni))
            descs.append(gp.draw_desc(idx, verts, gp.GP_SHADER_SKIN, uni, out, ids, binv))
        rng = np.random.default_rng(5)
        gp.gp_autotune(ctx, [descs[i] for i in rng.choice(len(descs), size=200, replace=False)], reps=1)
        frame = gp.gp_frame_create(ctx, descs)
        try:
            t = gp.gp_frame_submit(frame, ctx)
            assert gp.gp_sync(ctx, t) == gp.GP_OK
            torch.cuda.synchronize()
            for i, ((m, _, _, _), (_, _, _, ids, _, _)) in enumerate(zip(meshes, bufs)):
                assert np.array_equal(ids.cpu().numpy().view(np.uint32), m.indices), i
            names = {0: "naive", 1: "warp", 2: "sort", 3: "hash", 4: "phash"}
            for i in sorted(rng.choice(len(meshes), size=40, replace=False)):
                m, pal, M, N = meshes[i]
                _, _, out, _, binv, _ = bufs[i]
                cfg = gp.gp_frame_draw_config(frame, i)
                variant = names[cfg["variant"]]
                T = m.num_tris
                if variant == "naive":
                    st = list(range(0, T, 256)) + [T]
                elif variant == "warp" or cfg["mode"] == 0:
                    st = B.static_starts(T, cfg["batch_indices"])
                else:
                    st = B.dynamic_partition(m.indices, cfg["max_unique"], cfg["max_tris"], 4096)
                assert cfg["batches"] == len(st) - 1, (i, cfg)
                if variant in ("sort", "hash", "phash"):
                    want = B.unique_per_batch(m.indices, st)
                    assert np.array_equal(binv.cpu().numpy()[: len(st) - 1], want), (i, cfg)
                elif variant == "warp" and T <= 5000:  # the lane-by-lane replay is slow in Python
                    want = B.batch_invocations(m.indices, st, variant)
                    assert np.array_equal(binv.cpu().numpy()[: len(st) - 1], want), (i, cfg)
                tris = np.sort(rng.choice(T, size=min(T, 500), replace=False))
                got = out.cpu().numpy().reshape(T, 3, 7)[tris]
                ref = S.draw(m, S.SHADER_SKIN, {"M": M, "N": N, "palette": pal}, tris=tris)
                assert_attrs_close(got, ref, S.SHADER_SKIN, m)
        finally:
            gp.gp_frame_destroy(frame)
    finally:
        gp.gp_destroy(ctx)
