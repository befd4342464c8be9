"""Shared helpers for the GPU parity tests: run a draw through the C ABI and
compare it with the CPU oracle."""
import math

import numpy as np

import meshgen as mg
from oracle import batching as B
from oracle import shading as S

REL_TOL = 1e-5  # shaded FP32 attributes vs the float64 oracle (relative, with a scale floor)

SHADERS = {"mvp": S.SHADER_MVP, "skin": S.SHADER_SKIN, "envelope": S.SHADER_ENVELOPE, "load": S.SHADER_LOAD}


def uniforms_for(mesh, shader_id, seed=1, palette=None, steps=64):
    """(ctypes uniform blob for the library, dict for the oracle)."""
    import paper_1805_08893_gb300 as gp
    M, N = mg.mvp_uniforms(seed)
    if shader_id == S.SHADER_MVP:
        return gp.uniforms_mvp(M, N), {"M": M, "N": N}
    if shader_id == S.SHADER_SKIN:
        return gp.uniforms_skin(M, N, palette), {"M": M, "N": N, "palette": palette}
    if shader_id == S.SHADER_ENVELOPE:
        d = mg.envelope_offset(mesh)
        dirs = mg.envelope_directions()
        return gp.uniforms_envelope(d, dirs), {"d": d, "dirs": dirs}
    if shader_id == S.SHADER_LOAD:
        return gp.uniforms_load(M, N, steps), {"M": M, "N": N, "steps": steps}
    raise ValueError(shader_id)


def attr_floor(ref, shader_id, mesh):
    """Scale floor of the relative tolerance for each output value.

    clip x, y, z, w: |clip.w| (perspective divides by w); normals: 1;
    envelope positions: the mesh's bounding-box diagonal."""
    fl = np.ones_like(ref)
    if shader_id == S.SHADER_ENVELOPE:
        p = mesh.vertices[:, 0:3].astype(np.float64)
        fl[:] = np.linalg.norm(p.max(axis=0) - p.min(axis=0))
    else:
        fl[..., 0:4] = np.abs(ref[..., 3:4])
    return fl


def assert_attrs_close(gpu, ref, shader_id, mesh, rel=REL_TOL):
    gpu = np.asarray(gpu, np.float64)
    bound = rel * np.maximum(np.abs(ref), attr_floor(ref, shader_id, mesh))
    err = np.abs(gpu - ref)
    bad = err > bound
    if bad.any():
        i = np.argwhere(bad)[0]
        raise AssertionError(f"{bad.sum()} values out of tolerance; first at {tuple(i)}: gpu={gpu[tuple(i)]!r} "
                             f"ref={ref[tuple(i)]!r} bound={bound[tuple(i)]!r}")


class DrawResult:
    pass


def draw_gpu(mesh, variant, shader_id=S.SHADER_MVP, mode="static", uniforms=None, debug=True, device="cuda",
             **cfg):
    """One draw through the C ABI.  Returns out [T,3,K] (numpy), corner ids,
    per-batch invocations, batch starts (triangles) and stats."""
    import torch
    import paper_1805_08893_gb300 as gp
    T = mesh.num_tris
    K = gp.gp_out_floats(shader_id)
    idx = torch.from_numpy(mesh.indices.view(np.int32).copy()).to(device)
    verts = torch.from_numpy(mesh.vertices).to(device)
    out = torch.full((max(T, 1) * 3 * K,), float("nan"), dtype=torch.float32, device=device)
    ids = torch.full((max(T, 1) * 3,), -1, dtype=torch.int32, device=device) if debug else None
    md = gp.GP_BATCH_DYNAMIC if mode == "dynamic" else gp.GP_BATCH_STATIC
    stream = torch.cuda.current_stream()
    ctx = gp.gp_create(variant, mode=md, stream=stream, **cfg)
    r = DrawResult()
    try:
        handle = 0
        if md == gp.GP_BATCH_DYNAMIC:
            handle, nb = gp.gp_partition(ctx, idx)
            st = torch.zeros(nb + 1, dtype=torch.int32, device=device)
            gp.gp_partition_starts(ctx, handle, st)
            r.starts = st.cpu().numpy().astype(np.int64)
        elif variant == "multi":
            nb = 1 if T else 0
            r.starts = np.array([0, T] if T else [0], dtype=np.int64)
        elif variant == "naive":
            per = cfg.get("threads_per_group") or 256
            nb = (T + per - 1) // per
            r.starts = np.array(list(range(0, T, per)) + [T] if T else [0], dtype=np.int64)
        else:
            nb = gp.gp_static_batch_count(ctx, 3 * T)
            S_ = cfg.get("batch_indices") or (96 if variant == "warp" else 768)
            r.starts = np.asarray(B.static_starts(T, S_), dtype=np.int64)
        binv = torch.full((max(nb, 1),), -1, dtype=torch.int32, device=device) if debug else None
        r.ticket = gp.gp_submit_drawcall(ctx, idx, verts, shader_id, uniforms, out, ids, binv, partition=handle)
        r.status = gp.gp_sync(ctx, r.ticket, raise_on_error=False)
        torch.cuda.synchronize()
        r.stats = gp.gp_stats(ctx)
        r.out = out.cpu().numpy()[: T * 3 * K].reshape(T, 3, K)
        r.ids = ids.cpu().numpy()[: 3 * T].view(np.uint32) if debug else None
        r.inv = binv.cpu().numpy()[:nb].astype(np.int64) if debug else None
        r.num_batches = nb
        if handle:
            gp.gp_partition_release(ctx, handle)
    finally:
        gp.gp_destroy(ctx)
    return r


def expected_invocations(mesh, variant, starts):
    return B.batch_invocations(mesh.indices, list(starts), "naive" if variant == "naive" else variant)
