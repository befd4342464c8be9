"""The error model of the C ABI, exercised without a GPU fault.

* an allocation that fails (injected on the host: the context's allocation
  wrapper reports an exhausted device without allocating) returns
  GP_ERR_OOM, and the context then works normally;
* gp_sync with a limit shorter than the draw returns GP_ERR_TIMEOUT, and a
  later gp_sync without a limit returns GP_OK;
* a bounded device wait that runs out (injected: the kernel announces its
  first index window on the mbarrier but never copies it) stops the kernel,
  gp_sync returns GP_ERR_TIMEOUT, and the next draw on the same context
  equals the oracle.
"""
import numpy as np
import pytest

import meshgen as mg
from oracle import shading as S
from helpers_gp import assert_attrs_close, uniforms_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def grid():
    return mg.grid_mesh(64)


def _draw(gp, torch, ctx, mesh, uni, idx=None, partition=0):
    """One MVP draw; a partition handle belongs to the index tensor it was made for."""
    if idx is None:
        idx = torch.from_numpy(mesh.indices.view(np.int32)).cuda()
    verts = torch.from_numpy(mesh.vertices).cuda()
    out = torch.zeros(mesh.num_tris * 21, dtype=torch.float32, device="cuda")
    gp.gp_submit_drawcall(ctx, idx, verts, gp.GP_SHADER_MVP, uni, out, partition=partition)
    return idx, verts, out


def _check_mvp(out, mesh, ref_uni):
    ref = S.draw(mesh, S.SHADER_MVP, ref_uni)
    assert_attrs_close(out.cpu().numpy().reshape(mesh.num_tris, 3, 7), ref, S.SHADER_MVP, mesh)


def test_failed_allocation_reports_oom_and_context_recovers(grid):
    import torch
    import paper_1805_08893_gb300 as gp
    uni, ref_uni = uniforms_for(grid, S.SHADER_MVP)
    idx = torch.from_numpy(grid.indices.view(np.int32)).cuda()
    ctx = gp.gp_create("hash", mode=gp.GP_BATCH_DYNAMIC, stream=torch.cuda.current_stream())
    try:
        gp.gp_test_inject(ctx, gp.GP_TEST_FAIL_ALLOC, 1)
        with pytest.raises(gp.GpError) as e:
            gp.gp_partition(ctx, idx)
        assert e.value.status == gp.GP_ERR_OOM
        assert "GP_ERR_OOM" in gp.gp_last_error(ctx)
        # the injection is used up: the same call now succeeds and the draw is right
        h, nb = gp.gp_partition(ctx, idx)
        assert nb > 0
        _, _, out = _draw(gp, torch, ctx, grid, uni, idx, partition=h)
        assert gp.gp_sync(ctx) == gp.GP_OK
        _check_mvp(out, grid, ref_uni)
        gp.gp_partition_release(ctx, h)
    finally:
        gp.gp_destroy(ctx)


def test_failed_allocation_in_multi_kernel_draw(grid):
    import torch
    import paper_1805_08893_gb300 as gp
    uni, ref_uni = uniforms_for(grid, S.SHADER_MVP)
    ctx = gp.gp_create("multi", stream=torch.cuda.current_stream())
    try:
        gp.gp_test_inject(ctx, gp.GP_TEST_FAIL_ALLOC, 1)
        with pytest.raises(gp.GpError) as e:
            _draw(gp, torch, ctx, grid, uni)  # the shaded-row buffer is allocated at the first draw
        assert e.value.status == gp.GP_ERR_OOM
        _, _, out = _draw(gp, torch, ctx, grid, uni)
        assert gp.gp_sync(ctx) == gp.GP_OK
        _check_mvp(out, grid, ref_uni)
    finally:
        gp.gp_destroy(ctx)


def test_sync_limit_shorter_than_the_draw_times_out(grid):
    import torch
    import paper_1805_08893_gb300 as gp
    # a load of 2^24 dependent FMAs per shaded vertex: tens of milliseconds
    uni, _ = uniforms_for(grid, S.SHADER_LOAD, steps=1 << 24)
    idx = torch.from_numpy(grid.indices.view(np.int32)).cuda()
    verts = torch.from_numpy(grid.vertices).cuda()
    out = torch.zeros(grid.num_tris * 21, dtype=torch.float32, device="cuda")
    ctx = gp.gp_create("naive", stream=torch.cuda.current_stream())
    try:
        t = gp.gp_submit_drawcall(ctx, idx, verts, gp.GP_SHADER_LOAD, uni, out)
        assert gp.gp_sync(ctx, t, timeout_ms=1, raise_on_error=False) == gp.GP_ERR_TIMEOUT
        assert "did not complete in time" in gp.gp_last_error(ctx)
        assert gp.gp_sync(ctx, t) == gp.GP_OK
        assert gp.gp_stats(ctx)["draws"] == 1
    finally:
        gp.gp_destroy(ctx)


@pytest.mark.parametrize("variant", ["hash", "sort"])
def test_device_wait_that_runs_out_reports_timeout(grid, variant):
    import torch
    import paper_1805_08893_gb300 as gp
    uni, ref_uni = uniforms_for(grid, S.SHADER_MVP)
    idx = torch.from_numpy(grid.indices.view(np.int32)).cuda()
    ctx = gp.gp_create(variant, mode=gp.GP_BATCH_DYNAMIC, stream=torch.cuda.current_stream())
    try:
        h, _ = gp.gp_partition(ctx, idx)
        gp.gp_test_inject(ctx, gp.GP_TEST_STALL_WINDOW, 1)
        _draw(gp, torch, ctx, grid, uni, idx, partition=h)
        assert gp.gp_sync(ctx, raise_on_error=False) == gp.GP_ERR_TIMEOUT
        assert "bounded device wait" in gp.gp_last_error(ctx)
        # the context is still usable: the next draw runs and equals the oracle
        _, _, out = _draw(gp, torch, ctx, grid, uni, idx, partition=h)
        assert gp.gp_sync(ctx) == gp.GP_OK
        _check_mvp(out, grid, ref_uni)
        gp.gp_partition_release(ctx, h)
    finally:
        gp.gp_destroy(ctx)


def test_injection_rejects_unknown_kind(grid):
    import torch
    import paper_1805_08893_gb300 as gp
    ctx = gp.gp_create("hash", stream=torch.cuda.current_stream())
    try:
        with pytest.raises(gp.GpError) as e:
            gp.gp_test_inject(ctx, 99, 1)
        assert e.value.status == gp.GP_ERR_INVALID
    finally:
        gp.gp_destroy(ctx)
