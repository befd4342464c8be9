"""gp_partition_noalloc: the dynamic partition for callers that must not
allocate device memory (a real-time frame loop, or an application that owns
all device memory through its own pool).

Its batch starts must equal the oracle's greedy partition (Section 3.4, with
the segmented reading) and those of gp_partition, bit for bit, and repeated
calls must not be affected by what an earlier call left in the shared
scratch array.  This file is collected last so that a run stopping at the
first failure has already run every other test; it also passes alone in a
fresh process.
"""
import ctypes

import numpy as np
import pytest

import meshgen as mg
from oracle import batching as B

pytestmark = pytest.mark.gpu


def _reference_starts(gp, torch, idx, max_unique, max_tris, segment_tris):
    ctx = gp.gp_create("hash", mode=gp.GP_BATCH_DYNAMIC, max_unique=max_unique, max_tris=max_tris,
                       segment_tris=segment_tris, stream=torch.cuda.current_stream())
    try:
        h, nb = gp.gp_partition(ctx, idx)
        st = torch.zeros(nb + 1, dtype=torch.int32, device="cuda")
        gp.gp_partition_starts(ctx, h, st)
        gp.gp_partition_release(ctx, h)
    finally:
        gp.gp_destroy(ctx)
    return st.cpu().numpy()


def _noalloc_starts(gp, torch, idx, max_unique, max_tris, segment_tris):
    T = idx.numel() // 3
    starts = torch.full((T + 1,), -7, dtype=torch.int32, device="cuda")
    count = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    # straight through the C ABI
    rc = gp.lib.gp_partition_noalloc(ctypes.c_void_p(idx.data_ptr()), idx.numel(), max_unique, max_tris,
                                     segment_tris, ctypes.c_void_p(starts.data_ptr()), starts.numel(),
                                     ctypes.c_void_p(count.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    assert rc == gp.GP_OK, gp.gp_last_error(None)
    torch.cuda.synchronize()
    nb = int(count.item())
    return starts.cpu().numpy()[: nb + 1]


def test_noalloc_partition_matches_oracle_on_consecutive_calls():
    import torch
    import paper_1805_08893_gb300 as gp
    big = mg.geodesic_sphere(35, 5)      # 24,500 triangles: 6 segments
    small = mg.grid_mesh(64)             # 7,938 triangles, ragged index count
    cases = [(big, 256, 341, 4096), (small, 256, 341, 4096), (big, 64, 100, 1000)]
    for mesh, nu, mt, seg in cases:  # consecutive calls share the scratch array
        idx = torch.from_numpy(mesh.indices.view(np.int32)).cuda()
        oracle = np.asarray(B.dynamic_partition(mesh.indices, nu, mt, seg), dtype=np.int64)
        for rep in range(2):  # two calls in a row on the same input
            got = _noalloc_starts(gp, torch, idx, nu, mt, seg).astype(np.int64)
            assert np.array_equal(got, oracle), (mesh.name, nu, mt, seg, rep)
        want = _reference_starts(gp, torch, idx, nu, mt, seg).astype(np.int64)
        assert np.array_equal(want, oracle), (mesh.name, nu, mt, seg)


def test_noalloc_rejects_oversized_input():
    import torch
    import paper_1805_08893_gb300 as gp
    # a single unsegmented scan with one triangle per batch needs one start per
    # triangle in scratch: 2^20 triangles exceed the fixed 4 MiB array
    T = 1 << 20
    idx = torch.zeros(3 * T, dtype=torch.int32, device="cuda")
    starts = torch.zeros(T + 1, dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(gp.GpError) as e:
        gp.gp_partition_noalloc(idx, 3, 1, 0xFFFFFFFF, starts, count)
    assert e.value.status == gp.GP_ERR_INVALID
    assert "4 MiB" in gp.gp_last_error(None)
