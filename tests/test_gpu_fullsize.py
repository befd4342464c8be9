"""Parity at the benchmark's full size: the 7.2M-triangle geodesic sphere
(f = 600) in the launch configurations bench.py times (256 threads, segments
of 4096 triangles; dynamic batches of <= 320 unique / 426 triangles with a
2048-slot table for hash and phash, and of <= 256 unique / 341 triangles,
the paper's limits, for sort and for hash beside them).

Exact: the partition against the oracle's front-to-back scan, the vertex
behind every one of the 21.6M corners, and every batch's invocation count.
Sampled: the shaded attributes of 20,000 random triangles against the
float64 oracle (1e-5)."""
import numpy as np
import pytest

import meshgen as mg
from oracle import batching as B
from oracle import shading as S

from helpers_gp import assert_attrs_close, draw_gpu, uniforms_for

pytestmark = pytest.mark.gpu


# the dynamic-batch configurations bench.py draws with
TUNED = {"max_unique": 320, "max_tris": 426, "hash_slots": 2048}
PAPER = {"max_unique": 256, "max_tris": 341}
BENCH_DYNAMIC = [("hash", TUNED), ("phash", TUNED), ("sort", PAPER), ("hash", PAPER)]


def _partitions(mesh):
    return {(c["max_unique"], c["max_tris"]): B.dynamic_partition(mesh.indices, c["max_unique"], c["max_tris"], 4096)
            for c in (TUNED, PAPER)}


@pytest.fixture(scope="module")
def big():
    mesh = mg.geodesic_sphere(600, 2)
    return mesh, _partitions(mesh)


@pytest.mark.parametrize("variant,cfg", BENCH_DYNAMIC, ids=["hash", "phash", "sort", "hash-1023"])
def test_full_size_dynamic(big, variant, cfg):
    mesh, parts = big
    starts = parts[(cfg["max_unique"], cfg["max_tris"])]
    uni, uni_o = uniforms_for(mesh, S.SHADER_MVP, seed=2)
    r = draw_gpu(mesh, variant, S.SHADER_MVP, "dynamic", uni, threads_per_group=256, **cfg)
    assert r.status == 0
    assert r.starts.tolist() == starts
    assert np.array_equal(r.ids, mesh.indices)
    want = B.batch_invocations(mesh.indices, starts, variant)
    assert np.array_equal(r.inv, want)
    assert r.stats["invocations"] == int(want.sum())
    tris = np.sort(np.random.default_rng(5).choice(mesh.num_tris, size=20000, replace=False))
    assert_attrs_close(r.out[tris], S.draw(mesh, S.SHADER_MVP, uni_o, tris=tris), S.SHADER_MVP, mesh)


@pytest.mark.parametrize("variant", ["naive", "multi"])
def test_full_size_baselines(big, variant):
    mesh, _ = big
    uni, uni_o = uniforms_for(mesh, S.SHADER_MVP, seed=2)
    r = draw_gpu(mesh, variant, S.SHADER_MVP, "static", uni)
    assert r.status == 0
    assert np.array_equal(r.ids, mesh.indices)
    assert r.stats["invocations"] == (3 * mesh.num_tris if variant == "naive" else mesh.num_vertices)
    tris = np.sort(np.random.default_rng(6).choice(mesh.num_tris, size=20000, replace=False))
    assert_attrs_close(r.out[tris], S.draw(mesh, S.SHADER_MVP, uni_o, tris=tris), S.SHADER_MVP, mesh)


# ---------------------------------------------------------------------------
# the heavy-shader workload at its bench size: the envelope shader on the
# 2M-triangle geodesic sphere (f = 316), as bench.py's heavy section draws it
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def heavy():
    mesh = mg.geodesic_sphere(316, 4)
    return mesh, _partitions(mesh)


@pytest.mark.parametrize("variant,cfg", BENCH_DYNAMIC[:3], ids=["hash", "phash", "sort"])
def test_envelope_bench_size_dynamic(heavy, variant, cfg):
    mesh, parts = heavy
    starts = parts[(cfg["max_unique"], cfg["max_tris"])]
    uni, uni_o = uniforms_for(mesh, S.SHADER_ENVELOPE)
    r = draw_gpu(mesh, variant, S.SHADER_ENVELOPE, "dynamic", uni, threads_per_group=256, **cfg)
    assert r.status == 0
    assert r.starts.tolist() == starts
    assert np.array_equal(r.ids, mesh.indices)
    # sort/hash/phash shade each batch's distinct ids once: the plain definition
    want = B.unique_per_batch(mesh.indices, starts)
    assert np.array_equal(r.inv, want)
    assert r.stats["invocations"] == int(want.sum())
    tris = np.sort(np.random.default_rng(7).choice(mesh.num_tris, size=20000, replace=False))
    assert_attrs_close(r.out[tris], S.draw(mesh, S.SHADER_ENVELOPE, uni_o, tris=tris), S.SHADER_ENVELOPE, mesh)


@pytest.mark.parametrize("variant", ["naive", "multi", "warp"])
def test_envelope_bench_size_baselines(heavy, variant):
    mesh, _ = heavy
    uni, uni_o = uniforms_for(mesh, S.SHADER_ENVELOPE)
    r = draw_gpu(mesh, variant, S.SHADER_ENVELOPE, "static", uni)
    assert r.status == 0
    assert np.array_equal(r.ids, mesh.indices)
    if variant == "naive":
        assert r.stats["invocations"] == 3 * mesh.num_tris
    elif variant == "multi":
        assert r.stats["invocations"] == mesh.num_vertices
    tris = np.sort(np.random.default_rng(8).choice(mesh.num_tris, size=20000, replace=False))
    assert_attrs_close(r.out[tris], S.draw(mesh, S.SHADER_ENVELOPE, uni_o, tris=tris), S.SHADER_ENVELOPE, mesh)
