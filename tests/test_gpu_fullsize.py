"""Parity at the benchmark's full size: the 7.2M-triangle geodesic sphere
(f = 600) in the launch configuration bench.py times (dynamic batches of 256
unique / 341 triangles, 256 threads, segments of 4096 triangles).

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


@pytest.fixture(scope="module")
def big():
    mesh = mg.geodesic_sphere(600, 2)
    starts = B.dynamic_partition(mesh.indices, 256, 341, 4096)
    return mesh, starts


@pytest.mark.parametrize("variant", ["hash", "phash", "sort"])
def test_full_size_dynamic(big, variant):
    mesh, starts = big
    uni, uni_o = uniforms_for(mesh, S.SHADER_MVP, seed=2)
    r = draw_gpu(mesh, variant, S.SHADER_MVP, "dynamic", uni, threads_per_group=256)
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
    starts = B.dynamic_partition(mesh.indices, 256, 341, 4096)
    return mesh, starts


@pytest.mark.parametrize("variant", ["hash", "phash", "sort"])
def test_envelope_bench_size_dynamic(heavy, variant):
    mesh, starts = heavy
    uni, uni_o = uniforms_for(mesh, S.SHADER_ENVELOPE)
    r = draw_gpu(mesh, variant, S.SHADER_ENVELOPE, "dynamic", uni, threads_per_group=256)
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
