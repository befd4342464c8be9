"""Python binding of the GB300 vertex-reuse geometry stage (libgp.so).

Argument marshalling only: every step of the geometry stage runs in the CUDA
kernels behind the C ABI declared in ``include/gp.h``.  The functions keep the
C names (``gp_create``, ``gp_submit_drawcall``, ``gp_sync``, ...).  Device
buffers are torch CUDA tensors (PyTorch provides memory and streams); there is
no CPU fallback: if the library cannot be loaded, importing this package
raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

__all__ = [
    "GpError", "gp_create", "gp_destroy", "gp_partition", "gp_partition_starts", "gp_partition_release",
    "gp_submit_drawcall", "gp_sync", "gp_stats", "gp_draw_host", "gp_out_floats", "gp_static_batch_count",
    "gp_last_error", "gp_status_string", "gp_partition_noalloc", "gp_frame_create", "gp_frame_submit",
    "gp_frame_set_uniforms", "gp_frame_draw_config", "gp_frame_destroy", "gp_autotune", "gp_autotune_table",
    "gp_autotune_set_table", "draw_desc", "gp_server_create", "gp_server_add_mesh", "gp_server_submit",
    "gp_server_replay", "gp_server_wait", "gp_server_latency", "gp_server_stats", "gp_server_destroy", "uniforms_mvp", "uniforms_skin", "uniforms_envelope", "uniforms_load", "gp_test_inject",
    "Context", "lib", "library_path",
]

# enums (gp.h)
GP_OK, GP_ERR_INVALID, GP_ERR_OOM, GP_ERR_CUDA, GP_ERR_TIMEOUT, GP_ERR_BUSY, GP_ERR_INDEX_RANGE, \
    GP_ERR_UNSUPPORTED = range(8)
GP_NAIVE, GP_WARP, GP_SORT, GP_HASH, GP_PHASH, GP_AUTO, GP_MULTI = range(7)
GP_BATCH_STATIC, GP_BATCH_DYNAMIC = 0, 1
GP_SHADER_MVP, GP_SHADER_SKIN, GP_SHADER_ENVELOPE, GP_SHADER_LOAD = range(4)
GP_VFMT_PNU32, GP_VFMT_SKIN64 = 0, 1
GP_SEGMENT_NONE = 0xFFFFFFFF
GP_TEST_FAIL_ALLOC, GP_TEST_STALL_WINDOW = 1, 2

VARIANTS = {"naive": GP_NAIVE, "warp": GP_WARP, "sort": GP_SORT, "hash": GP_HASH, "phash": GP_PHASH,
            "multi": GP_MULTI}


class gp_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("variant", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("batch_indices", ctypes.c_uint32), ("max_unique", ctypes.c_uint32),
                ("max_tris", ctypes.c_uint32), ("threads_per_group", ctypes.c_uint32),
                ("probe_k", ctypes.c_uint32), ("hash_slots", ctypes.c_uint32),
                ("segment_tris", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("mem_budget_bytes", ctypes.c_uint64), ("stream", ctypes.c_void_p)]


class gp_index_buf(ctypes.Structure):
    _fields_ = [("d_indices", ctypes.c_void_p), ("num_indices", ctypes.c_uint64), ("partition", ctypes.c_uint64)]


class gp_vertex_buf(ctypes.Structure):
    _fields_ = [("d_vertices", ctypes.c_void_p), ("num_vertices", ctypes.c_uint64),
                ("stride_bytes", ctypes.c_uint32), ("format", ctypes.c_uint32)]


class gp_out_buf(ctypes.Structure):
    _fields_ = [("d_out", ctypes.c_void_p), ("capacity_bytes", ctypes.c_uint64),
                ("d_corner_ids", ctypes.c_void_p), ("d_batch_invocations", ctypes.c_void_p),
                ("batch_capacity", ctypes.c_uint64)]


class gp_uniforms_mvp(ctypes.Structure):
    _fields_ = [("mvp", ctypes.c_float * 16), ("normal", ctypes.c_float * 9)]


class gp_uniforms_skin(ctypes.Structure):
    _fields_ = [("mvp", ctypes.c_float * 16), ("normal", ctypes.c_float * 9), ("palette", ctypes.c_float * 768)]


class gp_uniforms_envelope(ctypes.Structure):
    _fields_ = [("d", ctypes.c_float), ("num_dirs", ctypes.c_uint32), ("dirs", ctypes.c_float * 48)]


class gp_uniforms_load(ctypes.Structure):
    _fields_ = [("mvp", ctypes.c_float * 16), ("normal", ctypes.c_float * 9), ("steps", ctypes.c_uint32)]


class gp_stats_t(ctypes.Structure):
    _fields_ = [("draws", ctypes.c_uint64), ("triangles", ctypes.c_uint64), ("indices", ctypes.c_uint64),
                ("invocations", ctypes.c_uint64), ("batches", ctypes.c_uint64), ("busy_ms", ctypes.c_double),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("bytes_moved", ctypes.c_uint64),
                ("last_error", ctypes.c_uint32)]


class gp_draw_desc(ctypes.Structure):
    _fields_ = [("index_buf", gp_index_buf), ("vertex_buf", gp_vertex_buf), ("out", gp_out_buf),
                ("shader_id", ctypes.c_uint32), ("uniforms_bytes", ctypes.c_uint32), ("uniforms", ctypes.c_void_p),
                ("variant", ctypes.c_int32), ("mode", ctypes.c_int32), ("batch_indices", ctypes.c_uint32),
                ("max_unique", ctypes.c_uint32), ("max_tris", ctypes.c_uint32),
                ("threads_per_group", ctypes.c_uint32)]


class gp_draw_config(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("mode", ctypes.c_int32), ("batch_indices", ctypes.c_uint32),
                ("max_unique", ctypes.c_uint32), ("max_tris", ctypes.c_uint32),
                ("threads_per_group", ctypes.c_uint32), ("batches", ctypes.c_uint64)]


class gp_autotune_entry(ctypes.Structure):
    _fields_ = [("shader_id", ctypes.c_uint32), ("tris_lo", ctypes.c_uint32), ("tris_hi", ctypes.c_uint32),
                ("pad", ctypes.c_uint32), ("config", gp_draw_config), ("us_per_draw", ctypes.c_double)]


class gp_serve_config(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_uint64), ("streams", ctypes.c_uint32),
                ("step_max_batches", ctypes.c_uint32), ("max_active", ctypes.c_uint32), ("variant", ctypes.c_int32),
                ("mode", ctypes.c_int32), ("batch_indices", ctypes.c_uint32), ("max_unique", ctypes.c_uint32),
                ("max_tris", ctypes.c_uint32), ("threads_per_group", ctypes.c_uint32)]


class gp_serve_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("triangles", ctypes.c_uint64),
                ("invocations", ctypes.c_uint64), ("steps", ctypes.c_uint64), ("uploads", ctypes.c_uint64),
                ("evictions", ctypes.c_uint64), ("resident_bytes", ctypes.c_uint64), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double), ("busy_ms", ctypes.c_double),
                ("wall_ms", ctypes.c_double), ("last_error", ctypes.c_uint32), ("pad", ctypes.c_uint32),
                ("device_ms", ctypes.c_double)]


class gp_walk_desc(ctypes.Structure):
    _fields_ = [("d_activity", ctypes.c_void_p), ("d_pos", ctypes.c_void_p), ("d_scratch", ctypes.c_void_p),
                ("d_counters", ctypes.c_void_p), ("stream", ctypes.c_void_p), ("seed", ctypes.c_uint64),
                ("width", ctypes.c_uint32), ("height", ctypes.c_uint32), ("num_agents", ctypes.c_uint32),
                ("variant", ctypes.c_int32), ("first_step", ctypes.c_uint32), ("steps", ctypes.c_uint32),
                ("batch_agents", ctypes.c_uint32), ("threads", ctypes.c_uint32)]


class gp_loop_desc(ctypes.Structure):
    _fields_ = [("d_indices", ctypes.c_void_p), ("d_vertices", ctypes.c_void_p), ("d_ring_offsets", ctypes.c_void_p),
                ("d_ring", ctypes.c_void_p), ("d_vertex_flags", ctypes.c_void_p), ("d_opposite", ctypes.c_void_p),
                ("d_out", ctypes.c_void_p), ("d_starts", ctypes.c_void_p), ("d_num_batches", ctypes.c_void_p),
                ("d_counters", ctypes.c_void_p), ("stream", ctypes.c_void_p), ("num_indices", ctypes.c_uint64),
                ("num_vertices", ctypes.c_uint64), ("ring_count", ctypes.c_uint64), ("stride_bytes", ctypes.c_uint32),
                ("variant", ctypes.c_int32), ("batch_indices", ctypes.c_uint32), ("max_batch_indices", ctypes.c_uint32),
                ("max_unique", ctypes.c_uint32), ("max_batches", ctypes.c_uint32), ("threads", ctypes.c_uint32)]


class GpError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(message)
        self.status = status


def library_path() -> str:
    return os.environ.get("GP_LIBRARY") or _build.LIB


def _load():
    """Loads libgp.so, building it first if it is missing or stale.
    GP_LIBRARY=<path> loads that build of the library instead."""
    path = os.environ.get("GP_LIBRARY") or _build.LIB
    if not os.environ.get("GP_LIBRARY") and (not os.path.exists(path) or
                                              os.environ.get("GP_BUILD_ON_IMPORT", "1") == "1"):
        _build.build()
    L = ctypes.CDLL(path)
    P, U64, U32, I = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
    sig = {
        "gp_create": ([ctypes.POINTER(gp_config), ctypes.POINTER(P)], I),
        "gp_destroy": ([P], I),
        "gp_partition": ([P, ctypes.POINTER(gp_index_buf), ctypes.POINTER(U64), ctypes.POINTER(U64)], I),
        "gp_partition_starts": ([P, U64, P, U64, ctypes.POINTER(U64)], I),
        "gp_partition_release": ([P, U64], I),
        "gp_submit_drawcall": ([P, ctypes.POINTER(gp_index_buf), ctypes.POINTER(gp_vertex_buf), U32, P, U32,
                                ctypes.POINTER(gp_out_buf), ctypes.POINTER(U64)], I),
        "gp_sync": ([P, U64, U32], I),
        "gp_stats": ([P, ctypes.POINTER(gp_stats_t), I], I),
        "gp_draw_host": ([P, P, U64, P, U64, U32, U32, U32, P, U32, P, U64], I),
        "gp_out_floats": ([U32], U32),
        "gp_static_batch_count": ([P, U64], U64),
        "gp_last_error": ([P], ctypes.c_char_p),
        "gp_status_string": ([I], ctypes.c_char_p),
        "gp_partition_noalloc": ([P, U64, U32, U32, U32, P, U64, P, P], I),
        "gp_test_inject": ([P, U32, U32], I),
        "gp_frame_create": ([P, ctypes.POINTER(gp_draw_desc), U32, ctypes.POINTER(P)], I),
        "gp_frame_submit": ([P, ctypes.POINTER(U64)], I),
        "gp_frame_set_uniforms": ([P, U32, P, U32], I),
        "gp_frame_draw_config": ([P, U32, ctypes.POINTER(gp_draw_config)], I),
        "gp_frame_destroy": ([P], I),
        "gp_autotune": ([P, ctypes.POINTER(gp_draw_desc), U32, U32], I),
        "gp_autotune_table": ([P, ctypes.POINTER(gp_autotune_entry), U32, ctypes.POINTER(U32)], I),
        "gp_autotune_set_table": ([P, ctypes.POINTER(gp_autotune_entry), U32], I),
        "gp_server_create": ([P, ctypes.POINTER(gp_serve_config), ctypes.POINTER(P)], I),
        "gp_server_add_mesh": ([P, P, U64, P, U64, U32, U32, ctypes.POINTER(U64)], I),
        "gp_server_submit": ([P, U64, U32, P, U32, P, U64, ctypes.POINTER(U64)], I),
        "gp_server_replay": ([P, U32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(U64), ctypes.POINTER(U32),
                              ctypes.POINTER(P), ctypes.POINTER(U32), ctypes.POINTER(P), ctypes.POINTER(U64),
                              ctypes.POINTER(U64)], I),
        "gp_server_wait": ([P, U64, U32], I),
        "gp_server_latency": ([P, U64, ctypes.POINTER(ctypes.c_double)], I),
        "gp_server_stats": ([P, ctypes.POINTER(gp_serve_stats), I], I),
        "gp_server_destroy": ([P], I),
        "gp_simulate_parallel_cache": ([ctypes.POINTER(U32), U64, U32, U32, U32, U32, ctypes.POINTER(U64)], I),
        "gp_random_walk": ([ctypes.POINTER(gp_walk_desc)], I),
        "gp_loop_adjacency": ([P, U64, U32, P, P, U64, P, P, ctypes.POINTER(U64)], I),
        "gp_loop_subdivide": ([ctypes.POINTER(gp_loop_desc)], I),
    }
    for name, (argt, rest) in sig.items():
        f = getattr(L, name)
        f.argtypes = argt
        f.restype = rest
    return L


lib = _load()


def gp_last_error(ctx=None) -> str:
    return lib.gp_last_error(ctx).decode()


def gp_status_string(status: int) -> str:
    return lib.gp_status_string(status).decode()


def _check(status: int, ctx=None):
    if status != GP_OK:
        raise GpError(status, gp_last_error(ctx) or gp_status_string(status))


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def gp_create(variant="hash", mode=GP_BATCH_STATIC, device=0, batch_indices=0, max_unique=0, max_tris=0,
              threads_per_group=0, probe_k=0, hash_slots=0, segment_tris=0, mem_budget_bytes=0, stream=None):
    """gp_create: returns an opaque context handle."""
    cfg = gp_config(device, VARIANTS.get(variant, variant), int(mode), batch_indices, max_unique, max_tris,
                    threads_per_group, probe_k, hash_slots, segment_tris, 0, mem_budget_bytes,
                    _stream_handle(stream))
    h = ctypes.c_void_p()
    _check(lib.gp_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def gp_destroy(ctx):
    _check(lib.gp_destroy(ctx))


def _index_buf(indices, partition=0):
    assert indices.is_cuda and indices.is_contiguous() and indices.element_size() == 4
    return gp_index_buf(indices.data_ptr(), indices.numel(), partition)


def gp_partition(ctx, indices, want_count=True):
    """gp_partition: returns (handle, number of batches or None)."""
    ib = _index_buf(indices)
    h = ctypes.c_uint64()
    n = ctypes.c_uint64()
    _check(lib.gp_partition(ctx, ctypes.byref(ib), ctypes.byref(h), ctypes.byref(n) if want_count else None), ctx)
    return h.value, (n.value if want_count else None)


def gp_partition_starts(ctx, handle, out=None):
    """gp_partition_starts: copies the starts into ``out`` (uint32/int32 CUDA
    tensor) if given; returns the number of batches."""
    n = ctypes.c_uint64()
    cap = 0 if out is None else out.numel()
    _check(lib.gp_partition_starts(ctx, handle, _ptr(out), cap, ctypes.byref(n)), ctx)
    return n.value


def gp_partition_release(ctx, handle):
    _check(lib.gp_partition_release(ctx, handle), ctx)


def _vertex_buf(vertices, num_vertices=None, fmt=None):
    assert vertices.is_cuda and vertices.is_contiguous() and vertices.dim() == 2
    stride = vertices.shape[1] * vertices.element_size()
    if fmt is None:
        fmt = GP_VFMT_SKIN64 if stride == 64 else GP_VFMT_PNU32
    nv = vertices.shape[0] if num_vertices is None else num_vertices
    return gp_vertex_buf(vertices.data_ptr(), nv, stride, fmt)


def gp_submit_drawcall(ctx, indices, vertices, shader_id, uniforms, out, corner_ids=None, batch_invocations=None,
                       partition=0, num_vertices=None, fmt=None):
    """gp_submit_drawcall: returns the ticket.  ``uniforms`` is one of the
    gp_uniforms_* ctypes structures."""
    ib = _index_buf(indices, partition)
    vb = _vertex_buf(vertices, num_vertices, fmt)
    ob = gp_out_buf(out.data_ptr(), out.numel() * out.element_size(),
                    None if corner_ids is None else corner_ids.data_ptr(),
                    None if batch_invocations is None else batch_invocations.data_ptr(),
                    0 if batch_invocations is None else batch_invocations.numel())
    t = ctypes.c_uint64()
    _check(lib.gp_submit_drawcall(ctx, ctypes.byref(ib), ctypes.byref(vb), shader_id,
                                  ctypes.cast(ctypes.byref(uniforms), ctypes.c_void_p), ctypes.sizeof(uniforms),
                                  ctypes.byref(ob), ctypes.byref(t)), ctx)
    return t.value


def gp_sync(ctx, ticket=0, timeout_ms=0, raise_on_error=True):
    """gp_sync: returns the status (raises GpError on a non-OK status unless
    ``raise_on_error`` is False)."""
    s = lib.gp_sync(ctx, ticket, timeout_ms)
    if raise_on_error:
        _check(s, ctx)
    return s


def gp_stats(ctx, reset=False) -> dict:
    st = gp_stats_t()
    _check(lib.gp_stats(ctx, ctypes.byref(st), 1 if reset else 0), ctx)
    return {name: getattr(st, name) for name, _ in gp_stats_t._fields_}


def gp_draw_host(ctx, indices, vertices, shader_id, uniforms, out, fmt=None):
    """gp_draw_host: end-to-end draw from host memory (numpy arrays or CPU
    tensors, ideally pinned).  ``out`` receives the triangles."""
    def addr(x):
        return x.ctypes.data if isinstance(x, np.ndarray) else x.data_ptr()

    def nbytes(x):
        return x.nbytes if isinstance(x, np.ndarray) else x.numel() * x.element_size()
    nidx = indices.size if isinstance(indices, np.ndarray) else indices.numel()
    nv = vertices.shape[0]
    stride = nbytes(vertices) // max(nv, 1)
    if fmt is None:
        fmt = GP_VFMT_SKIN64 if stride == 64 else GP_VFMT_PNU32
    s = lib.gp_draw_host(ctx, addr(indices), nidx, addr(vertices), nv, stride, fmt, shader_id,
                         ctypes.cast(ctypes.byref(uniforms), ctypes.c_void_p), ctypes.sizeof(uniforms),
                         addr(out), nbytes(out))
    _check(s, ctx)


def gp_test_inject(ctx, what, count=1):
    """gp_test_inject: failure injection for tests (GP_TEST_FAIL_ALLOC,
    GP_TEST_STALL_WINDOW)."""
    _check(lib.gp_test_inject(ctx, what, count), ctx)


def gp_partition_noalloc(indices, max_unique, max_tris, segment_tris, starts, num_batches, stream=None):
    """gp_partition_noalloc: batch starts into ``starts`` (int32 CUDA tensor,
    at least T + 1 entries) and the count into ``num_batches`` (1 entry), with
    no device allocation.  Asynchronous on ``stream``."""
    s = lib.gp_partition_noalloc(ctypes.c_void_p(indices.data_ptr()), indices.numel(), max_unique, max_tris,
                                 segment_tris, ctypes.c_void_p(starts.data_ptr()), starts.numel(),
                                 ctypes.c_void_p(num_batches.data_ptr()), _stream_handle(stream))
    _check(s)


# ---------------------------------------------------------------------------
# frames and the autotuner
# ---------------------------------------------------------------------------

def draw_desc(indices, vertices, shader_id, uniforms, out, corner_ids=None, batch_invocations=None,
              variant=GP_AUTO, mode=GP_BATCH_STATIC, batch_indices=0, max_unique=0, max_tris=0,
              threads_per_group=0, num_vertices=None, fmt=None):
    """A gp_draw_desc for gp_frame_create / gp_autotune (keeps ``uniforms``
    referenced until the call that copies it)."""
    d = gp_draw_desc()
    d.index_buf = _index_buf(indices)
    d.vertex_buf = _vertex_buf(vertices, num_vertices, fmt)
    d.out = gp_out_buf(out.data_ptr(), out.numel() * out.element_size(),
                       None if corner_ids is None else corner_ids.data_ptr(),
                       None if batch_invocations is None else batch_invocations.data_ptr(),
                       0 if batch_invocations is None else batch_invocations.numel())
    d.shader_id = shader_id
    d.uniforms_bytes = ctypes.sizeof(uniforms)
    d.uniforms = ctypes.cast(ctypes.byref(uniforms), ctypes.c_void_p)
    d.variant = VARIANTS.get(variant, variant) if isinstance(variant, str) else variant
    d.mode = mode
    d.batch_indices = batch_indices
    d.max_unique = max_unique
    d.max_tris = max_tris
    d.threads_per_group = threads_per_group
    d._keep = uniforms  # the blob must outlive the C call
    return d


def _desc_array(descs):
    arr = (gp_draw_desc * max(1, len(descs)))()
    for i, d in enumerate(descs):
        arr[i] = d
    return arr


def gp_frame_create(ctx, descs):
    """gp_frame_create: ``descs`` is a list of draw_desc(...) entries."""
    arr = _desc_array(descs)
    h = ctypes.c_void_p()
    _check(lib.gp_frame_create(ctx, arr, len(descs), ctypes.byref(h)), ctx)
    return h


def gp_frame_submit(frame, ctx=None):
    t = ctypes.c_uint64()
    _check(lib.gp_frame_submit(frame, ctypes.byref(t)), ctx)
    return t.value


def gp_frame_set_uniforms(frame, draw, uniforms, ctx=None):
    _check(lib.gp_frame_set_uniforms(frame, draw, ctypes.cast(ctypes.byref(uniforms), ctypes.c_void_p),
                                     ctypes.sizeof(uniforms)), ctx)


def _config_dict(k):
    return {name: getattr(k, name) for name, _ in gp_draw_config._fields_}


def gp_frame_draw_config(frame, draw) -> dict:
    k = gp_draw_config()
    _check(lib.gp_frame_draw_config(frame, draw, ctypes.byref(k)))
    return _config_dict(k)


def gp_frame_destroy(frame):
    _check(lib.gp_frame_destroy(frame))


def gp_autotune(ctx, descs, reps=3):
    arr = _desc_array(descs)
    _check(lib.gp_autotune(ctx, arr, len(descs), reps), ctx)


def gp_autotune_table(ctx) -> list:
    n = ctypes.c_uint32()
    _check(lib.gp_autotune_table(ctx, None, 0, ctypes.byref(n)), ctx)
    arr = (gp_autotune_entry * max(1, n.value))()
    _check(lib.gp_autotune_table(ctx, arr, n.value, ctypes.byref(n)), ctx)
    return [{"shader_id": e.shader_id, "tris_lo": e.tris_lo, "tris_hi": e.tris_hi, "config": _config_dict(e.config),
             "us_per_draw": e.us_per_draw} for e in arr[: n.value]]


def gp_autotune_set_table(ctx, rows):
    arr = (gp_autotune_entry * max(1, len(rows)))()
    for i, r in enumerate(rows):
        arr[i].shader_id = r["shader_id"]
        arr[i].tris_lo = r["tris_lo"]
        arr[i].tris_hi = r["tris_hi"]
        for name, _ in gp_draw_config._fields_:
            setattr(arr[i].config, name, r["config"][name])
        arr[i].us_per_draw = r.get("us_per_draw", 0.0)
    _check(lib.gp_autotune_set_table(ctx, arr, len(rows)), ctx)


# ---------------------------------------------------------------------------
# serving
# ---------------------------------------------------------------------------

def gp_server_create(ctx, mem_budget_bytes=0, streams=0, step_max_batches=0, max_active=0, variant="hash",
                     mode=GP_BATCH_DYNAMIC, batch_indices=0, max_unique=0, max_tris=0, threads_per_group=0):
    cfg = gp_serve_config(mem_budget_bytes, streams, step_max_batches, max_active,
                          VARIANTS.get(variant, variant) if isinstance(variant, str) else variant, mode, batch_indices,
                          max_unique, max_tris, threads_per_group)
    h = ctypes.c_void_p()
    _check(lib.gp_server_create(ctx, ctypes.byref(cfg), ctypes.byref(h)), ctx)
    return h


def gp_server_add_mesh(server, indices, vertices, fmt=None):
    """Registers a mesh from host arrays (numpy); returns its id."""
    idx = np.ascontiguousarray(indices, dtype=np.uint32)
    vtx = np.ascontiguousarray(vertices)
    stride = vtx.shape[1] * vtx.itemsize
    if fmt is None:
        fmt = GP_VFMT_SKIN64 if stride == 64 else GP_VFMT_PNU32
    m = ctypes.c_uint64()
    _check(lib.gp_server_add_mesh(server, idx.ctypes.data, idx.size, vtx.ctypes.data, vtx.shape[0], stride, fmt,
                                  ctypes.byref(m)))
    return m.value


def gp_server_submit(server, mesh, shader_id, uniforms, out):
    r = ctypes.c_uint64()
    _check(lib.gp_server_submit(server, mesh, shader_id, ctypes.cast(ctypes.byref(uniforms), ctypes.c_void_p),
                                ctypes.sizeof(uniforms), ctypes.c_void_p(out.data_ptr()),
                                out.numel() * out.element_size(), ctypes.byref(r)))
    return r.value


def gp_server_replay(server, arrivals_s, meshes, shader_ids, uniforms, outs):
    """Submits requests at their arrival times (seconds from the call) from the
    native side; returns their ids once all are submitted."""
    n = len(arrivals_s)
    arr = (ctypes.c_double * n)(*[float(x) for x in arrivals_s])
    ms = (ctypes.c_uint64 * n)(*[int(x) for x in meshes])
    sh = (ctypes.c_uint32 * n)(*[int(x) for x in shader_ids])
    up = (ctypes.c_void_p * n)(*[ctypes.cast(ctypes.byref(u), ctypes.c_void_p).value for u in uniforms])
    ub = (ctypes.c_uint32 * n)(*[ctypes.sizeof(u) for u in uniforms])
    op = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
    oc = (ctypes.c_uint64 * n)(*[o.numel() * o.element_size() for o in outs])
    ids = (ctypes.c_uint64 * n)()
    _check(lib.gp_server_replay(server, n, arr, ms, sh, up, ub, op, oc, ids))
    return list(ids)


def gp_server_wait(server, request=0, timeout_ms=0, raise_on_error=True):
    s = lib.gp_server_wait(server, request, timeout_ms)
    if raise_on_error:
        _check(s)
    return s


def gp_server_latency(server, request) -> float:
    v = ctypes.c_double()
    _check(lib.gp_server_latency(server, request, ctypes.byref(v)))
    return v.value


def gp_server_stats(server, reset=False) -> dict:
    st = gp_serve_stats()
    _check(lib.gp_server_stats(server, ctypes.byref(st), 1 if reset else 0))
    return {name: getattr(st, name) for name, _ in gp_serve_stats._fields_ if name != "pad"}


def gp_server_destroy(server):
    _check(lib.gp_server_destroy(server))


def gp_simulate_parallel_cache(indices, num_sms=28, concurrent=1024, capacity_entries=512, threads=0) -> int:
    """gp_simulate_parallel_cache: hits of the per-multiprocessor LRU cache
    (Section 5.1).  ``indices``: host uint32 array (numpy)."""
    a = np.ascontiguousarray(indices, dtype=np.uint32)
    hits = ctypes.c_uint64()
    _check(lib.gp_simulate_parallel_cache(a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), a.size, num_sms,
                                          concurrent, capacity_entries, threads, ctypes.byref(hits)))
    return hits.value


def gp_random_walk(activity, pos, scratch, counters, steps, seed, variant="hash", first_step=0, batch_agents=0,
                   threads=0, stream=None):
    """gp_random_walk: ``activity`` uint32/int32 CUDA tensor [height, width];
    ``pos``/``scratch`` uint32/int32 CUDA tensors [num_agents] (pos is updated
    in place); ``counters`` int64 CUDA tensor [3] (accumulated)."""
    for t in (activity, pos, scratch, counters):
        assert t.is_cuda and t.is_contiguous()
    assert activity.element_size() == 4 and pos.element_size() == 4 and counters.element_size() == 8
    h, w = activity.shape
    d = gp_walk_desc(activity.data_ptr(), pos.data_ptr(), scratch.data_ptr(), counters.data_ptr(),
                     _stream_handle(stream), seed, w, h, pos.numel(), VARIANTS.get(variant, variant), first_step,
                     steps, batch_agents, threads)
    _check(lib.gp_random_walk(ctypes.byref(d)))


def gp_loop_adjacency(indices, num_vertices):
    """gp_loop_adjacency on host arrays: returns (ring_offsets, ring,
    opposite, vertex_flags) as uint32 numpy arrays."""
    idx = np.ascontiguousarray(indices, dtype=np.uint32)
    off = np.zeros(num_vertices + 1, dtype=np.uint32)
    opp = np.zeros(max(idx.size, 1), dtype=np.uint32)
    flags = np.zeros(max(num_vertices, 1), dtype=np.uint32)
    cnt = ctypes.c_uint64()
    _check(lib.gp_loop_adjacency(idx.ctypes.data, idx.size, num_vertices, off.ctypes.data, None, 0,
                                 opp.ctypes.data, flags.ctypes.data, ctypes.byref(cnt)))
    ring = np.zeros(max(cnt.value, 1), dtype=np.uint32)
    _check(lib.gp_loop_adjacency(idx.ctypes.data, idx.size, num_vertices, off.ctypes.data, ring.ctypes.data,
                                 ring.size, opp.ctypes.data, flags.ctypes.data, ctypes.byref(cnt)))
    return off, ring[:cnt.value], opp[:idx.size], flags[:num_vertices]


def gp_loop_subdivide(indices, vertices, adjacency, out, counters, variant="hash", batch_indices=0, starts=None,
                      num_batches=None, max_batches=0, max_batch_indices=0, max_unique=0, threads=0, stream=None):
    """gp_loop_subdivide: ``adjacency`` = (ring_offsets, ring, opposite,
    vertex_flags) as CUDA tensors; ``out`` float32 CUDA tensor of T*36
    floats; ``counters`` int64 CUDA tensor [3]; dynamic batches: ``starts``
    and ``num_batches`` (CUDA tensors from a partition) with their limits."""
    off, ring, opp, flags = adjacency
    d = gp_loop_desc(indices.data_ptr(), vertices.data_ptr(), off.data_ptr(), ring.data_ptr(), flags.data_ptr(),
                     opp.data_ptr(), out.data_ptr(), None if starts is None else starts.data_ptr(),
                     None if num_batches is None else num_batches.data_ptr(), counters.data_ptr(),
                     _stream_handle(stream), indices.numel(), vertices.shape[0], ring.numel(),
                     vertices.shape[1] * vertices.element_size(), VARIANTS.get(variant, variant), batch_indices,
                     max_batch_indices, max_unique, max_batches, threads)
    _check(lib.gp_loop_subdivide(ctypes.byref(d)))


def gp_out_floats(shader_id: int) -> int:
    return lib.gp_out_floats(shader_id)


def gp_static_batch_count(ctx, num_indices: int) -> int:
    return lib.gp_static_batch_count(ctx, num_indices)


# ---------------------------------------------------------------------------
# uniform blobs
# ---------------------------------------------------------------------------

def _fill(arr, values):
    v = np.ascontiguousarray(np.asarray(values, dtype=np.float32).reshape(-1))
    assert v.size == len(arr), (v.size, len(arr))
    ctypes.memmove(arr, v.ctypes.data, v.nbytes)


def uniforms_mvp(M, N) -> gp_uniforms_mvp:
    u = gp_uniforms_mvp()
    _fill(u.mvp, M)
    _fill(u.normal, N)
    return u


def uniforms_skin(M, N, palette) -> gp_uniforms_skin:
    u = gp_uniforms_skin()
    _fill(u.mvp, M)
    _fill(u.normal, N)
    _fill(u.palette, palette)
    return u


def uniforms_envelope(d, dirs) -> gp_uniforms_envelope:
    u = gp_uniforms_envelope()
    dirs = np.asarray(dirs, dtype=np.float32).reshape(-1, 3)
    u.d = float(d)
    u.num_dirs = dirs.shape[0]
    full = np.zeros((16, 3), np.float32)
    full[: dirs.shape[0]] = dirs
    _fill(u.dirs, full)
    return u


def uniforms_load(M, N, steps) -> gp_uniforms_load:
    u = gp_uniforms_load()
    _fill(u.mvp, M)
    _fill(u.normal, N)
    u.steps = int(steps)
    return u


class Context:
    """Owns a gp_ctx handle (``with Context(...) as c:``)."""

    def __init__(self, variant="hash", **kw):
        self.handle = gp_create(variant, **kw)

    def close(self):
        if self.handle:
            gp_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
