/*
 * gp.h -- C ABI of a GB300 (sm_103a) software geometry stage with batch-based
 * on-the-fly vertex reuse (Kenzel et al., "On-the-fly Vertex Reuse for
 * Massively-Parallel Software Geometry Processing").
 *
 * The stage is given an index stream and a vertex buffer (Section 4.2).  The
 * index stream is cut into batches, each handled by one thread group
 * (Section 3.2): static batches of a fixed number of indices (Section 3.3)
 * or dynamic batches formed by a load-time scan (Section 3.4).  Inside a batch
 * the unique vertex indices are found by warp voting (Algorithm 1), sorting
 * (Algorithm 2), hashing (Algorithm 3) or two-tier parallel hashing
 * (Section 3.4); each unique vertex is shaded once and triangles are
 * assembled from the shared results.  The naive method (Section 3.3) shades
 * every corner.
 *
 * Conventions for every entry point:
 *  - All calls return a gp_status and never abort the process.
 *  - Buffers named d_* are device pointers owned by the caller; they must
 *    stay valid until gp_sync has covered the ticket of the draw that uses
 *    them.  Host pointers are read before the call returns unless stated.
 *  - Work is enqueued on the context's stream (gp_config.stream, a
 *    cudaStream_t; NULL means the legacy default stream) and runs
 *    asynchronously; errors found on the device are reported by gp_sync.
 *  - A context is internally locked; calls on one context from several host
 *    threads are serialised.
 *  - Index value 0xFFFFFFFF is reserved (it is the empty marker of the
 *    paper's tables) and, like any index >= num_vertices, is an index-range
 *    error: the affected corners are written as zeros and gp_sync returns
 *    GP_ERR_INDEX_RANGE.  Invocation counts of such a draw are unspecified.
 *
 * Output layout: triangle t, corner k (k = 0,1,2, input order) occupies
 * floats [(3t + k) * K, (3t + k + 1) * K) of d_out, K = gp_out_floats(shader).
 *   K = 7 (MVP, SKIN, LOAD): clip x, y, z, w, normal x, y, z.
 *   K = 8 (ENVELOPE): inner x, y, z, 1, outer x, y, z, 1.
 * The paper's output queue (Section 4.2) is replaced by this positional
 * layout, which is deterministic.
 */
#ifndef GP_H
#define GP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gp_status {
  GP_OK = 0,
  GP_ERR_INVALID = 1,      /* bad argument (null pointer, size, alignment, enum) */
  GP_ERR_OOM = 2,          /* a context-owned allocation failed */
  GP_ERR_CUDA = 3,         /* a CUDA runtime call failed; see gp_last_error */
  GP_ERR_TIMEOUT = 4,      /* gp_sync timed out, or a bounded device wait gave up */
  GP_ERR_BUSY = 5,         /* admission refused: over the memory budget or queue full */
  GP_ERR_INDEX_RANGE = 6,  /* an index was >= num_vertices (or 0xFFFFFFFF) */
  GP_ERR_UNSUPPORTED = 7   /* valid request this build cannot run */
} gp_status;

/* Vertex-reuse method.  GP_NAIVE: Section 3.3 "statically batched naive";
 * GP_WARP: Algorithm 1; GP_SORT: Algorithm 2; GP_HASH: Algorithm 3;
 * GP_PHASH: Section 3.4 parallel hashing; GP_AUTO: chosen per draw by the
 * context's autotune table. */
typedef enum gp_variant {
  GP_NAIVE = 0, GP_WARP = 1, GP_SORT = 2, GP_HASH = 3, GP_PHASH = 4, GP_AUTO = 5
} gp_variant;

/* Section 3.3 (static) and Section 3.4 (dynamic).  GP_WARP and GP_NAIVE are
 * static-only, as in the paper. */
typedef enum gp_batch_mode { GP_BATCH_STATIC = 0, GP_BATCH_DYNAMIC = 1 } gp_batch_mode;

/* Vertex shaders (Section 4.2 "simple" matrix multiplication and synthetic
 * loads; Section 5 skinning/envelope applications).  Uniform blobs below. */
typedef enum gp_shader_id {
  GP_SHADER_MVP = 0, GP_SHADER_SKIN = 1, GP_SHADER_ENVELOPE = 2, GP_SHADER_LOAD = 3
} gp_shader_id;

/* Vertex layouts: PNU32 = 8 floats (pos xyz, normal xyz, uv); SKIN64 = PNU32
 * followed by 4 uint8 bone ids (one 32-bit word), 4 float weights and 12
 * bytes of padding.  The vertex pointer must be 16-byte aligned. */
typedef enum gp_vertex_format { GP_VFMT_PNU32 = 0, GP_VFMT_SKIN64 = 1 } gp_vertex_format;

enum {
  GP_FLAG_NONE = 0,
  GP_SEGMENT_NONE = 0xFFFFFFFFu /* gp_config.segment_tris: one unsegmented scan */
};

typedef struct gp_ctx gp_ctx;

/* Context configuration.  Zero fields take the defaults in brackets. */
typedef struct gp_config {
  int32_t device;             /* CUDA device ordinal */
  int32_t variant;            /* gp_variant (0 = GP_NAIVE) */
  int32_t mode;               /* gp_batch_mode */
  uint32_t batch_indices;     /* static batch size S in indices, a multiple of 3
                                 [warp 96, naive 3*threads, sort/hash/phash 768];
                                 Section 3.3 */
  uint32_t max_unique;        /* dynamic N: unique indices per batch [256]; Section 3.4 */
  uint32_t max_tris;          /* dynamic triangle cap per batch [341 = 1023 indices]; Section 4.1 */
  uint32_t threads_per_group; /* threads per batch for sort/hash/phash [256],
                                 warps per block for warp [2], block size for naive [256] */
  uint32_t probe_k;           /* parallel hash: per-thread probes before the warp
                                 cooperates [4]; Section 3.4 */
  uint32_t hash_slots;        /* hash table slots, a power of two >= unique capacity
                                 [next power of two >= 2 x capacity] */
  uint32_t segment_tris;      /* dynamic partition: also cut at every multiple of this
                                 many triangles [4096]; GP_SEGMENT_NONE = single scan */
  uint32_t flags;             /* reserved, 0 */
  uint64_t mem_budget_bytes;  /* admission budget for resident meshes [0 = unlimited] */
  void* stream;               /* cudaStream_t the context enqueues on */
} gp_config;

typedef struct gp_index_buf {
  const uint32_t* d_indices;  /* 3T indices, triangle list; 16-byte aligned */
  uint64_t num_indices;       /* multiple of 3, < 2^32 */
  uint64_t partition;         /* dynamic mode: handle from gp_partition for exactly
                                 this buffer, or 0 to partition at submit */
} gp_index_buf;

typedef struct gp_vertex_buf {
  const void* d_vertices;     /* num_vertices rows of stride_bytes; 16-byte aligned */
  uint64_t num_vertices;      /* < 2^31 */
  uint32_t stride_bytes;      /* 32 for PNU32, 64 for SKIN64 */
  uint32_t format;            /* gp_vertex_format; must match the shader's needs */
} gp_vertex_buf;

typedef struct gp_out_buf {
  float* d_out;               /* T * 3 * K floats; 16-byte aligned */
  uint64_t capacity_bytes;    /* must be >= T * 3 * K * 4 */
  uint32_t* d_corner_ids;     /* optional (NULL): per output corner, the vertex id
                                 whose shaded result was written there */
  uint32_t* d_batch_invocations; /* optional (NULL): shader invocations per batch */
  uint64_t batch_capacity;    /* entries available in d_batch_invocations */
} gp_out_buf;

/* Uniform blobs (row-major matrices), copied by value at submit. */
typedef struct gp_uniforms_mvp {
  float mvp[16];              /* clip = mvp * (p, 1) */
  float normal[9];            /* n' = normal * n */
} gp_uniforms_mvp;

typedef struct gp_uniforms_skin {
  float mvp[16];
  float normal[9];
  float palette[64 * 12];     /* 64 bones, each a 3x4 [R | t] */
} gp_uniforms_skin;

typedef struct gp_uniforms_envelope {
  float d;                    /* offset distance */
  uint32_t num_dirs;          /* 1..16 */
  float dirs[16 * 3];         /* unit directions a_j */
} gp_uniforms_envelope;

typedef struct gp_uniforms_load {
  float mvp[16];
  float normal[9];
  uint32_t steps;             /* length of the dependent multiply-add chain */
} gp_uniforms_load;

typedef struct gp_stats_t {
  uint64_t draws;             /* completed draws since the last reset */
  uint64_t triangles;         /* triangles assembled */
  uint64_t indices;           /* indices read */
  uint64_t invocations;       /* vertex shader invocations */
  uint64_t batches;           /* batches processed */
  double busy_ms;             /* sum of device time of completed draws */
  double p50_ms, p99_ms;      /* per-draw device time percentiles */
  uint64_t bytes_moved;       /* algorithmic bytes: indices + vertices fetched + output */
  uint32_t last_error;        /* gp_status of the last failed call, or GP_OK */
} gp_stats_t;

/* Creates a context on cfg->device.  Allocates small device scratch (error
 * word, counters).  *out is NULL on failure.  GP_ERR_INVALID on a bad
 * configuration (e.g. batch_indices not a multiple of 3, max_unique < 3). */
gp_status gp_create(const gp_config* cfg, gp_ctx** out);

/* Waits for all work of the context, then frees it and its partitions. */
gp_status gp_destroy(gp_ctx* ctx);

/* Dynamic batching preprocessing (Section 3.4): scans the triangles front to
 * back and starts a new batch when the next triangle would exceed max_unique
 * unique indices or max_tris triangles (and at every multiple of
 * segment_tris).  The batch starts are kept in context-owned device memory
 * under *out_handle.  If out_num_batches is non-NULL the call waits for the
 * scan and reports the batch count.  The index buffer must not change while
 * the handle is used. */
gp_status gp_partition(gp_ctx* ctx, const gp_index_buf* index_buf, uint64_t* out_handle,
                       uint64_t* out_num_batches);

/* Copies the batch starts of a partition (in triangles, count + 1 entries, the
 * last one = T) to device memory d_starts (capacity in entries) and reports
 * the count.  Waits for the partition. */
gp_status gp_partition_starts(gp_ctx* ctx, uint64_t handle, uint32_t* d_starts, uint64_t capacity,
                              uint64_t* out_num_batches);

/* Frees a partition (after the draws that use it have been synced). */
gp_status gp_partition_release(gp_ctx* ctx, uint64_t handle);

/* Enqueues one draw call (Section 4.2: index stream + vertex buffer + shader)
 * with the context's variant and batching.  uniforms points to the blob of
 * shader_id (uniforms_bytes = its sizeof).  *out_ticket identifies the draw
 * for gp_sync.  GP_ERR_INVALID for sizes, alignment, a too-small output or a
 * variant/mode/format the shader cannot use. */
gp_status gp_submit_drawcall(gp_ctx* ctx, const gp_index_buf* index_buf, const gp_vertex_buf* vertex_buf,
                             uint32_t shader_id, const void* uniforms, uint32_t uniforms_bytes,
                             const gp_out_buf* out_tris, uint64_t* out_ticket);

/* Waits up to timeout_ms (0 = no limit) for the draw with this ticket
 * (0 = every submitted draw), folds it into the statistics and reports any
 * device-side error of the draws it covers: GP_ERR_INDEX_RANGE, or
 * GP_ERR_TIMEOUT (host wait expired, or a bounded device wait gave up). */
gp_status gp_sync(gp_ctx* ctx, uint64_t ticket, uint32_t timeout_ms);

/* Reads the statistics of completed draws (syncs the context first).
 * reset != 0 clears them afterwards. */
gp_status gp_stats(gp_ctx* ctx, gp_stats_t* out, int reset);

/* End-to-end draw from HOST memory: copies the indices and vertices to
 * context-owned device buffers, partitions (dynamic mode), draws, copies the
 * output back to out_host (capacity in bytes) and waits.  Pinned host memory
 * gives full copy bandwidth; pageable memory works but is slower. */
gp_status gp_draw_host(gp_ctx* ctx, const uint32_t* indices_host, uint64_t num_indices,
                       const void* vertices_host, uint64_t num_vertices, uint32_t stride_bytes,
                       uint32_t format, uint32_t shader_id, const void* uniforms, uint32_t uniforms_bytes,
                       float* out_host, uint64_t out_capacity_bytes);

/* Dynamic partition without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that must not allocate
 * device memory -- a real-time frame loop, where cudaMalloc can synchronise
 * the device and stall a frame, or an application that owns all device
 * memory through its own pool.  It computes the same batch starts as
 * gp_partition (same rule, same segmentation; segment_tris 0 means 4096) and
 * needs no context.  Its scratch is one fixed 4 MiB array in the library's
 * device memory, held on every GPU that loads the library until the process
 * exits; inputs whose scratch would not fit (about 80 million triangles at
 * the default limits) return GP_ERR_INVALID -- use gp_partition for those.
 *   d_indices      device, num_indices indices, 16-byte aligned (read only)
 *   d_starts       device, receives count + 1 batch starts in triangles; the
 *                  capacity must be at least num_indices / 3 + 1 entries
 *   d_num_batches  device, receives the batch count
 *   stream         cudaStream_t for the work (NULL = legacy default stream)
 * The work is asynchronous on the stream.  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  All calls on a
 * device share the array and it keeps the last call's contents: calls whose
 * work overlaps on the GPU race on it, calls ordered on one stream do not.
 * Returns GP_ERR_INVALID for bad arguments or sizes, GP_ERR_CUDA for a failed
 * CUDA call, GP_OK otherwise; gp_last_error(NULL) then gives the reason on
 * the calling thread.  It calls no cudaMalloc or cudaFree. */
gp_status gp_partition_noalloc(const uint32_t* d_indices, uint64_t num_indices, uint32_t max_unique,
                               uint32_t max_tris, uint32_t segment_tris, uint32_t* d_starts,
                               uint64_t starts_capacity, uint32_t* d_num_batches, void* stream);

/* Floats per output corner for a shader (7 or 8), 0 for an unknown id. */
uint32_t gp_out_floats(uint32_t shader_id);

/* Batches a draw of num_indices indices will use under the context's static
 * configuration (ceil(num_indices / S)); 0 for dynamic mode. */
uint64_t gp_static_batch_count(gp_ctx* ctx, uint64_t num_indices);

/* Human-readable text of the context's last error ("" if none); valid until
 * the next call on the context.  ctx may be NULL for creation errors. */
const char* gp_last_error(gp_ctx* ctx);

/* Name of a status code. */
const char* gp_status_string(gp_status status);

#ifdef __cplusplus
}
#endif

#endif /* GP_H */
