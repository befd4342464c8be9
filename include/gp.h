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
  GP_ERR_UNSUPPORTED = 7   /* a valid request the library cannot run (a capacity or limit) */
} gp_status;

/* Vertex-reuse method.  GP_NAIVE: Section 3.3 "statically batched naive";
 * GP_WARP: Algorithm 1; GP_SORT: Algorithm 2; GP_HASH: Algorithm 3;
 * GP_PHASH: Section 3.4 parallel hashing; GP_AUTO: chosen per draw by the
 * context's autotune table (frames only).  GP_MULTI: the non-streaming
 * multi-kernel comparator of Section 5 (Table 2 "multi"): one kernel shades
 * every vertex of the vertex buffer once into a context-owned buffer
 * (32 bytes per vertex, grown on demand), a second assembles the triangles
 * from it; single draws only, static mode, invocations = num_vertices. */
typedef enum gp_variant {
  GP_NAIVE = 0, GP_WARP = 1, GP_SORT = 2, GP_HASH = 3, GP_PHASH = 4, GP_AUTO = 5, GP_MULTI = 6
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
  uint32_t max_unique;        /* dynamic N: unique indices per batch [256], 3..4096; Section 3.4 */
  uint32_t max_tris;          /* dynamic triangle cap per batch [341 = 1023 indices], 1..1365;
                                 Section 4.1.  On GB300 hash/phash draws are fastest at
                                 max_unique 320, max_tris 426, hash_slots 2048 (one
                                 producer pass of a 256-thread block per batch) */
  uint32_t threads_per_group; /* threads per batch for sort/hash/phash, a power of two
                                 <= 512 [256]; block size for warp voting (one warp per
                                 batch), a multiple of 32 <= 256 [64]; block size for
                                 naive and multi, a multiple of 32 <= 256 [256] */
  uint32_t probe_k;           /* parallel hash: per-thread probes before the warp
                                 cooperates [4]; Section 3.4 */
  uint32_t hash_slots;        /* hash table slots, a power of two >= unique capacity and
                                 <= 32768 [the larger of the next power of two >= 2 x
                                 capacity and of min(next power of two >= 4 x capacity,
                                 1024)] */
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
/* Per-batch debug information.  There is no separate gp_batch_info call: a
 * draw writes the invocations of batch b to d_batch_invocations[b] (device,
 * for b < batch_capacity; sort/hash/phash/warp kernels) when the caller
 * passes that buffer, and the batch boundaries are either static (batch b =
 * triangles [b*S/3, min((b+1)*S/3, T)), S = batch_indices) or those of the
 * dynamic partition, which gp_partition_starts copies out.  Both are final
 * once gp_sync has covered the draw's ticket. */

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
 * output back to out_host (capacity in bytes) and waits.  The triangles go in
 * chunks of about 2^20, each a whole number of batches (segments for dynamic
 * mode, static batches, naive blocks), so the batches and the output are
 * those of one draw; each chunk's upload, draw and read-back overlap those of
 * its neighbours on separate streams, and each chunk counts as one draw in
 * gp_stats.  GP_MULTI and the unsegmented partition run as one chunk.
 * Pinned host memory gives full copy bandwidth; pageable memory works but is
 * slower. */
gp_status gp_draw_host(gp_ctx* ctx, const uint32_t* indices_host, uint64_t num_indices,
                       const void* vertices_host, uint64_t num_vertices, uint32_t stride_bytes,
                       uint32_t format, uint32_t shader_id, const void* uniforms, uint32_t uniforms_bytes,
                       float* out_host, uint64_t out_capacity_bytes);

/* ---------------------------------------------------------------------------
 * Frames: many draw calls in one persistent launch.
 *
 * The draws of a frame are fused into one persistent kernel launch, replayed
 * from a captured CUDA graph.  Each draw keeps its own method, batch size and
 * threads per group; GP_AUTO takes them from the context's autotune table
 * (gp_autotune).  The batches of every draw are handled exactly as in a
 * single draw of that configuration (Sections 3.3-3.4), so each draw's
 * output is the same as its single-draw output.
 * ------------------------------------------------------------------------- */

/* One draw of a frame.  Buffers follow the single-draw rules (gp_index_buf's
 * partition field is ignored: the frame partitions its dynamic draws when it
 * is created). */
typedef struct gp_draw_desc {
  gp_index_buf index_buf;
  gp_vertex_buf vertex_buf;
  gp_out_buf out;
  uint32_t shader_id;
  uint32_t uniforms_bytes;
  const void* uniforms;
  int32_t variant;            /* GP_NAIVE..GP_PHASH, or GP_AUTO (autotune table) */
  int32_t mode;               /* gp_batch_mode for sort/hash/phash */
  uint32_t batch_indices;     /* static S [warp 96, sort/hash/phash 255] */
  uint32_t max_unique;        /* dynamic N [256] */
  uint32_t max_tris;          /* dynamic triangle cap [floor((4N - 1) / 3)] */
  uint32_t threads_per_group; /* sort/hash/phash: 64, 128 or 256 [256]; 256 runs the draw's batches in runs
                                 through the two-stage pipeline of the single-draw kernel.  A batch must fit
                                 64 KB of shared memory per block (else GP_ERR_UNSUPPORTED at frame creation) */
} gp_draw_desc;

/* The configuration a frame draw runs with (after GP_AUTO is resolved). */
typedef struct gp_draw_config {
  int32_t variant;
  int32_t mode;
  uint32_t batch_indices;
  uint32_t max_unique;
  uint32_t max_tris;
  uint32_t threads_per_group;
  uint64_t batches;           /* batches of the draw in this frame */
} gp_draw_config;

/* One row of the autotune table: draws with this shader and a triangle count
 * in [tris_lo, tris_hi) run with 'config' (its 'batches' field unused). */
typedef struct gp_autotune_entry {
  uint32_t shader_id;
  uint32_t tris_lo, tris_hi;
  uint32_t pad;
  gp_draw_config config;
  double us_per_draw;         /* measured time of the winning configuration */
} gp_autotune_entry;

typedef struct gp_frame gp_frame;

/* Builds a frame: validates every draw, resolves GP_AUTO, partitions the
 * dynamic draws (load-time preprocessing, Section 3.4), uploads the draw
 * table and captures the launch in a CUDA graph.  The buffers and uniforms
 * are referenced (buffers) or copied (uniforms) as in gp_submit_drawcall; the
 * buffers must stay valid for the frame's lifetime.  Waits for the
 * partitions.  GP_ERR_INVALID / GP_ERR_UNSUPPORTED name the first bad draw in
 * gp_last_error. */
gp_status gp_frame_create(gp_ctx* ctx, const gp_draw_desc* draws, uint32_t num_draws, gp_frame** out);

/* Launches the frame on the context's stream (a graph launch).  The ticket
 * works with gp_sync and gp_stats like a draw's; its statistics count every
 * draw of the frame.  A frame's previous launch is waited for first. */
gp_status gp_frame_submit(gp_frame* frame, uint64_t* out_ticket);

/* Replaces one draw's uniforms (copied, ordered before the next launch). */
gp_status gp_frame_set_uniforms(gp_frame* frame, uint32_t draw, const void* uniforms, uint32_t uniforms_bytes);

/* The configuration draw 'draw' runs with. */
gp_status gp_frame_draw_config(gp_frame* frame, uint32_t draw, gp_draw_config* out);

/* Waits for the frame's last launch and frees it. */
gp_status gp_frame_destroy(gp_frame* frame);

/* Autotuner: groups the sample draws by shader and power-of-two triangle
 * count, times candidate configurations (method; static batch size or
 * dynamic unique limit; threads per group) on up to four samples of each
 * group with the frame kernel, 'reps' launches each, and stores the fastest
 * per group in the context's table (replacing rows of the same group).
 * Draws referenced here are read and their outputs overwritten. */
gp_status gp_autotune(gp_ctx* ctx, const gp_draw_desc* samples, uint32_t num_samples, uint32_t reps);

/* Copies the autotune table (count rows; up to capacity are written). */
gp_status gp_autotune_table(gp_ctx* ctx, gp_autotune_entry* out, uint32_t capacity, uint32_t* count);

/* Replaces the autotune table (e.g. one saved from an earlier run). */
gp_status gp_autotune_set_table(gp_ctx* ctx, const gp_autotune_entry* entries, uint32_t count);

/* ---------------------------------------------------------------------------
 * Serving: a persistent request loop with continuous batching.
 *
 * Meshes are registered once (host copies); a mesh is made resident on the
 * device when a request needs it, within a memory budget, and the least
 * recently used meshes without active requests are evicted to make room.
 * Requests (mesh, shader, uniforms, output) queue up; a native server thread
 * admits them as memory and slots free up, and every step launches one
 * persistent kernel over batches taken from all active requests, so requests
 * that arrive while others are on the GPU join the next step.  Batches stay
 * request-local: each request's output is the same as its single draw.  Up
 * to 'streams' steps are in flight on the device at once.  Latency is
 * measured from submission to the completion of the request's last batch.
 * ------------------------------------------------------------------------- */

typedef struct gp_server gp_server;

typedef struct gp_serve_config {
  uint64_t mem_budget_bytes;  /* device bytes for resident meshes [20 GiB] */
  uint32_t streams;           /* steps in flight at once [2] */
  uint32_t step_max_batches;  /* batches per step [32768]: small steps under load leave the device underused */
  uint32_t max_active;        /* requests admitted at once [4096] */
  int32_t variant;            /* method for every request: GP_NAIVE..GP_PHASH or GP_AUTO [GP_HASH] */
  int32_t mode;               /* gp_batch_mode (sort/hash/phash) [GP_BATCH_DYNAMIC] */
  uint32_t batch_indices;     /* as in gp_draw_desc */
  uint32_t max_unique;
  uint32_t max_tris;
  uint32_t threads_per_group;
} gp_serve_config;

typedef struct gp_serve_stats {
  uint64_t submitted, completed;
  uint64_t triangles, invocations, steps;
  uint64_t uploads, evictions, resident_bytes;
  double p50_ms, p99_ms, max_ms; /* request latency */
  double busy_ms;                /* summed device time of the steps */
  double wall_ms;                /* first submission to last completion */
  uint32_t last_error;           /* gp_status of the last failed step, or GP_OK */
  uint32_t pad;
  double device_ms;              /* union of the steps' device intervals: time with >= 1 step in flight */
} gp_serve_stats;

/* Starts a server (and its thread) on the context's device.  The context
 * must outlive the server.  GP_ERR_INVALID for a malformed configuration
 * (threads_per_group of sort/hash/phash other than 64, 128 or 256);
 * GP_ERR_UNSUPPORTED when a batch of the configuration does not fit the
 * frame kernel's shared memory. */
gp_status gp_server_create(gp_ctx* ctx, const gp_serve_config* cfg, gp_server** out);

/* Registers a mesh: the host buffers are copied; the mesh is uploaded on
 * first use.  Returns its id in *out_mesh. */
gp_status gp_server_add_mesh(gp_server* server, const uint32_t* indices_host, uint64_t num_indices,
                             const void* vertices_host, uint64_t num_vertices, uint32_t stride_bytes,
                             uint32_t format, uint64_t* out_mesh);

/* Queues a request: draw 'mesh' with the shader into d_out (device, caller-
 * owned, valid until the request completes).  Uniforms are copied.
 * GP_ERR_BUSY if the mesh alone exceeds the memory budget. */
gp_status gp_server_submit(gp_server* server, uint64_t mesh, uint32_t shader_id, const void* uniforms,
                           uint32_t uniforms_bytes, float* d_out, uint64_t out_capacity_bytes,
                           uint64_t* out_request);

/* Submits n requests at their arrival times (seconds after the call starts)
 * from the calling thread; returns after the last submission.  The request
 * ids go to out_requests (may be NULL). */
gp_status gp_server_replay(gp_server* server, uint32_t n, const double* arrival_s, const uint64_t* meshes,
                           const uint32_t* shader_ids, const void* const* uniforms, const uint32_t* uniforms_bytes,
                           float* const* d_outs, const uint64_t* out_capacity_bytes, uint64_t* out_requests);

/* Waits until request 'request' (0 = every request submitted so far) has
 * completed, up to timeout_ms (0 = no limit).  Returns the request's status. */
gp_status gp_server_wait(gp_server* server, uint64_t request, uint32_t timeout_ms);

/* Latency of a completed request, in ms. */
gp_status gp_server_latency(gp_server* server, uint64_t request, double* out_ms);

/* Statistics of completed requests; reset != 0 clears them afterwards. */
gp_status gp_server_stats(gp_server* server, gp_serve_stats* out, int reset);

/* Waits for all requests, stops the thread and frees device memory. */
gp_status gp_server_destroy(gp_server* server);

/* Failure injection, for testing the error paths without a GPU fault.
 * The paper has no counterpart.  what:
 *   GP_TEST_FAIL_ALLOC    the context's next `count` device allocations
 *                         (partition buffers, host-draw staging, the
 *                         multi-kernel comparator's rows) report an
 *                         exhausted device without allocating; the call that
 *                         needed them returns GP_ERR_OOM and the context
 *                         stays usable;
 *   GP_TEST_STALL_WINDOW  the next `count` sort/hash/phash draws announce
 *                         each block's first index window on its mbarrier
 *                         but never copy it, so the kernel's bounded wait
 *                         runs out (about a second) and the block stops;
 *                         gp_sync reports GP_ERR_TIMEOUT for the draw and
 *                         later draws run normally.
 * count = 0 clears the injection.  GP_ERR_INVALID for an unknown kind or a
 * NULL context. */
enum { GP_TEST_FAIL_ALLOC = 1, GP_TEST_STALL_WINDOW = 2 };
gp_status gp_test_inject(gp_ctx* ctx, uint32_t what, uint32_t count);

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
 * current and keeps it for later calls; make that first call before any
 * stream capture.  The kept address does not survive a device reset: after
 * cudaDeviceReset (or any other reset of the device's primary context) this
 * entry point must not be called again in the same process.  All calls on a
 * device share the array and it keeps the last call's contents: calls whose
 * work overlaps on the GPU race on it, calls ordered on one stream do not.
 * Device-side errors are not reported: the partition kernels' error word
 * lives in the shared array and is not read back.  None can arise here, since
 * the scratch is sized so that every segment's batch-start list has room for
 * its worst case (one batch per min(max_tris, max_unique / 3) triangles).
 * Returns GP_ERR_INVALID for bad arguments or sizes, GP_ERR_CUDA for a failed
 * CUDA call, GP_OK otherwise; gp_last_error(NULL) then gives the reason on
 * the calling thread.  It calls no cudaMalloc or cudaFree. */
gp_status gp_partition_noalloc(const uint32_t* d_indices, uint64_t num_indices, uint32_t max_unique,
                               uint32_t max_tris, uint32_t segment_tris, uint32_t* d_starts,
                               uint64_t starts_capacity, uint32_t* d_num_batches, void* stream);

/* ---------------------------------------------------------------------
 * Cache comparator (host only, no GPU needed)
 * ------------------------------------------------------------------- */

/* The per-multiprocessor LRU vertex cache the paper compares batching with
 * (Section 5.1, Table 1 "Parallel Cache"; 28 multiprocessors, 1024
 * concurrent invocations, 16/32/64 KB in the paper).
 *
 * indices:          HOST pointer to num_indices vertex ids (the index
 *                   buffer); read only.
 * num_sms:          simulated multiprocessors; the buffer is split into
 *                   num_sms contiguous parts of ceil(num_indices / num_sms)
 *                   indices, each worked through in shading cycles of
 *                   `concurrent` consecutive indices.
 * concurrent:       invocations a multiprocessor runs at once.  A duplicate
 *                   index hits only if its vertex was shaded in an EARLIER
 *                   cycle of the same multiprocessor; the ids that miss are
 *                   inserted when their cycle ends, in index order.
 * capacity_entries: cached vertices per multiprocessor (cache bytes / bytes
 *                   per shaded vertex), <= 2^30.
 * threads:          host threads simulating multiprocessors side by side
 *                   (0 = all hardware threads).
 * *hits:            indices served from a cache; reuse = hits / num_indices.
 * Returns GP_ERR_INVALID for a NULL pointer or a zero count. */
gp_status gp_simulate_parallel_cache(const uint32_t* indices, uint64_t num_indices, uint32_t num_sms,
                                     uint32_t concurrent, uint32_t capacity_entries, uint32_t threads,
                                     uint64_t* hits);

/* ---------------------------------------------------------------------
 * Parallel random walk with reuse (Section 5.4)
 * ------------------------------------------------------------------- */

/* Agents on a toroidal width x height grid, each the packed key
 * (x << 16) | y.  Per step every agent evaluates the moves (dx, dy) with
 * 1 <= dx^2 + dy^2 <= 16^2 -- likelihood activity[target] * (65536 / r^2),
 * exact integers -- keeps the 8 largest (on equal likelihoods the earlier
 * move in (dy, dx) row-major order from (-16, -16)), and takes one with
 * probability proportional to its likelihood: u = splitmix64(seed ^
 * ((step << 32) | agent)), the first kept move whose running sum exceeds
 * u mod total (no move if the total is 0).  The kept moves depend only on
 * the cell, so the key is the reuse methods' "index": naive evaluates per
 * agent, warp per unique key of each 32 agents, sort/hash/phash per unique
 * key of each static batch of batch_agents agents. */
typedef struct gp_walk_desc {
  const uint32_t* d_activity;       /* device [height][width] activity, caller-owned */
  uint32_t* d_pos;                  /* device [num_agents] keys; in: positions, out: after `steps` steps */
  uint32_t* d_scratch;              /* device [num_agents], caller-owned scratch */
  unsigned long long* d_counters;   /* device [3]: += cell evaluations, += batches, |= error bits */
  void* stream;                     /* cudaStream_t (NULL = default stream) */
  uint64_t seed;
  uint32_t width, height;           /* 17..32768 */
  uint32_t num_agents;
  int32_t variant;                  /* GP_NAIVE, GP_WARP, GP_SORT, GP_HASH or GP_PHASH */
  uint32_t first_step;              /* step number of the first step (the random numbers use it) */
  uint32_t steps;
  uint32_t batch_agents;            /* agents per batch, a multiple of 32 [576]; <= 1024 for sort/hash/phash */
  uint32_t threads;                 /* sort/hash/phash: threads per block, a power of two <= 512 [256] */
} gp_walk_desc;

/* Enqueues `steps` steps on the stream (asynchronous; the counters and
 * d_pos are final when the stream reaches this point).  Returns
 * GP_ERR_INVALID for bad sizes, pointers or variants, GP_ERR_CUDA if a launch
 * fails. */
gp_status gp_random_walk(const gp_walk_desc* desc);

/* ---------------------------------------------------------------------
 * Loop subdivision with reuse (Section 5.2)
 * ------------------------------------------------------------------- */

/* Adjacency for gp_loop_subdivide, built on the host from HOST arrays:
 *   ring_offsets [num_vertices + 1], ring [ring_capacity]: vertex v's 1-ring
 *     is ring[ring_offsets[v] .. ring_offsets[v+1]): its distinct neighbours
 *     in order of first appearance, or -- for a boundary vertex (an edge
 *     used by one triangle; vertex_flags[v] bit 0 set) -- its two boundary
 *     neighbours (a vertex with more than two is treated as interior);
 *   opposite [num_indices]: for edge (v_k, v_k+1) of triangle t, the third
 *     vertex of the other triangle on that edge, 0xFFFFFFFF on a boundary;
 *   *ring_count: entries the rings need.  ring may be NULL (or too small:
 *     GP_ERR_INVALID) to query the size first.
 * GP_ERR_INDEX_RANGE for an index >= num_vertices. */
gp_status gp_loop_adjacency(const uint32_t* indices, uint64_t num_indices, uint32_t num_vertices,
                            uint32_t* ring_offsets, uint32_t* ring, uint64_t ring_capacity, uint32_t* opposite,
                            uint32_t* vertex_flags, uint64_t* ring_count);

/* One Loop subdivision step, streamed triangle by triangle (Section 5.2, after
 * Loop's thesis).  Triangle t = (v0, v1, v2) yields output triangles
 * 4t..4t+3 = (E0, M0, M2), (E1, M1, M0), (E2, M2, M1), (M0, M1, M2):
 *   E_k = (1 - n beta) v_k + beta * sum of its n ring neighbours, beta =
 *         (5/8 - (3/8 + cos(2 pi / n) / 4)^2) / n; boundary vertices:
 *         3/4 v + 1/8 (b0 + b1);
 *   M_k = 3/8 (v_k + v_k+1) + 1/8 (v_k+2 + opposite vertex); boundary edges:
 *         the midpoint.
 * Positions are the first three floats of each vertex row.  The vertex rule
 * reads a whole ring, so it is what the methods reuse: GP_NAIVE evaluates it
 * per corner; GP_WARP once per vertex of each round of Algorithm 1 (one warp
 * per static batch of batch_indices <= 384 [96]); GP_SORT / GP_HASH /
 * GP_PHASH once per unique vertex of a batch (static batches of
 * batch_indices, or the dynamic batches of a partition passed in d_starts).  All device buffers are caller-owned; the
 * call enqueues on `stream` and returns. */
typedef struct gp_loop_desc {
  const uint32_t* d_indices;         /* [num_indices], 16-byte aligned */
  const void* d_vertices;            /* rows of stride_bytes; position = floats 0..2 */
  const uint32_t* d_ring_offsets;    /* [num_vertices + 1] */
  const uint32_t* d_ring;            /* [ring_count] */
  const uint32_t* d_vertex_flags;    /* [num_vertices] */
  const uint32_t* d_opposite;        /* [num_indices] */
  float* d_out;                      /* [T][4][3][3], 16-byte aligned */
  const uint32_t* d_starts;          /* dynamic batch starts (triangles), or NULL for static batches */
  const uint32_t* d_num_batches;     /* dynamic: device batch count */
  unsigned long long* d_counters;    /* [3]: += vertex-rule evaluations, += batches, |= error bits */
  void* stream;                      /* cudaStream_t */
  uint64_t num_indices, num_vertices, ring_count;
  uint32_t stride_bytes;             /* >= 12, a multiple of 4 */
  int32_t variant;                   /* GP_NAIVE, GP_WARP, GP_SORT, GP_HASH or GP_PHASH */
  uint32_t batch_indices;            /* static: indices per batch, a multiple of 3, <= 4095 [768; warp: 96] */
  uint32_t max_batch_indices;        /* dynamic: 3 x the partition's triangle limit */
  uint32_t max_unique;               /* dynamic: the partition's unique limit [max_batch_indices] */
  uint32_t max_batches;              /* dynamic: the number of batches (or more) */
  uint32_t threads;                  /* sort/hash/phash: threads per block, a power of two <= 512 [256];
                                        warp: a multiple of 32 <= 256 [64] */
} gp_loop_desc;

/* GP_ERR_INVALID for bad sizes, pointers, variants or batch limits. */
gp_status gp_loop_subdivide(const gp_loop_desc* desc);

/* Floats per output corner for a shader (7 or 8), 0 for an unknown id. */
uint32_t gp_out_floats(uint32_t shader_id);

/* Batches a draw of num_indices indices will use under the context's static
 * configuration (ceil(num_indices / S); GP_MULTI: 1 for a non-empty draw);
 * 0 for dynamic mode. */
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
