// C-ABI runtime of the geometry stage: contexts, argument checking, kernel
// selection and sizing, tickets, partitions and statistics.  Every compute
// step runs in the kernels of gp_draw_*.cu and gp_partition.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <cstdio>
#include <cstdlib>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "gp_context.h"

using namespace gp;

namespace {
thread_local std::string g_create_error;
// gp_draw_host: triangles per chunk (rounded to whole batches); uploads,
// draws and read-backs of consecutive chunks overlap.  The host link bounds
// this path; smaller chunks start the read-back earlier but add per-chunk
// partition and launch work (2^18 measured slower than 2^20).
constexpr uint64_t kHostChunkTris = 1u << 20;
}  // namespace

namespace gp {
namespace rt {

uint32_t next_pow2(uint32_t x) {
  uint32_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

uint32_t log2u(uint32_t x) {
  uint32_t b = 0;
  while ((1u << b) < x) ++b;
  return b;
}

const char* status_name(gp_status s) {
  switch (s) {
    case GP_OK: return "GP_OK";
    case GP_ERR_INVALID: return "GP_ERR_INVALID";
    case GP_ERR_OOM: return "GP_ERR_OOM";
    case GP_ERR_CUDA: return "GP_ERR_CUDA";
    case GP_ERR_TIMEOUT: return "GP_ERR_TIMEOUT";
    case GP_ERR_BUSY: return "GP_ERR_BUSY";
    case GP_ERR_INDEX_RANGE: return "GP_ERR_INDEX_RANGE";
    case GP_ERR_UNSUPPORTED: return "GP_ERR_UNSUPPORTED";
  }
  return "GP_ERR_UNKNOWN";
}

}  // namespace rt
}  // namespace gp

void gp::set_thread_error(const char* msg) { g_create_error = msg; }

namespace gp {
namespace rt {

gp_status fail(gp_ctx* c, gp_status s, const std::string& msg) {
  if (c) {
    c->last_status = s;
    c->last_error = std::string(status_name(s)) + ": " + msg;
  } else {
    g_create_error = std::string(status_name(s)) + ": " + msg;
  }
  return s;
}

// Device allocation on behalf of a context; reports an exhausted device
// without allocating while failure injection asks for it (gp_test_inject).
cudaError_t ctx_malloc(gp_ctx* c, void** p, size_t bytes) {
  if (c && c->test_fail_allocs) {
    --c->test_fail_allocs;
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

gp_status cuda_fail(gp_ctx* c, cudaError_t e, const char* what) {
  return fail(c, e == cudaErrorMemoryAllocation ? GP_ERR_OOM : GP_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}


cudaEvent_t get_event(gp_ctx* c) {
  if (!c->events.empty()) {
    cudaEvent_t e = c->events.back();
    c->events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

void put_event(gp_ctx* c, cudaEvent_t e) {
  if (e) c->events.push_back(e);
}

void release_partition(Partition& p) {
  if (p.d_starts) cudaFree(p.d_starts);
  if (p.d_seg) cudaFree(p.d_seg);
  if (p.done) cudaEventDestroy(p.done);
  p = Partition{};
}

// Wait for an event with an optional limit (ms; 0 = none).
gp_status wait_event(gp_ctx* c, cudaEvent_t e, uint32_t timeout_ms) {
  if (timeout_ms == 0) {
    GP_CUDA(c, cudaEventSynchronize(e));
    return GP_OK;
  }
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t q = cudaEventQuery(e);
    if (q == cudaSuccess) return GP_OK;
    if (q != cudaErrorNotReady) return cuda_fail(c, q, "cudaEventQuery");
    const auto ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (ms > timeout_ms) return fail(c, GP_ERR_TIMEOUT, "draw did not complete in time");
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

// Folds completed tickets (front of the queue, up to and including 'upto')
// into the statistics.  Their events must have completed.
gp_status fold(gp_ctx* c, uint64_t upto) {
  gp_status worst = GP_OK;
  if (c->inflight.empty() || c->inflight.front().id > upto) return GP_OK;
  // the records of the folded tickets are consecutive ring slots (maybe wrapping)
  {
    const uint32_t first = c->inflight.front().slot;
    uint64_t n = 0;
    for (const Ticket& t : c->inflight)
      if (t.id <= upto) ++n;
    const uint32_t run1 = (uint32_t)std::min<uint64_t>(n, kRing - first);
    GP_CUDA(c, cudaMemcpyAsync(c->h_rec + first, c->d_rec + first, sizeof(DevRec) * run1, cudaMemcpyDeviceToHost,
                               c->aux));
    if (n > run1)
      GP_CUDA(c, cudaMemcpyAsync(c->h_rec, c->d_rec, sizeof(DevRec) * (n - run1), cudaMemcpyDeviceToHost, c->aux));
    GP_CUDA(c, cudaMemcpyAsync(c->h_rec + kRing, c->d_rec + kRing, sizeof(DevRec), cudaMemcpyDeviceToHost, c->aux));
    GP_CUDA(c, cudaStreamSynchronize(c->aux));
    if (c->h_rec[kRing].err) worst = fail(c, GP_ERR_UNSUPPORTED, "the dynamic partition exceeded a capacity");
  }
  while (!c->inflight.empty() && c->inflight.front().id <= upto) {
    Ticket t = c->inflight.front();
    c->inflight.pop_front();
    DevRec ext{};
    if (t.ext_rec) {  // a frame keeps its own record
      GP_CUDA(c, cudaMemcpyAsync(&c->h_rec[t.slot], t.ext_rec, sizeof(DevRec), cudaMemcpyDeviceToHost, c->aux));
      GP_CUDA(c, cudaStreamSynchronize(c->aux));
      ext = c->h_rec[t.slot];
    }
    const DevRec& r = t.ext_rec ? ext : c->h_rec[t.slot];
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t.ev0, t.ev1);
    put_event(c, t.ev0);
    put_event(c, t.ev1);
    const uint64_t inv = t.device_counts ? r.cnt[CNT_INVOCATIONS] : t.host_inv;
    const uint64_t bat = t.device_counts ? r.cnt[CNT_BATCHES] : t.host_batches;
    c->s_draws += t.draws;
    c->s_tris += t.tris;
    c->s_idx += t.indices;
    c->s_inv += inv;
    c->s_batches += bat;
    c->s_bytes += 4 * t.indices + t.vertex_bytes_per_inv * inv + t.out_bytes;
    c->s_busy += ms;
    c->s_lat.push_back(ms);
    gp_status s = GP_OK;
    if (r.err & EBIT_TIMEOUT) s = fail(c, GP_ERR_TIMEOUT, "a bounded device wait gave up");
    else if (r.err & EBIT_CAPACITY) s = fail(c, GP_ERR_UNSUPPORTED, "a batch exceeded a shared-memory capacity");
    else if (r.err & EBIT_INDEX_RANGE) s = fail(c, GP_ERR_INDEX_RANGE, "index >= num_vertices in a draw");
    if (worst == GP_OK) worst = s;
  }
  return worst;
}

gp_status sync_locked(gp_ctx* c, uint64_t ticket, uint32_t timeout_ms) {
  if (c->inflight.empty()) return GP_OK;
  if (ticket == 0) ticket = c->inflight.back().id;
  // the newest ticket <= 'ticket'
  const Ticket* last = nullptr;
  for (const Ticket& t : c->inflight)
    if (t.id <= ticket) last = &t;
  if (!last) return GP_OK;  // already folded
  gp_status s = wait_event(c, last->ev1, timeout_ms);
  if (s != GP_OK) return s;
  return fold(c, last->id);
}

uint32_t default_batch(const gp_config& cfg) {
  if (cfg.batch_indices) return cfg.batch_indices;
  switch (cfg.variant) {
    case GP_WARP: return 96;
    case GP_NAIVE:
    case GP_MULTI: return 3 * (cfg.threads_per_group ? cfg.threads_per_group : 256);
    default: return 768;
  }
}

gp_status make_uniforms(gp_ctx* c, uint32_t shader, const void* blob, uint32_t bytes, Uniforms& u) {
  std::memset(&u, 0, sizeof(u));
  if (!blob) return fail(c, GP_ERR_INVALID, "uniforms is NULL");
  switch (shader) {
    case GP_SHADER_MVP: {
      if (bytes != sizeof(gp_uniforms_mvp)) return fail(c, GP_ERR_INVALID, "uniforms_bytes != sizeof(gp_uniforms_mvp)");
      const gp_uniforms_mvp* m = static_cast<const gp_uniforms_mvp*>(blob);
      std::memcpy(u.mvp, m->mvp, sizeof(u.mvp));
      std::memcpy(u.nrm, m->normal, sizeof(u.nrm));
      return GP_OK;
    }
    case GP_SHADER_SKIN: {
      if (bytes != sizeof(gp_uniforms_skin)) return fail(c, GP_ERR_INVALID, "uniforms_bytes != sizeof(gp_uniforms_skin)");
      const gp_uniforms_skin* m = static_cast<const gp_uniforms_skin*>(blob);
      std::memcpy(u.mvp, m->mvp, sizeof(u.mvp));
      std::memcpy(u.nrm, m->normal, sizeof(u.nrm));
      std::memcpy(u.palette, m->palette, sizeof(u.palette));
      return GP_OK;
    }
    case GP_SHADER_ENVELOPE: {
      if (bytes != sizeof(gp_uniforms_envelope))
        return fail(c, GP_ERR_INVALID, "uniforms_bytes != sizeof(gp_uniforms_envelope)");
      const gp_uniforms_envelope* m = static_cast<const gp_uniforms_envelope*>(blob);
      if (m->num_dirs < 1 || m->num_dirs > (uint32_t)kMaxEnvelopeDirs)
        return fail(c, GP_ERR_INVALID, "envelope num_dirs must be in 1..16");
      u.d = m->d;
      u.num_dirs = m->num_dirs;
      u.inv_dirs = (float)(1.0 / (double)m->num_dirs);
      std::memcpy(u.dirs, m->dirs, sizeof(u.dirs));
      double f = 1.0;  // k!
      for (int k = 0; k < kEnvelopeTerms; ++k) {
        if (k > 0) f *= (double)k;
        u.coef[k] = (float)(1.0 / f);
      }
      return GP_OK;
    }
    case GP_SHADER_LOAD: {
      if (bytes != sizeof(gp_uniforms_load)) return fail(c, GP_ERR_INVALID, "uniforms_bytes != sizeof(gp_uniforms_load)");
      const gp_uniforms_load* m = static_cast<const gp_uniforms_load*>(blob);
      std::memcpy(u.mvp, m->mvp, sizeof(u.mvp));
      std::memcpy(u.nrm, m->normal, sizeof(u.nrm));
      u.steps = m->steps;
      return GP_OK;
    }
  }
  return fail(c, GP_ERR_INVALID, "unknown shader_id");
}

// Enqueues the partition kernels for 'p' (already sized) on the stream.
gp_status run_partition(gp_ctx* c, Partition& p, const uint32_t* idx, uint64_t num_idx, cudaStream_t stream) {
  PartitionArgs a{};
  a.idx = idx;
  a.num_tris = (uint32_t)(num_idx / 3);
  a.max_unique = p.max_unique;
  a.max_tris = p.max_tris;
  a.segment_tris = p.segment_tris;
  a.num_segments = p.num_segments;
  a.seg_cap = p.seg_cap;
  a.table_slots = next_pow2(2 * (p.max_unique + 96));
  a.table_bits = log2u(a.table_slots);
  a.seg_starts = p.d_seg;
  a.seg_counts = p.d_seg + (size_t)p.num_segments * p.seg_cap;
  a.starts = p.d_starts;
  a.num_batches = p.d_count;
  a.err = &c->d_rec[kRing].err;  // the record after the draw ring collects partition errors
  GP_CUDA(c, launch_partition(a, 4, stream));
  return GP_OK;
}

// Sizes (and allocates if needed) a partition for num_idx indices.
gp_status size_partition(gp_ctx* c, Partition& p, uint64_t num_idx, bool reuse_alloc, uint32_t max_unique,
                         uint32_t max_tris, uint32_t segment_tris) {
  const uint32_t T = (uint32_t)(num_idx / 3);
  const uint32_t nu = max_unique, mt = max_tris;
  const uint32_t seg = segment_tris == GP_SEGMENT_NONE ? std::max(T, 1u) : segment_tris;
  const uint32_t min_tris = std::max(1u, std::min(mt, (nu - 2 + 2) / 3));
  const uint32_t nseg = T ? (T + seg - 1) / seg : 0;
  const uint32_t seg_cap = (std::min(seg, std::max(T, 1u)) + min_tris - 1) / min_tris + 1;
  const uint64_t max_b = (uint64_t)nseg * seg_cap;
  const size_t need_seg = ((size_t)nseg * seg_cap + 2 * (size_t)nseg + 1) * 4;
  const size_t need_starts = (max_b + 2) * 4;
  const bool fits = reuse_alloc && p.d_starts && p.max_batches >= max_b &&
                    (size_t)p.num_segments * p.seg_cap + 2 * (size_t)p.num_segments + 1 >= need_seg / 4;
  if (!fits) {
    if (p.d_starts) cudaFree(p.d_starts);
    if (p.d_seg) cudaFree(p.d_seg);
    p.d_starts = nullptr;
    p.d_seg = nullptr;
    void* ptr = nullptr;
    GP_CUDA(c, ctx_malloc(c, &ptr, need_starts + 16));
    p.d_starts = static_cast<uint32_t*>(ptr);
    GP_CUDA(c, ctx_malloc(c, &ptr, need_seg + 16));
    p.d_seg = static_cast<uint32_t*>(ptr);
    p.max_batches = (uint32_t)max_b;
  }
  p.d_count = p.d_starts + max_b + 1;
  p.num_segments = nseg;
  p.seg_cap = seg_cap;
  p.max_unique = nu;
  p.max_tris = mt;
  p.segment_tris = seg;
  p.num_idx = num_idx;
  return GP_OK;
}

gp_status check_index_buf(gp_ctx* c, const gp_index_buf* ib) {
  if (!ib) return fail(c, GP_ERR_INVALID, "index_buf is NULL");
  if (ib->num_indices % 3) return fail(c, GP_ERR_INVALID, "num_indices is not a multiple of 3");
  if (ib->num_indices >= 0xFFFFFFF0ull) return fail(c, GP_ERR_INVALID, "num_indices must be < 2^32 - 16");
  if (ib->num_indices && !ib->d_indices) return fail(c, GP_ERR_INVALID, "d_indices is NULL");
  if (reinterpret_cast<uintptr_t>(ib->d_indices) % 16)
    return fail(c, GP_ERR_INVALID, "d_indices must be 16-byte aligned");
  return GP_OK;
}

// Enqueues one draw (after validation); fills the ticket's counters.
gp_status enqueue_draw(gp_ctx* c, const gp_index_buf* ib, const gp_vertex_buf* vb, uint32_t shader,
                       const Uniforms& u, const gp_out_buf* ob, Ticket& t, DevRec* rec, Partition* pre) {
  const gp_config& cfg = c->cfg;
  const uint32_t T = (uint32_t)(ib->num_indices / 3);
  DrawArgs a{};
  a.idx = ib->d_indices;
  a.num_idx = (uint32_t)ib->num_indices;
  a.num_tris = T;
  a.verts = static_cast<const unsigned char*>(vb->d_vertices);
  a.num_verts = (uint32_t)vb->num_vertices;
  a.stride = vb->stride_bytes;
  a.vec8 = (reinterpret_cast<uintptr_t>(vb->d_vertices) % 32 == 0 && vb->stride_bytes % 32 == 0) ? 1u : 0u;
  a.out = ob->d_out;
  a.corner_ids = ob->d_corner_ids;
  a.batch_inv = ob->d_batch_invocations;
  a.batch_cap = (uint32_t)std::min<uint64_t>(ob->batch_capacity, 0xFFFFFFFFu);
  a.counters = rec->cnt;
  a.err = &rec->err;
  a.probe_k = cfg.probe_k;
  t.tris = T;
  t.indices = ib->num_indices;
  t.vertex_bytes_per_inv = vb->stride_bytes;
  t.out_bytes = (uint64_t)T * 3 * out_floats((int)shader) * 4;
  if (T == 0) return GP_OK;
  const uint32_t threads = cfg.threads_per_group;

  if (cfg.variant == GP_NAIVE) {
    const int block = threads;
    t.host_inv = 3ull * T;
    t.host_batches = (T + block - 1) / block;
    GP_CUDA(c, launch_naive(a, u, (int)shader, block, c->stream));
    return GP_OK;
  }
  if (cfg.variant == GP_MULTI) {
    const uint64_t V = vb->num_vertices;
    if (V > c->shaded_cap) {  // grow the shaded-row buffer (cudaFree waits for draws still using it)
      if (c->d_shaded) cudaFree(c->d_shaded);
      c->d_shaded = nullptr;
      c->shaded_cap = 0;
      cudaError_t e = ctx_malloc(c, reinterpret_cast<void**>(&c->d_shaded), V * 2 * sizeof(float4));
      if (e != cudaSuccess) return cuda_fail(c, e, "cudaMalloc (shaded vertex rows)");
      c->shaded_cap = V;
    }
    t.host_inv = V;  // every vertex of the buffer is shaded once, referenced or not
    t.host_batches = 1;
    GP_CUDA(c, launch_multi(a, u, (int)shader, c->d_shaded, (int)threads, c->stream));
    return GP_OK;
  }
  if (cfg.variant == GP_WARP) {
    const uint32_t S = default_batch(cfg);
    a.static_batch_tris = S / 3;
    a.num_batches = (T + a.static_batch_tris - 1) / a.static_batch_tris;
    const int wpb = std::max(1u, threads / 32);
    const uint64_t key = (1ull << 40) | ((uint64_t)shader << 32) | (uint64_t)wpb;
    auto it = c->occ.find(key);
    const int bpsm = it != c->occ.end() ? it->second : (c->occ[key] = warp_kernel_blocks_per_sm((int)shader, wpb));
    const uint64_t want = ((uint64_t)a.num_batches + wpb - 1) / wpb;
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)c->sms * bpsm, want));
    if (std::getenv("GP_VERBOSE") && c->logged.insert(key).second)
      std::fprintf(stderr, "[gp] warp shader=%u warps/block=%d blocks/SM=%d grid=%d batch=%u\n", shader, wpb, bpsm,
                   grid, S);
    t.device_counts = true;
    GP_CUDA(c, launch_warp(a, u, (int)shader, wpb, grid, c->stream));
    return GP_OK;
  }
  // sort / hash / phash
  const int dedup = cfg.variant == GP_SORT ? DEDUP_SORT : (cfg.variant == GP_HASH ? DEDUP_HASH : DEDUP_PHASH);
  const bool dyn = cfg.mode == GP_BATCH_DYNAMIC;
  if (dyn) {
    Partition* p = nullptr;
    if (pre) {  // gp_draw_host: the chunk's partition, on its own stream
      p = pre;
      GP_CUDA(c, cudaStreamWaitEvent(c->stream, p->done, 0));
    } else if (ib->partition) {
      auto it = c->parts.find(ib->partition);
      if (it == c->parts.end()) return fail(c, GP_ERR_INVALID, "unknown partition handle");
      p = &it->second;
      if (p->idx != ib->d_indices || p->num_idx != ib->num_indices)
        return fail(c, GP_ERR_INVALID, "partition handle belongs to another index buffer");
    } else {
      p = &c->temp_part;
      gp_status s = size_partition(c, *p, ib->num_indices, true, cfg.max_unique, cfg.max_tris, cfg.segment_tris);
      if (s != GP_OK) return s;
      p->idx = ib->d_indices;
      s = run_partition(c, *p, ib->d_indices, ib->num_indices, c->stream);
      if (s != GP_OK) return s;
    }
    a.starts = p->d_starts;
    a.num_batches_dev = p->d_count;
    a.max_batch_idx = 3 * cfg.max_tris;
    a.ucap = cfg.max_unique;
  } else {
    const uint32_t S = default_batch(cfg);
    a.static_batch_tris = S / 3;
    a.num_batches = (T + a.static_batch_tris - 1) / a.static_batch_tris;
    a.max_batch_idx = S;
    a.ucap = S;
  }
  if (cfg.hash_slots && cfg.hash_slots < a.ucap)
    return fail(c, GP_ERR_INVALID, "hash_slots must be at least the unique-vertex capacity of a batch");
  // default: at least 2x the unique capacity, and 4x up to 1024 slots (fewer
  // collisions, so shorter probe sequences, where the table stays small)
  a.hash_slots = cfg.hash_slots ? cfg.hash_slots : std::max(next_pow2(2 * a.ucap), std::min(next_pow2(4 * a.ucap), 1024u));
  a.hash_slots = std::max(a.hash_slots, next_pow2(threads));
  if (a.hash_slots > 32768u)  // slots are stored in 15 bits
    return fail(c, GP_ERR_UNSUPPORTED, "hash_slots may be at most 32768");
  a.hash_bits = log2u(a.hash_slots);
  a.sort_n = next_pow2(a.max_batch_idx);
  {  // 32-bit sort keys when every id (plus one value for "out of range") fits beside the position
    const uint32_t pb = std::max(1u, log2u(a.sort_n));
    a.sort_pos_bits = (pb < 32 && (uint64_t)a.num_verts + 1 < (1ull << (32 - pb))) ? pb : 0u;
  }
  // the kernel splits its block into producer and consumer warps: at least two warps
  const uint32_t block = std::max(64u, threads);
  const size_t smem = reuse_smem_bytes(dedup, (int)shader, a, (int)block);
  if (smem > 227 * 1024)
    return fail(c, GP_ERR_UNSUPPORTED, "batch configuration needs more than 227 KB of shared memory");
  const uint64_t key = (2ull << 56) | ((uint64_t)dedup << 48) | ((uint64_t)dyn << 47) | ((uint64_t)shader << 40) |
                       ((uint64_t)threads << 24) | (uint64_t)smem;  // smem < 2^24
  int bpsm;
  bool wide = false;
  auto it = c->occ.find(key);
  if (it != c->occ.end()) {
    bpsm = it->second & 0xFF;
    wide = (it->second >> 8) != 0;
  } else {
    bpsm = reuse_blocks_per_sm(dedup, dyn, (int)shader, (int)block, smem, &wide);
    c->occ[key] = bpsm | (wide ? 0x100 : 0);
  }
  if (bpsm <= 0) return fail(c, GP_ERR_UNSUPPORTED, "draw kernel cannot be resident with this configuration");
  uint64_t grid = (uint64_t)c->sms * bpsm;
  if (!dyn) grid = std::min<uint64_t>(grid, a.num_batches);
  if (std::getenv("GP_VERBOSE") && c->logged.insert(key).second)
    std::fprintf(stderr, "[gp] reuse dedup=%d dyn=%d shader=%u threads=%u smem=%zu blocks/SM=%d grid=%llu slots=%u regs=%d\n",
                 dedup, (int)dyn, shader, block, smem, bpsm, (unsigned long long)grid, a.hash_slots, wide ? 80 : 64);
  if (c->test_stall_draws) {  // failure injection: this draw's bounded window wait runs out
    --c->test_stall_draws;
    a.test_stall = 1;
  }
  t.device_counts = true;
  GP_CUDA(c, launch_reuse(dedup, dyn, wide, a, u, (int)shader, (int)block, (int)std::max<uint64_t>(grid, 1), smem,
                          c->stream));
  return GP_OK;
}

gp_status check_draw(gp_ctx* c, const gp_index_buf* ib, const gp_vertex_buf* vb, uint32_t shader,
                     const gp_out_buf* ob) {
  gp_status s = check_index_buf(c, ib);
  if (s != GP_OK) return s;
  if (!vb || !ob) return fail(c, GP_ERR_INVALID, "vertex_buf or out_tris is NULL");
  if (shader > GP_SHADER_LOAD) return fail(c, GP_ERR_INVALID, "unknown shader_id");
  if (vb->num_vertices >= 0x80000000ull) return fail(c, GP_ERR_INVALID, "num_vertices must be < 2^31");
  const uint32_t need_stride = shader == GP_SHADER_SKIN ? 64 : 32;
  const uint32_t need_fmt = shader == GP_SHADER_SKIN ? GP_VFMT_SKIN64 : vb->format;
  if (vb->format != GP_VFMT_PNU32 && vb->format != GP_VFMT_SKIN64)
    return fail(c, GP_ERR_INVALID, "unknown vertex format");
  if (vb->format != need_fmt) return fail(c, GP_ERR_INVALID, "the skinning shader needs GP_VFMT_SKIN64 vertices");
  if (vb->stride_bytes < need_stride || vb->stride_bytes % 16)
    return fail(c, GP_ERR_INVALID, "stride_bytes too small for the format or not a multiple of 16");
  if (vb->num_vertices && (!vb->d_vertices || reinterpret_cast<uintptr_t>(vb->d_vertices) % 16))
    return fail(c, GP_ERR_INVALID, "d_vertices NULL or not 16-byte aligned");
  const uint64_t T = ib->num_indices / 3;
  const uint64_t need = T * 3 * out_floats((int)shader) * 4;
  if (T && (!ob->d_out || reinterpret_cast<uintptr_t>(ob->d_out) % 16))
    return fail(c, GP_ERR_INVALID, "d_out NULL or not 16-byte aligned");
  if (ob->capacity_bytes < need) return fail(c, GP_ERR_INVALID, "out_tris capacity_bytes too small");
  return GP_OK;
}

gp_status new_ticket(gp_ctx* c, Ticket& t) {
  // a free device record: fold the oldest draw if the ring is full
  if (c->inflight.size() >= kRing) {
    gp_status s = sync_locked(c, c->inflight.front().id, 0);
    if (s != GP_OK && s != GP_ERR_INDEX_RANGE) return s;
  }
  t.id = c->next_ticket++;
  t.slot = (uint32_t)(t.id % kRing);
  t.ev0 = get_event(c);
  t.ev1 = get_event(c);
  if (!t.ev0 || !t.ev1) {
    put_event(c, t.ev0);
    put_event(c, t.ev1);
    return fail(c, GP_ERR_CUDA, "cudaEventCreate failed");
  }
  return GP_OK;
}

gp_status submit_locked(gp_ctx* c, const gp_index_buf* ib, const gp_vertex_buf* vb, uint32_t shader,
                        const void* uniforms, uint32_t ubytes, const gp_out_buf* ob, uint64_t* out_ticket,
                        Partition* pre) {
  gp_status s = check_draw(c, ib, vb, shader, ob);
  if (s != GP_OK) return s;
  Uniforms u;
  s = make_uniforms(c, shader, uniforms, ubytes, u);
  if (s != GP_OK) return s;
  Ticket t;
  s = new_ticket(c, t);
  if (s != GP_OK) return s;
  DevRec* rec = c->d_rec + t.slot;
  GP_CUDA(c, cudaEventRecord(t.ev0, c->stream));
  GP_CUDA(c, cudaMemsetAsync(rec, 0, sizeof(DevRec), c->stream));
  s = enqueue_draw(c, ib, vb, shader, u, ob, t, rec, pre);
  if (s != GP_OK) {
    put_event(c, t.ev0);
    put_event(c, t.ev1);
    return s;
  }
  GP_CUDA(c, cudaEventRecord(t.ev1, c->stream));
  c->inflight.push_back(t);
  if (out_ticket) *out_ticket = t.id;
  return GP_OK;
}

gp_status ensure_buf(gp_ctx* c, void** p, size_t* cap, size_t need) {
  if (*cap >= need && *p) return GP_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  GP_CUDA(c, ctx_malloc(c, p, std::max<size_t>(need, 256)));
  *cap = std::max<size_t>(need, 256);
  return GP_OK;
}

}  // namespace rt
}  // namespace gp

using namespace gp::rt;

extern "C" {

gp_status gp_create(const gp_config* cfg_in, gp_ctx** out) {
  if (!out) return fail(nullptr, GP_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!cfg_in) return fail(nullptr, GP_ERR_INVALID, "cfg is NULL");
  gp_config cfg = *cfg_in;
  if ((cfg.variant < GP_NAIVE || cfg.variant > GP_PHASH) && cfg.variant != GP_MULTI)
    return fail(nullptr, cfg.variant == GP_AUTO ? GP_ERR_UNSUPPORTED : GP_ERR_INVALID,
                "variant must be GP_NAIVE..GP_PHASH or GP_MULTI for a single-draw context");
  if (cfg.mode != GP_BATCH_STATIC && cfg.mode != GP_BATCH_DYNAMIC) return fail(nullptr, GP_ERR_INVALID, "bad mode");
  if (!cfg.max_unique) cfg.max_unique = 256;
  if (!cfg.max_tris) cfg.max_tris = 341;
  if (!cfg.probe_k) cfg.probe_k = 4;
  if (!cfg.segment_tris) cfg.segment_tris = 4096;
  if (!cfg.threads_per_group) cfg.threads_per_group = cfg.variant == GP_WARP ? 64 : 256;
  cfg.batch_indices = default_batch(cfg);
  const uint32_t th = cfg.threads_per_group;
  if (th % 32 || th == 0) return fail(nullptr, GP_ERR_INVALID, "threads_per_group must be a multiple of 32");
  if (cfg.variant == GP_NAIVE || cfg.variant == GP_WARP || cfg.variant == GP_MULTI) {
    if (th > 256) return fail(nullptr, GP_ERR_INVALID, "naive/warp/multi blocks are at most 256 threads");
  } else if ((th & (th - 1)) || th > 512) {
    return fail(nullptr, GP_ERR_INVALID, "sort/hash/phash threads_per_group must be a power of two <= 512");
  }
  if (cfg.batch_indices % 3) return fail(nullptr, GP_ERR_INVALID, "batch_indices must be a multiple of 3");
  if (cfg.mode == GP_BATCH_DYNAMIC && (cfg.variant == GP_NAIVE || cfg.variant == GP_WARP || cfg.variant == GP_MULTI))
    return fail(nullptr, GP_ERR_INVALID, "naive, warp voting and multi-kernel use static batches");
  if (cfg.variant == GP_WARP && cfg.batch_indices > 384)
    return fail(nullptr, GP_ERR_INVALID, "warp voting batches are at most 384 indices");
  if (cfg.variant >= GP_SORT && cfg.variant <= GP_PHASH && cfg.mode == GP_BATCH_STATIC && cfg.batch_indices > 4095)
    return fail(nullptr, GP_ERR_INVALID, "static batches are at most 4095 indices");
  if (cfg.max_unique < 3 || cfg.max_unique > 4096) return fail(nullptr, GP_ERR_INVALID, "max_unique must be in 3..4096");
  if (cfg.max_tris < 1 || cfg.max_tris > 1365) return fail(nullptr, GP_ERR_INVALID, "max_tris must be in 1..1365");
  if (cfg.hash_slots && (cfg.hash_slots & (cfg.hash_slots - 1)))
    return fail(nullptr, GP_ERR_INVALID, "hash_slots must be a power of two");
  if (cfg.variant == GP_NAIVE && cfg.batch_indices != 3 * th)
    return fail(nullptr, GP_ERR_INVALID, "naive batch_indices is 3 x threads_per_group");

  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0)
    return fail(nullptr, GP_ERR_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
  if (cfg.device < 0 || cfg.device >= ndev) return fail(nullptr, GP_ERR_INVALID, "bad device ordinal");
  e = cudaSetDevice(cfg.device);
  if (e != cudaSuccess) return fail(nullptr, GP_ERR_CUDA, cudaGetErrorString(e));
  gp_ctx* c = new gp_ctx();
  c->cfg = cfg;
  c->device = cfg.device;
  c->stream = static_cast<cudaStream_t>(cfg.stream);
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, cfg.device);
  if ((e = cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaMalloc(&c->d_rec, sizeof(DevRec) * (kRing + 1))) != cudaSuccess ||
      (e = cudaMallocHost(&c->h_rec, sizeof(DevRec) * (kRing + 1))) != cudaSuccess ||
      (e = cudaMemset(c->d_rec, 0, sizeof(DevRec) * (kRing + 1))) != cudaSuccess) {
    gp_status s = fail(nullptr, e == cudaErrorMemoryAllocation ? GP_ERR_OOM : GP_ERR_CUDA, cudaGetErrorString(e));
    gp_destroy(c);
    return s;
  }
  *out = c;
  return GP_OK;
}

gp_status gp_destroy(gp_ctx* c) {
  if (!c) return GP_ERR_INVALID;
  {
    std::lock_guard<std::mutex> lk(c->mu);
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    for (Ticket& t : c->inflight) {
      put_event(c, t.ev0);
      put_event(c, t.ev1);
    }
    c->inflight.clear();
    for (auto& kv : c->parts) release_partition(kv.second);
    release_partition(c->temp_part);
    for (Partition& p : c->host_parts) release_partition(p);
    for (cudaEvent_t e : c->events) cudaEventDestroy(e);
    if (c->d_rec) cudaFree(c->d_rec);
    if (c->h_rec) cudaFreeHost(c->h_rec);
    if (c->h_idx) cudaFree(c->h_idx);
    if (c->h_vtx) cudaFree(c->h_vtx);
    if (c->h_out) cudaFree(c->h_out);
    if (c->d_shaded) cudaFree(c->d_shaded);
    if (c->copy_in) cudaStreamDestroy(c->copy_in);
    if (c->copy_out) cudaStreamDestroy(c->copy_out);
    if (c->part_stream) cudaStreamDestroy(c->part_stream);
    if (c->aux) cudaStreamDestroy(c->aux);
  }
  delete c;
  return GP_OK;
}

gp_status gp_partition(gp_ctx* c, const gp_index_buf* ib, uint64_t* out_handle, uint64_t* out_num_batches) {
  if (!c) return GP_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  if (!out_handle) return fail(c, GP_ERR_INVALID, "out_handle is NULL");
  gp_status s = check_index_buf(c, ib);
  if (s != GP_OK) return s;
  Partition p;
  s = size_partition(c, p, ib->num_indices, false, c->cfg.max_unique, c->cfg.max_tris, c->cfg.segment_tris);
  if (s != GP_OK) {
    release_partition(p);
    return s;
  }
  p.idx = ib->d_indices;
  s = run_partition(c, p, ib->d_indices, ib->num_indices, c->stream);
  if (s != GP_OK) {
    release_partition(p);
    return s;
  }
  if (cudaEventCreateWithFlags(&p.done, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventRecord(p.done, c->stream) != cudaSuccess) {
    release_partition(p);
    return fail(c, GP_ERR_CUDA, "event for the partition");
  }
  const uint64_t h = c->next_part++;
  c->parts[h] = p;
  *out_handle = h;
  if (out_num_batches) {
    Partition& q = c->parts[h];
    GP_CUDA(c, cudaEventSynchronize(q.done));
    uint32_t cnt = 0;
    GP_CUDA(c, cudaMemcpy(&cnt, q.d_count, 4, cudaMemcpyDeviceToHost));
    q.count = cnt;
    q.count_known = true;
    *out_num_batches = cnt;
  }
  return GP_OK;
}

gp_status gp_partition_starts(gp_ctx* c, uint64_t handle, uint32_t* d_starts, uint64_t capacity,
                              uint64_t* out_num_batches) {
  if (!c) return GP_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  auto it = c->parts.find(handle);
  if (it == c->parts.end()) return fail(c, GP_ERR_INVALID, "unknown partition handle");
  Partition& p = it->second;
  GP_CUDA(c, cudaEventSynchronize(p.done));
  uint32_t cnt = 0;
  GP_CUDA(c, cudaMemcpy(&cnt, p.d_count, 4, cudaMemcpyDeviceToHost));
  p.count = cnt;
  p.count_known = true;
  if (out_num_batches) *out_num_batches = cnt;
  if (d_starts) {
    if (capacity < (uint64_t)cnt + 1) return fail(c, GP_ERR_INVALID, "capacity < batches + 1");
    GP_CUDA(c, cudaMemcpy(d_starts, p.d_starts, ((size_t)cnt + 1) * 4, cudaMemcpyDeviceToDevice));
  }
  return GP_OK;
}

gp_status gp_partition_release(gp_ctx* c, uint64_t handle) {
  if (!c) return GP_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  auto it = c->parts.find(handle);
  if (it == c->parts.end()) return fail(c, GP_ERR_INVALID, "unknown partition handle");
  cudaEventSynchronize(it->second.done);
  cudaStreamSynchronize(c->stream);  // draws that read the starts are done
  release_partition(it->second);
  c->parts.erase(it);
  return GP_OK;
}

gp_status gp_submit_drawcall(gp_ctx* c, const gp_index_buf* ib, const gp_vertex_buf* vb, uint32_t shader_id,
                             const void* uniforms, uint32_t uniforms_bytes, const gp_out_buf* out_tris,
                             uint64_t* out_ticket) {
  if (!c) return GP_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  return submit_locked(c, ib, vb, shader_id, uniforms, uniforms_bytes, out_tris, out_ticket, nullptr);
}

gp_status gp_sync(gp_ctx* c, uint64_t ticket, uint32_t timeout_ms) {
  if (!c) return GP_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  return sync_locked(c, ticket, timeout_ms);
}

gp_status gp_test_inject(gp_ctx* c, uint32_t what, uint32_t count) {
  if (!c) return fail(nullptr, GP_ERR_INVALID, "gp_test_inject: ctx is NULL");
  std::lock_guard<std::mutex> lk(c->mu);
  switch (what) {
    case GP_TEST_FAIL_ALLOC: c->test_fail_allocs = count; return GP_OK;
    case GP_TEST_STALL_WINDOW: c->test_stall_draws = count; return GP_OK;
    default: return fail(c, GP_ERR_INVALID, "gp_test_inject: unknown failure kind");
  }
}

gp_status gp_stats(gp_ctx* c, gp_stats_t* out, int reset) {
  if (!c || !out) return GP_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  gp_status s = sync_locked(c, 0, 0);
  std::memset(out, 0, sizeof(*out));
  out->draws = c->s_draws;
  out->triangles = c->s_tris;
  out->indices = c->s_idx;
  out->invocations = c->s_inv;
  out->batches = c->s_batches;
  out->busy_ms = c->s_busy;
  out->bytes_moved = c->s_bytes;
  out->last_error = (uint32_t)c->last_status;
  if (!c->s_lat.empty()) {
    std::vector<float> v = c->s_lat;
    std::sort(v.begin(), v.end());
    auto pct = [&](double q) {
      const size_t i = (size_t)std::min<double>(v.size() - 1, std::ceil(q * v.size()) - 1);
      return (double)v[i];
    };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
  }
  if (reset) {
    c->s_draws = c->s_tris = c->s_idx = c->s_inv = c->s_batches = c->s_bytes = 0;
    c->s_busy = 0.0;
    c->s_lat.clear();
    c->last_status = GP_OK;
    c->last_error.clear();
  }
  return s == GP_ERR_INDEX_RANGE ? GP_OK : s;
}

gp_status gp_draw_host(gp_ctx* c, const uint32_t* indices_host, uint64_t num_indices, const void* vertices_host,
                       uint64_t num_vertices, uint32_t stride_bytes, uint32_t format, uint32_t shader_id,
                       const void* uniforms, uint32_t uniforms_bytes, float* out_host, uint64_t out_capacity_bytes) {
  if (!c) return GP_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  if ((num_indices && !indices_host) || (num_vertices && !vertices_host) || (num_indices && !out_host))
    return fail(c, GP_ERR_INVALID, "NULL host buffer");
  if (shader_id > GP_SHADER_LOAD) return fail(c, GP_ERR_INVALID, "unknown shader_id");
  if (num_indices % 3) return fail(c, GP_ERR_INVALID, "num_indices is not a multiple of 3");
  const uint64_t T = num_indices / 3;
  const uint32_t K = (uint32_t)out_floats((int)shader_id);
  const size_t out_bytes = (size_t)T * 3 * K * 4;
  if (out_capacity_bytes < out_bytes) return fail(c, GP_ERR_INVALID, "out capacity too small");
  gp_status s;
  if ((s = ensure_buf(c, &c->h_idx, &c->h_idx_cap, num_indices * 4)) != GP_OK) return s;
  if ((s = ensure_buf(c, &c->h_vtx, &c->h_vtx_cap, num_vertices * stride_bytes)) != GP_OK) return s;
  if ((s = ensure_buf(c, &c->h_out, &c->h_out_cap, out_bytes)) != GP_OK) return s;
  if (!c->copy_in) GP_CUDA(c, cudaStreamCreateWithFlags(&c->copy_in, cudaStreamNonBlocking));
  if (!c->copy_out) GP_CUDA(c, cudaStreamCreateWithFlags(&c->copy_out, cudaStreamNonBlocking));

  // Chunks of whole batches, so that each chunk's batches are exactly those of
  // the whole draw: multiples of the segment (dynamic), of the static batch
  // (sort/hash/phash/warp) or of the block (naive).  The multi-kernel
  // comparator and the unsegmented partition run as one chunk.
  const gp_config& cfg = c->cfg;
  uint64_t granule = 0;
  if (cfg.variant == GP_MULTI) granule = 0;
  else if (cfg.mode == GP_BATCH_DYNAMIC) granule = cfg.segment_tris == GP_SEGMENT_NONE ? 0 : cfg.segment_tris;
  else if (cfg.variant == GP_NAIVE) granule = cfg.threads_per_group;
  else granule = default_batch(cfg) / 3;
  uint64_t chunk = T;
  if (granule) chunk = std::max<uint64_t>(1, (kHostChunkTris + granule / 2) / granule) * granule;
  if (chunk == 0) chunk = 1;

  // dynamic batches: one partition per chunk on its own stream, started as
  // soon as the chunk's indices have arrived; the first chunk's indices go up
  // before the vertices, so its partition overlaps the vertex upload
  const bool pre_part = cfg.mode == GP_BATCH_DYNAMIC && cfg.variant >= GP_SORT && cfg.variant <= GP_PHASH &&
                        granule && T > 0;
  const uint64_t nchunks = T ? (T + chunk - 1) / chunk : 1;
  if (pre_part) {
    if (!c->part_stream) GP_CUDA(c, cudaStreamCreateWithFlags(&c->part_stream, cudaStreamNonBlocking));
    if (c->host_parts.size() < nchunks) c->host_parts.resize(nchunks);
  }

  std::vector<cudaEvent_t> evs;
  auto new_event = [&]() {
    cudaEvent_t e = get_event(c);
    if (e) evs.push_back(e);
    return e;
  };
  auto finish = [&](gp_status st) {
    cudaStreamSynchronize(c->copy_in);
    if (c->part_stream) cudaStreamSynchronize(c->part_stream);
    cudaStreamSynchronize(c->stream);
    cudaStreamSynchronize(c->copy_out);
    for (cudaEvent_t e : evs) put_event(c, e);
    return st;
  };
  std::vector<cudaEvent_t> ev_in(nchunks, nullptr);
  auto upload_indices = [&](uint64_t k) -> gp_status {
    const uint64_t t0 = k * chunk, nt = T ? std::min<uint64_t>(chunk, T - t0) : 0;
    uint32_t* d_idx = static_cast<uint32_t*>(c->h_idx) + 3 * t0;
    if (!(ev_in[k] = new_event())) return fail(c, GP_ERR_CUDA, "cudaEventCreate failed");
    if (nt) GP_CUDA(c, cudaMemcpyAsync(d_idx, indices_host + 3 * t0, nt * 12, cudaMemcpyHostToDevice, c->copy_in));
    GP_CUDA(c, cudaEventRecord(ev_in[k], c->copy_in));
    if (pre_part) {
      Partition& p = c->host_parts[k];
      gp_status st = size_partition(c, p, 3 * nt, true, cfg.max_unique, cfg.max_tris, cfg.segment_tris);
      if (st != GP_OK) return st;
      p.idx = d_idx;
      if (!p.done) GP_CUDA(c, cudaEventCreateWithFlags(&p.done, cudaEventDisableTiming));
      GP_CUDA(c, cudaStreamWaitEvent(c->part_stream, ev_in[k], 0));
      if ((st = run_partition(c, p, d_idx, 3 * nt, c->part_stream)) != GP_OK) return st;
      GP_CUDA(c, cudaEventRecord(p.done, c->part_stream));
    }
    return GP_OK;
  };
  if (pre_part && (s = upload_indices(0)) != GP_OK) return finish(s);
  cudaEvent_t ev_v = new_event();
  if (!ev_v) return finish(fail(c, GP_ERR_CUDA, "cudaEventCreate failed"));
  if (num_vertices)
    GP_CUDA(c, cudaMemcpyAsync(c->h_vtx, vertices_host, num_vertices * stride_bytes, cudaMemcpyHostToDevice,
                               c->copy_in));
  GP_CUDA(c, cudaEventRecord(ev_v, c->copy_in));
  GP_CUDA(c, cudaStreamWaitEvent(c->stream, ev_v, 0));
  for (uint64_t k = pre_part ? 1 : 0; k < nchunks; ++k)
    if ((s = upload_indices(k)) != GP_OK) return finish(s);
  uint64_t ticket = 0;
  gp_vertex_buf vb{c->h_vtx, num_vertices, stride_bytes, format};
  for (uint64_t k = 0; k < nchunks; ++k) {
    const uint64_t t0 = k * chunk, nt = T ? std::min<uint64_t>(chunk, T - t0) : 0;
    uint32_t* d_idx = static_cast<uint32_t*>(c->h_idx) + 3 * t0;
    float* d_out = static_cast<float*>(c->h_out) + 3 * K * t0;
    cudaEvent_t ev_done = new_event();
    if (!ev_done) return finish(fail(c, GP_ERR_CUDA, "cudaEventCreate failed"));
    GP_CUDA(c, cudaStreamWaitEvent(c->stream, ev_in[k], 0));
    gp_index_buf ib{d_idx, 3 * nt, 0};
    gp_out_buf ob{d_out, nt * 3 * K * 4, nullptr, nullptr, 0};
    s = submit_locked(c, &ib, &vb, shader_id, uniforms, uniforms_bytes, &ob, &ticket,
                      pre_part ? &c->host_parts[k] : nullptr);
    if (s != GP_OK) return finish(s);
    GP_CUDA(c, cudaEventRecord(ev_done, c->stream));
    GP_CUDA(c, cudaStreamWaitEvent(c->copy_out, ev_done, 0));
    if (nt) GP_CUDA(c, cudaMemcpyAsync(out_host + 3 * K * t0, d_out, nt * 3 * K * 4, cudaMemcpyDeviceToHost, c->copy_out));
  }
  s = finish(GP_OK);
  return sync_locked(c, ticket, 0);
}

uint32_t gp_out_floats(uint32_t shader_id) { return shader_id <= GP_SHADER_LOAD ? (uint32_t)out_floats((int)shader_id) : 0u; }

uint64_t gp_static_batch_count(gp_ctx* c, uint64_t num_indices) {
  if (!c || c->cfg.mode != GP_BATCH_STATIC) return 0;
  if (c->cfg.variant == GP_MULTI) return num_indices ? 1 : 0;  // the whole draw
  const uint64_t S = c->cfg.batch_indices;
  return (num_indices + S - 1) / S;
}

const char* gp_last_error(gp_ctx* c) {
  if (!c) return g_create_error.c_str();
  return c->last_error.c_str();
}

const char* gp_status_string(gp_status s) { return status_name(s); }

}  // extern "C"
