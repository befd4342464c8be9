// C-ABI of frames (many draw calls in one persistent launch, replayed from a
// captured CUDA graph) and of the autotuner that picks each draw's method,
// batch size and threads per group.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>
#include <string>
#include <vector>

#include "gp_context.h"

using namespace gp;
using namespace gp::rt;

struct gp_frame {
  gp_ctx* ctx = nullptr;
  std::vector<gp_draw_desc> desc;
  std::vector<gp_draw_config> cfg;
  std::vector<FrameDraw> h_draws;
  std::vector<Uniforms> h_uni;
  std::vector<Partition> parts;  // one per draw (empty for static draws)
  FrameDraw* d_draws = nullptr;
  uint32_t* d_item_draw = nullptr;  // work item -> draw
  Uniforms* d_uni = nullptr;
  uint32_t* d_work = nullptr;
  DevRec* d_rec = nullptr;
  uint32_t total_items = 0;
  uint64_t tris = 0, indices = 0, out_bytes = 0, vertex_bytes = 0;
  int grid = 0;
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t last_ticket = 0;
};

namespace gp {
namespace rt {

uint32_t frame_capacities(DrawArgs& a, int method, uint32_t shader, uint32_t group) {
  const bool pipe = group == kFrameThreads;
  // the whole-block path sizes its table like the single-draw kernel
  a.hash_slots = pipe ? std::max(next_pow2(2 * a.ucap), std::min(next_pow2(4 * a.ucap), 1024u)) : next_pow2(2 * a.ucap);
  a.hash_slots = std::max(a.hash_slots, next_pow2(group));
  a.hash_bits = log2u(a.hash_slots);
  a.sort_n = next_pow2(a.max_batch_idx);
  {  // 32-bit sort keys when every id (plus one value for "out of range") fits beside the position
    const uint32_t pb = std::max(1u, log2u(a.sort_n));
    a.sort_pos_bits = (pb < 32 && (uint64_t)a.num_verts + 1 < (1ull << (32 - pb))) ? pb : 0u;
  }
  if (!pipe) return frame_slice_bytes(method, (int)shader, a.max_batch_idx, a.ucap, a.hash_slots, a.sort_n, group, 0);
  // a thread numbers at most 32 positions; slots are stored in 15 bits
  if (method != kFrameSort && (a.max_batch_idx > 32u * group || a.hash_slots > 32768u)) return 0;
  // the largest output chunk (the whole batch, a half, a quarter, ...) that fits
  for (uint32_t chunk = (a.max_batch_idx + 2) / 3;; chunk = (chunk + 1) / 2) {
    a.out_chunk = chunk;
    const uint32_t bytes = frame_pipe_bytes(method, (int)shader, a);
    if (bytes <= kFrameSliceBytes) return bytes;
    if (chunk <= 16) return 0;
  }
}

}  // namespace rt
}  // namespace gp

namespace {

int method_of(int32_t variant) {
  switch (variant) {
    case GP_NAIVE: return kFrameNaive;
    case GP_WARP: return kFrameWarp;
    case GP_SORT: return kFrameSort;
    case GP_HASH: return kFrameHash;
    default: return kFramePHash;
  }
}

// Defaults for fields left at 0, and the checks of a concrete configuration.
gp_status normalize_config(gp_ctx* c, gp_draw_config& k, uint32_t draw) {
  auto bad = [&](const char* why) {
    return fail(c, GP_ERR_INVALID, "frame draw " + std::to_string(draw) + ": " + why);
  };
  if (k.variant < GP_NAIVE || k.variant > GP_PHASH) return bad("variant must be GP_NAIVE..GP_PHASH or GP_AUTO");
  if (k.variant == GP_NAIVE || k.variant == GP_WARP) {
    if (k.mode != GP_BATCH_STATIC) return bad("naive and warp voting use static batches");
    if (k.variant == GP_NAIVE) {
      k.threads_per_group = kFrameThreads;
      k.batch_indices = 3 * kFrameThreads;
    } else {
      k.threads_per_group = 32;
      if (!k.batch_indices) k.batch_indices = 96;
      if (k.batch_indices % 3 || k.batch_indices > 384) return bad("warp voting batches are multiples of 3, <= 384");
    }
    return GP_OK;
  }
  if (!k.threads_per_group) k.threads_per_group = 256;
  if (k.threads_per_group != 64 && k.threads_per_group != 128 && k.threads_per_group != 256)
    return bad("threads_per_group must be 64, 128 or 256 for sort/hash/phash");
  if (k.mode == GP_BATCH_STATIC) {
    if (!k.batch_indices) k.batch_indices = 255;
    if (k.batch_indices % 3 || k.batch_indices > 4095) return bad("batch_indices must be a multiple of 3, <= 4095");
  } else if (k.mode == GP_BATCH_DYNAMIC) {
    if (!k.max_unique) k.max_unique = 256;
    if (!k.max_tris) k.max_tris = (4 * k.max_unique - 1) / 3;
    if (k.max_unique < 3 || k.max_unique > 4096 || k.max_tris < 1 || k.max_tris > 1365)
      return bad("need 3 <= max_unique <= 4096 and 1 <= max_tris <= 1365");
  } else {
    return bad("bad mode");
  }
  return GP_OK;
}

// Fills the capacities of a sort/hash/phash draw and checks that one group's
// working set fits its share of the block's shared memory.
gp_status capacities(gp_ctx* c, const gp_draw_config& k, uint32_t shader, DrawArgs& a, uint32_t draw) {
  const int method = method_of(k.variant);
  if (method == kFrameNaive || method == kFrameWarp) {
    const uint32_t bytes = frame_slice_bytes(method, (int)shader, 0, 0, 0, 0, k.threads_per_group, k.batch_indices);
    if (bytes > kFrameSliceBytes)
      return fail(c, GP_ERR_UNSUPPORTED, "frame draw " + std::to_string(draw) + ": batch too large for the frame");
    return GP_OK;
  }
  if (k.mode == GP_BATCH_STATIC) {
    a.max_batch_idx = k.batch_indices;
    a.ucap = k.batch_indices;
  } else {
    a.max_batch_idx = 3 * k.max_tris;
    a.ucap = k.max_unique;
  }
  const uint32_t bytes = frame_capacities(a, method, shader, k.threads_per_group);
  if (bytes == 0 || bytes > kFrameSliceBytes)
    return fail(c, GP_ERR_UNSUPPORTED,
                "frame draw " + std::to_string(draw) + ": batch too large for " +
                    std::to_string(k.threads_per_group) + " threads per group");
  return GP_OK;
}

// The autotune table's configuration for a draw, or a default.
gp_draw_config resolve_auto(const gp_ctx* c, uint32_t shader, uint64_t tris) {
  for (const gp_autotune_entry& e : c->tune)
    if (e.shader_id == shader && tris >= e.tris_lo && tris < e.tris_hi) return e.config;
  gp_draw_config k{};
  k.variant = GP_HASH;
  k.mode = tris >= 1024 ? GP_BATCH_DYNAMIC : GP_BATCH_STATIC;
  k.max_unique = 256;
  k.threads_per_group = 256;
  k.batch_indices = 255;
  return k;
}

void free_frame(gp_frame* f) {
  if (f->exec) cudaGraphExecDestroy(f->exec);
  if (f->graph) cudaGraphDestroy(f->graph);
  if (f->cap_stream) cudaStreamDestroy(f->cap_stream);
  if (f->d_draws) cudaFree(f->d_draws);
  if (f->d_item_draw) cudaFree(f->d_item_draw);
  if (f->d_uni) cudaFree(f->d_uni);
  if (f->d_work) cudaFree(f->d_work);
  if (f->d_rec) cudaFree(f->d_rec);
  for (Partition& p : f->parts) release_partition(p);
  delete f;
}

gp_status frame_create_locked(gp_ctx* c, const gp_draw_desc* draws, uint32_t n, gp_frame** out) {
  if (!out) return fail(c, GP_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (n && !draws) return fail(c, GP_ERR_INVALID, "draws is NULL");
  gp_frame* f = new gp_frame();
  f->ctx = c;
  f->desc.assign(draws, draws + n);
  f->cfg.resize(n);
  f->h_draws.resize(n);
  f->h_uni.resize(n);
  f->parts.resize(n);
  auto abort = [&](gp_status s) {
    cudaStreamSynchronize(c->stream);
    free_frame(f);
    return s;
  };
  cudaError_t e;
  if ((e = cudaMalloc(&f->d_rec, sizeof(DevRec))) != cudaSuccess ||
      (e = cudaMalloc(&f->d_work, 16)) != cudaSuccess)
    return abort(cuda_fail(c, e, "cudaMalloc"));
  std::map<std::tuple<uintptr_t, uint64_t, uint32_t, uint32_t>, uint32_t> shared_part;
  std::vector<uint32_t> part_src(n, 0);

  for (uint32_t i = 0; i < n; ++i) {
    const gp_draw_desc& d = draws[i];
    gp_status s = check_draw(c, &d.index_buf, &d.vertex_buf, d.shader_id, &d.out);
    if (s != GP_OK) return abort(fail(c, s, "frame draw " + std::to_string(i) + ": " + c->last_error));
    if ((s = make_uniforms(c, d.shader_id, d.uniforms, d.uniforms_bytes, f->h_uni[i])) != GP_OK)
      return abort(fail(c, s, "frame draw " + std::to_string(i) + ": " + c->last_error));
    const uint64_t T = d.index_buf.num_indices / 3;
    gp_draw_config k{};
    if (d.variant == GP_AUTO) {
      k = resolve_auto(c, d.shader_id, T);
    } else {
      k.variant = d.variant;
      k.mode = d.mode;
      k.batch_indices = d.batch_indices;
      k.max_unique = d.max_unique;
      k.max_tris = d.max_tris;
      k.threads_per_group = d.threads_per_group;
    }
    if ((s = normalize_config(c, k, i)) != GP_OK) return abort(s);
    FrameDraw& D = f->h_draws[i];
    std::memset(&D, 0, sizeof(D));
    DrawArgs& a = D.a;
    a.idx = d.index_buf.d_indices;
    a.num_idx = (uint32_t)d.index_buf.num_indices;
    a.num_tris = (uint32_t)T;
    a.verts = static_cast<const unsigned char*>(d.vertex_buf.d_vertices);
    a.num_verts = (uint32_t)d.vertex_buf.num_vertices;
    a.stride = d.vertex_buf.stride_bytes;
    a.vec8 = (reinterpret_cast<uintptr_t>(d.vertex_buf.d_vertices) % 32 == 0 && a.stride % 32 == 0) ? 1u : 0u;
    a.out = d.out.d_out;
    a.corner_ids = d.out.d_corner_ids;
    a.batch_inv = d.out.d_batch_invocations;
    a.batch_cap = (uint32_t)std::min<uint64_t>(d.out.batch_capacity, 0xFFFFFFFFu);
    a.probe_k = c->cfg.probe_k;
    a.counters = f->d_rec->cnt;
    a.err = &f->d_rec->err;
    D.method = (uint32_t)method_of(k.variant);
    D.shader = d.shader_id;
    D.group = k.threads_per_group;
    if ((s = capacities(c, k, d.shader_id, a, i)) != GP_OK) return abort(s);
    if (k.variant == GP_NAIVE) {
      D.num_batches = (uint32_t)((T + kFrameThreads - 1) / kFrameThreads);
    } else if (k.mode == GP_BATCH_STATIC) {
      a.static_batch_tris = k.batch_indices / 3;
      D.num_batches = (uint32_t)((T + a.static_batch_tris - 1) / a.static_batch_tris);
      a.num_batches = D.num_batches;
    } else {
      D.dynamic = 1;
      // draws over the same index buffer with the same limits share one partition
      const auto key = std::make_tuple(reinterpret_cast<uintptr_t>(d.index_buf.d_indices), d.index_buf.num_indices,
                                       k.max_unique, k.max_tris);
      const auto it = shared_part.find(key);
      if (it != shared_part.end()) {
        part_src[i] = it->second;
        a.starts = f->parts[it->second].d_starts;
        a.num_batches_dev = f->parts[it->second].d_count;
      } else {
        Partition& p = f->parts[i];
        if ((s = size_partition(c, p, d.index_buf.num_indices, false, k.max_unique, k.max_tris,
                                c->cfg.segment_tris)) != GP_OK)
          return abort(s);
        p.idx = d.index_buf.d_indices;
        if (T && (s = run_partition(c, p, d.index_buf.d_indices, d.index_buf.num_indices, c->stream)) != GP_OK)
          return abort(s);
        a.starts = p.d_starts;
        a.num_batches_dev = p.d_count;
        shared_part.emplace(key, i);
        part_src[i] = i;
      }
    }
    f->cfg[i] = k;
    f->tris += T;
    f->indices += d.index_buf.num_indices;
    f->out_bytes += T * 3 * out_floats((int)d.shader_id) * 4;
    f->vertex_bytes += (uint64_t)a.stride;  // per invocation (averaged below)
  }
  if (n) f->vertex_bytes /= n;
  // batch counts of the dynamic draws (the partitions ran on the stream)
  if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return abort(cuda_fail(c, e, "partition"));
  uint32_t item = 0;
  for (uint32_t i = 0; i < n; ++i) {
    FrameDraw& D = f->h_draws[i];
    if (D.dynamic) {
      uint32_t cnt = 0;
      if (D.a.num_tris) {
        if (part_src[i] != i) {
          cnt = f->h_draws[part_src[i]].num_batches;  // set earlier in this loop (part_src[i] < i)
        } else if ((e = cudaMemcpy(&cnt, f->parts[i].d_count, 4, cudaMemcpyDeviceToHost)) != cudaSuccess) {
          return abort(cuda_fail(c, e, "partition count"));
        }
      }
      D.num_batches = cnt;
    }
    const uint32_t per_item = D.method == kFrameNaive ? 1u : (D.method == kFrameWarp ? kFrameThreads / 32 : kFrameThreads / D.group);
    D.items = (D.num_batches + per_item - 1) / per_item;
    D.item_begin = item;
    item += D.items;
    f->cfg[i].batches = D.num_batches;
  }
  f->total_items = item;
  if (item) {
    std::vector<uint32_t> h_item_draw(item);
    for (uint32_t i = 0; i < n; ++i)
      for (uint32_t j = 0; j < f->h_draws[i].items; ++j) h_item_draw[f->h_draws[i].item_begin + j] = i;
    if ((e = cudaMalloc(&f->d_item_draw, sizeof(uint32_t) * item)) != cudaSuccess ||
        (e = cudaMemcpy(f->d_item_draw, h_item_draw.data(), sizeof(uint32_t) * item, cudaMemcpyHostToDevice)) !=
            cudaSuccess)
      return abort(cuda_fail(c, e, "item table"));
  }
  if (n) {
    if ((e = cudaMalloc(&f->d_draws, sizeof(FrameDraw) * n)) != cudaSuccess ||
        (e = cudaMalloc(&f->d_uni, sizeof(Uniforms) * n)) != cudaSuccess)
      return abort(cuda_fail(c, e, "cudaMalloc"));
    for (uint32_t i = 0; i < n; ++i) f->h_draws[i].u = f->d_uni + i;
    if ((e = cudaMemcpy(f->d_draws, f->h_draws.data(), sizeof(FrameDraw) * n, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(f->d_uni, f->h_uni.data(), sizeof(Uniforms) * n, cudaMemcpyHostToDevice)) != cudaSuccess)
      return abort(cuda_fail(c, e, "cudaMemcpy"));
  }
  const int bpsm = frame_blocks_per_sm();
  if (bpsm <= 0) return abort(fail(c, GP_ERR_UNSUPPORTED, "frame kernel cannot be resident"));
  f->grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)c->sms * bpsm, std::max(1u, f->total_items)));
  // capture: reset the work counter and the record, then the persistent launch
  if ((e = cudaStreamCreateWithFlags(&f->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return abort(cuda_fail(c, e, "cudaStreamCreate"));
  if ((e = cudaStreamBeginCapture(f->cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
    return abort(cuda_fail(c, e, "cudaStreamBeginCapture"));
  cudaError_t e1 = cudaMemsetAsync(f->d_work, 0, 16, f->cap_stream);
  cudaError_t e2 = cudaMemsetAsync(f->d_rec, 0, sizeof(DevRec), f->cap_stream);
  cudaError_t e3 = f->total_items ? launch_frame(f->d_draws, f->d_item_draw, f->total_items, f->d_work,
                                                f->d_rec->cnt, f->grid, f->cap_stream)
                                  : cudaSuccess;
  e = cudaStreamEndCapture(f->cap_stream, &f->graph);
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess || e != cudaSuccess)
    return abort(cuda_fail(c, e3 != cudaSuccess ? e3 : (e != cudaSuccess ? e : (e1 != cudaSuccess ? e1 : e2)),
                           "frame capture"));
  if ((e = cudaGraphInstantiate(&f->exec, f->graph, 0)) != cudaSuccess)
    return abort(cuda_fail(c, e, "cudaGraphInstantiate"));
  *out = f;
  return GP_OK;
}

gp_status frame_submit_locked(gp_frame* f, uint64_t* out_ticket) {
  gp_ctx* c = f->ctx;
  // the frame's record is shared by its launches: the previous one must be folded
  if (f->last_ticket) {
    gp_status s = sync_locked(c, f->last_ticket, 0);
    if (s != GP_OK && s != GP_ERR_INDEX_RANGE) return s;
  }
  Ticket t;
  gp_status s = new_ticket(c, t);
  if (s != GP_OK) return s;
  GP_CUDA(c, cudaEventRecord(t.ev0, c->stream));
  GP_CUDA(c, cudaGraphLaunch(f->exec, c->stream));
  GP_CUDA(c, cudaEventRecord(t.ev1, c->stream));
  t.draws = f->desc.size();
  t.tris = f->tris;
  t.indices = f->indices;
  t.out_bytes = f->out_bytes;
  t.vertex_bytes_per_inv = f->vertex_bytes;
  t.device_counts = true;
  t.ext_rec = f->d_rec;
  c->inflight.push_back(t);
  f->last_ticket = t.id;
  if (out_ticket) *out_ticket = t.id;
  return GP_OK;
}

}  // namespace

extern "C" {

gp_status gp_frame_create(gp_ctx* c, const gp_draw_desc* draws, uint32_t num_draws, gp_frame** out) {
  if (!c) return GP_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  return frame_create_locked(c, draws, num_draws, out);
}

gp_status gp_frame_submit(gp_frame* f, uint64_t* out_ticket) {
  if (!f) return GP_ERR_INVALID;
  std::lock_guard<std::mutex> lk(f->ctx->mu);
  cudaSetDevice(f->ctx->device);
  return frame_submit_locked(f, out_ticket);
}

gp_status gp_frame_set_uniforms(gp_frame* f, uint32_t draw, const void* uniforms, uint32_t uniforms_bytes) {
  if (!f) return GP_ERR_INVALID;
  gp_ctx* c = f->ctx;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  if (draw >= f->desc.size()) return fail(c, GP_ERR_INVALID, "draw index out of range");
  Uniforms u;
  gp_status s = make_uniforms(c, f->desc[draw].shader_id, uniforms, uniforms_bytes, u);
  if (s != GP_OK) return s;
  // the host copy must outlive the asynchronous upload: wait for launches in flight
  if (f->last_ticket) {
    s = sync_locked(c, f->last_ticket, 0);
    if (s != GP_OK && s != GP_ERR_INDEX_RANGE) return s;
  }
  f->h_uni[draw] = u;
  GP_CUDA(c, cudaMemcpyAsync(f->d_uni + draw, &f->h_uni[draw], sizeof(Uniforms), cudaMemcpyHostToDevice, c->stream));
  return GP_OK;
}

gp_status gp_frame_draw_config(gp_frame* f, uint32_t draw, gp_draw_config* out) {
  if (!f || !out) return GP_ERR_INVALID;
  if (draw >= f->cfg.size()) return fail(f->ctx, GP_ERR_INVALID, "draw index out of range");
  *out = f->cfg[draw];
  return GP_OK;
}

gp_status gp_frame_destroy(gp_frame* f) {
  if (!f) return GP_ERR_INVALID;
  gp_ctx* c = f->ctx;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  if (f->last_ticket) sync_locked(c, f->last_ticket, 0);
  cudaStreamSynchronize(c->stream);
  free_frame(f);
  return GP_OK;
}

// ---------------------------------------------------------------------------
// autotuner
// ---------------------------------------------------------------------------

// Size of a tuning frame: about this many triangles, in at most this many draws.
constexpr uint64_t kTuneTris = 1u << 22;
constexpr uint64_t kTuneMaxDraws = 4096;

gp_status gp_autotune(gp_ctx* c, const gp_draw_desc* samples, uint32_t num_samples, uint32_t reps) {
  if (!c) return GP_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  if (num_samples && !samples) return fail(c, GP_ERR_INVALID, "samples is NULL");
  if (reps == 0) reps = 3;
  // groups: (shader, floor(log2 T))
  std::map<std::pair<uint32_t, uint32_t>, std::vector<uint32_t>> groups;
  for (uint32_t i = 0; i < num_samples; ++i) {
    const uint64_t T = samples[i].index_buf.num_indices / 3;
    if (T == 0) continue;
    uint32_t lg = 0;
    while ((2ull << lg) <= T) ++lg;
    groups[{samples[i].shader_id, lg}].push_back(i);
  }
  // candidate configurations
  std::vector<gp_draw_config> cand;
  {
    gp_draw_config k{};
    k.variant = GP_NAIVE;
    cand.push_back(k);
    for (uint32_t S : {96u, 192u}) {
      k = gp_draw_config{};
      k.variant = GP_WARP;
      k.batch_indices = S;
      cand.push_back(k);
    }
    for (int32_t v : {GP_HASH, GP_PHASH, GP_SORT}) {
      for (uint32_t G : {64u, 128u, 256u}) {
        for (uint32_t S : {63u, 126u, 255u, 510u}) {
          k = gp_draw_config{};
          k.variant = v;
          k.mode = GP_BATCH_STATIC;
          k.batch_indices = S;
          k.threads_per_group = G;
          cand.push_back(k);
        }
        for (uint32_t N : {64u, 128u, 256u}) {
          k = gp_draw_config{};
          k.variant = v;
          k.mode = GP_BATCH_DYNAMIC;
          k.max_unique = N;
          k.max_tris = (4 * N - 1) / 3;
          k.threads_per_group = G;
          cand.push_back(k);
        }
      }
    }
  }
  // the tuning launches do not count in the context's statistics
  gp_status s0 = sync_locked(c, 0, 0);
  if (s0 != GP_OK && s0 != GP_ERR_INDEX_RANGE) return s0;
  const uint64_t sv[6] = {c->s_draws, c->s_tris, c->s_idx, c->s_inv, c->s_batches, c->s_bytes};
  const double sv_busy = c->s_busy;
  const size_t sv_lat = c->s_lat.size();
  {  // store candidates in their normalised form (what a frame reports)
    std::vector<gp_draw_config> ok;
    const std::string saved = c->last_error;
    for (gp_draw_config k : cand)
      if (normalize_config(c, k, 0) == GP_OK) ok.push_back(k);
    c->last_error = saved;
    c->last_status = GP_OK;
    cand.swap(ok);
  }
  std::vector<gp_autotune_entry> found;
  for (auto& kv : groups) {
    const uint32_t shader = kv.first.first, lg = kv.first.second;
    std::vector<uint32_t>& ids = kv.second;
    // up to four samples of the group, closest to its median size
    std::sort(ids.begin(), ids.end(), [&](uint32_t x, uint32_t y) {
      return samples[x].index_buf.num_indices < samples[y].index_buf.num_indices;
    });
    const size_t mid = ids.size() / 2, lo = mid >= 2 ? mid - 2 : 0;
    std::vector<gp_draw_desc> pick;
    for (size_t j = lo; j < ids.size() && pick.size() < 4; ++j) pick.push_back(samples[ids[j]]);
    // Candidates are ranked by throughput, the quantity a frame of many draws
    // sees: the samples are repeated until the tuning frame holds enough
    // triangles to fill every SM several times over (a handful of small
    // draws would rank configurations by latency instead).  Repeats of a
    // draw write the same values to the same output.
    uint64_t pick_tris = 0;
    for (const gp_draw_desc& d : pick) pick_tris += d.index_buf.num_indices / 3;
    const uint64_t copies = std::min<uint64_t>(std::max<uint64_t>(1, (kTuneTris + pick_tris - 1) / pick_tris),
                                               kTuneMaxDraws / pick.size());
    const size_t nunique = pick.size();
    for (uint64_t r = 1; r < copies; ++r)
      for (size_t j = 0; j < nunique; ++j) pick.push_back(pick[j]);
    double best = 1e30;
    gp_draw_config best_k{};
    for (const gp_draw_config& k0 : cand) {
      std::vector<gp_draw_desc> ds = pick;
      for (gp_draw_desc& d : ds) {
        d.variant = k0.variant;
        d.mode = k0.mode;
        d.batch_indices = k0.batch_indices;
        d.max_unique = k0.max_unique;
        d.max_tris = k0.max_tris;
        d.threads_per_group = k0.threads_per_group;
      }
      gp_frame* f = nullptr;
      const std::string saved = c->last_error;
      if (frame_create_locked(c, ds.data(), (uint32_t)ds.size(), &f) != GP_OK) {
        c->last_error = saved;  // a candidate that does not fit is skipped
        c->last_status = GP_OK;
        continue;
      }
      double ms_best = 1e30;
      for (uint32_t r = 0; r < reps + 1; ++r) {  // the first launch warms up
        uint64_t t = 0;
        if (frame_submit_locked(f, &t) != GP_OK) break;
        if (sync_locked(c, t, 0) != GP_OK) break;
        if (r > 0 && !c->s_lat.empty()) ms_best = std::min<double>(ms_best, c->s_lat.back());
      }
      free_frame(f);
      if (ms_best < best) {
        best = ms_best;
        best_k = k0;
      }
    }
    if (best < 1e30) {
      gp_autotune_entry en{};
      en.shader_id = shader;
      en.tris_lo = 1u << lg;
      en.tris_hi = lg >= 31 ? 0xFFFFFFFFu : (2u << lg);
      en.config = best_k;
      en.us_per_draw = best * 1e3 / (double)pick.size();
      found.push_back(en);
    }
  }
  c->s_draws = sv[0];
  c->s_tris = sv[1];
  c->s_idx = sv[2];
  c->s_inv = sv[3];
  c->s_batches = sv[4];
  c->s_bytes = sv[5];
  c->s_busy = sv_busy;
  c->s_lat.resize(sv_lat);
  // merge: new rows replace rows of the same group
  for (const gp_autotune_entry& en : found) {
    c->tune.erase(std::remove_if(c->tune.begin(), c->tune.end(),
                                 [&](const gp_autotune_entry& x) {
                                   return x.shader_id == en.shader_id && x.tris_lo == en.tris_lo;
                                 }),
                  c->tune.end());
    c->tune.push_back(en);
  }
  return GP_OK;
}

gp_status gp_autotune_table(gp_ctx* c, gp_autotune_entry* out, uint32_t capacity, uint32_t* count) {
  if (!c) return GP_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  if (count) *count = (uint32_t)c->tune.size();
  if (out)
    for (uint32_t i = 0; i < capacity && i < c->tune.size(); ++i) out[i] = c->tune[i];
  return GP_OK;
}

gp_status gp_autotune_set_table(gp_ctx* c, const gp_autotune_entry* entries, uint32_t count) {
  if (!c) return GP_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  if (count && !entries) return fail(c, GP_ERR_INVALID, "entries is NULL");
  c->tune.assign(entries, entries + count);
  return GP_OK;
}

}  // extern "C"
