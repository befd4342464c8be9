// C-ABI of the serving loop: a native server thread that admits draw-call
// requests under a device-memory budget, keeps their meshes resident (LRU
// eviction of meshes without active requests) and runs continuous-batching
// steps: every step is one launch of the frame kernel over batch ranges taken
// from all active requests, so requests that arrive while others are on the
// GPU join the next step.  Batches never span requests.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gp_context.h"

using namespace gp;
using namespace gp::rt;

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Mesh {
  uint64_t id = 0;
  uint32_t* h_idx = nullptr;  // pinned host copies
  void* h_vtx = nullptr;
  uint64_t num_idx = 0, num_verts = 0;
  uint32_t stride = 0, format = 0;
  // resident state
  bool resident = false;
  uint32_t* d_idx = nullptr;
  void* d_vtx = nullptr;
  Partition part;
  uint32_t batches = 0;
  uint64_t bytes = 0;
  uint32_t active = 0;  // requests using it
  gp_draw_config k{};   // configuration the mesh was made resident with (batches, partition)
  std::list<uint64_t>::iterator lru;
};

struct Request {
  uint64_t id = 0;
  uint64_t mesh = 0;
  uint32_t shader = 0;
  Uniforms uni;
  float* d_out = nullptr;
  Clock::time_point arrival;
  Clock::time_point done_at;
  uint32_t slot = 0;           // admission slot (at most max_active requests at once)
  uint32_t batches = 0, next = 0, done = 0;
  bool finished = false;
  gp_status status = GP_OK;
};

// A step's inputs travel to the device in one copy: the pinned host block
// and the device block share one layout, packed per step as
//   entries' FrameDraw | entries' Uniforms | item -> entry table | work
//   counter (16 zero bytes) | DevRec (zeroed)
// with each part 256-byte aligned.
struct StepSlot {
  cudaStream_t stream = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  unsigned char* h_block = nullptr;  // pinned
  unsigned char* d_block = nullptr;
  size_t block_bytes = 0;
  DevRec* h_rec = nullptr;           // pinned read-back of the step's record
  bool busy = false;
  std::vector<std::pair<uint64_t, uint32_t>> parts;  // (request, batches in this step)
};

inline size_t step_align(size_t x) { return (x + 255) & ~(size_t)255; }

// Bytes of a step block for n entries and `items` work items.
inline size_t step_block_bytes(uint32_t n, uint32_t items) {
  return step_align(sizeof(FrameDraw) * n) + step_align(sizeof(Uniforms) * n) + step_align(4ull * items) + 256 +
         step_align(sizeof(DevRec));
}

}  // namespace

struct gp_server {
  gp_ctx* ctx = nullptr;
  gp_serve_config cfg{};
  gp_draw_config k{};  // resolved per request when GP_AUTO
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread thread;
  bool stop = false;
  // meshes
  std::unordered_map<uint64_t, Mesh> meshes;
  uint64_t next_mesh = 1;
  std::list<uint64_t> lru;  // resident meshes, most recently used at the back
  uint64_t resident_bytes = 0;
  cudaStream_t upload = nullptr;
  // requests
  std::deque<uint64_t> pending;
  std::deque<uint64_t> active;  // admission order
  std::unordered_map<uint64_t, Request> reqs;
  uint64_t next_req = 1;
  uint64_t submitted = 0, completed = 0;
  std::vector<uint32_t> free_slots;
  std::vector<uint32_t> item_scratch;  // launch_step's work item -> entry table
  std::vector<StepSlot> steps;
  int frame_bpsm = 1;
  // statistics
  std::vector<double> lat;
  uint64_t s_tris = 0, s_inv = 0, s_steps = 0, s_uploads = 0, s_evictions = 0;
  double s_busy = 0.0;
  // device time of the steps as intervals against a reference event recorded
  // before the first step after the last idle point (their union is the time
  // the device had at least one step in flight); dev_folded holds the union
  // of the intervals folded away (at idle points, or the oldest ones when
  // many accumulate under continuous load)
  cudaEvent_t ev_ref = nullptr;
  bool ref_set = false;
  std::vector<std::pair<float, float>> step_iv;
  double dev_folded = 0.0;
  bool have_first = false;
  Clock::time_point first_submit, last_done;
  gp_status last_error = GP_OK;
};

namespace {

constexpr uint32_t kStepMaxEntries = 4096;

gp_draw_config request_config(gp_server* s, uint32_t shader, uint64_t tris) {
  gp_draw_config k = s->k;
  if (s->cfg.variant == GP_AUTO) {
    bool hit = false;
    for (const gp_autotune_entry& e : s->ctx->tune)
      if (e.shader_id == shader && tris >= e.tris_lo && tris < e.tris_hi) {
        k = e.config;
        hit = true;
        break;
      }
    if (!hit) {
      k = gp_draw_config{};
      k.variant = GP_HASH;
      k.mode = GP_BATCH_DYNAMIC;
      k.max_unique = 256;
      k.max_tris = 341;
      k.threads_per_group = 256;
    }
  }
  return k;
}

void evict(gp_server* s, Mesh& m) {
  if (m.d_idx) cudaFree(m.d_idx);
  if (m.d_vtx) cudaFree(m.d_vtx);
  release_partition(m.part);
  m.d_idx = nullptr;
  m.d_vtx = nullptr;
  m.resident = false;
  s->resident_bytes -= m.bytes;
  m.bytes = 0;
  s->lru.erase(m.lru);
  s->s_evictions += 1;
}

// Makes the mesh resident for a request of configuration k.  Returns false
// (without side effects) if the budget cannot be met right now.
bool make_resident(gp_server* s, Mesh& m, const gp_draw_config& k, gp_status* err) {
  if (m.resident) {
    s->lru.erase(m.lru);
    m.lru = s->lru.insert(s->lru.end(), m.id);
    return true;
  }
  const uint64_t T = m.num_idx / 3;
  const uint64_t need = m.num_idx * 4 + m.num_verts * m.stride + (k.mode == GP_BATCH_DYNAMIC ? (T / 32 + 64) * 4 : 0);
  // evict least recently used meshes that no active request uses
  for (auto it = s->lru.begin(); s->resident_bytes + need > s->cfg.mem_budget_bytes && it != s->lru.end();) {
    Mesh& v = s->meshes[*it];
    ++it;
    if (v.active == 0) evict(s, v);
  }
  if (s->resident_bytes + need > s->cfg.mem_budget_bytes) return false;
  cudaError_t e;
  void* p = nullptr;
  if ((e = cudaMalloc(&p, std::max<uint64_t>(m.num_idx * 4, 16))) != cudaSuccess) {
    *err = GP_ERR_OOM;
    return false;
  }
  m.d_idx = static_cast<uint32_t*>(p);
  if ((e = cudaMalloc(&m.d_vtx, std::max<uint64_t>(m.num_verts * m.stride, 16))) != cudaSuccess) {
    cudaFree(m.d_idx);
    m.d_idx = nullptr;
    *err = GP_ERR_OOM;
    return false;
  }
  cudaMemcpyAsync(m.d_idx, m.h_idx, m.num_idx * 4, cudaMemcpyHostToDevice, s->upload);
  cudaMemcpyAsync(m.d_vtx, m.h_vtx, m.num_verts * m.stride, cudaMemcpyHostToDevice, s->upload);
  if (k.variant == GP_NAIVE) {
    m.batches = (uint32_t)((T + kFrameThreads - 1) / kFrameThreads);
  } else if (k.variant == GP_WARP || k.mode == GP_BATCH_STATIC) {
    const uint32_t per = k.batch_indices / 3;
    m.batches = (uint32_t)((T + per - 1) / per);
  } else {
    // load-time partition on the upload stream (Section 3.4)
    gp_ctx* c = s->ctx;
    gp_status st;
    {
      std::lock_guard<std::mutex> clk(c->mu);  // error text and scratch sizing use the context
      st = size_partition(c, m.part, m.num_idx, false, k.max_unique, k.max_tris, c->cfg.segment_tris);
      if (st == GP_OK && T) st = run_partition(c, m.part, m.d_idx, m.num_idx, s->upload);
    }
    uint32_t cnt = 0;
    if (st == GP_OK) cudaStreamSynchronize(s->upload);
    if (st == GP_OK && T && cudaMemcpy(&cnt, m.part.d_count, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
      st = GP_ERR_CUDA;
    if (st != GP_OK) {
      cudaFree(m.d_idx);
      cudaFree(m.d_vtx);
      release_partition(m.part);
      m.d_idx = nullptr;
      m.d_vtx = nullptr;
      *err = st;
      return false;
    }
    m.batches = cnt;
  }
  cudaStreamSynchronize(s->upload);
  m.resident = true;
  m.k = k;
  m.bytes = need;
  s->resident_bytes += need;
  m.lru = s->lru.insert(s->lru.end(), m.id);
  s->s_uploads += 1;
  return true;
}

void finish_request(gp_server* s, Request& r) {
  r.finished = true;
  r.done_at = Clock::now();
  s->lat.push_back(ms_between(r.arrival, r.done_at));
  s->last_done = r.done_at;
  s->completed += 1;
  Mesh& m = s->meshes[r.mesh];
  if (m.active) m.active -= 1;
  s->free_slots.push_back(r.slot);
}

// Admission, in arrival order: a request needs a free slot and its mesh
// resident within the budget.  Called with s->mu held.
void admit(gp_server* s) {
  while (!s->pending.empty() && !s->free_slots.empty()) {
    Request& r = s->reqs[s->pending.front()];
    Mesh& m = s->meshes[r.mesh];
    const gp_draw_config k = request_config(s, r.shader, m.num_idx / 3);
    gp_status err = GP_OK;
    if (!make_resident(s, m, k, &err)) {
      if (err != GP_OK) {  // allocation failure: the request fails, others go on
        r.status = err;
        s->pending.pop_front();
        r.slot = 0;
        r.finished = true;
        r.done_at = Clock::now();
        s->completed += 1;
        s->last_error = err;
        s->cv_done.notify_all();
        continue;
      }
      return;  // wait until memory frees up
    }
    s->pending.pop_front();
    m.active += 1;
    r.slot = s->free_slots.back();
    s->free_slots.pop_back();
    r.batches = m.batches;
    r.next = 0;
    r.done = 0;
    if (r.batches == 0) {
      finish_request(s, r);
      s->cv_done.notify_all();
      continue;
    }
    s->active.push_back(r.id);
  }
}

// Builds and launches one step on a free slot.  Called with s->mu held.
bool launch_step(gp_server* s, StepSlot& st) {
  uint32_t n = 0, items = 0, batches = 0;
  st.parts.clear();
  // entries first (FrameDraw and Uniforms at capacity offsets), then packed
  FrameDraw* h_draws = reinterpret_cast<FrameDraw*>(st.h_block);
  Uniforms* h_uni = reinterpret_cast<Uniforms*>(st.h_block + step_align(sizeof(FrameDraw) * kStepMaxEntries));
  std::vector<uint32_t>& item_draw = s->item_scratch;
  item_draw.clear();
  for (uint64_t rid : s->active) {
    if (batches >= s->cfg.step_max_batches || n >= kStepMaxEntries) break;
    Request& r = s->reqs[rid];
    if (r.next >= r.batches) continue;
    Mesh& m = s->meshes[r.mesh];
    const gp_draw_config& k = m.k;  // every request on a mesh uses its resident configuration
    const uint32_t take = std::min(r.batches - r.next, s->cfg.step_max_batches - batches);
    FrameDraw& D = h_draws[n];
    std::memset(&D, 0, sizeof(D));
    DrawArgs& a = D.a;
    a.idx = m.d_idx;
    a.num_idx = (uint32_t)m.num_idx;
    a.num_tris = (uint32_t)(m.num_idx / 3);
    a.verts = static_cast<const unsigned char*>(m.d_vtx);
    a.num_verts = (uint32_t)m.num_verts;
    a.stride = m.stride;
    a.vec8 = (reinterpret_cast<uintptr_t>(m.d_vtx) % 32 == 0 && m.stride % 32 == 0) ? 1u : 0u;
    a.out = r.d_out;
    a.probe_k = s->ctx->cfg.probe_k;
    D.method = k.variant == GP_NAIVE ? kFrameNaive
               : k.variant == GP_WARP ? kFrameWarp
               : k.variant == GP_SORT ? kFrameSort
               : k.variant == GP_HASH ? kFrameHash
                                      : kFramePHash;
    D.shader = r.shader;
    D.group = k.variant == GP_WARP ? 32u : (k.variant == GP_NAIVE ? kFrameThreads : k.threads_per_group);
    if (k.variant != GP_NAIVE && k.variant != GP_WARP) {
      if (k.mode == GP_BATCH_STATIC) {
        a.max_batch_idx = k.batch_indices;
        a.ucap = k.batch_indices;
        a.static_batch_tris = k.batch_indices / 3;
      } else {
        a.max_batch_idx = 3 * k.max_tris;
        a.ucap = k.max_unique;
        a.starts = m.part.d_starts;
        D.dynamic = 1;
      }
      frame_capacities(a, (int)D.method, r.shader, D.group);  // checked when the mesh became resident
    } else if (k.variant == GP_WARP) {
      a.static_batch_tris = k.batch_indices / 3;
    }
    h_uni[n] = r.uni;
    D.batch_begin = r.next;
    D.num_batches = take;
    const uint32_t per = D.method == kFrameNaive ? 1u : (D.method == kFrameWarp ? kFrameThreads / 32 : kFrameThreads / D.group);
    D.items = (take + per - 1) / per;
    D.item_begin = items;
    for (uint32_t j = 0; j < D.items; ++j) item_draw.push_back(n);
    items += D.items;
    r.next += take;
    batches += take;
    st.parts.push_back({rid, take});
    ++n;
  }
  if (n == 0) return false;
  // pack: move the uniforms down behind the n entries, then the item table,
  // the zeroed work counter and record; point the entries at the device copy
  const size_t o_uni = step_align(sizeof(FrameDraw) * n);
  const size_t o_items = o_uni + step_align(sizeof(Uniforms) * n);
  const size_t o_work = o_items + step_align(4ull * items);
  const size_t o_rec = o_work + 256;
  const size_t bytes = o_rec + sizeof(DevRec);
  std::memmove(st.h_block + o_uni, h_uni, sizeof(Uniforms) * n);
  std::memcpy(st.h_block + o_items, item_draw.data(), 4ull * items);
  std::memset(st.h_block + o_work, 0, 256 + sizeof(DevRec));
  const Uniforms* d_uni = reinterpret_cast<const Uniforms*>(st.d_block + o_uni);
  DevRec* d_rec = reinterpret_cast<DevRec*>(st.d_block + o_rec);
  for (uint32_t i = 0; i < n; ++i) {
    h_draws[i].u = d_uni + i;
    h_draws[i].a.counters = d_rec->cnt;
    h_draws[i].a.err = &d_rec->err;
  }
  cudaStream_t q = st.stream;
  if (!s->ref_set) {
    cudaEventRecord(s->ev_ref, q);
    s->ref_set = true;
  }
  cudaEventRecord(st.ev0, q);
  cudaMemcpyAsync(st.d_block, st.h_block, bytes, cudaMemcpyHostToDevice, q);
  const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)s->ctx->sms * s->frame_bpsm, items));
  cudaError_t e = launch_frame(reinterpret_cast<const FrameDraw*>(st.d_block),
                               reinterpret_cast<const uint32_t*>(st.d_block + o_items), items,
                               reinterpret_cast<uint32_t*>(st.d_block + o_work), d_rec->cnt, grid, q);
  cudaMemcpyAsync(st.h_rec, d_rec, sizeof(DevRec), cudaMemcpyDeviceToHost, q);
  cudaEventRecord(st.ev1, q);
  if (e != cudaSuccess) s->last_error = GP_ERR_CUDA;
  st.busy = true;
  s->s_steps += 1;
  return true;
}

// Total length of the union of intervals (sorts them).
double union_ms(std::vector<std::pair<float, float>>& iv) {
  std::sort(iv.begin(), iv.end());
  double total = 0.0, lo = 0.0, hi = 0.0;
  bool open = false;
  for (const auto& x : iv) {
    if (open && x.first <= hi) {
      hi = std::max<double>(hi, x.second);
    } else {
      if (open) total += hi - lo;
      lo = x.first;
      hi = x.second;
      open = true;
    }
  }
  if (open) total += hi - lo;
  return total;
}

// Keeps the interval list short.  With no step in flight every interval is
// folded into dev_folded and the next step records a new reference event
// (so the timestamps stay small and precise).  Under continuous load, once
// kMaxIntervals accumulate, the merged intervals that end before the start of
// the 1024 latest ones are folded: a step still in flight (at most one per
// stream) overlaps only recent ones.  Called with s->mu held.
constexpr size_t kMaxIntervals = 1u << 16;
void fold_intervals(gp_server* s, bool idle) {
  auto& iv = s->step_iv;
  if (iv.empty()) return;
  if (idle) {
    s->dev_folded += union_ms(iv);
    iv.clear();
    s->ref_set = false;
    return;
  }
  if (iv.size() < kMaxIntervals) return;
  std::sort(iv.begin(), iv.end());
  const float keep_from = iv[iv.size() - 1024].first;
  std::vector<std::pair<float, float>> kept, old;
  for (const auto& x : iv) (x.second < keep_from ? old : kept).push_back(x);
  s->dev_folded += union_ms(old);
  iv.swap(kept);
}

// Folds a completed step.  Called with s->mu held.
void complete_step(gp_server* s, StepSlot& st) {
  float ms = 0.f;
  cudaEventElapsedTime(&ms, st.ev0, st.ev1);
  s->s_busy += ms;
  float a = 0.f, b = 0.f;
  if (cudaEventElapsedTime(&a, s->ev_ref, st.ev0) == cudaSuccess &&
      cudaEventElapsedTime(&b, s->ev_ref, st.ev1) == cudaSuccess)
    s->step_iv.push_back({a, b});
  s->s_inv += st.h_rec->cnt[CNT_INVOCATIONS];
  gp_status err = GP_OK;
  if (st.h_rec->err & EBIT_INDEX_RANGE) err = GP_ERR_INDEX_RANGE;
  if (st.h_rec->err & (EBIT_CAPACITY | EBIT_TIMEOUT)) err = GP_ERR_UNSUPPORTED;
  if (err != GP_OK) s->last_error = err;
  for (auto& pr : st.parts) {
    Request& r = s->reqs[pr.first];
    r.done += pr.second;
    if (err != GP_OK) r.status = err;
    if (r.done >= r.batches && !r.finished) {
      s->s_tris += s->meshes[r.mesh].num_idx / 3;
      finish_request(s, r);
    }
  }
  // drop finished requests from the active list
  s->active.erase(std::remove_if(s->active.begin(), s->active.end(),
                                 [&](uint64_t id) { return s->reqs[id].finished; }),
                  s->active.end());
  st.busy = false;
  st.parts.clear();
}

void server_loop(gp_server* s) {
  cudaSetDevice(s->ctx->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    bool progressed = false;
    for (StepSlot& st : s->steps) {
      if (st.busy && cudaEventQuery(st.ev1) == cudaSuccess) {
        complete_step(s, st);
        progressed = true;
      }
    }
    {
      bool in_flight = false;
      for (StepSlot& st : s->steps) in_flight |= st.busy;
      fold_intervals(s, !in_flight);
    }
    if (progressed) s->cv_done.notify_all();
    admit(s);
    for (StepSlot& st : s->steps)
      if (!st.busy && launch_step(s, st)) progressed = true;
    bool busy = false;
    for (StepSlot& st : s->steps) busy |= st.busy;
    if (s->stop && !busy && s->pending.empty()) break;
    if (!busy && s->pending.empty() && !progressed) {
      s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
    } else if (!progressed) {
      // steps in flight: poll briefly without holding the lock
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(5));
      lk.lock();
    }
  }
}

void free_server(gp_server* s) {
  if (s->ev_ref) cudaEventDestroy(s->ev_ref);
  for (StepSlot& st : s->steps) {
    if (st.stream) cudaStreamDestroy(st.stream);
    if (st.ev0) cudaEventDestroy(st.ev0);
    if (st.ev1) cudaEventDestroy(st.ev1);
    if (st.h_block) cudaFreeHost(st.h_block);
    if (st.d_block) cudaFree(st.d_block);
    if (st.h_rec) cudaFreeHost(st.h_rec);
  }
  for (auto& kv : s->meshes) {
    Mesh& m = kv.second;
    if (m.resident) {
      if (m.d_idx) cudaFree(m.d_idx);
      if (m.d_vtx) cudaFree(m.d_vtx);
      release_partition(m.part);
    }
    if (m.h_idx) cudaFreeHost(m.h_idx);
    if (m.h_vtx) cudaFreeHost(m.h_vtx);
  }
  if (s->upload) cudaStreamDestroy(s->upload);
  delete s;
}

gp_status submit_one(gp_server* s, uint64_t mesh, uint32_t shader, const void* uniforms, uint32_t ubytes,
                     float* d_out, uint64_t cap, uint64_t* out_req) {
  gp_ctx* c = s->ctx;
  Uniforms u;
  {
    std::lock_guard<std::mutex> clk(c->mu);
    gp_status st = make_uniforms(c, shader, uniforms, ubytes, u);
    if (st != GP_OK) return st;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->meshes.find(mesh);
  if (it == s->meshes.end()) return GP_ERR_INVALID;
  Mesh& m = it->second;
  const uint64_t T = m.num_idx / 3;
  if (shader > GP_SHADER_LOAD) return GP_ERR_INVALID;
  if ((shader == GP_SHADER_SKIN) != (m.format == GP_VFMT_SKIN64)) return GP_ERR_INVALID;
  if (T && (!d_out || reinterpret_cast<uintptr_t>(d_out) % 16)) return GP_ERR_INVALID;
  if (cap < T * 3 * out_floats((int)shader) * 4) return GP_ERR_INVALID;
  if (m.num_idx * 4 + m.num_verts * m.stride > s->cfg.mem_budget_bytes) return GP_ERR_BUSY;
  Request r;
  r.id = s->next_req++;
  r.mesh = mesh;
  r.shader = shader;
  r.uni = u;
  r.d_out = d_out;
  r.arrival = Clock::now();
  if (!s->have_first) {
    s->first_submit = r.arrival;
    s->have_first = true;
  }
  s->reqs[r.id] = r;
  s->pending.push_back(r.id);
  s->submitted += 1;
  if (out_req) *out_req = r.id;
  s->cv_work.notify_one();
  return GP_OK;
}

}  // namespace

extern "C" {

gp_status gp_server_create(gp_ctx* c, const gp_serve_config* cfg_in, gp_server** out) {
  if (!c || !out) return GP_ERR_INVALID;
  *out = nullptr;
  gp_server* s = new gp_server();
  s->ctx = c;
  if (cfg_in) s->cfg = *cfg_in;
  gp_serve_config& cfg = s->cfg;
  if (!cfg.mem_budget_bytes) cfg.mem_budget_bytes = 20ull << 30;
  if (!cfg.streams) cfg.streams = 2;
  if (!cfg.step_max_batches) cfg.step_max_batches = 32768;
  if (!cfg.max_active) cfg.max_active = 4096;
  if (!cfg_in) {
    cfg.variant = GP_HASH;
    cfg.mode = GP_BATCH_DYNAMIC;
  }
  gp_draw_config k{};
  k.variant = cfg.variant == GP_AUTO ? GP_HASH : cfg.variant;
  k.mode = cfg.mode;
  k.batch_indices = cfg.batch_indices;
  k.max_unique = cfg.max_unique;
  k.max_tris = cfg.max_tris;
  k.threads_per_group = cfg.threads_per_group;
  if (cfg.variant < GP_NAIVE || cfg.variant > GP_AUTO || cfg.streams > 16 || cfg.step_max_batches > (1u << 20)) {
    delete s;
    return GP_ERR_INVALID;
  }
  // defaults of a concrete method (the same rules as frame draws)
  if (k.variant == GP_NAIVE) {
    k.mode = GP_BATCH_STATIC;
  } else if (k.variant == GP_WARP) {
    k.mode = GP_BATCH_STATIC;
    if (!k.batch_indices) k.batch_indices = 96;
  } else {
    if (!k.threads_per_group) k.threads_per_group = 256;
    if (k.mode == GP_BATCH_STATIC && !k.batch_indices) k.batch_indices = 255;
    if (k.mode == GP_BATCH_DYNAMIC) {
      if (!k.max_unique) k.max_unique = 256;
      if (!k.max_tris) k.max_tris = (4 * k.max_unique - 1) / 3;
    }
  }
  if ((k.batch_indices % 3) || (k.variant == GP_WARP && k.batch_indices > 384)) {
    delete s;
    return GP_ERR_INVALID;
  }
  if (k.variant >= GP_SORT && k.variant <= GP_PHASH) {  // the groups' shared memory in the frame kernel
    if (k.threads_per_group != 64 && k.threads_per_group != 128 && k.threads_per_group != kFrameThreads) {
      delete s;
      return GP_ERR_INVALID;
    }
    const int method = k.variant == GP_SORT ? kFrameSort : (k.variant == GP_HASH ? kFrameHash : kFramePHash);
    for (uint32_t sh = 0; sh < 4; ++sh) {
      DrawArgs a{};
      a.max_batch_idx = k.mode == GP_BATCH_STATIC ? k.batch_indices : 3 * k.max_tris;
      a.ucap = k.mode == GP_BATCH_STATIC ? k.batch_indices : k.max_unique;
      const uint32_t need = frame_capacities(a, method, sh, k.threads_per_group);
      if (need == 0 || need > kFrameSliceBytes) {
        delete s;
        return GP_ERR_UNSUPPORTED;
      }
    }
  }
  s->k = k;
  cudaSetDevice(c->device);
  cudaError_t e = cudaStreamCreateWithFlags(&s->upload, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&s->ev_ref);
  s->steps.resize(cfg.streams);
  for (StepSlot& st : s->steps) {
    if (e != cudaSuccess) break;
    if ((e = cudaStreamCreateWithFlags(&st.stream, cudaStreamNonBlocking)) != cudaSuccess) break;
    if ((e = cudaEventCreate(&st.ev0)) != cudaSuccess) break;
    if ((e = cudaEventCreate(&st.ev1)) != cudaSuccess) break;
    st.block_bytes = step_block_bytes(kStepMaxEntries, cfg.step_max_batches);
    if ((e = cudaMallocHost(&st.h_block, st.block_bytes)) != cudaSuccess) break;
    if ((e = cudaMalloc(&st.d_block, st.block_bytes)) != cudaSuccess) break;
    if ((e = cudaMallocHost(&st.h_rec, sizeof(DevRec))) != cudaSuccess) break;
  }
  if (e != cudaSuccess) {
    free_server(s);
    return e == cudaErrorMemoryAllocation ? GP_ERR_OOM : GP_ERR_CUDA;
  }
  for (uint32_t i = 0; i < cfg.max_active; ++i) s->free_slots.push_back(cfg.max_active - 1 - i);
  s->frame_bpsm = std::max(1, frame_blocks_per_sm());
  s->thread = std::thread(server_loop, s);
  *out = s;
  return GP_OK;
}

gp_status gp_server_add_mesh(gp_server* s, const uint32_t* indices_host, uint64_t num_indices,
                             const void* vertices_host, uint64_t num_vertices, uint32_t stride_bytes, uint32_t format,
                             uint64_t* out_mesh) {
  if (!s || !out_mesh) return GP_ERR_INVALID;
  if (num_indices % 3 || num_indices >= 0xFFFFFFF0ull || num_vertices >= 0x80000000ull) return GP_ERR_INVALID;
  if ((num_indices && !indices_host) || (num_vertices && !vertices_host)) return GP_ERR_INVALID;
  if (format != GP_VFMT_PNU32 && format != GP_VFMT_SKIN64) return GP_ERR_INVALID;
  if (stride_bytes % 16 || stride_bytes < (format == GP_VFMT_SKIN64 ? 64u : 32u)) return GP_ERR_INVALID;
  Mesh m;
  cudaSetDevice(s->ctx->device);
  if (cudaMallocHost(reinterpret_cast<void**>(&m.h_idx), std::max<uint64_t>(num_indices * 4, 16)) != cudaSuccess ||
      cudaMallocHost(&m.h_vtx, std::max<uint64_t>(num_vertices * stride_bytes, 16)) != cudaSuccess) {
    if (m.h_idx) cudaFreeHost(m.h_idx);
    return GP_ERR_OOM;
  }
  if (num_indices) std::memcpy(m.h_idx, indices_host, num_indices * 4);
  if (num_vertices) std::memcpy(m.h_vtx, vertices_host, num_vertices * stride_bytes);
  m.num_idx = num_indices;
  m.num_verts = num_vertices;
  m.stride = stride_bytes;
  m.format = format;
  std::lock_guard<std::mutex> lk(s->mu);
  m.id = s->next_mesh++;
  s->meshes[m.id] = m;
  *out_mesh = m.id;
  return GP_OK;
}

gp_status gp_server_submit(gp_server* s, uint64_t mesh, uint32_t shader_id, const void* uniforms,
                           uint32_t uniforms_bytes, float* d_out, uint64_t out_capacity_bytes, uint64_t* out_request) {
  if (!s) return GP_ERR_INVALID;
  return submit_one(s, mesh, shader_id, uniforms, uniforms_bytes, d_out, out_capacity_bytes, out_request);
}

gp_status gp_server_replay(gp_server* s, uint32_t n, const double* arrival_s, const uint64_t* meshes,
                           const uint32_t* shader_ids, const void* const* uniforms, const uint32_t* uniforms_bytes,
                           float* const* d_outs, const uint64_t* out_capacity_bytes, uint64_t* out_requests) {
  if (!s) return GP_ERR_INVALID;
  if (n && (!arrival_s || !meshes || !shader_ids || !uniforms || !uniforms_bytes || !d_outs || !out_capacity_bytes))
    return GP_ERR_INVALID;
  const Clock::time_point t0 = Clock::now();
  for (uint32_t i = 0; i < n; ++i) {
    const Clock::time_point due = t0 + std::chrono::duration_cast<Clock::duration>(
                                           std::chrono::duration<double>(arrival_s[i]));
    while (Clock::now() < due) {
      const auto left = due - Clock::now();
      if (left > std::chrono::microseconds(200)) std::this_thread::sleep_for(left - std::chrono::microseconds(100));
      else std::this_thread::yield();
    }
    uint64_t id = 0;
    gp_status st = submit_one(s, meshes[i], shader_ids[i], uniforms[i], uniforms_bytes[i], d_outs[i],
                              out_capacity_bytes[i], &id);
    if (st != GP_OK) return st;
    if (out_requests) out_requests[i] = id;
  }
  return GP_OK;
}

gp_status gp_server_wait(gp_server* s, uint64_t request, uint32_t timeout_ms) {
  if (!s) return GP_ERR_INVALID;
  std::unique_lock<std::mutex> lk(s->mu);
  auto ready = [&]() {
    if (request == 0) return s->completed >= s->submitted;
    auto it = s->reqs.find(request);
    return it == s->reqs.end() || it->second.finished;
  };
  if (timeout_ms == 0) {
    s->cv_done.wait(lk, ready);
  } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
    return GP_ERR_TIMEOUT;
  }
  if (request == 0) return s->last_error == GP_ERR_INDEX_RANGE ? GP_ERR_INDEX_RANGE : GP_OK;
  auto it = s->reqs.find(request);
  if (it == s->reqs.end()) return GP_ERR_INVALID;
  return it->second.status;
}

gp_status gp_server_latency(gp_server* s, uint64_t request, double* out_ms) {
  if (!s || !out_ms) return GP_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(request);
  if (it == s->reqs.end() || !it->second.finished) return GP_ERR_INVALID;
  *out_ms = ms_between(it->second.arrival, it->second.done_at);
  return GP_OK;
}

gp_status gp_server_stats(gp_server* s, gp_serve_stats* out, int reset) {
  if (!s || !out) return GP_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(out, 0, sizeof(*out));
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->triangles = s->s_tris;
  out->invocations = s->s_inv;
  out->steps = s->s_steps;
  out->uploads = s->s_uploads;
  out->evictions = s->s_evictions;
  out->resident_bytes = s->resident_bytes;
  out->busy_ms = s->s_busy;
  {  // union of the step intervals
    std::vector<std::pair<float, float>> iv = s->step_iv;
    out->device_ms = s->dev_folded + union_ms(iv);
  }
  out->last_error = (uint32_t)s->last_error;
  if (s->have_first && s->completed) out->wall_ms = ms_between(s->first_submit, s->last_done);
  if (!s->lat.empty()) {
    std::vector<double> v = s->lat;
    std::sort(v.begin(), v.end());
    auto pct = [&](double q) { return v[(size_t)std::min<double>(v.size() - 1, std::ceil(q * v.size()) - 1)]; };
    out->p50_ms = pct(0.5);
    out->p99_ms = pct(0.99);
    out->max_ms = v.back();
  }
  if (reset) {
    s->lat.clear();
    s->s_tris = s->s_inv = s->s_steps = s->s_uploads = s->s_evictions = 0;
    s->s_busy = 0.0;
    s->step_iv.clear();
    s->dev_folded = 0.0;
    s->ref_set = false;
    s->have_first = false;
    s->last_error = GP_OK;
    // forget finished requests (their ids stay unique)
    for (auto it = s->reqs.begin(); it != s->reqs.end();) {
      if (it->second.finished) it = s->reqs.erase(it);
      else ++it;
    }
    s->submitted -= s->completed;
    s->completed = 0;
  }
  return GP_OK;
}

gp_status gp_server_destroy(gp_server* s) {
  if (!s) return GP_ERR_INVALID;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->thread.joinable()) s->thread.join();
  cudaSetDevice(s->ctx->device);
  for (StepSlot& st : s->steps)
    if (st.stream) cudaStreamSynchronize(st.stream);
  free_server(s);
  return GP_OK;
}

}  // extern "C"
