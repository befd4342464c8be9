// Internal runtime state shared by the C-ABI translation units (single
// draws, frames, the serving loop): the context, tickets, partitions and the
// helpers that act on them.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <deque>
#include <mutex>
#include <string>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "gp.h"
#include "gp_internal.h"

namespace gp {
namespace rt {

constexpr uint32_t kRing = 1024;  // in-flight draws with their own device record

// Per-draw device record: error word and counters (CNT_* slots).
struct alignas(128) DevRec {
  uint32_t err;
  uint32_t pad;
  unsigned long long cnt[15];
};
static_assert(sizeof(DevRec) == 128, "device record layout");

struct Ticket {
  uint64_t id = 0;
  uint32_t slot = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  uint64_t draws = 1;
  uint64_t tris = 0, indices = 0;
  uint64_t host_inv = 0, host_batches = 0;  // counts known on the host (naive)
  bool device_counts = false;
  uint64_t out_bytes = 0;
  uint64_t vertex_bytes_per_inv = 0;
  const DevRec* ext_rec = nullptr;          // a frame's own record instead of the ring slot
};

struct Partition {
  const uint32_t* idx = nullptr;
  uint64_t num_idx = 0;
  uint32_t* d_starts = nullptr;  // count + 1 entries
  uint32_t* d_count = nullptr;
  uint32_t* d_seg = nullptr;     // seg_starts, then seg_counts (2 x nseg)
  uint32_t max_batches = 0;
  uint32_t num_segments = 0, seg_cap = 0;
  uint32_t max_unique = 0, max_tris = 0, segment_tris = 0;
  cudaEvent_t done = nullptr;
  bool count_known = false;
  uint64_t count = 0;
};

// Capacities of a sort/hash/phash frame draw whose max_batch_idx, ucap and
// num_verts are set: hash table, sort keys and, when the group is the whole
// block (the pipelined path), the output chunk.  Returns the shared memory
// its groups need in a block (at most kFrameSliceBytes to run), 0 if a
// batch cannot run that way.
uint32_t frame_capacities(DrawArgs& a, int method, uint32_t shader, uint32_t group);
uint32_t next_pow2(uint32_t x);
uint32_t log2u(uint32_t x);
const char* status_name(gp_status s);

}  // namespace rt
}  // namespace gp

struct gp_ctx {
  std::mutex mu;
  gp_config cfg{};
  cudaStream_t stream = nullptr;
  cudaStream_t aux = nullptr;
  int device = 0;
  int sms = 0;
  gp::rt::DevRec* d_rec = nullptr;
  gp::rt::DevRec* h_rec = nullptr;  // pinned mirror
  std::deque<gp::rt::Ticket> inflight;
  uint64_t next_ticket = 1;
  std::vector<cudaEvent_t> events;
  std::unordered_map<uint64_t, gp::rt::Partition> parts;
  uint64_t next_part = 1;
  gp::rt::Partition temp_part;  // submit-time partition scratch (dynamic draw without a handle)
  // statistics of folded draws
  uint64_t s_draws = 0, s_tris = 0, s_idx = 0, s_inv = 0, s_batches = 0, s_bytes = 0;
  double s_busy = 0.0;
  std::vector<float> s_lat;
  // errors
  gp_status last_status = GP_OK;
  std::string last_error;
  // failure injection (gp_test_inject): allocations to fail, draws whose
  // kernel is to stall on its first index window
  uint32_t test_fail_allocs = 0;
  uint32_t test_stall_draws = 0;
  // host-draw staging
  void* h_idx = nullptr;
  size_t h_idx_cap = 0;
  void* h_vtx = nullptr;
  size_t h_vtx_cap = 0;
  void* h_out = nullptr;
  size_t h_out_cap = 0;
  // occupancy cache: key -> blocks per SM
  std::unordered_map<uint64_t, int> occ;
  std::unordered_set<uint64_t> logged;
  // autotune table (frame draws with GP_AUTO), see gp_frame_api.cpp
  std::vector<gp_autotune_entry> tune;
  // gp_draw_host: copy streams (created on first use), so that uploads, draws
  // and read-backs of consecutive chunks overlap; dynamic batches: one
  // partition per chunk, run on their own stream as the chunk's indices arrive
  cudaStream_t copy_in = nullptr, copy_out = nullptr, part_stream = nullptr;
  std::vector<gp::rt::Partition> host_parts;
  // GP_MULTI: shaded vertex rows (32 B each), grown to the largest vertex buffer drawn
  float4* d_shaded = nullptr;
  size_t shaded_cap = 0;  // vertices
};

namespace gp {
namespace rt {

gp_status fail(gp_ctx* c, gp_status s, const std::string& msg);
gp_status cuda_fail(gp_ctx* c, cudaError_t e, const char* what);
cudaEvent_t get_event(gp_ctx* c);
void put_event(gp_ctx* c, cudaEvent_t e);
void release_partition(Partition& p);
gp_status wait_event(gp_ctx* c, cudaEvent_t e, uint32_t timeout_ms);
gp_status sync_locked(gp_ctx* c, uint64_t ticket, uint32_t timeout_ms);
gp_status make_uniforms(gp_ctx* c, uint32_t shader, const void* blob, uint32_t bytes, Uniforms& u);
gp_status size_partition(gp_ctx* c, Partition& p, uint64_t num_idx, bool reuse_alloc, uint32_t max_unique,
                         uint32_t max_tris, uint32_t segment_tris);
gp_status run_partition(gp_ctx* c, Partition& p, const uint32_t* idx, uint64_t num_idx, cudaStream_t stream);
gp_status check_index_buf(gp_ctx* c, const gp_index_buf* ib);
gp_status check_draw(gp_ctx* c, const gp_index_buf* ib, const gp_vertex_buf* vb, uint32_t shader,
                     const gp_out_buf* ob);
// Reserves a ticket id and a ring slot (folding the oldest draw if the ring is full).
gp_status new_ticket(gp_ctx* c, Ticket& t);

}  // namespace rt
}  // namespace gp

#define GP_CUDA(ctx, call)                                                \
  do {                                                                    \
    cudaError_t e_ = (call);                                              \
    if (e_ != cudaSuccess) return gp::rt::cuda_fail(ctx, e_, #call);      \
  } while (0)
