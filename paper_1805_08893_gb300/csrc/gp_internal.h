// Internal interface between the C-ABI runtime (gp_api.cpp) and the kernel
// launchers (*.cu).  Plain structs, passed by value to the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gp {

// Device error word bits (OR-ed by kernels, read by gp_sync).
enum : uint32_t {
  EBIT_INDEX_RANGE = 1u,  // an index >= num_vertices
  EBIT_TIMEOUT = 2u,      // a bounded mbarrier wait gave up
  EBIT_CAPACITY = 4u,     // a batch exceeded a table/buffer capacity (internal)
};

// Counter slots in the context's device counter array (uint64).
enum : int {
  CNT_INVOCATIONS = 0,
  CNT_BATCHES = 1,
  CNT_UNIQUE = 2,
  CNT_WORK = 3,  // batches claimed beyond the first wave (single-draw reuse kernel)
  CNT_SLOTS = 8,
};

constexpr uint32_t kInvalidId = 0xFFFFFFFEu;  // canonical out-of-range id
constexpr uint32_t kEmpty = 0xFFFFFFFFu;      // empty hash slot / padding key
constexpr int kMaxEnvelopeDirs = 16;
constexpr int kEnvelopeTerms = 32;

// Shader uniforms as the kernels see them (kernel parameter, by value).
struct Uniforms {
  float mvp[16];
  float nrm[9];
  uint32_t steps;        // LOAD
  float d;               // ENVELOPE
  uint32_t num_dirs;     // ENVELOPE
  float inv_dirs;        // ENVELOPE: 1 / num_dirs
  float dirs[kMaxEnvelopeDirs * 3];
  float coef[kEnvelopeTerms];  // ENVELOPE: 1/k!, k = 0..31
  float palette[64 * 12];      // SKIN
};

// One draw as the kernels see it.
struct DrawArgs {
  const uint32_t* idx;           // index buffer
  uint32_t num_idx;              // 3T
  uint32_t num_tris;             // T
  const unsigned char* verts;    // vertex buffer
  uint32_t num_verts;
  uint32_t stride;               // bytes
  uint32_t vec8;                 // 1: vertex rows are 32-byte aligned (256-bit loads)
  float* out;                    // T * 3 * K floats
  uint32_t* corner_ids;          // optional
  uint32_t* batch_inv;           // optional
  uint32_t batch_cap;            // entries in batch_inv
  // batching
  uint32_t static_batch_tris;    // static: triangles per batch (S / 3)
  uint32_t num_batches;          // static: batch count
  const uint32_t* starts;        // dynamic: batch starts (triangles), count+1 entries
  const uint32_t* num_batches_dev;  // dynamic: device batch count
  uint32_t max_batch_idx;        // capacity: indices per batch
  uint32_t ucap;                 // capacity: unique vertices per batch
  uint32_t hash_slots;           // power of two
  uint32_t hash_bits;            // log2(hash_slots)
  uint32_t sort_n;               // power of two >= max_batch_idx
  uint32_t sort_pos_bits;        // sort: 32-bit keys (id << bits | position) with this many position bits; 0 = 64-bit
  uint32_t probe_k;
  uint32_t out_chunk;            // triangles per output bulk store (staging buffer size)
  // bookkeeping
  unsigned long long* counters;  // CNT_* slots
  uint32_t* err;                 // error word
  uint32_t test_stall;           // 1: failure injection, the first index window is never copied
};

struct PartitionArgs {
  const uint32_t* idx;
  uint32_t num_tris;
  uint32_t max_unique;
  uint32_t max_tris;
  uint32_t segment_tris;     // > 0
  uint32_t num_segments;
  uint32_t seg_cap;          // batch-start slots per segment
  uint32_t table_slots;      // per-warp hash slots (power of two)
  uint32_t table_bits;
  uint32_t* seg_starts;      // [num_segments * seg_cap]
  uint32_t* seg_counts;      // [num_segments]
  uint32_t* starts;          // out: [total + 1]
  uint32_t* num_batches;     // out: total (device)
  uint32_t* err;
};

enum Dedup : int { DEDUP_SORT = 0, DEDUP_HASH = 1, DEDUP_PHASH = 2 };

// Launchers (return the launch error).  'shader' is a gp_shader_id.
cudaError_t launch_naive(const DrawArgs& a, const Uniforms& u, int shader, int block, cudaStream_t s);
// Multi-kernel comparator: shade all num_verts vertices into rows (2 float4
// per vertex, caller-owned), then assemble the triangles from them.
cudaError_t launch_multi(const DrawArgs& a, const Uniforms& u, int shader, float4* rows, int block,
                         cudaStream_t s);
cudaError_t launch_warp(const DrawArgs& a, const Uniforms& u, int shader, int warps_per_block,
                        int grid, cudaStream_t s);
int warp_kernel_blocks_per_sm(int shader, int warps_per_block);
size_t warp_kernel_smem(int shader, int warps_per_block, uint32_t batch_idx);

// Single-draw sort/hash/phash kernel (gp_reuse.cu).
size_t reuse_smem_bytes(int dedup, int shader, const DrawArgs& a, int threads);
// Blocks per SM of the 64-register kernel; *wide: the 80-register kernel
// exists for this draw and fits as many (launch it instead).
int reuse_blocks_per_sm(int dedup, bool dynamic, int shader, int threads, size_t smem, bool* wide);
cudaError_t launch_reuse(int dedup, bool dynamic, bool wide, const DrawArgs& a, const Uniforms& u, int shader,
                         int threads, int grid, size_t smem, cudaStream_t s);

size_t partition_smem_bytes(const PartitionArgs& p, int warps);
cudaError_t launch_partition(const PartitionArgs& p, int warps_per_block, cudaStream_t s);

int out_floats(int shader);  // K

// ---- multi-draw frame (gp_frame.cu)
enum FrameMethod : int { kFrameNaive = 0, kFrameWarp = 1, kFrameSort = 2, kFrameHash = 3, kFramePHash = 4 };
constexpr uint32_t kFrameThreads = 256;          // threads per block of the frame kernel
constexpr uint32_t kFrameSliceBytes = 64 * 1024;  // shared memory for the groups of one block
constexpr uint32_t kFrameUniBytes = (sizeof(Uniforms) + 127) / 128 * 128;  // the current draw's uniforms

struct FrameDraw {
  DrawArgs a;               // buffers, batching and capacities of the draw (err/counters: the frame's record)
  const Uniforms* u;        // device copy of the draw's uniforms
  uint32_t method;          // FrameMethod
  uint32_t shader;          // gp_shader_id
  uint32_t dynamic;         // batches from a.starts
  uint32_t group;           // threads per group G (sort/hash/phash)
  uint32_t num_batches;     // batches of this entry: [batch_begin, batch_begin + num_batches)
  uint32_t item_begin;      // first work item of the entry
  uint32_t items;           // work items of the entry
  uint32_t batch_begin;     // first batch (a serving step runs a sub-range of a draw)
};

uint32_t frame_slice_bytes(int method, int shader, uint32_t max_idx, uint32_t ucap, uint32_t slots, uint32_t sort_n,
                           uint32_t group, uint32_t batch_idx);
// Shared memory of a sort/hash/phash draw whose group is the whole block
// (the pipelined path), with the capacities and out_chunk set in 'a'.
uint32_t frame_pipe_bytes(int method, int shader, const DrawArgs& a);
size_t frame_smem_bytes();
int frame_blocks_per_sm();
// item_draw[i]: the entry of draws[] that work item i belongs to.
cudaError_t launch_frame(const FrameDraw* d_draws, const uint32_t* d_item_draw, uint32_t total_items,
                         uint32_t* d_work, unsigned long long* d_counters, int grid, cudaStream_t s);

// Sets the calling thread's context-free error text (gp_last_error(NULL)).
void set_thread_error(const char* msg);

}  // namespace gp
