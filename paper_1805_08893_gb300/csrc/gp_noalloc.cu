// gp_partition_noalloc: the dynamic batch partition for callers that must not
// allocate device memory.
//
// Some callers cannot call cudaMalloc: a real-time frame loop, where an
// allocation can synchronise the device and stall a frame, or a host
// application that owns all device memory through its own pool and forbids
// allocations outside it.  gp_partition needs a context, and a context
// allocates its scratch.  This entry point runs the same partition kernels
// with their scratch (per-segment batch-start lists, counts, offsets and an
// error word) in one file-scope device array instead, so the call allocates
// nothing; the caller passes the index buffer and the output buffers.
//
// The array is fixed at kNoAllocScratchBytes per device and every GPU that
// loads the library keeps it until the process exits.  All calls on a device
// share it, and it keeps the last call's contents, so calls whose work
// overlaps on the GPU (on different streams, or from different threads)
// race on it; calls on one stream are ordered and safe.
#include <algorithm>
#include <mutex>
#include <string>

#include "gp.h"
#include "gp_device.cuh"

namespace gp {

constexpr size_t kNoAllocScratchBytes = 4u << 20;  // 4 MiB
constexpr size_t kNoAllocScratchWords = kNoAllocScratchBytes / 4;

static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocScratchWords];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
uint32_t* g_noalloc_ptr[kMaxDevices] = {};  // device address of the array, per device

// The array's name in host code is only a host-side stand-in; the device
// address comes from cudaGetSymbolAddress, once per device, with that device
// current.
cudaError_t scratch_address(int device, uint32_t** out) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[device] = static_cast<uint32_t*>(p);
  }
  *out = g_noalloc_ptr[device];
  return cudaSuccess;
}

uint32_t next_pow2_u32(uint32_t x) {
  uint32_t p = 1;
  while (p < x) p <<= 1;
  return p;
}
}  // namespace

}  // namespace gp

extern "C" gp_status gp_partition_noalloc(const uint32_t* d_indices, uint64_t num_indices, uint32_t max_unique,
                                          uint32_t max_tris, uint32_t segment_tris, uint32_t* d_starts,
                                          uint64_t starts_capacity, uint32_t* d_num_batches, void* stream) {
  using namespace gp;
  auto invalid = [](const char* why) {
    set_thread_error(why);
    return GP_ERR_INVALID;
  };
  if (num_indices % 3 || num_indices >= 0xFFFFFFF0ull)
    return invalid("gp_partition_noalloc: num_indices must be a multiple of 3 and < 2^32 - 16");
  if ((num_indices && !d_indices) || !d_starts || !d_num_batches)
    return invalid("gp_partition_noalloc: NULL buffer");
  if (reinterpret_cast<uintptr_t>(d_indices) % 16)
    return invalid("gp_partition_noalloc: d_indices must be 16-byte aligned");
  if (max_unique < 3 || max_unique > 4096 || max_tris < 1 || max_tris > 1365)
    return invalid("gp_partition_noalloc: need 3 <= max_unique <= 4096 and 1 <= max_tris <= 1365");
  const uint32_t T = (uint32_t)(num_indices / 3);
  if (starts_capacity < (uint64_t)T + 1)
    return invalid("gp_partition_noalloc: starts_capacity must be at least num_indices / 3 + 1");
  if (segment_tris == 0) segment_tris = 4096;
  const uint32_t seg = segment_tris == GP_SEGMENT_NONE ? (T > 0 ? T : 1u) : segment_tris;
  const uint32_t min_tris = std::max(1u, std::min(max_tris, max_unique / 3));
  const uint32_t nseg = T ? (T + seg - 1) / seg : 0;
  const uint32_t seg_cap = (std::min(seg, std::max(T, 1u)) + min_tris - 1) / min_tris + 1;
  // error word, segment start lists, counts, offsets
  const uint64_t words = 1 + (uint64_t)nseg * seg_cap + 2ull * nseg;
  if (words > kNoAllocScratchWords)
    return invalid("gp_partition_noalloc: this input needs more scratch than the fixed 4 MiB array "
                   "(too many triangles for these limits); use gp_partition");

  int device = 0;
  auto cuda_err = [](const char* what, cudaError_t e) {
    set_thread_error((std::string("gp_partition_noalloc: ") + what + ": " + cudaGetErrorString(e)).c_str());
    return GP_ERR_CUDA;
  };
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return cuda_err("cudaGetDevice", e);
  if (device < 0 || device >= kMaxDevices) return invalid("gp_partition_noalloc: device ordinal out of range");
  uint32_t* scratch = nullptr;
  if ((e = scratch_address(device, &scratch)) != cudaSuccess) return cuda_err("cudaGetSymbolAddress", e);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the error word must start at zero; the other words are written before read
  if ((e = cudaMemsetAsync(scratch, 0, 4, s)) != cudaSuccess) return cuda_err("cudaMemsetAsync", e);

  PartitionArgs a{};
  a.idx = d_indices;
  a.num_tris = T;
  a.max_unique = max_unique;
  a.max_tris = max_tris;
  a.segment_tris = seg;
  a.num_segments = nseg;
  a.seg_cap = seg_cap;
  a.table_slots = next_pow2_u32(2 * (max_unique + 96));
  a.table_bits = 0;
  while ((1u << a.table_bits) < a.table_slots) ++a.table_bits;
  a.err = scratch;
  a.seg_starts = scratch + 1;
  a.seg_counts = scratch + 1 + (size_t)nseg * seg_cap;
  a.starts = d_starts;
  a.num_batches = d_num_batches;
  if ((e = launch_partition(a, 4, s)) != cudaSuccess) return cuda_err("partition launch", e);
  return GP_OK;
}
