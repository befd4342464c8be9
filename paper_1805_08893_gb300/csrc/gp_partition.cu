// Dynamic batching preprocessing (Section 3.4): scan the triangles front to
// back, counting the unique indices of the open batch; close it before the
// triangle that would make it exceed N unique indices or the triangle cap.
//
// The scan is sequential by nature.  To use the whole GPU the triangle list
// is cut into segments of segment_tris triangles, a batch is also closed at
// every segment boundary, and each warp scans one segment:
//   * the batch's maximal window (max_tris triangles) is read into the
//     warp's shared memory in one coalesced pass;
//   * 32 triangles are examined per step, one per lane: each of their three
//     indices goes into a warp-private hash table that keeps, per id, the
//     smallest position at which it occurs in the batch (atomicMin), so an
//     index is new exactly when its position is that minimum;
//   * an inclusive warp scan of the new-index counts gives the unique count
//     after each lane's triangle; the first lane whose count exceeds N ends
//     the batch there.
// A second kernel turns the per-segment lists into one array of batch
// starts (exclusive scan of the segment counts, then a copy).
#include <algorithm>

#include "gp_device.cuh"

namespace gp {

struct PartLayout {
  uint32_t win_words, keys_off, pos_off, per_warp;
};

__host__ __device__ inline PartLayout part_layout(uint32_t max_tris, uint32_t slots) {
  PartLayout L;
  L.win_words = (3 * max_tris + 3) & ~3u;
  L.keys_off = L.win_words * 4;
  L.pos_off = L.keys_off + slots * 4;
  L.per_warp = L.pos_off + slots * 4;
  return L;
}

__device__ __forceinline__ uint32_t part_hash(uint32_t id, uint32_t bits) {
  return bits ? (id * 2654435769u) >> (32 - bits) : 0u;
}

__global__ void __launch_bounds__(256) partition_segments_kernel(const __grid_constant__ PartitionArgs p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const PartLayout L = part_layout(p.max_tris, p.table_slots);
  const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
  const uint32_t seg = blockIdx.x * (blockDim.x >> 5) + warp;
  if (seg >= p.num_segments) return;  // warp-uniform; no block barrier in this kernel
  unsigned char* wb = smem + warp * L.per_warp;
  uint32_t* win = reinterpret_cast<uint32_t*>(wb);
  uint32_t* keys = reinterpret_cast<uint32_t*>(wb + L.keys_off);
  uint32_t* pos = reinterpret_cast<uint32_t*>(wb + L.pos_off);
  const uint32_t mask = p.table_slots - 1;

  const uint32_t seg_begin = seg * p.segment_tris;
  const uint32_t seg_end = min(seg_begin + p.segment_tris, p.num_tris);
  uint32_t* out = p.seg_starts + (size_t)seg * p.seg_cap;
  uint32_t count = 0;
  uint32_t t = seg_begin;
  while (t < seg_end) {
    if (count >= p.seg_cap) {  // cannot happen: seg_cap bounds the batches of a segment
      if (lane == 0) atomicOr(p.err, EBIT_CAPACITY);
      break;
    }
    if (lane == 0) out[count] = t;
    ++count;
    const uint32_t wt = min(p.max_tris, seg_end - t);
    const uint32_t nidx = 3 * wt;
    const uint32_t* src = p.idx + 3 * (size_t)t;
    for (uint32_t i = lane; i < nidx; i += 32) {
      const uint32_t x = __ldg(src + i);
      win[i] = x == kEmpty ? kInvalidId : x;
    }
    for (uint32_t s = lane; s < p.table_slots; s += 32) {
      keys[s] = kEmpty;
      pos[s] = 0xFFFFFFFFu;
    }
    __syncwarp();
    uint32_t nu = 0;    // unique ids of the batch so far
    uint32_t cut = wt;  // triangles the batch takes
    for (uint32_t c = 0; c < wt; c += 32) {
      const uint32_t j = c + lane;
      const bool valid = j < wt;
      // the triangle's three ids: insert them (three independent CAS, then
      // the rare collisions), record their positions (three independent
      // atomicMin), and count the ids whose smallest position is here
      uint32_t x[3], h[3], prev[3];
      if (valid) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          x[k] = win[3 * j + k];
          h[k] = part_hash(x[k], p.table_bits);
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) prev[k] = atomicCAS(&keys[h[k]], kEmpty, x[k]);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          for (uint32_t probes = 0; prev[k] != kEmpty && prev[k] != x[k]; ++probes) {
            if (probes > p.table_slots) {  // cannot happen: the table has room
              atomicOr(p.err, EBIT_CAPACITY);
              break;
            }
            h[k] = (h[k] + 1) & mask;
            prev[k] = atomicCAS(&keys[h[k]], kEmpty, x[k]);
          }
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) atomicMin(&pos[h[k]], 3 * j + k);
      }
      __syncwarp();
      uint32_t fresh = 0;
      if (valid) {
#pragma unroll
        for (int k = 0; k < 3; ++k) fresh += pos[h[k]] == 3 * j + k;
      }
      const uint32_t cum = warp_inclusive_scan(fresh);
      const uint32_t over = __ballot_sync(kFull, valid && nu + cum > p.max_unique);
      if (over) {
        cut = max(1u, c + (uint32_t)(__ffs(over) - 1));
        break;
      }
      nu += __shfl_sync(kFull, cum, 31);
      __syncwarp();
    }
    t += cut;
    __syncwarp();
  }
  if (lane == 0) p.seg_counts[seg] = count;
}

// One block: exclusive scan of the segment counts, then every warp copies
// segments' starts into the final array; starts[total] = T.
__global__ void __launch_bounds__(1024) partition_gather_kernel(const __grid_constant__ PartitionArgs p,
                                                                uint32_t* seg_offsets) {
  __shared__ uint32_t warp_sums[33];
  uint32_t carry = 0;
  for (uint32_t base = 0; base < p.num_segments; base += blockDim.x) {
    const uint32_t s = base + threadIdx.x;
    const uint32_t c = s < p.num_segments ? min(p.seg_counts[s], p.seg_cap) : 0u;
    uint32_t total;
    const uint32_t ex = block_exclusive_scan(c, warp_sums, &total);
    if (s < p.num_segments) seg_offsets[s] = carry + ex;
    carry += total;
    __syncthreads();
  }
  __syncthreads();
  const uint32_t warp = threadIdx.x >> 5, lane = lane_id(), nw = blockDim.x >> 5;
  for (uint32_t s = warp; s < p.num_segments; s += nw) {
    const uint32_t c = min(p.seg_counts[s], p.seg_cap);
    const uint32_t o = seg_offsets[s];
    const uint32_t* src = p.seg_starts + (size_t)s * p.seg_cap;
    for (uint32_t k = lane; k < c; k += 32) p.starts[o + k] = src[k];
  }
  if (threadIdx.x == 0) {
    p.starts[carry] = p.num_tris;
    *p.num_batches = carry;
  }
}

size_t partition_smem_bytes(const PartitionArgs& p, int warps) {
  return (size_t)warps * part_layout(p.max_tris, p.table_slots).per_warp;
}

cudaError_t launch_partition(const PartitionArgs& p, int warps_per_block, cudaStream_t s) {
  if (p.num_segments == 0) {
    // empty index buffer: zero batches
    partition_gather_kernel<<<1, 32, 0, s>>>(p, p.seg_counts);
    return cudaGetLastError();
  }
  // as many warps per block as fit in shared memory (large unique limits
  // need large per-warp tables)
  const size_t per_warp = partition_smem_bytes(p, 1);
  warps_per_block = (int)std::min<size_t>((size_t)warps_per_block, (227u * 1024u) / per_warp);
  if (warps_per_block < 1) return cudaErrorInvalidValue;
  const size_t smem = partition_smem_bytes(p, warps_per_block);
  cudaError_t e = cudaFuncSetAttribute(partition_segments_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const uint32_t blocks = (p.num_segments + warps_per_block - 1) / warps_per_block;
  partition_segments_kernel<<<blocks, warps_per_block * 32, smem, s>>>(p);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // the per-segment offsets reuse the tail of the segment-start scratch
  partition_gather_kernel<<<1, 1024, 0, s>>>(p, p.seg_counts + p.num_segments);
  return cudaGetLastError();
}

}  // namespace gp
