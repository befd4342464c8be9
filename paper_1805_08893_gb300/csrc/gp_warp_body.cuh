// One static batch of statically batched warp voting (Algorithm 1,
// Section 3.3), processed by one warp: shared by the single-draw warp kernel
// and the multi-draw frame kernel.
//
// A round assigns each new vertex index to the lowest free lane, in index
// order, until all 32 lanes hold a vertex or the batch ends; the corners
// before the first index that found no lane are "done"; floor(done/3)
// triangles are assembled from the shaded lanes through shuffles, and the
// next round starts after them (so a vertex of a cut-off triangle is shaded
// again).  The paper finds duplicates with a 32-step shuffle+ballot loop per
// chunk; here the chunk-internal duplicates come from one __match_any_sync,
// the new lanes are ranked with a ballot + popc, and the check against the
// vertices already held in earlier chunks of the round reads the warp's
// held-id list in shared memory.  The lane assignment is exactly the paper's:
// the k-th new index of the round goes to lane k.
#pragma once

#include "gp_device.cuh"

namespace gp {

constexpr uint32_t kWarpMaxBatch = 384;  // indices per warp batch (multiple of 3)

// Per-warp shared memory: stage[32*F + 4] f32, held[32] u32, idx[batch] u32,
// map[batch] u8; every part a multiple of 16 bytes.
template <int SH>
struct WarpSmem {
  static constexpr int K = ShaderTraits<SH>::K;
  static constexpr int F = 3 * K;
  __host__ __device__ static uint32_t idx_words(uint32_t batch) { return (batch + 3) & ~3u; }
  __host__ __device__ static uint32_t map_bytes(uint32_t batch) { return (batch + 15) & ~15u; }
  __host__ __device__ static uint32_t stage_floats() { return 32 * F + 4; }
  __host__ __device__ static uint32_t per_warp_bytes(uint32_t batch) {
    return idx_words(batch) * 4 + map_bytes(batch) + 32 * 4 + stage_floats() * 4;
  }
};

// One round of Algorithm 1 over the batch's ids widx[0..n), starting at
// index c: assigns each new id to the lowest free lane (held[lane] = id) in
// index order until 32 lanes are held or the batch ends, and records for the
// round's "done" indices (those before the first index that found no lane)
// the lane holding their id (map[0..done)).  Every lane of the warp calls it.
__device__ __forceinline__ void warp_vote_round(const uint32_t* widx, uint32_t n, uint32_t c, uint32_t* held,
                                                unsigned char* map, uint32_t lane, uint32_t& fill_out,
                                                uint32_t& done_out) {
  uint32_t fill = 0, done = 0, off = c;
  while (off < n && fill < 32) {
    const uint32_t pos = off + lane;
    const bool valid = pos < n;
    const uint32_t x = valid ? widx[pos] : kEmpty;
    int hs = -1;  // lane already holding x (earlier chunks of the round)
    for (uint32_t h = 0; h < fill; ++h)
      if (held[h] == x) hs = (int)h;
    const uint32_t grp = __match_any_sync(kFull, x);
    const uint32_t leader = __ffs(grp) - 1;
    const bool is_new = valid && hs < 0 && leader == lane;
    const uint32_t newmask = __ballot_sync(kFull, is_new);
    const uint32_t rank = __popc(newmask & lanemask_lt());
    const int myslot = (is_new && fill + rank < 32) ? (int)(fill + rank) : -1;
    if (myslot >= 0) held[myslot] = x;
    const int ls = __shfl_sync(kFull, myslot, leader);
    const int slot = !valid ? -1 : (hs >= 0 ? hs : ls);
    const uint32_t stop = __ballot_sync(kFull, slot < 0);
    const uint32_t fb = stop ? (uint32_t)(__ffs(stop) - 1) : 32u;
    if (lane < fb) map[done + lane] = (unsigned char)slot;
    done += fb;
    fill = min(32u, fill + __popc(newmask));
    off += 32;
    __syncwarp();
  }
  fill_out = fill;
  done_out = done;
}

// Processes static batch b (indices [b*S, min((b+1)*S, 3T))) with the warp's
// shared memory at wp; returns the shader invocations.
template <int SH>
__device__ __forceinline__ uint32_t warp_vote_batch(const DrawArgs& a, const Uniforms& u, const float* palette,
                                                    uint32_t b, unsigned char* wp, uint32_t lane) {
  using L = WarpSmem<SH>;
  constexpr int K = L::K;
  constexpr int F = L::F;
  const uint32_t S = 3u * a.static_batch_tris;
  float* stage = reinterpret_cast<float*>(wp);
  uint32_t* held = reinterpret_cast<uint32_t*>(wp + L::stage_floats() * 4);
  uint32_t* widx = held + 32;
  unsigned char* map = reinterpret_cast<unsigned char*>(widx + L::idx_words(S));
  const uint32_t B0 = b * S;
  const uint32_t B1 = min(B0 + S, a.num_idx);
  const uint32_t n = B1 - B0;
  for (uint32_t i = lane; i < n; i += 32) {
    uint32_t id = __ldg(a.idx + B0 + i);
    widx[i] = id < a.num_verts ? id : kInvalidId;
  }
  __syncwarp();
  uint32_t inv = 0;
  uint32_t c = 0;  // round start, relative to B0
  while (c < n) {
    uint32_t fill, done;
    warp_vote_round(widx, n, c, held, map, lane, fill, done);
    const uint32_t tris = done / 3;
    if (tris == 0) {  // cannot happen: a round's first chunk always places its lanes
      if (lane == 0) atomicOr(a.err, EBIT_CAPACITY);
      break;
    }
    float v[K];
    if (lane < fill) {
      fetch_and_shade<SH>(a, u, palette, held[lane], v);
    } else {
#pragma unroll
      for (int k = 0; k < K; ++k) v[k] = 0.f;
    }
    inv += fill;
    // emit triangles [ (B0 + c)/3, +tris ) in passes of up to 32 triangles
    const uint32_t tfirst = (B0 + c) / 3;
    for (uint32_t p = 0; p < tris; p += 32) {
      const uint32_t np = min(32u, tris - p);
      const size_t g0 = (size_t)(tfirst + p) * F;
      const uint32_t pad = (uint32_t)(g0 & 3);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const uint32_t cc = q * 32 + lane;
        const bool live = cc < 3 * np;
        const uint32_t s = live ? map[3 * p + cc] : 0u;
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const float val = __shfl_sync(kFull, v[k], s);
          if (live) stage[pad + cc * K + k] = val;
        }
        if (live && a.corner_ids != nullptr) a.corner_ids[B0 + c + 3 * p + cc] = held[s];
      }
      __syncwarp();
      const uint32_t nfl = np * F;
      const uint32_t head = min(nfl, (4u - pad) & 3u);
      float* dst = a.out + g0;
      const float* src = stage + pad;
      if (lane < head) dst[lane] = src[lane];
      const uint32_t n4 = (nfl - head) >> 2;
      float4* d4 = reinterpret_cast<float4*>(dst + head);
      const float4* s4 = reinterpret_cast<const float4*>(src + head);
      for (uint32_t i = lane; i < n4; i += 32) __stcs(d4 + i, s4[i]);
      for (uint32_t i = head + (n4 << 2) + lane; i < nfl; i += 32) dst[i] = src[i];
      __syncwarp();
    }
    c += 3 * tris;
  }
  return inv;
}

}  // namespace gp
