// Multi-draw frame: every draw call of a frame in one persistent launch.
//
// The draws' batches are cut into work items.  Blocks of 256 threads pull
// chunks of consecutive items from a global counter.  An item belongs to one draw and is split
// among the block's thread groups of that draw's size G (threads per group,
// chosen per draw; named barriers keep the groups independent):
//   naive -- one group of 256 threads, one triangle per thread (Section 3.3);
//   warp  -- eight warps, each runs one static batch by warp voting
//            (Algorithm 1);
//   sort / hash / phash, G < 256 -- 256/G groups, each runs one batch
//            (static, or a dynamic batch from the draw's partition) through
//            the dedup-and-shade body of gp_batch_body.cuh;
//   sort / hash / phash, G = 256 -- the whole block runs the batches of
//            consecutive items of the draw through the two-stage pipeline of
//            the single-draw kernel (gp_batch_pipeline.cuh).
// Each group works in its own slice of the block's shared memory, assembles
// its triangles there and writes them with 16-byte streaming stores (the
// pipeline: bulk stores).  The current draw's uniforms (and palette) are
// copied into shared memory when the draw changes.
#include <cstddef>

#include "gp_batch_pipeline.cuh"
#include "gp_warp_body.cuh"

namespace gp {

struct FrameSlice {
  uint32_t off_misc, off_win, off_map, off_keys, off_table, off_dense, off_uniq, off_v, off_stage, total;
};

__host__ __device__ inline uint32_t fr_align(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

// Shared memory of one dedup group (sort/hash/phash).
__host__ __device__ inline FrameSlice frame_slice(int method, int K, int KS, uint32_t max_idx, uint32_t ucap,
                                                  uint32_t slots, uint32_t sort_n, uint32_t group) {
  FrameSlice L;
  uint32_t o = 0;
  L.off_misc = o; o += 32 * 4;
  L.off_win = o; o = fr_align(o + max_idx * 4, 16);
  L.off_map = o; o = fr_align(o + max_idx * 2, 16);
  if (method == kFrameSort) {
    L.off_keys = o; o += sort_n * 8;
    L.off_table = L.off_dense = 0;
  } else {
    L.off_keys = 0;
    L.off_table = o; o += slots * 4;
    L.off_dense = o; o = fr_align(o + slots * 2, 16);
  }
  L.off_uniq = o; o = fr_align(o + ucap * 4, 16);
  L.off_v = o; o = fr_align(o + ucap * KS * 4, 16);
  L.off_stage = o; o = fr_align(o + (fr_align(max_idx, 3) * K + 4) * 4, 16);
  L.total = o;
  return L;
}

uint32_t frame_slice_bytes(int method, int shader, uint32_t max_idx, uint32_t ucap, uint32_t slots, uint32_t sort_n,
                           uint32_t group, uint32_t batch_idx) {
  const int K = shader == 2 ? 8 : 7;
  if (method == kFrameNaive) return (kFrameThreads / 32) * 32 * 3 * K * 4;
  if (method == kFrameWarp) {
    switch (shader) {
      case 0: return (kFrameThreads / 32) * WarpSmem<0>::per_warp_bytes(batch_idx);
      case 1: return (kFrameThreads / 32) * WarpSmem<1>::per_warp_bytes(batch_idx);
      case 2: return (kFrameThreads / 32) * WarpSmem<2>::per_warp_bytes(batch_idx);
      default: return (kFrameThreads / 32) * WarpSmem<3>::per_warp_bytes(batch_idx);
    }
  }
  return frame_slice(method, K, K, max_idx, ucap, slots, sort_n, group).total * (kFrameThreads / group);
}

// 16-byte streaming copy of nfl floats staged at src (16-byte aligned) + pad
// to dst (= out + g0, with pad = g0 mod 4) by nthreads threads.
__device__ __forceinline__ void store_staged(float* dst, const float* src, uint32_t pad, uint32_t nfl, uint32_t t,
                                             uint32_t nthreads) {
  const float* s = src + pad;
  const uint32_t head = min(nfl, (4u - pad) & 3u);
  if (t < head) dst[t] = s[t];
  const uint32_t n4 = (nfl - head) >> 2;
  float4* d4 = reinterpret_cast<float4*>(dst + head);
  const float4* s4 = reinterpret_cast<const float4*>(s + head);
  for (uint32_t i = t; i < n4; i += nthreads) __stcs(d4 + i, s4[i]);
  for (uint32_t i = head + (n4 << 2) + t; i < nfl; i += nthreads) dst[i] = s[i];
}

template <int SH>
__device__ __noinline__ uint2 frame_naive(const FrameDraw& D, const Uniforms& u, uint32_t b, unsigned char* slices) {
  constexpr int K = ShaderTraits<SH>::K;
  constexpr int F = 3 * K;
  const DrawArgs& a = D.a;
  const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = lane_id();
  float* stage = reinterpret_cast<float*>(slices) + warp * (32 * F);
  const uint32_t tb0 = b * kFrameThreads;
  const uint32_t ntb = min(kFrameThreads, a.num_tris - tb0);
  uint2 r = make_uint2(0, 0);
  if (tid == 0) {
    r = make_uint2(3u * ntb, 1u);
    if (a.batch_inv != nullptr && b < a.batch_cap) a.batch_inv[b] = 3u * ntb;
  }
  const uint32_t tw0 = tb0 + warp * 32;
  if (tw0 >= a.num_tris) return r;
  const uint32_t ntw = min(32u, a.num_tris - tw0);
  const uint32_t t = tw0 + lane;
  if (lane < ntw) {
    // the three corners' indices first, so their load latencies overlap
    uint32_t id[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) id[k] = __ldg(a.idx + 3u * t + k);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float o[K];
      fetch_and_shade<SH>(a, u, u.palette, id[k], o);
#pragma unroll
      for (int c = 0; c < K; ++c) stage[lane * F + k * K + c] = o[c];
      if (a.corner_ids != nullptr) a.corner_ids[3u * t + k] = id[k];
    }
  }
  __syncwarp();
  store_staged(a.out + (size_t)tw0 * F, stage, 0, ntw * F, lane, 32);
  return r;
}

template <int SH>
__device__ __noinline__ uint2 frame_warp(const FrameDraw& D, const Uniforms& u, uint32_t item, unsigned char* slices) {
  const DrawArgs& a = D.a;
  const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
  const uint32_t j = item * (kFrameThreads / 32) + warp;
  if (j >= D.num_batches) return make_uint2(0, 0);
  const uint32_t b = D.batch_begin + j;
  unsigned char* wp = slices + warp * WarpSmem<SH>::per_warp_bytes(3u * a.static_batch_tris);
  const uint32_t n = warp_vote_batch<SH>(a, u, u.palette, b, wp, lane);
  if (lane != 0) return make_uint2(0, 0);
  if (a.batch_inv != nullptr && b < a.batch_cap) a.batch_inv[b] = n;
  return make_uint2(n, 1u);
}

template <int METHOD, int SH>
__device__ __noinline__ uint2 frame_group(const FrameDraw& D, const Uniforms& u, uint32_t item,
                                          unsigned char* slices) {
  constexpr int DEDUP = METHOD == kFrameSort ? DEDUP_SORT : (METHOD == kFrameHash ? DEDUP_HASH : DEDUP_PHASH);
  constexpr int K = ShaderTraits<SH>::K;
  constexpr int KS = ShaderTraits<SH>::KS;
  constexpr int F = 3 * K;
  const DrawArgs& a = D.a;
  const uint32_t G = D.group;
  const uint32_t g = threadIdx.x / G, gt = threadIdx.x % G;
  const uint32_t j = item * (kFrameThreads / G) + g;
  if (j >= D.num_batches) return make_uint2(0, 0);  // the whole group is idle; its barrier is not used
  const uint32_t b = D.batch_begin + j;
  const GroupSync sync{g + 1, G};
  const FrameSlice L = frame_slice(METHOD, K, KS, a.max_batch_idx, a.ucap, a.hash_slots, a.sort_n, G);
  unsigned char* base = slices + g * L.total;
  uint32_t* misc = reinterpret_cast<uint32_t*>(base + L.off_misc);
  uint32_t* win = reinterpret_cast<uint32_t*>(base + L.off_win);
  float* stage = reinterpret_cast<float*>(base + L.off_stage);
  BatchSmem S;
  S.map = reinterpret_cast<uint16_t*>(base + L.off_map);
  S.keys = reinterpret_cast<unsigned long long*>(base + L.off_keys);
  S.table = reinterpret_cast<uint32_t*>(base + L.off_table);
  S.dense = reinterpret_cast<uint16_t*>(base + L.off_dense);
  S.uniq = reinterpret_cast<uint32_t*>(base + L.off_uniq);
  S.vsh = reinterpret_cast<float*>(base + L.off_v);
  S.ucount = misc;
  S.wsum = misc + 8;

  uint32_t t0, t1;
  if (D.dynamic) {
    t0 = __ldg(a.starts + b);
    t1 = __ldg(a.starts + b + 1);
  } else {
    t0 = b * a.static_batch_tris;
    t1 = min(t0 + a.static_batch_tris, a.num_tris);
  }
  const uint32_t n = 3 * (t1 - t0);
  if (n > a.max_batch_idx) {  // cannot happen with a consistent configuration
    if (gt == 0) atomicOr(a.err, EBIT_CAPACITY);
    return make_uint2(0, 0);
  }
  for (uint32_t i = gt; i < n; i += G) win[i] = __ldg(a.idx + 3 * t0 + i);
  if (DEDUP != DEDUP_SORT)
    for (uint32_t s = gt; s < a.hash_slots; s += G) S.table[s] = kEmpty;
  if (gt == 0) *S.ucount = 0;
  sync();
  dedup_and_shade<DEDUP, SH>(a, u, u.palette, S, win, n, gt, G, sync);
  sync();
  const uint32_t U = min(*S.ucount, a.ucap);
  const size_t g0 = (size_t)t0 * F;
  const uint32_t pad = (uint32_t)(g0 & 3);
  fill_stage<DEDUP, SH>(a, S, stage + pad, 0, n, U, 3ull * t0, gt, G, pad == 0);
  sync();
  store_staged(a.out + g0, stage, pad, (t1 - t0) * F, gt, G);
  if (gt != 0) return make_uint2(0, 0);
  if (a.batch_inv != nullptr && b < a.batch_cap) a.batch_inv[b] = U;
  return make_uint2(U, 1u);
}

// Per-method bodies are separate (not inlined) functions, each with its own
// register allocation, so the heaviest path does not make every path spill.
template <int SH>
__device__ __forceinline__ uint2 frame_item(const FrameDraw& D, const Uniforms& u, uint32_t item,
                                            unsigned char* slices) {
  switch (D.method) {
    case kFrameNaive: return frame_naive<SH>(D, u, D.batch_begin + item, slices);
    case kFrameWarp: return frame_warp<SH>(D, u, item, slices);
    case kFrameSort: return frame_group<kFrameSort, SH>(D, u, item, slices);
    case kFrameHash: return frame_group<kFrameHash, SH>(D, u, item, slices);
    default: return frame_group<kFramePHash, SH>(D, u, item, slices);
  }
}

// Shared memory of the pipelined path (the layout of the single-draw kernel
// without its palette, which the frame keeps beside the uniforms).
__host__ __device__ inline BatchLayout frame_pipe_layout(int dedup, int shader, const DrawArgs& a) {
  const uint32_t K = shader == 2 ? 8u : 7u;
  return batch_layout(dedup, K, K | 1u, shader == 1 ? 64u : 32u, false, a.max_batch_idx, a.ucap, a.hash_slots,
                      a.sort_n, a.out_chunk);
}

// Batches [b0, b1) of a sort/hash/phash draw whose groups are the whole
// block, through the pipeline.  Returns (unique vertices, batches) for
// thread 0; (~0u, ~0u) on every thread after an aborted run.
template <int DEDUP, int SH, bool DYN>
__device__ __noinline__ uint2 frame_pipe(const FrameDraw& D, const Uniforms& u, unsigned char* slices, PipeBars& pb,
                                         uint32_t b0, uint32_t b1) {
  const BatchLayout L = frame_pipe_layout(DEDUP, SH, D.a);
  unsigned long long inv = 0, nbat = 0;
  if (!pipeline_run<DEDUP, SH, DYN>(D.a, u, u.palette, slices, L, pb, b0, 1u, b1, inv, nbat))
    return make_uint2(~0u, ~0u);
  return make_uint2((uint32_t)inv, (uint32_t)nbat);
}

template <int DEDUP, int SH>
__device__ __forceinline__ uint2 frame_pipe_mode(const FrameDraw& D, const Uniforms& u, unsigned char* slices,
                                                 PipeBars& pb, uint32_t b0, uint32_t b1) {
  return D.dynamic ? frame_pipe<DEDUP, SH, true>(D, u, slices, pb, b0, b1)
                   : frame_pipe<DEDUP, SH, false>(D, u, slices, pb, b0, b1);
}

template <int SH>
__device__ __forceinline__ uint2 frame_pipe_any(const FrameDraw& D, const Uniforms& u, unsigned char* slices,
                                                PipeBars& pb, uint32_t b0, uint32_t b1) {
  switch (D.method) {
    case kFrameSort: return frame_pipe_mode<DEDUP_SORT, SH>(D, u, slices, pb, b0, b1);
    case kFrameHash: return frame_pipe_mode<DEDUP_HASH, SH>(D, u, slices, pb, b0, b1);
    default: return frame_pipe_mode<DEDUP_PHASH, SH>(D, u, slices, pb, b0, b1);
  }
}

// Work items are handed out in chunks of consecutive items from a global
// counter (guided self-scheduling): a chunk is about 1/(4 x blocks) of the
// items left, at least kFrameChunk and at most kFrameMaxChunk, so long runs
// of a draw's batches go through the pipeline while much work is left and
// the last chunks are short.  item_draw[item] names an item's draw, and the
// draw's descriptor is copied to shared memory only when it changes.
constexpr uint32_t kFrameChunk = 8;
constexpr uint32_t kFrameMaxChunk = 64;

// Thread 0: claims the next chunk; returns its first item (>= total when the
// work is done) and its length in *take.
__device__ __forceinline__ uint32_t claim_chunk(uint32_t* work, uint32_t total, uint32_t* take) {
  volatile uint32_t* vw = work;
  uint32_t base = *vw;
  for (uint32_t tries = 0; base < total; ++tries) {
    const uint32_t t = min(kFrameMaxChunk, max(kFrameChunk, (total - base) / (4u * gridDim.x)));
    if (tries == 64) break;  // heavy contention: take a fixed chunk instead
    const uint32_t prev = atomicCAS(work, base, base + t);
    if (prev == base) {
      *take = t;
      return base;
    }
    base = prev;
  }
  *take = kFrameChunk;
  return base < total ? atomicAdd(work, kFrameChunk) : base;
}

__global__ void __launch_bounds__(kFrameThreads, 3) frame_kernel(const FrameDraw* __restrict__ draws,
                                                                 const uint32_t* __restrict__ item_draw,
                                                                 uint32_t total_items, uint32_t* work,
                                                                 unsigned long long* counters) {
  extern __shared__ __align__(128) unsigned char smem[];
  Uniforms* su = reinterpret_cast<Uniforms*>(smem);  // the current draw's uniforms (and palette)
  unsigned char* slices = smem + kFrameUniBytes;
  __shared__ uint32_t s_base, s_take;
  __shared__ __align__(16) FrameDraw s_draw;  // the current item's draw, read from shared memory
  __shared__ __align__(8) uint64_t s_bars[2];  // index-window mbarriers of the pipelined path
  if (threadIdx.x == 0) {
    mbar_init(&s_bars[0], 1);
    mbar_init(&s_bars[1], 1);
    fence_mbar_init();
  }
  PipeBars pb{s_bars, 0u, 0u};
  unsigned long long inv = 0, nbat = 0;
  uint32_t cur_draw = 0xFFFFFFFFu;
  bool aborted = false;
  while (!aborted) {
    if (threadIdx.x == 0) s_base = claim_chunk(work, total_items, &s_take);
    __syncthreads();
    const uint32_t base = s_base;
    if (base >= total_items) break;
    const uint32_t end = min(base + s_take, total_items);
    for (uint32_t item = base; item < end;) {
      const uint32_t d = __ldg(item_draw + item);  // uniform across the block
      if (d != cur_draw) {
        constexpr uint32_t kWords = sizeof(FrameDraw) / 4;
        const uint32_t* src = reinterpret_cast<const uint32_t*>(draws + d);
        uint32_t* dst = reinterpret_cast<uint32_t*>(&s_draw);
        for (uint32_t i = threadIdx.x; i < kWords; i += blockDim.x) dst[i] = src[i];
        // the uniforms; the palette only for skinning
        const FrameDraw* dg = draws + d;
        const uint32_t uw = (dg->shader == 1 ? sizeof(Uniforms) : offsetof(Uniforms, palette)) / 4;
        const uint32_t* usrc = reinterpret_cast<const uint32_t*>(dg->u);
        uint32_t* udst = reinterpret_cast<uint32_t*>(su);
        for (uint32_t i = threadIdx.x; i < uw; i += blockDim.x) udst[i] = usrc[i];
        cur_draw = d;
        __syncthreads();
      }
      const FrameDraw& D = s_draw;
      const Uniforms& u = *su;
      const uint32_t local = item - D.item_begin;
      uint2 r;
      if (D.method >= kFrameSort && D.group == kFrameThreads) {
        // one batch per item: the chunk's items of this draw are one run
        const uint32_t last = min(end, D.item_begin + D.items);
        const uint32_t b0 = D.batch_begin + local, b1 = D.batch_begin + (last - D.item_begin);
        switch (D.shader) {
          case 0: r = frame_pipe_any<0>(D, u, slices, pb, b0, b1); break;
          case 1: r = frame_pipe_any<1>(D, u, slices, pb, b0, b1); break;
          case 2: r = frame_pipe_any<2>(D, u, slices, pb, b0, b1); break;
          default: r = frame_pipe_any<3>(D, u, slices, pb, b0, b1); break;
        }
        if (r.x == ~0u && r.y == ~0u) {  // flagged in the draw's error word; the other blocks go on
          aborted = true;
          break;
        }
        item = last;
      } else {
        switch (D.shader) {
          case 0: r = frame_item<0>(D, u, local, slices); break;
          case 1: r = frame_item<1>(D, u, local, slices); break;
          case 2: r = frame_item<2>(D, u, local, slices); break;
          default: r = frame_item<3>(D, u, local, slices); break;
        }
        ++item;
      }
      inv += r.x;
      nbat += r.y;
      __syncthreads();  // the slices (and possibly the descriptor) are reused by the next item
    }
  }
  if (threadIdx.x == 0) bulk_wait_all<0>();
  // per-thread partial counts (group leaders, warp leaders) into the record
  if (inv) atomicAdd(counters + CNT_INVOCATIONS, inv);
  if (nbat) atomicAdd(counters + CNT_BATCHES, nbat);
}

size_t frame_smem_bytes() { return kFrameUniBytes + kFrameSliceBytes; }

uint32_t frame_pipe_bytes(int method, int shader, const DrawArgs& a) {
  const int dedup = method == kFrameSort ? DEDUP_SORT : (method == kFrameHash ? DEDUP_HASH : DEDUP_PHASH);
  return frame_pipe_layout(dedup, shader, a).total;
}

int frame_blocks_per_sm() {
  const size_t smem = frame_smem_bytes();
  if (cudaFuncSetAttribute(frame_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  cudaFuncSetAttribute(frame_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, frame_kernel, kFrameThreads, smem) != cudaSuccess) return 0;
  return nb;
}

cudaError_t launch_frame(const FrameDraw* d_draws, const uint32_t* d_item_draw, uint32_t total_items,
                         uint32_t* d_work, unsigned long long* d_counters, int grid, cudaStream_t s) {
  const size_t smem = frame_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(frame_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  frame_kernel<<<grid, kFrameThreads, smem, s>>>(d_draws, d_item_draw, total_items, d_work, d_counters);
  return cudaGetLastError();
}

}  // namespace gp
