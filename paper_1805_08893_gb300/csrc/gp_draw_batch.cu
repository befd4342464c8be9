// Block-per-batch vertex reuse: sorting (Algorithm 2), hashing (Algorithm 3)
// and parallel hashing (Section 3.4), over static batches (Section 3.3) or
// the dynamic batches of the partition (Section 3.4).
//
// Per batch, one thread block:
//   1. has the batch's index window in shared memory (bulk copy issued one
//      batch ahead on an mbarrier, so the load overlaps the previous batch);
//   2. finds the unique indices and shades each one once (gp_batch_body.cuh):
//        hash  -- open addressing, multiplicative hash, linear probing with
//                 atomicCAS (map[position] = slot).  The thread whose CAS
//                 stores a new id takes the next dense rank (one shared
//                 counter, warp-aggregated); each warp then shades its new
//                 vertices in full-warp passes;
//        phash -- as hash, but each thread probes at most probe_k slots, then
//                 the warp probes 32 consecutive slots at a time for its
//                 remaining indices (ballot/shuffle);
//        sort  -- bitonic sort of (id, position) keys, tail flags, exclusive
//                 prefix sum: map[position] = rank of the id (ascending ids);
//                 the owner of a group's tail element queues that vertex;
//   3. assembles triangles in input order into a shared staging buffer and
//      writes it with one bulk (TMA) store per chunk (by default the whole
//      batch); the ragged 1..3 floats at an unaligned edge use plain stores.
//
// Three block barriers per batch for hash/phash (window ready; all vertices
// shaded; staging filled), plus the sort network and one scan barrier for sort.
// Blocks are persistent (grid = SMs x resident blocks) and walk the batches
// with a grid stride.
#include "gp_batch_body.cuh"

namespace gp {

struct BatchLayout {
  uint32_t off_bars, off_misc, off_idx, idx_words, off_map, off_keys, off_table, off_dense, off_uniq, off_v,
      off_stage, stage_floats, off_pal, off_wq, total;
};

__host__ __device__ inline uint32_t align_up_u32(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

__host__ __device__ inline BatchLayout batch_layout(int dedup, int K, int KS, bool skin, uint32_t max_idx,
                                                    uint32_t ucap, uint32_t slots, uint32_t sort_n,
                                                    uint32_t out_chunk, uint32_t nthreads) {
  BatchLayout L;
  uint32_t o = 0;
  L.off_bars = o; o += 16;
  L.off_misc = o; o += 64 * 4;
  L.idx_words = align_up_u32(max_idx + 8, 4);
  L.off_idx = o; o += 2 * L.idx_words * 4;
  L.off_map = o; o = align_up_u32(o + max_idx * 2, 16);
  if (dedup == DEDUP_SORT) {
    L.off_keys = o; o += sort_n * 8;
    L.off_table = L.off_dense = 0;
  } else {
    L.off_keys = 0;
    L.off_table = o; o += slots * 4;
    L.off_dense = o; o = align_up_u32(o + slots * 2, 16);
  }
  L.off_uniq = o; o = align_up_u32(o + ucap * 4, 16);
  L.off_v = o; o = align_up_u32(o + ucap * KS * 4, 16);
  L.stage_floats = align_up_u32(out_chunk * 3 * K + 4, 4);
  L.off_stage = o; o += L.stage_floats * 4;
  L.off_pal = o; o += skin ? 768 * 4 : 0;
  L.off_wq = o; o += align_up_u32(nthreads * kIdsPerRound * 2, 16);  // per warp: 32 x kIdsPerRound ranks
  L.total = o;
  return L;
}

template <int DEDUP, int SH, bool DYN>
__global__ void __launch_bounds__(512, 2) batched_kernel(const __grid_constant__ DrawArgs a,
                                                         const __grid_constant__ Uniforms u) {
  constexpr int K = ShaderTraits<SH>::K;
  constexpr int KS = ShaderTraits<SH>::KS;
  constexpr int F = 3 * K;
  extern __shared__ __align__(128) unsigned char smem[];
  const BatchLayout L = batch_layout(DEDUP, K, KS, ShaderTraits<SH>::kSkin, a.max_batch_idx, a.ucap,
                                     a.hash_slots, a.sort_n, a.out_chunk, blockDim.x);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.off_bars);
  uint32_t* misc = reinterpret_cast<uint32_t*>(smem + L.off_misc);  // [0] unique counter, [8..] scan
  uint32_t* idxbuf = reinterpret_cast<uint32_t*>(smem + L.off_idx);
  float* stage = reinterpret_cast<float*>(smem + L.off_stage);
  float* palette = reinterpret_cast<float*>(smem + L.off_pal);
  BatchSmem S;
  S.map = reinterpret_cast<uint16_t*>(smem + L.off_map);
  S.keys = reinterpret_cast<unsigned long long*>(smem + L.off_keys);
  S.table = reinterpret_cast<uint32_t*>(smem + L.off_table);
  S.dense = reinterpret_cast<uint16_t*>(smem + L.off_dense);
  S.uniq = reinterpret_cast<uint32_t*>(smem + L.off_uniq);
  S.vsh = reinterpret_cast<float*>(smem + L.off_v);
  S.wq = reinterpret_cast<uint16_t*>(smem + L.off_wq) + (threadIdx.x >> 5) * (32 * kIdsPerRound);
  S.ucount = misc;
  S.wsum = misc + 8;

  const uint32_t tid = threadIdx.x, NT = blockDim.x;
  const uint32_t nb = DYN ? *a.num_batches_dev : a.num_batches;
  const uint32_t n4 = a.num_idx & ~3u;  // end of the 16-byte-granular part of the index buffer

  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
    *S.ucount = 0;
  }
  if (ShaderTraits<SH>::kSkin)
    for (uint32_t i = tid; i < 768; i += NT) palette[i] = u.palette[i];
  if (DEDUP != DEDUP_SORT)
    for (uint32_t s = tid; s < a.hash_slots; s += NT) S.table[s] = kEmpty;
  __syncthreads();

  auto batch_range = [&](uint32_t b, uint32_t& t0, uint32_t& t1) {
    if (DYN) {
      t0 = __ldg(a.starts + b);
      t1 = __ldg(a.starts + b + 1);
    } else {
      t0 = b * a.static_batch_tris;
      t1 = min(t0 + a.static_batch_tris, a.num_tris);
    }
  };
  // Bulk-copies the 16-byte-aligned superset of the batch's index window
  // (clipped to the 16-byte-granular part of the buffer).  Thread 0 only.
  auto issue_window = [&](uint32_t b, uint32_t buf) {
    uint32_t t0, t1;
    batch_range(b, t0, t1);
    const uint32_t i0 = 3 * t0, i1 = 3 * t1, base = i0 & ~3u;
    const uint32_t end = min((i1 + 3) & ~3u, n4);
    // a window larger than the buffer is refused here and flagged by the consumer
    const uint32_t bytes = (end > base && end - base <= L.idx_words) ? (end - base) * 4 : 0;
    mbar_arrive_expect_tx(&bars[buf], bytes);
    if (bytes) bulk_load(idxbuf + buf * L.idx_words, a.idx + base, bytes, &bars[buf]);
  };

  uint32_t phase0 = 0, phase1 = 0;
  unsigned long long inv_total = 0, nbatches = 0;
  uint32_t buf = 0;
  uint32_t b = blockIdx.x;
  bool aborted = false, next_inflight = false;
  if (tid == 0 && b < nb) issue_window(b, 0);
  for (; b < nb; b += gridDim.x, buf ^= 1) {
    const uint32_t bn = b + gridDim.x;
    next_inflight = bn < nb;
    if (tid == 0 && next_inflight) issue_window(bn, buf ^ 1);
    uint32_t t0, t1;
    batch_range(b, t0, t1);
    const uint32_t i0 = 3 * t0, i1 = 3 * t1, base = i0 & ~3u, n = i1 - i0;
    uint32_t* win = idxbuf + buf * L.idx_words;
    bool bad = n > a.max_batch_idx;  // cannot happen with a consistent partition
    {
      const uint32_t par = buf ? phase1 : phase0;
      bad |= !mbar_wait_bounded(&bars[buf], par, a.err);
      if (buf) phase1 ^= 1; else phase0 ^= 1;
      if (!bad) {
        // indices past the 16-byte-granular part of the buffer (last batch only)
        const uint32_t end = min((i1 + 3) & ~3u, n4);
        const uint32_t p0 = max(i0, end > base ? end : base);
        for (uint32_t i = p0 + tid; i < i1; i += NT) win[i - base] = __ldg(a.idx + i);
      }
      if (__syncthreads_or(bad)) {  // barrier 1: window ready
        if (tid == 0) atomicOr(a.err, EBIT_CAPACITY);
        aborted = true;
        break;
      }
    }
    dedup_and_shade<DEDUP, SH>(a, u, palette, S, win + (i0 - base), n, tid, NT, BlockSync());
    // the previous batch's bulk store must have read the staging buffer
    // before this batch fills it (after the barrier below)
    if (tid == 0) bulk_wait_read<0>();
    __syncthreads();  // barrier 2: every unique vertex shaded, map/dense/uniq complete
    const uint32_t U = min(*S.ucount, a.ucap);
    if (DEDUP != DEDUP_SORT)  // the table is done: clear it for the next batch
      for (uint32_t s = tid; s < a.hash_slots; s += NT) S.table[s] = kEmpty;

    // --- assemble triangles in input order, chunk by chunk
    for (uint32_t ta = t0; ta < t1; ta += a.out_chunk) {
      const uint32_t tb = min(ta + a.out_chunk, t1);
      if (ta != t0) {
        if (tid == 0) bulk_wait_read<0>();
        __syncthreads();  // the previous chunk's bulk store has read the staging buffer
      }
      const size_t g0 = (size_t)ta * F;
      const uint32_t pad = (uint32_t)(g0 & 3);
      float* st = stage + pad;
      fill_stage<DEDUP, SH>(a, S, st, 3 * (ta - t0), 3 * (tb - ta), U, 3ull * ta, tid, NT, pad == 0);
      fence_proxy_async_smem();
      __syncthreads();  // barrier 3: staging filled
      const uint32_t nfl = (tb - ta) * F;
      const uint32_t head = min(nfl, (4u - pad) & 3u);
      const uint32_t nv4 = (nfl - head) >> 2;
      if (tid == 0) {
        if (nv4) bulk_store(a.out + g0 + head, st + head, nv4 * 16);
        bulk_commit();
      }
      if (tid < head) a.out[g0 + tid] = st[tid];
      const uint32_t tail0 = head + (nv4 << 2);
      if (tid < nfl - tail0) a.out[g0 + tail0 + tid] = st[tail0 + tid];
    }
    if (tid == 0) {
      inv_total += U;
      nbatches += 1;
      if (a.batch_inv != nullptr && b < a.batch_cap) a.batch_inv[b] = U;
      *S.ucount = 0;  // every thread read U before barrier 3
    }
  }
  if (aborted && next_inflight) {
    // never leave a bulk load in flight into this block's shared memory
    const uint32_t nbuf = buf ^ 1;
    mbar_wait_bounded(&bars[nbuf], nbuf ? phase1 : phase0, a.err);
  }
  if (tid == 0) {
    bulk_wait_all<0>();
    if (nbatches) {
      atomicAdd(a.counters + CNT_INVOCATIONS, inv_total);
      atomicAdd(a.counters + CNT_BATCHES, nbatches);
      atomicAdd(a.counters + CNT_UNIQUE, inv_total);
    }
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

template <int D, int SH, bool DYN>
static const void* batched_fn() {
  return reinterpret_cast<const void*>(&batched_kernel<D, SH, DYN>);
}

template <int D, bool DYN>
static const void* batched_fn_sh(int shader) {
  switch (shader) {
    case 0: return batched_fn<D, 0, DYN>();
    case 1: return batched_fn<D, 1, DYN>();
    case 2: return batched_fn<D, 2, DYN>();
    default: return batched_fn<D, 3, DYN>();
  }
}

static const void* batched_kernel_ptr(int dedup, bool dyn, int shader) {
  if (dyn) {
    switch (dedup) {
      case DEDUP_SORT: return batched_fn_sh<DEDUP_SORT, true>(shader);
      case DEDUP_HASH: return batched_fn_sh<DEDUP_HASH, true>(shader);
      default: return batched_fn_sh<DEDUP_PHASH, true>(shader);
    }
  }
  switch (dedup) {
    case DEDUP_SORT: return batched_fn_sh<DEDUP_SORT, false>(shader);
    case DEDUP_HASH: return batched_fn_sh<DEDUP_HASH, false>(shader);
    default: return batched_fn_sh<DEDUP_PHASH, false>(shader);
  }
}

size_t batched_smem_bytes(int dedup, int shader, const DrawArgs& a, int threads) {
  const int K = shader == 2 ? 8 : 7;
  const BatchLayout L = batch_layout(dedup, K, K, shader == 1, a.max_batch_idx, a.ucap, a.hash_slots, a.sort_n,
                                     a.out_chunk, (uint32_t)threads);
  return L.total;
}

int batched_blocks_per_sm(int dedup, bool dynamic, int shader, int threads, size_t smem) {
  const void* fn = batched_kernel_ptr(dedup, dynamic, shader);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, smem) != cudaSuccess) return 0;
  return nb;
}

cudaError_t launch_batched(int dedup, bool dynamic, const DrawArgs& a, const Uniforms& u, int shader, int threads,
                           int grid, size_t smem, cudaStream_t s) {
  const void* fn = batched_kernel_ptr(dedup, dynamic, shader);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  void* args[] = {const_cast<DrawArgs*>(&a), const_cast<Uniforms*>(&u)};
  return cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, smem, s);
}

}  // namespace gp
