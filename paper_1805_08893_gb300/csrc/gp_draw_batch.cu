// Block-per-batch vertex reuse: sorting (Algorithm 2), hashing (Algorithm 3)
// and parallel hashing (Section 3.4), over static batches (Section 3.3) or
// the dynamic batches of the partition (Section 3.4).
//
// Per batch, one thread block:
//   1. has the batch's index window in shared memory (bulk copy issued one
//      batch ahead on an mbarrier, so the load overlaps the previous batch);
//   2. finds the unique indices and shades each one once:
//        hash  -- open addressing, multiplicative hash, linear probing with
//                 atomicCAS (map[position] = slot).  The thread whose CAS
//                 stores a new id takes the next dense rank (one shared
//                 counter, warp-aggregated), fetches that vertex and shades
//                 it at once, so vertex loads overlap the other insertions;
//        phash -- as hash, but each thread probes at most probe_k slots, then
//                 the warp probes 32 consecutive slots at a time for its
//                 remaining indices (ballot/shuffle);
//        sort  -- bitonic sort of (id, position) keys, tail flags, exclusive
//                 prefix sum: map[position] = rank of the id (ascending ids);
//                 the owner of a group's tail element shades that vertex;
//   3. assembles triangles in input order into a shared staging buffer and
//      writes it with one bulk (TMA) store per chunk (by default the whole
//      batch); the ragged 1..3 floats at an unaligned edge use plain stores.
//
// Three block barriers per batch for hash/phash (window ready; all vertices
// shaded; staging filled), plus the sort network and one scan barrier for sort.
// Blocks are persistent (grid = SMs x resident blocks) and walk the batches
// with a grid stride.
#include "gp_device.cuh"

namespace gp {

constexpr int kIdsPerRound = 4;  // indices a thread handles before shading its new ones

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

__device__ __forceinline__ uint32_t hash_slot(uint32_t id, uint32_t bits) {
  return bits ? (id * 2654435769u) >> (32 - bits) : 0u;
}

template <int SH>
__device__ __forceinline__ void store_shaded(float* vsh, uint32_t k, const float* o) {
  constexpr int K = ShaderTraits<SH>::K;
  constexpr int KS = ShaderTraits<SH>::KS;
  if (K == 8) {
    float4* dv = reinterpret_cast<float4*>(vsh + k * KS);
    dv[0] = make_float4(o[0], o[1], o[2], o[3]);
    dv[1] = make_float4(o[4], o[5], o[6], o[7]);
  } else {
#pragma unroll
    for (int c = 0; c < K; ++c) vsh[k * KS + c] = o[c];
  }
}

constexpr uint16_t kNoRank = 0xFFFFu;

// One compare-exchange of the bitonic network seen from element i holding x,
// whose partner (i ^ j) holds y: ascending runs where (i & k) == 0; the lower
// index of a pair keeps the smaller key in an ascending run.
__device__ __forceinline__ unsigned long long bitonic_keep(unsigned long long x, unsigned long long y, uint32_t i,
                                                           uint32_t j, uint32_t k) {
  const bool asc = (i & k) == 0;
  const bool lower = (i & j) == 0;
  const bool take_min = lower == asc;
  const unsigned long long mn = x < y ? x : y, mx = x < y ? y : x;
  return take_min ? mn : mx;
}

// Bitonic sort of N = 4 * blockDim.x keys, 4 consecutive keys per thread in
// registers.  Stages with j <= 2 stay inside a thread, 4 <= j <= 64 exchange
// within the warp by shuffles (partner lane = lane ^ j/4), and only j >= 128
// goes through shared memory.  Reads keys[] and leaves the sorted keys there.
__device__ __forceinline__ void bitonic_sort_regs4(unsigned long long* keys, uint32_t N, uint32_t tid) {
  unsigned long long r[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) r[e] = keys[4 * tid + e];
  for (uint32_t k = 2; k <= N; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      if (j >= 128) {
        __syncthreads();  // every thread has read the previous contents
#pragma unroll
        for (int e = 0; e < 4; ++e) keys[4 * tid + e] = r[e];
        __syncthreads();
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const uint32_t i = 4 * tid + e;
          r[e] = bitonic_keep(r[e], keys[i ^ j], i, j, k);
        }
      } else if (j >= 4) {
        const uint32_t lm = j >> 2;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const unsigned long long y = __shfl_xor_sync(kFull, r[e], lm);
          r[e] = bitonic_keep(r[e], y, 4 * tid + e, j, k);
        }
      } else if (j == 2) {
        unsigned long long s[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) s[e] = bitonic_keep(r[e], r[e ^ 2], 4 * tid + e, 2, k);
#pragma unroll
        for (int e = 0; e < 4; ++e) r[e] = s[e];
      } else {
        unsigned long long s[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) s[e] = bitonic_keep(r[e], r[e ^ 1], 4 * tid + e, 1, k);
#pragma unroll
        for (int e = 0; e < 4; ++e) r[e] = s[e];
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int e = 0; e < 4; ++e) keys[4 * tid + e] = r[e];
  __syncthreads();
}

// Shades the warp's queue of new vertices (their ranks; the id is uniq[rank])
// in full-warp passes: two vertices per lane per pass, both loads issued
// before the math.
template <int SH>
__device__ __forceinline__ void shade_queue(const DrawArgs& a, const Uniforms& u, const float* palette, float* vsh,
                                            const uint32_t* uniq, const uint16_t* q, uint32_t qn, uint32_t lane) {
  constexpr int K = ShaderTraits<SH>::K;
  for (uint32_t e = lane; e < qn; e += 64) {
    const bool has1 = e + 32 < qn;
    const uint32_t r0 = q[e], r1 = has1 ? q[e + 32] : kNoRank;
    const uint2 e0 = make_uint2(r0 != kNoRank ? uniq[r0] : kInvalidId, r0 != kNoRank ? r0 : 0xFFFFFFFFu);
    const uint2 e1 = make_uint2(r1 != kNoRank ? uniq[r1] : kInvalidId, r1 != kNoRank ? r1 : 0xFFFFFFFFu);
    VertexIn v0, v1;
    const bool ok0 = e0.x < a.num_verts, ok1 = has1 && e1.x < a.num_verts;
    if (ok0) fetch_vertex<SH>(a.verts, a.stride, e0.x, v0, a.vec8 != 0);
    if (ok1) fetch_vertex<SH>(a.verts, a.stride, e1.x, v1, a.vec8 != 0);
    float o[K];
    if (e0.y != 0xFFFFFFFFu) {
      if (ok0) {
        shade_vertex<SH>(u, palette, v0, o);
      } else {
#pragma unroll
        for (int c = 0; c < K; ++c) o[c] = 0.f;
        atomicOr(a.err, EBIT_INDEX_RANGE);
      }
      store_shaded<SH>(vsh, e0.y, o);
    }
    if (has1 && e1.y != 0xFFFFFFFFu) {
      if (ok1) {
        shade_vertex<SH>(u, palette, v1, o);
      } else {
#pragma unroll
        for (int c = 0; c < K; ++c) o[c] = 0.f;
        atomicOr(a.err, EBIT_INDEX_RANGE);
      }
      store_shaded<SH>(vsh, e1.y, o);
    }
  }
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
  uint16_t* map = reinterpret_cast<uint16_t*>(smem + L.off_map);
  unsigned long long* keys = reinterpret_cast<unsigned long long*>(smem + L.off_keys);
  uint32_t* table = reinterpret_cast<uint32_t*>(smem + L.off_table);
  uint16_t* dense = reinterpret_cast<uint16_t*>(smem + L.off_dense);
  uint32_t* uniq = reinterpret_cast<uint32_t*>(smem + L.off_uniq);
  float* vsh = reinterpret_cast<float*>(smem + L.off_v);
  float* stage = reinterpret_cast<float*>(smem + L.off_stage);
  float* palette = reinterpret_cast<float*>(smem + L.off_pal);
  uint32_t* ucount = misc;
  uint16_t* wq = reinterpret_cast<uint16_t*>(smem + L.off_wq) + (threadIdx.x >> 5) * (32 * kIdsPerRound);

  const uint32_t tid = threadIdx.x, NT = blockDim.x, lane = lane_id(), warp = tid >> 5;
  const uint32_t nb = DYN ? *a.num_batches_dev : a.num_batches;
  const uint32_t n4 = a.num_idx & ~3u;  // end of the 16-byte-granular part of the index buffer

  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
    *ucount = 0;
  }
  if (ShaderTraits<SH>::kSkin)
    for (uint32_t i = tid; i < 768; i += NT) palette[i] = u.palette[i];
  if (DEDUP != DEDUP_SORT)
    for (uint32_t s = tid; s < a.hash_slots; s += NT) table[s] = kEmpty;
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
    const uint32_t* ids = win + (i0 - base);

    if (DEDUP == DEDUP_SORT) {
      // --- Algorithm 2: sort (id, position), tail flags, exclusive prefix sum
      for (uint32_t i = tid; i < a.sort_n; i += NT) {
        if (i < n) {
          uint32_t id = ids[i];
          id = id < a.num_verts ? id : kInvalidId;
          keys[i] = ((unsigned long long)id << 32) | i;
        } else {
          keys[i] = ~0ull;
        }
      }
      __syncthreads();
      // Bitonic network.  For j <= 32 the pairs (i, i + j) touched by the
      // threads of one warp stay inside that warp's 64-key blocks (i = 2t -
      // (t mod j), t = 32q + r), so those stages need only a warp barrier;
      // a block barrier separates a stage from one with j >= 64.
      const uint32_t N = a.sort_n;
      if (N == 4 * NT) {
        bitonic_sort_regs4(keys, N, tid);
      } else {
      for (uint32_t k = 2; k <= N; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
          for (uint32_t t = tid; t < N / 2; t += NT) {
            const uint32_t i = 2 * t - (t & (j - 1));
            const uint32_t l = i + j;
            const bool up = (i & k) == 0;
            const unsigned long long x = keys[i], y = keys[l];
            if ((x > y) == up) {
              keys[i] = y;
              keys[l] = x;
            }
          }
          const uint32_t nj = j > 1 ? (j >> 1) : k;  // j of the next stage
          if (j >= 64 || nj >= 64) __syncthreads();
          else __syncwarp();
        }
      }
      __syncthreads();
      }
      // tail flags over each thread's contiguous run, then a block scan with
      // one barrier: every thread adds up the totals of the warps before its own
      const uint32_t ipt = (n + NT - 1) / NT;
      const uint32_t lo = min(tid * ipt, n), hi = min(lo + ipt, n);
      uint32_t cnt = 0;
      for (uint32_t i = lo; i < hi; ++i)
        cnt += (i == n - 1 || (uint32_t)(keys[i] >> 32) != (uint32_t)(keys[i + 1] >> 32)) ? 1u : 0u;
      const uint32_t inc = warp_inclusive_scan(cnt);
      uint32_t* wsum = misc + 8;
      if (lane == 31) wsum[warp] = inc;
      __syncthreads();
      uint32_t r = inc - cnt;
      for (uint32_t w = 0; w < warp; ++w) r += wsum[w];
      if (tid == NT - 1) *ucount = r + cnt;
      // walk the run in rounds of kIdsPerRound elements (ipt is the same for
      // every thread, so the warp's ballots line up); tails go to the warp's
      // shading queue
      for (uint32_t off = 0; off < ipt; off += kIdsPerRound) {
        uint32_t qn = 0;
#pragma unroll
        for (int q = 0; q < kIdsPerRound; ++q) {
          const uint32_t i = lo + off + q;
          bool tail = false;
          uint32_t id = 0;
          if (off + q < ipt && i < hi) {
            id = (uint32_t)(keys[i] >> 32);
            map[(uint32_t)(keys[i] & 0xFFFFu)] = (uint16_t)r;
            tail = (i == n - 1) || id != (uint32_t)(keys[i + 1] >> 32);
          }
          const uint32_t tm = __ballot_sync(kFull, tail);
          if (tail) {
            uint16_t rk = (uint16_t)r;
            if (r < a.ucap) {
              uniq[r] = id;
            } else {
              atomicOr(a.err, EBIT_CAPACITY);
              rk = kNoRank;
            }
            wq[qn + __popc(tm & lanemask_lt())] = rk;
            ++r;
          }
          qn += __popc(tm);
        }
        __syncwarp();
        shade_queue<SH>(a, u, palette, vsh, uniq, wq, qn, lane);
        __syncwarp();
      }
    } else {
      // --- Algorithm 3 / Section 3.4: insert; the thread storing a new id
      // takes its rank and shades it
      const uint32_t mask = a.hash_slots - 1;
      for (uint32_t rbase = 0; rbase < n; rbase += kIdsPerRound * NT) {
        uint32_t qn = 0;  // the warp's queue of new (id, rank) pairs
#pragma unroll
        for (int q = 0; q < kIdsPerRound; ++q) {
          const uint32_t i = rbase + q * NT + tid;
          const bool active = i < n;
          uint32_t id = active ? ids[i] : 0u;
          id = id < a.num_verts ? id : kInvalidId;
          uint32_t h = hash_slot(id, a.hash_bits);
          bool is_new = false;
          if (DEDUP == DEDUP_HASH) {
            if (active) {
              for (uint32_t probes = 0;; ++probes) {
                const uint32_t prev = atomicCAS(&table[h], kEmpty, id);
                if (prev == kEmpty) {
                  is_new = true;
                  break;
                }
                if (prev == id) break;
                h = (h + 1) & mask;
                if (probes > a.hash_slots) {  // table full: cannot happen within capacity
                  atomicOr(a.err, EBIT_CAPACITY);
                  h = 0;
                  break;
                }
              }
            }
          } else {
            bool placed = !active;
            for (uint32_t p = 0; p < a.probe_k && !placed; ++p) {
              const uint32_t prev = atomicCAS(&table[h], kEmpty, id);
              if (prev == kEmpty) is_new = true;
              if (prev == kEmpty || prev == id) placed = true;
              else h = (h + 1) & mask;
            }
            uint32_t pending = __ballot_sync(kFull, !placed);
            while (pending) {
              const uint32_t leader = __ffs(pending) - 1;
              const uint32_t lid = __shfl_sync(kFull, id, leader);
              uint32_t lh = __shfl_sync(kFull, h, leader);
              uint32_t found = kEmpty;
              bool fresh = false;
              for (uint32_t guard = 0; found == kEmpty; ++guard) {
                if (guard > a.hash_slots / 16 + 64) {  // table full: cannot happen within capacity
                  if (lane == 0) atomicOr(a.err, EBIT_CAPACITY);
                  found = 0;
                  break;
                }
                const uint32_t s = (lh + lane) & mask;
                const uint32_t val = table[s];
                const uint32_t hit = __ballot_sync(kFull, val == lid);
                if (hit) {
                  found = (lh + __ffs(hit) - 1) & mask;
                  break;
                }
                const uint32_t emp = __ballot_sync(kFull, val == kEmpty);
                if (emp) {
                  const uint32_t fl = __ffs(emp) - 1;
                  const uint32_t cs = (lh + fl) & mask;
                  uint32_t prev = 0;
                  if (lane == fl) prev = atomicCAS(&table[cs], kEmpty, lid);
                  prev = __shfl_sync(kFull, prev, fl);
                  if (prev == kEmpty || prev == lid) {
                    found = cs;
                    fresh = prev == kEmpty;
                  } else {
                    lh = cs;  // the slot was just taken: continue probing from it
                  }
                } else {
                  lh = (lh + 32) & mask;
                }
              }
              if (lane == leader) {
                h = found;
                is_new = fresh;
              }
              pending &= pending - 1;
            }
          }
          // warp-aggregated dense ranks for the new ids
          const uint32_t newmask = __ballot_sync(kFull, is_new);
          uint32_t wbase = 0;
          if (newmask) {
            const uint32_t leader = __ffs(newmask) - 1;
            if (lane == leader) wbase = atomicAdd(ucount, __popc(newmask));
            wbase = __shfl_sync(kFull, wbase, leader);
          }
          if (is_new) {
            const uint32_t pos = __popc(newmask & lanemask_lt());
            const uint32_t rk = wbase + pos;
            if (rk < a.ucap) {
              dense[h] = (uint16_t)rk;
              uniq[rk] = id;
              wq[qn + pos] = (uint16_t)rk;
            } else {
              atomicOr(a.err, EBIT_CAPACITY);
              wq[qn + pos] = kNoRank;
            }
          }
          qn += __popc(newmask);
          if (active) map[i] = (uint16_t)h;
        }
        __syncwarp();
        shade_queue<SH>(a, u, palette, vsh, uniq, wq, qn, lane);
        __syncwarp();
      }
    }
    // the previous batch's bulk store must have read the staging buffer
    // before this batch fills it (after the barrier below)
    if (tid == 0) bulk_wait_read<0>();
    __syncthreads();  // barrier 2: every unique vertex shaded, map/dense/uniq complete
    const uint32_t U = min(*ucount, a.ucap);
    if (DEDUP != DEDUP_SORT)  // the table is done: clear it for the next batch
      for (uint32_t s = tid; s < a.hash_slots; s += NT) table[s] = kEmpty;

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
      const uint32_t nc = 3 * (tb - ta);
      const uint32_t cbase = 3 * (ta - t0);
      for (uint32_t lc = tid; lc < nc; lc += NT) {
        const uint32_t m = map[cbase + lc];
        uint32_t s = (DEDUP == DEDUP_SORT) ? m : dense[m];
        s = s < U ? s : 0u;  // only reachable after a flagged capacity error; keeps reads in bounds
        if (K == 8 && pad == 0) {
          const float4* sv = reinterpret_cast<const float4*>(vsh + s * KS);
          float4* dv = reinterpret_cast<float4*>(st + lc * K);
          dv[0] = sv[0];
          dv[1] = sv[1];
        } else {
#pragma unroll
          for (int c = 0; c < K; ++c) st[lc * K + c] = vsh[s * KS + c];
        }
        if (a.corner_ids != nullptr) a.corner_ids[3 * ta + lc] = uniq[s];
      }
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
      *ucount = 0;  // every thread read U before barrier 3
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
