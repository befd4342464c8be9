// Block-per-batch vertex reuse: sorting (Algorithm 2), hashing (Algorithm 3)
// and parallel hashing (Section 3.4), over static batches (Section 3.3) or
// the dynamic batches of the partition (Section 3.4).
//
// pipeline_run walks a block's batches b_0, b_1, ... (first, first + stride,
// ...) as a two-stage pipeline: while batch
// b_k is shaded and written, the unique vertices of b_{k+1} are already on
// their way into shared memory.  One iteration of the loop:
//   A. waits for the index window of b_{k+1} (a bulk copy on an mbarrier,
//      issued one iteration earlier) and issues the window of b_{k+2};
//   B. finds the unique indices of b_{k+1} (gp_batch_body.cuh):
//        hash  -- open addressing, multiplicative hash, linear probing with
//                 atomicCAS (map[position] = slot);
//        phash -- as hash, but each thread probes at most probe_k slots, then
//                 the warp probes 32 consecutive slots at a time for its
//                 remaining indices (ballot/shuffle);
//        sort  -- bitonic sort of (id, position) keys, tail flags, exclusive
//                 prefix sum: map[position] = rank of the id (ascending ids);
//      then waits for the rows of b_k, whose copies started one iteration
//      earlier;
//   C. shades each unique vertex of b_k once, from its raw row, into the
//      shaded buffer; then (hash/phash) numbers b_{k+1}'s vertices in the
//      order of the positions whose CAS stored them (a block scan: slot ->
//      dense rank, rank -> id), clears the table, and starts cp.async copies
//      of b_{k+1}'s rows into the raw buffer, which the shading has just
//      released;
//   D. assembles b_k's triangles in input order into a staging buffer (each
//      corner's shaded row, found through the map, then slot -> rank for
//      hash/phash) and writes it with one bulk (TMA) store per chunk -- by
//      default the whole batch; the 1..3 floats at an unaligned edge use
//      plain stores.
// Block barriers per iteration: after A, B and C, one inside C and one per
// output chunk, plus the sort network and one scan barrier for sort.
#pragma once

#include "gp_batch_body.cuh"

namespace gp {

struct BatchLayout {
  uint32_t off_bars, off_misc, off_idx, idx_words, off_map, map_elems, off_keys, off_table, off_dense, off_uniq,
      uniq_words, off_raw, off_v, off_pal, off_stage, stage_floats, total;
};

__host__ __device__ inline uint32_t align_up_u32(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

// K: floats per output corner; KV: shared-memory stride (floats) of a shaded
// vertex; RB: bytes of a raw row; out_chunk: triangles per output bulk store.
__host__ __device__ inline BatchLayout batch_layout(int dedup, uint32_t K, uint32_t KV, uint32_t RB, bool skin,
                                                    uint32_t max_idx, uint32_t ucap, uint32_t slots,
                                                    uint32_t sort_n, uint32_t out_chunk) {
  BatchLayout L;
  uint32_t o = 0;
  L.off_bars = o; o += 16;
  L.off_misc = o; o += 64 * 4;
  L.idx_words = align_up_u32(max_idx + 8, 4);
  L.off_idx = o; o += 2 * L.idx_words * 4;
  L.map_elems = align_up_u32(max_idx, 8);
  L.off_map = o; o += 2 * L.map_elems * 2;
  if (dedup == DEDUP_SORT) {
    L.off_keys = o; o += sort_n * 8;
    L.off_table = L.off_dense = 0;
  } else {
    L.off_keys = 0;
    L.off_table = o; o += slots * 4;
    L.off_dense = o; o = align_up_u32(o + 2 * slots * 2, 16);  // one slot -> rank map per buffer
  }
  L.uniq_words = align_up_u32(ucap, 4);
  L.off_uniq = o; o += 2 * L.uniq_words * 4;
  L.off_raw = o; o += ucap * RB;
  L.off_v = o; o = align_up_u32(o + ucap * KV * 4, 16);
  L.off_pal = o; o += skin ? 768 * 4 : 0;
  L.stage_floats = align_up_u32(out_chunk * 3 * K + 4, 4);
  L.off_stage = o; o += L.stage_floats * 4;
  L.total = o;
  return L;
}

// Rank of a batch corner (its vertex's row in the shaded buffer): the map
// holds it (sort) or the corner's hash slot, numbered by the slot -> rank map.
// Ranks at or above U only follow a flagged capacity error; they read row 0.
template <int DEDUP>
struct CornerRank {
  const uint16_t* map;
  const uint16_t* dense;
  uint32_t U;
  __device__ __forceinline__ uint32_t operator()(uint32_t lc) const {
    uint32_t r = map[lc];
    if (DEDUP != DEDUP_SORT) r = dense[r & ~kNewFlag];
    return r < U ? r : 0u;
  }
};

// The two index-window mbarriers of a block and their phase bits, kept
// across pipeline runs (initialised once per block).
struct PipeBars {
  uint64_t* bars;
  uint32_t phase0, phase1;
};

// Runs batches first, first + stride, ... (< nb) of draw 'a' through the
// pipeline, in the shared memory 'smem' laid out by L (its palette region is
// not used: 'palette' points to the skinning palette, SH == 1).  Every thread
// of the block calls it.  Adds the unique vertices and the batches it shaded
// to inv_total / nbatches (thread 0).  Returns false after a capacity error
// or a window that did not land (flagged in a.err), with every copy into
// shared memory drained.  On return the shared memory is free for reuse.
template <int DEDUP, int SH, bool DYN>
__device__ __forceinline__ bool pipeline_run(const DrawArgs& a, const Uniforms& u, const float* palette,
                                             unsigned char* smem, const BatchLayout& L, PipeBars& pb,
                                             uint32_t first, uint32_t stride, uint32_t nb,
                                             unsigned long long& inv_total, unsigned long long& nbatches) {
  constexpr int K = ShaderTraits<SH>::K;
  constexpr int KV = K | 1;  // odd stride: random ranks spread over the banks
  constexpr int F = 3 * K;
  constexpr uint32_t RB = RawTraits<SH>::kBytes;
  uint64_t* bars = pb.bars;
  uint32_t* misc = reinterpret_cast<uint32_t*>(smem + L.off_misc);  // [0] unique counter, [8..] scan
  uint32_t* wrange = misc + 48;  // [2 buf + 0/1]: triangle range of the window in flight into buffer buf
  uint32_t* idxbuf = reinterpret_cast<uint32_t*>(smem + L.off_idx);
  uint16_t* mapbuf = reinterpret_cast<uint16_t*>(smem + L.off_map);
  uint16_t* densebuf = reinterpret_cast<uint16_t*>(smem + L.off_dense);
  uint32_t* uniqbuf = reinterpret_cast<uint32_t*>(smem + L.off_uniq);
  unsigned char* raw = smem + L.off_raw;
  float* vsh = reinterpret_cast<float*>(smem + L.off_v);
  float* stage = reinterpret_cast<float*>(smem + L.off_stage);
  BatchSmem S;
  S.keys = reinterpret_cast<unsigned long long*>(smem + L.off_keys);
  S.table = reinterpret_cast<uint32_t*>(smem + L.off_table);
  S.vsh = vsh;
  S.ucount = misc;
  S.wsum = misc + 8;

  const uint32_t tid = threadIdx.x, NT = blockDim.x;
  const uint32_t n4 = a.num_idx & ~3u;  // end of the 16-byte-granular part of the index buffer
  if (DEDUP != DEDUP_SORT)
    for (uint32_t s = tid; s < a.hash_slots; s += NT) S.table[s] = kEmpty;

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
  // (clipped to the 16-byte-granular part of the buffer) and records the
  // batch's triangle range for the other threads.  Thread 0 only.
  auto issue_window = [&](uint32_t b, uint32_t buf) {
    uint32_t t0, t1;
    batch_range(b, t0, t1);
    wrange[2 * buf] = t0;
    wrange[2 * buf + 1] = t1;
    const uint32_t i0 = 3 * t0, i1 = 3 * t1, base = i0 & ~3u;
    const uint32_t end = min((i1 + 3) & ~3u, n4);
    // a window larger than the buffer is refused here and flagged by the consumer
    const uint32_t bytes = (end > base && end - base <= L.idx_words) ? (end - base) * 4 : 0;
    mbar_arrive_expect_tx(&bars[buf], bytes);
    if (bytes) bulk_load(idxbuf + buf * L.idx_words, a.idx + base, bytes, &bars[buf]);
  };

  uint32_t& phase0 = pb.phase0;
  uint32_t& phase1 = pb.phase1;
  bool aborted = false, window_inflight = false, window_timed_out = false;
  uint32_t inflight_buf = 0, waited_buf = 0;
  uint32_t U_cur = 0, U_next = 0;
  uint32_t cur_t0 = 0, cur_t1 = 0;  // the current batch's triangles (the previous iteration's next batch)
  if (tid == 0) {
    *S.ucount = 0;
    issue_window(first, 0);
  }
  __syncthreads();  // table cleared, first window range recorded
  // iteration 'it': the current batch is first + (it - 1) stride (none for
  // it == 0), the next one first + it stride; their buffers alternate.
  for (uint32_t it = 0;; ++it) {
    const uint32_t nbuf = it & 1u, cbuf = nbuf ^ 1u;
    const bool has_cur = it > 0;
    const uint32_t cur = first + (it - 1) * stride, nxt = first + it * stride;
    const bool has_next = nxt < nb;
    window_inflight = false;
    // --- A: the next batch's index window
    uint32_t n = 0, i0 = 0, base = 0;
    bool bad = false;
    uint32_t nt0 = 0, nt1 = 0;
    if (has_next) {
      nt0 = wrange[2 * nbuf];
      nt1 = wrange[2 * nbuf + 1];
      const uint32_t t0 = nt0, t1 = nt1;
      i0 = 3 * t0;
      n = 3 * (t1 - t0);
      base = i0 & ~3u;
      bad = n > a.max_batch_idx;  // cannot happen with a consistent partition
      const uint32_t par = nbuf ? phase1 : phase0;
      const bool landed = mbar_wait_bounded(&bars[nbuf], par, a.err);
      window_timed_out = !landed;
      waited_buf = nbuf;
      bad |= !landed;
      if (nbuf) phase1 ^= 1; else phase0 ^= 1;
      if (!bad) {
        // indices past the 16-byte-granular part of the buffer (last batch only)
        const uint32_t i1 = i0 + n, end = min((i1 + 3) & ~3u, n4);
        const uint32_t p0 = max(i0, end > base ? end : base);
        for (uint32_t i = p0 + tid; i < i1; i += NT) idxbuf[nbuf * L.idx_words + i - base] = __ldg(a.idx + i);
      }
      if (tid == 0 && nxt + stride < nb) {
        issue_window(nxt + stride, cbuf);  // the current batch's window was consumed in the previous iteration
        window_inflight = true;
        inflight_buf = cbuf;
      }
    }
    if (__syncthreads_or(bad)) {  // barrier 1: window ready
      if (tid == 0) atomicOr(a.err, EBIT_CAPACITY);
      aborted = true;
      break;
    }
    // --- B: dedup of the next batch
    uint16_t* nmap = mapbuf + nbuf * L.map_elems;
    uint32_t* nuniq = uniqbuf + nbuf * L.uniq_words;
    if (has_next) {
      S.map = nmap;
      S.uniq = nuniq;
      // sort: ranks and uniq; hash/phash: the table and the slots only (numbered in C)
      dedup<DEDUP, DEDUP == DEDUP_SORT>(a, S, idxbuf + nbuf * L.idx_words + (i0 - base), n, tid, NT, BlockSync(),
                                        NoConsume());
    }
    cp_async_wait<0>();  // this thread's copies of the current batch's rows (started in C) have landed
    __syncthreads();     // barrier 2: dedup done; the current batch's rows are in shared memory
    // --- C: shade the current batch; number the next batch's vertices and
    // start the copies of their rows
    // hash/phash: the vertices are numbered in the order of the positions
    // whose CAS stored them, so a run of corners mostly refers to nearby
    // ranks (fewer bank conflicts when D reads their rows).  Each thread owns
    // the contiguous positions [p0, p0 + ppt) (ppt <= 32); bit j of 'won' =
    // position p0 + j stored its id.
    const uint32_t ppt = (n + NT - 1) / NT, p0 = min(tid * ppt, n), p1 = min(p0 + ppt, n);
    uint32_t won = 0, occ_inc = 0;
    if (has_next) {
      if (DEDUP == DEDUP_SORT) {
        U_next = min(*S.ucount, a.ucap);
      } else {
        for (uint32_t p = p0; p < p1; ++p) won |= (uint32_t)(nmap[p] >> 15) << (p - p0);
        occ_inc = warp_inclusive_scan(__popc(won));
        if ((tid & 31) == 31) S.wsum[tid >> 5] = occ_inc;
      }
    }
    const uint32_t* cuniq = uniqbuf + cbuf * L.uniq_words;
    if (has_cur) {
      for (uint32_t r = tid; r < U_cur; r += NT) {
        float o[K];
        if (cuniq[r] < a.num_verts) {
          VertexIn v;
          load_raw<SH>(raw + r * RB, v);
          shade_vertex<SH>(u, palette, v, o);
        } else {
#pragma unroll
          for (int c = 0; c < K; ++c) o[c] = 0.f;
          atomicOr(a.err, EBIT_INDEX_RANGE);
        }
#pragma unroll
        for (int c = 0; c < K; ++c) vsh[r * KV + c] = o[c];
      }
    }
    if (has_next) {
      __syncthreads();  // the raw rows are shaded (the buffer is free); the per-warp counts are in S.wsum
      if (DEDUP == DEDUP_SORT) {
        for (uint32_t e = tid; e < U_next * RawTraits<SH>::kChunks; e += NT) {
          const uint32_t r = e / RawTraits<SH>::kChunks, c = e % RawTraits<SH>::kChunks;
          const uint32_t id = nuniq[r];
          if (id < a.num_verts) cp_async16(raw + r * RB + c * 16, a.verts + (size_t)id * a.stride + c * 16);
        }
      } else {
        // the warps' totals, scanned within each warp (NT / 32 <= 32 of them)
        const uint32_t lane = tid & 31, nw = NT >> 5;
        const uint32_t wv = lane < nw ? S.wsum[lane] : 0u;
        const uint32_t wi = warp_inclusive_scan(wv);
        const uint32_t total = __shfl_sync(kFull, wi, 31);
        uint32_t r = __shfl_sync(kFull, wi - wv, tid >> 5) + occ_inc - __popc(won);
        uint16_t* ndense = densebuf + nbuf * a.hash_slots;
        for (uint32_t f = won; f; f &= f - 1, ++r) {
          const uint32_t sl = nmap[p0 + __ffs(f) - 1] & ~kNewFlag;
          const uint32_t id = S.table[sl];
          S.table[sl] = kEmpty;  // the table is done: clear it for the batch after
          if (r < a.ucap) {
            ndense[sl] = (uint16_t)r;
            nuniq[r] = id;
            if (id < a.num_verts)
#pragma unroll
              for (uint32_t c = 0; c < RawTraits<SH>::kChunks; ++c)
                cp_async16(raw + r * RB + c * 16, a.verts + (size_t)id * a.stride + c * 16);
          } else {
            atomicOr(a.err, EBIT_CAPACITY);
          }
        }
        U_next = min(total, a.ucap);
      }
      cp_async_commit();
    }
    // the previous batch's last bulk store must have read the staging buffer
    if (tid == 0) bulk_wait_read<0>();
    __syncthreads();  // barrier 3: every unique vertex of the current batch shaded; counter read
    if (tid == 0) *S.ucount = 0;
    // --- D: the current batch's triangles, in input order, chunk by chunk
    if (has_cur) {
      const uint32_t t0 = cur_t0, t1 = cur_t1;
      const CornerRank<DEDUP> rank{mapbuf + cbuf * L.map_elems, densebuf + cbuf * a.hash_slots, U_cur};
      for (uint32_t ta = t0; ta < t1; ta += a.out_chunk) {
        const uint32_t tb = min(ta + a.out_chunk, t1);
        if (ta != t0) {
          if (tid == 0) bulk_wait_read<0>();
          __syncthreads();  // the previous chunk's bulk store has read the staging buffer
        }
        const size_t g0 = (size_t)ta * F;
        const uint32_t pad = (uint32_t)(g0 & 3);
        float* st = stage + pad;
        const uint32_t cbase = 3 * (ta - t0), nc = 3 * (tb - ta);
        for (uint32_t lc = tid; lc < nc; lc += NT) {
          const uint32_t r = rank(cbase + lc);
          const float* row = vsh + r * KV;
#pragma unroll
          for (int k = 0; k < K; ++k) st[lc * K + k] = row[k];
          if (a.corner_ids != nullptr) a.corner_ids[3ull * ta + lc] = cuniq[r];
        }
        fence_proxy_async_smem();
        __syncthreads();  // staging filled
        const uint32_t nfl = nc * K;
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
        inv_total += U_cur;
        nbatches += 1;
        if (a.batch_inv != nullptr && cur < a.batch_cap) a.batch_inv[cur] = U_cur;
      }
    }
    U_cur = U_next;
    cur_t0 = nt0;
    cur_t1 = nt1;
    if (!has_next) break;
  }
  if (aborted) {
    // never leave a copy in flight into this block's shared memory
    cp_async_wait<0>();
    if (tid == 0) {
      if (window_inflight) mbar_wait_bounded(&bars[inflight_buf], inflight_buf ? phase1 : phase0, a.err);
      if (window_timed_out)  // the window that did not land (its phase bit was already advanced)
        mbar_wait_bounded(&bars[waited_buf], (waited_buf ? phase1 : phase0) ^ 1u, a.err);
    }
  }
  if (tid == 0) bulk_wait_read<0>();  // the last bulk store has read the staging buffer
  __syncthreads();
  return !aborted;
}

}  // namespace gp
