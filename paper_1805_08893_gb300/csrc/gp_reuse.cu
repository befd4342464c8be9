// Single-draw vertex reuse: sorting (Algorithm 2), hashing (Algorithm 3) and
// parallel hashing (Section 3.4), over static batches (Section 3.3) or the
// dynamic batches of the partition (Section 3.4).
//
// Each block is persistent (grid = SMs x resident blocks): it takes batches
// blockIdx.x, blockIdx.x + gridDim.x, ... in turn, and for the last few
// rounds of the draw claims batches from a per-draw counter, one at a time,
// so blocks that run faster take more of them and all finish together.
// Its warps have two roles that run side by side, handing batches over
// through a two-deep ring of shared-memory slots guarded by mbarriers
// ("full": deduplicated, rows landed; "empty": assembled, slot free):
//
//   producer warps (five eighths of the block; sort: half) deduplicate
//     batch j into slot j mod 2: the index window (bulk-copied on an
//     mbarrier one batch ahead, its triangle range left beside it) is read
//     from the 16-byte boundary at or below the batch's first index, 4 words
//     per thread ("a group"); hash/phash -- each position's id is inserted
//     into the shared open-addressing table with atomicCAS (multiplicative
//     hash, linear probing; phash: at most probe_k probes alone, then 32
//     slots at a time with the whole warp), and the thread whose CAS stored
//     an id takes the next unique rank from the slot's counter (one
//     atomicAdd per warp step), records slot -> rank and rank -> id and
//     starts the cp.async copy of the vertex row into the slot; sort --
//     bitonic sort of (id, position) keys, tail flags, prefix sum
//     (gp_batch_body.cuh), each warp copying the rows of the ranks it
//     created.  Each group's 4 slots (hash) or ranks (sort) go to the map as
//     u16 x 4.  The "full" mbarrier completes when every producer thread has
//     arrived and every row copy has landed.
//   consumer warps (the rest) take batch j from its slot: each unique
//     vertex is shaded once, in place in its row; then every warp assembles
//     its groups (4 corners' shaded rows per lane) through a per-warp staging
//     area (a transpose): with 7 floats per corner a span that lies inside
//     the batch leaves in one bulk (TMA) store per warp, otherwise through
//     coalesced 16-byte streaming stores -- only the float4 at the batch's
//     two ends that the neighbouring batch shares are written float by
//     float -- and arrives on the slot's "empty" mbarrier.
//
// Deduplication (shared-memory atomics) and shading/assembly (shared-memory
// reads, FP32, stores) thus overlap across warps instead of alternating
// between block barriers; each role synchronises only its own warps (named
// barriers 1 and 2).  Every wait is bounded; a wait that gives up sets
// EBIT_TIMEOUT and stops the block.
#include "gp_batch_body.cuh"

namespace gp {

constexpr uint32_t kNoBatch = 0xFFFFFFFFu;  // a ring slot that ends the block's work
constexpr uint32_t kDynamicRounds = 6;       // rounds of batches per block claimed from the counter
constexpr uint32_t kBarProducers = 1;  // named barrier of the producer warps
constexpr uint32_t kBarConsumers = 2;  // named barrier of the consumer warps

struct ReuseLayout {
  uint32_t off_bar, off_misc, groups, win_words, off_win, off_scratch, map_elems, uniq_words, rb, off_ring,
      ring_map, ring_dense, ring_uniq, ring_rows, ring_bytes, off_stage, off_pal, total;
};

__host__ __device__ inline uint32_t reuse_align16(uint32_t x) { return (x + 15u) & ~15u; }

// Producer warps of a block of NT threads (at least 64): hash/phash five
// eighths, rounded down (5 of 8 warps) -- deduplication is the longer chain
// of dependent shared-memory round trips; sort half (4 of 8), so that a
// 1024-key network keeps 8 keys per producer thread in registers.  The rest
// are consumers.
__host__ __device__ inline uint32_t reuse_producer_warps(uint32_t NT, int dedup) {
  const uint32_t w = NT / 32, p = dedup == DEDUP_SORT ? w / 2 : (5 * w) / 8;
  return p < 1 ? 1 : (p >= w ? w - 1 : p);
}
// Groups (4 positions) a producer thread inserts per pass, all CAS in flight.
constexpr int kGroupsPerPass = 2;

// Shared-memory layout for NT threads.  K: floats per output corner.
__host__ __device__ inline ReuseLayout reuse_layout(int dedup, int shader, const DrawArgs& a, uint32_t NT) {
  const uint32_t K = shader == 2 ? 8u : 7u;
  const uint32_t consumer_warps = NT / 32 - reuse_producer_warps(NT, dedup);
  ReuseLayout L;
  uint32_t o = 0;
  L.off_bar = o; o += 64;       // window[2], full[2], empty[2]
  L.off_misc = o; o += 64 * 4;  // [0], [1]: unique counters of the two slots; [2]: abort; [4], [5]: each slot's
                                // batch; [6], [7]: the producers' next batch; [8..31]: sort scan; [32..35]: first
                                // and end triangle of the batch in each window buffer; [36..39]: of each slot's batch
  L.groups = (a.max_batch_idx + 6) / 4;  // pad (<= 3) + indices, in 4-word groups
  L.win_words = 4 * L.groups;
  L.off_win = o; o += 2 * L.win_words * 4;
  L.off_scratch = o;  // two hash tables (batches alternate), or the sort keys
  {
    const uint32_t table = dedup == DEDUP_SORT ? 0u : 2 * a.hash_slots * 4;
    const uint32_t keys = dedup == DEDUP_SORT ? a.sort_n * (a.sort_pos_bits ? 4u : 8u) : 0u;
    o += reuse_align16(table > keys ? table : keys);
  }
  L.map_elems = 4 * L.groups;
  L.uniq_words = (a.ucap + 3) & ~3u;
  L.rb = shader == 1 ? 64u : 32u;
  L.off_ring = o;
  L.ring_map = 0;
  L.ring_dense = reuse_align16(L.map_elems * 2);
  L.ring_uniq = L.ring_dense + reuse_align16(dedup == DEDUP_SORT ? 0u : a.hash_slots * 2);
  L.ring_rows = L.ring_uniq + L.uniq_words * 4;  // uniq_words is a multiple of 4
  L.ring_bytes = L.ring_rows + a.ucap * L.rb;     // rows are 32 or 64 bytes
  o += 2 * L.ring_bytes;
  L.off_stage = o; o += consumer_warps * 32 * K * 16;
  L.off_pal = o; o += shader == 1 ? 768 * 4 : 0;
  L.total = o;
  return L;
}

// Float4 slot (within a slot's rows) of half h of the shaded vertex r, shaded
// in place over its raw row: the halves are placed so that 8 consecutive
// ranks' same halves fall into 8 different bank groups.
template <int SH>
__device__ __forceinline__ uint32_t row_slot(uint32_t r, uint32_t h) {
  return ShaderTraits<SH>::kSkin ? 4u * r + h + 2u * ((r >> 1) & 1u) : 2u * r + (h ^ ((r >> 2) & 1u));
}

// Per-warp staging: lane l writes its K float4 (4 corners) at put(l, j); the
// warp then reads float4 q = 32 j + lane of its span at get(q).  Both sides
// are free of bank conflicts (K = 7: odd stride; K = 8: xor swizzle).
template <int K>
__device__ __forceinline__ uint32_t stage_put(uint32_t lane, uint32_t j) {
  return K == 8 ? lane * 8u + (j ^ (lane & 7u)) : lane * (uint32_t)K + j;
}
template <int K>
__device__ __forceinline__ uint32_t stage_get(uint32_t q) {
  if (K == 8) {
    const uint32_t o = q >> 3, e = q & 7u;
    return o * 8u + (e ^ (o & 7u));
  }
  return q;
}

__device__ __forceinline__ void st_stream4(float* p, const float4& v) {
  asm volatile("st.global.cs.v4.f32 [%0], {%1,%2,%3,%4};" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w));
}

__device__ __forceinline__ void named_sync(uint32_t id, uint32_t nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Bounded wait on an mbarrier phase that also gives up once another thread
// has stopped the block (*abort != 0).  The waiting thread sleeps in steps
// of at most 50 us (waking as soon as the phase completes), so a waiting
// warp takes no issue slots from the other role; after 2^14 steps (at most
// ~0.8 s) it sets EBIT_TIMEOUT and *abort and gives up.
__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, volatile uint32_t* abort,
                                              uint32_t* err) {
  for (uint32_t it = 0; it < (1u << 14); ++it) {
    if (mbar_try_wait_sleep(bar, parity, 50000u)) return true;
    if (*abort) return false;
  }
  atomicOr(err, EBIT_TIMEOUT);
  *abort = 1u;
  return false;
}

// Copies the raw row of vertex id into row r of a slot (cp.async, 16 bytes
// at a time; ids out of range are not copied, their rank is shaded as zeros).
template <int SH>
__device__ __forceinline__ void copy_row(const DrawArgs& a, unsigned char* rows, uint32_t r, uint32_t id) {
  if (id < a.num_verts) {
    constexpr uint32_t RB = ShaderTraits<SH>::kSkin ? 64u : 32u;
#pragma unroll
    for (uint32_t c = 0; c < RB / 16; ++c) cp_async16(rows + r * RB + c * 16, a.verts + (size_t)id * a.stride + c * 16);
  }
}

// Sort: each warp copies the rows of the ranks it has just created.
template <int SH>
struct RowCopy {
  const DrawArgs& a;
  unsigned char* rows;
  const uint32_t* uniq;
  __device__ __forceinline__ void operator()(uint32_t rb, uint32_t re, uint32_t lane) const {
    re = min(re, a.ucap);
    for (uint32_t r = rb + lane; r < re; r += 32) copy_row<SH>(a, rows, r, uniq[r]);
  }
};

template <int DEDUP, int SH, bool DYN>
__device__ __forceinline__ void reuse_body(const DrawArgs& a, const Uniforms& u) {
  constexpr int K = ShaderTraits<SH>::K;
  constexpr uint32_t RB = ShaderTraits<SH>::kSkin ? 64u : 32u;
  extern __shared__ __align__(128) unsigned char smem[];
  const uint32_t tid = threadIdx.x, NT = blockDim.x, lane = tid & 31u, warp = tid >> 5;
  const uint32_t NPW = reuse_producer_warps(NT, DEDUP), NP = 32 * NPW, NC = NT - NP;
  const ReuseLayout L = reuse_layout(DEDUP, SH, a, NT);
  const uint32_t nb = DYN ? *a.num_batches_dev : a.num_batches;
  if (blockIdx.x >= nb) return;

  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.off_bar);  // [0,1] window, [2,3] full, [4,5] empty
  uint32_t* misc = reinterpret_cast<uint32_t*>(smem + L.off_misc);
  volatile uint32_t* abort_flag = misc + 2;
  uint32_t* winbuf = reinterpret_cast<uint32_t*>(smem + L.off_win);
  uint32_t* table = reinterpret_cast<uint32_t*>(smem + L.off_scratch);
  float* palette = reinterpret_cast<float*>(smem + L.off_pal);
  auto ring = [&](uint32_t s) { return smem + L.off_ring + s * L.ring_bytes; };

  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_init(&bars[2], NP);
    mbar_init(&bars[3], NP);
    mbar_init(&bars[4], NC);
    mbar_init(&bars[5], NC);
    fence_mbar_init();
    misc[0] = 0;
    misc[1] = 0;
    misc[2] = 0;
  }
  if (ShaderTraits<SH>::kSkin)
    for (uint32_t i = tid; i < 768; i += NT) palette[i] = u.palette[i];
  if (DEDUP != DEDUP_SORT)
    for (uint32_t s = tid; s < 2 * a.hash_slots; s += NT) table[s] = kEmpty;

  const uint32_t n4 = a.num_idx & ~3u;  // end of the 16-byte-granular part of the index buffer
  auto batch_range = [&](uint32_t b, uint32_t& t0, uint32_t& t1) {
    if (DYN) {
      t0 = __ldg(a.starts + b);
      t1 = __ldg(a.starts + b + 1);
    } else {
      t0 = b * a.static_batch_tris;
      t1 = min(t0 + a.static_batch_tris, a.num_tris);
    }
  };
  // Thread 0: bulk copy of the 16-byte-aligned superset of batch b's window,
  // clipped to the 16-byte-granular part of the buffer (the rest is loaded
  // by plain loads).  A window larger than the buffer is refused here and
  // flagged by the producers.  The batch's triangle range goes beside it in
  // shared memory, so that no producer waits on a global load for it.
  auto issue_window = [&](uint32_t t0, uint32_t t1, uint32_t buf, bool copy) {
    misc[32 + 2 * buf] = t0;
    misc[33 + 2 * buf] = t1;
    const uint32_t base = (3 * t0) & ~3u, end = min((3 * t1 + 3) & ~3u, n4);
    const uint32_t bytes = (end > base && end - base <= L.win_words) ? (end - base) * 4 : 0;
    if (!copy) {  // failure injection: bytes that never come
      mbar_arrive_expect_tx(&bars[buf], 16);
      return;
    }
    mbar_arrive_expect_tx(&bars[buf], bytes);
    if (bytes) bulk_load(winbuf + buf * L.win_words, a.idx + base, bytes, &bars[buf]);
  };
  if (tid == 0) {
    uint32_t t0, t1;
    batch_range(blockIdx.x, t0, t1);
    issue_window(t0, t1, 0, !a.test_stall);
  }
  __syncthreads();
  // batches [0, nstatic) go to the blocks in turn (block i: i, i + grid,
  // ...); the last rounds, from nstatic on, are claimed from the per-draw
  // counter, so blocks that run faster take more of them and all finish
  // together -- and the claim's global atomic stays out of most batches
  const uint32_t G = gridDim.x;
  const uint32_t nstatic = G * max(1u, nb / G > kDynamicRounds ? nb / G - kDynamicRounds : 1u);

  if (warp < NPW) {
    // ======================= producers =======================
    const uint32_t pw = warp;
    uint32_t wph = 0u, eph = 0u;  // bit s: parity of window[s] / empty[s]
    bool window_pending = tid == 0;  // thread 0: a window copy may be in flight into pending_buf
    uint32_t pending_buf = 0;
    uint32_t b = blockIdx.x;  // the batch this iteration deduplicates
    for (uint32_t j = 0;; ++j) {
      const uint32_t s = j & 1u;
      // (a block stopped by another thread is noticed in the waits below)
      if (b >= nb) {  // no batch left: hand the consumers a slot that says so
        if (j >= 2 && !wait_or_abort(&bars[4 + s], (eph >> s) & 1u, abort_flag, a.err)) break;
        if (tid == 0) misc[4 + s] = kNoBatch;
        mbar_arrive(&bars[2 + s]);
        break;
      }
      const uint32_t t0 = misc[32 + 2 * s], t1 = misc[33 + 2 * s];  // left by thread 0 with the window
      const uint32_t i0 = 3 * t0, n = 3 * (t1 - t0), base = i0 & ~3u, pad = i0 - base;
      const uint32_t ngroups = (pad + n + 3) >> 2;
      unsigned char* slot_p = ring(s);
      uint16_t* map = reinterpret_cast<uint16_t*>(slot_p + L.ring_map);
      uint16_t* dense = reinterpret_cast<uint16_t*>(slot_p + L.ring_dense);
      uint32_t* uniq = reinterpret_cast<uint32_t*>(slot_p + L.ring_uniq);
      unsigned char* rows = slot_p + L.ring_rows;
      uint32_t* counter = misc + s;
      uint32_t* win = winbuf + s * L.win_words;
      // the slot is free once the consumers have assembled the batch two back
      if (j >= 2) {
        if (!wait_or_abort(&bars[4 + s], (eph >> s) & 1u, abort_flag, a.err)) break;
        eph ^= 1u << s;
      }
      if (!wait_or_abort(&bars[s], (wph >> s) & 1u, abort_flag, a.err)) break;
      wph ^= 1u << s;
      window_pending = false;
      if (tid == 0) {
        // the next batch's window goes into the other buffer, which was read
        // before the last batch's barrier
        const uint32_t next =
            b + G < nstatic ? b + G : nstatic + atomicAdd(reinterpret_cast<unsigned int*>(a.counters + CNT_WORK), 1u);
        misc[6 + (s ^ 1u)] = next;
        misc[4 + s] = b;
        misc[36 + 2 * s] = t0;  // the slot's batch, for the consumers
        misc[37 + 2 * s] = t1;
        if (next < nb) {
          uint32_t nt0, nt1;
          batch_range(next, nt0, nt1);
          issue_window(nt0, nt1, s ^ 1u, true);
          window_pending = true;
          pending_buf = s ^ 1u;
        }
      }
      if (n > a.max_batch_idx) {  // cannot happen with a consistent partition; uniform
        if (tid == 0) atomicOr(a.err, EBIT_CAPACITY);
        *abort_flag = 1u;
        break;
      }
      {  // indices past the 16-byte-granular part of the buffer (the buffer's last batch only)
        const uint32_t end = min((3 * t1 + 3) & ~3u, n4);
        const uint32_t p0 = max(end, base);
        if (p0 < i0 + n) {  // uniform per batch
          for (uint32_t i = p0 + tid; i < i0 + n; i += NP) win[i - base] = __ldg(a.idx + i);
          named_sync(kBarProducers, NP);
        }
      }
      uint32_t* tbl = table + (DEDUP == DEDUP_SORT ? 0u : s * a.hash_slots);  // this batch's hash table
      if (DEDUP == DEDUP_SORT) {
        BatchSmem S;
        S.map = map + pad;
        S.keys = reinterpret_cast<unsigned long long*>(table);
        S.uniq = uniq;
        S.ucount = counter;
        S.wsum = misc + 8;
        const RowCopy<SH> consume{a, rows, uniq};
        if (a.sort_pos_bits)
          sort_dedup<uint32_t>(a, S, win + pad, n, tid, NP, GroupSync{kBarProducers, NP}, consume, a.sort_pos_bits);
        else
          sort_dedup<unsigned long long>(a, S, win + pad, n, tid, NP, GroupSync{kBarProducers, NP}, consume, 32);
      } else {
        const uint32_t mask = a.hash_slots - 1;
        constexpr int Q = 4 * kGroupsPerPass;  // positions per thread and pass
        for (uint32_t gb = 0; gb < ngroups; gb += kGroupsPerPass * NP) {  // warp-uniform
          // a thread's groups: the lanes of a warp take groups NPW apart, so
          // one CAS instruction meets fewer repeats of the same id
          uint32_t id[Q], sl[Q], prev[Q];
          uint32_t act = 0, newmask = 0, pend = 0;  // bit q: position q
#pragma unroll
          for (int k = 0; k < kGroupsPerPass; ++k) {
            const uint32_t g = gb + k * NP + lane * NPW + pw;
            uint4 w = make_uint4(0, 0, 0, 0);
            if (g < ngroups) w = reinterpret_cast<const uint4*>(win)[g];
            const uint32_t raw[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const uint32_t p = 4 * g + e;
              act |= (g < ngroups && p >= pad && p < pad + n ? 1u : 0u) << (4 * k + e);
              id[4 * k + e] = raw[e] < a.num_verts ? raw[e] : kInvalidId;
              sl[4 * k + e] = hash_slot(id[4 * k + e], a.hash_bits);
            }
          }
          // the first probe of every position, issued before any result is used
#pragma unroll
          for (int q = 0; q < Q; ++q) prev[q] = (act >> q) & 1u ? atomicCAS(&tbl[sl[q]], kEmpty, id[q]) : kEmpty;
          // resolve collisions: every position still probing advances one
          // slot per round, the round's CAS all in flight together
          uint32_t probing = 0;
#pragma unroll
          for (int q = 0; q < Q; ++q) {
            if (!((act >> q) & 1u)) sl[q] = 0;
            else if (prev[q] == kEmpty) newmask |= 1u << q;
            else if (prev[q] != id[q]) probing |= 1u << q;
          }
          const uint32_t rounds = DEDUP == DEDUP_HASH ? a.hash_slots : a.probe_k;  // per-thread probes
          for (uint32_t round = 1; probing && round < rounds; ++round) {
#pragma unroll
            for (int q = 0; q < Q; ++q)
              if ((probing >> q) & 1u) {
                sl[q] = (sl[q] + 1) & mask;
                prev[q] = atomicCAS(&tbl[sl[q]], kEmpty, id[q]);
              }
#pragma unroll
            for (int q = 0; q < Q; ++q)
              if ((probing >> q) & 1u) {
                if (prev[q] == kEmpty) newmask |= 1u << q;
                if (prev[q] == kEmpty || prev[q] == id[q]) probing &= ~(1u << q);
              }
          }
          if (DEDUP == DEDUP_HASH) {
            if (probing) {  // table full: cannot happen within capacity
              atomicOr(a.err, EBIT_CAPACITY);
#pragma unroll
              for (int q = 0; q < Q; ++q)
                if ((probing >> q) & 1u) sl[q] = 0;
            }
          } else {
#pragma unroll
            for (int q = 0; q < Q; ++q)
              if ((probing >> q) & 1u) sl[q] = (sl[q] + 1) & mask;  // the next slot to probe
            pend = probing;
          }
          if (DEDUP == DEDUP_PHASH) {
            // the positions still pending (rare), one at a time -- the lowest
            // lane's lowest position first -- probed by the whole warp 32
            // consecutive slots at a time; one loop for all Q positions keeps
            // this cold path small
            for (uint32_t anyp = __ballot_sync(kFull, pend != 0u); anyp; anyp = __ballot_sync(kFull, pend != 0u)) {
              const uint32_t leader = __ffs(anyp) - 1;
              const uint32_t q = __ffs(__shfl_sync(kFull, pend, leader)) - 1;  // uniform
              uint32_t myid = id[0], mysl = sl[0];
#pragma unroll
              for (int k = 1; k < Q; ++k)
                if (q == (uint32_t)k) {
                  myid = id[k];
                  mysl = sl[k];
                }
              const uint32_t lid = __shfl_sync(kFull, myid, leader);
              uint32_t lh = __shfl_sync(kFull, mysl, leader);
              uint32_t found = 0;
              bool fresh = false;
              for (uint32_t guard = 0;; ++guard) {
                if (guard > a.hash_slots / 16 + 64) {  // table full: cannot happen within capacity
                  if (lane == 0) atomicOr(a.err, EBIT_CAPACITY);
                  found = 0;
                  break;
                }
                const uint32_t ps = (lh + lane) & mask;
                const uint32_t val = tbl[ps];
                const uint32_t hit = __ballot_sync(kFull, val == lid);
                if (hit) {
                  found = (lh + __ffs(hit) - 1) & mask;
                  break;
                }
                const uint32_t emp = __ballot_sync(kFull, val == kEmpty);
                if (emp) {
                  const uint32_t fl = __ffs(emp) - 1;
                  const uint32_t cs = (lh + fl) & mask;
                  uint32_t cv = 0;
                  if (lane == fl) cv = atomicCAS(&tbl[cs], kEmpty, lid);
                  cv = __shfl_sync(kFull, cv, fl);
                  if (cv == kEmpty || cv == lid) {
                    found = cs;
                    fresh = cv == kEmpty;
                    break;
                  }
                  lh = cs;  // the slot was just taken: probe on from it
                } else {
                  lh = (lh + 32) & mask;
                }
              }
              if (lane == leader) {
#pragma unroll
                for (int k = 0; k < Q; ++k)
                  if (q == (uint32_t)k) sl[k] = found;
                newmask |= (fresh ? 1u : 0u) << q;
                pend &= ~(1u << q);
              }
            }
          }
          // ranks for this pass's new ids (lane order, then position order);
          // each new vertex's row starts on its way into the slot at once
          const uint32_t cnt = __popc(newmask);
          const uint32_t b0 = __ballot_sync(kFull, cnt & 1u), b1 = __ballot_sync(kFull, cnt & 2u),
                         b2 = __ballot_sync(kFull, cnt & 4u), b3 = __ballot_sync(kFull, cnt & 8u);
          const uint32_t lt = lanemask_lt();
          const uint32_t total = __popc(b0) + 2 * __popc(b1) + 4 * __popc(b2) + 8 * __popc(b3);
          uint32_t r = 0;
          if (lane == 0 && total) r = atomicAdd(counter, total);
          r = __shfl_sync(kFull, r, 0) + __popc(b0 & lt) + 2 * __popc(b1 & lt) + 4 * __popc(b2 & lt) +
              8 * __popc(b3 & lt);
#pragma unroll
          for (int q = 0; q < Q; ++q) {
            if ((newmask >> q) & 1u) {
              if (r < a.ucap) {
                dense[sl[q]] = (uint16_t)r;
                uniq[r] = id[q];
                copy_row<SH>(a, rows, r, id[q]);
              } else {
                atomicOr(a.err, EBIT_CAPACITY);
              }
              ++r;
            }
          }
#pragma unroll
          for (int k = 0; k < kGroupsPerPass; ++k) {
            const uint32_t g = gb + k * NP + lane * NPW + pw;
            if (g < ngroups)
              reinterpret_cast<uint2*>(map)[g] =
                  make_uint2(sl[4 * k] | (sl[4 * k + 1] << 16), sl[4 * k + 2] | (sl[4 * k + 3] << 16));
          }
        }
      }
      // hand the slot over: its phase completes once every producer has
      // arrived and this thread's row copies have landed
      cp_async_mbar_arrive(&bars[2 + s]);
      mbar_arrive(&bars[2 + s]);
      if (DEDUP != DEDUP_SORT) {
        // empty the other table for the next batch (the last batch used it),
        // after this batch's insertions so that the stores do not queue
        // ahead of its atomics
        uint32_t* other = table + (s ^ 1u) * a.hash_slots;
        for (uint32_t sl = 4 * tid; sl < a.hash_slots; sl += 4 * NP)
          *reinterpret_cast<uint4*>(other + sl) = make_uint4(kEmpty, kEmpty, kEmpty, kEmpty);
      }
      // every id of the batch inserted, the other table empty again; the
      // window and the sort keys are free; the next batch is known
      named_sync(kBarProducers, NP);
      b = misc[6 + (s ^ 1u)];
    }
    // never leave a copy in flight into this block's shared memory
    cp_async_wait<0>();
    if (tid == 0 && window_pending && *abort_flag)  // sleeps in steps, at most ~0.8 s
      for (uint32_t it = 0; it < (1u << 14); ++it)
        if (mbar_try_wait_sleep(&bars[pending_buf], (wph >> pending_buf) & 1u, 50000u)) break;
  } else {
    // ======================= consumers =======================
    const uint32_t ctid = tid - NP, cw = warp - NPW;
    float4* stage = reinterpret_cast<float4*>(smem + L.off_stage) + cw * 32u * K;
    unsigned long long inv_total = 0, nbatches = 0;
    bool bulk_pending = false;  // a bulk store of this warp may still read its staging area
    uint32_t fph = 0u;  // bit s: parity of full[s]
    for (uint32_t j = 0;; ++j) {
      const uint32_t s = j & 1u;
      if (!wait_or_abort(&bars[2 + s], (fph >> s) & 1u, abort_flag, a.err)) break;
      fph ^= 1u << s;
      const uint32_t b = misc[4 + s];  // the slot's batch
      if (b == kNoBatch) break;
      const uint32_t t0 = misc[36 + 2 * s], t1 = misc[37 + 2 * s];
      const uint32_t i0 = 3 * t0, n = 3 * (t1 - t0), base = i0 & ~3u, pad = i0 - base;
      const uint32_t ngroups = (pad + n + 3) >> 2;
      unsigned char* slot_p = ring(s);
      const uint16_t* map = reinterpret_cast<const uint16_t*>(slot_p + L.ring_map);
      const uint16_t* dense = reinterpret_cast<const uint16_t*>(slot_p + L.ring_dense);
      const uint32_t* uniq = reinterpret_cast<const uint32_t*>(slot_p + L.ring_uniq);
      unsigned char* rows = slot_p + L.ring_rows;
      float4* vsh = reinterpret_cast<float4*>(rows);
      const uint32_t U = min(misc[s], a.ucap);

      // --- shade each unique vertex once, in place
      for (uint32_t r = ctid; r < U; r += NC) {
        float o[8];
        const uint32_t id = uniq[r];
        if (id < a.num_verts) {
          VertexIn v;
          load_raw<SH>(rows + r * RB, v);
          shade_vertex<SH>(u, palette, v, o);
        } else {
#pragma unroll
          for (int c = 0; c < 8; ++c) o[c] = 0.f;
          atomicOr(a.err, EBIT_INDEX_RANGE);
        }
        if (K == 7) o[7] = 0.f;
        vsh[row_slot<SH>(r, 0)] = make_float4(o[0], o[1], o[2], o[3]);
        vsh[row_slot<SH>(r, 1)] = make_float4(o[4], o[5], o[6], o[7]);
      }
      named_sync(kBarConsumers, NC);  // every unique vertex shaded; every consumer has read the counter
      if (ctid == 0) {
        misc[s] = 0;  // the slot's counter, for the batch two on
        inv_total += U;
        nbatches += 1;
        if (a.batch_inv != nullptr && b < a.batch_cap) a.batch_inv[b] = U;
      }

      // --- assemble the batch's triangles in input order
      if (n <= a.max_batch_idx) {  // a larger batch was flagged and stopped by the producers
        const size_t f_lo = (size_t)K * i0, f_hi = (size_t)K * (i0 + n);  // the batch's output floats
        for (uint32_t gw = cw * 32u; gw < ngroups; gw += NC) {  // warp-uniform
          const uint32_t g = gw + lane;
          uint2 m = make_uint2(0, 0);
          if (g < ngroups) m = reinterpret_cast<const uint2*>(map)[g];
          const uint32_t sl[4] = {m.x & 0xFFFFu, m.x >> 16, m.y & 0xFFFFu, m.y >> 16};
          float f[4 * 7];  // K = 7: the 4 corners' floats, regrouped into 7 float4
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            uint32_t r = (DEDUP == DEDUP_SORT) ? sl[e] : (uint32_t)dense[sl[e]];
            r = r < U ? r : 0u;  // positions outside the batch (never written) and flagged capacity errors
            const float4 lo = vsh[row_slot<SH>(r, 0)], hi = vsh[row_slot<SH>(r, 1)];
            if (K == 8) {  // a corner is two whole float4
              stage[stage_put<K>(lane, 2 * e)] = lo;
              stage[stage_put<K>(lane, 2 * e + 1)] = hi;
            } else {
              f[7 * e + 0] = lo.x; f[7 * e + 1] = lo.y; f[7 * e + 2] = lo.z; f[7 * e + 3] = lo.w;
              f[7 * e + 4] = hi.x; f[7 * e + 5] = hi.y; f[7 * e + 6] = hi.z;
            }
            if (a.corner_ids != nullptr) {
              const uint32_t p = 4 * g + e;
              if (g < ngroups && p >= pad && p < pad + n) a.corner_ids[base + p] = uniq[r];
            }
          }
          const size_t F0 = (size_t)K * (base + 4 * gw);  // first float of the warp's span (16-byte aligned)
          const bool interior = F0 >= f_lo && F0 + 128 * K <= f_hi;  // the whole span lies in the batch
          if (K == 7) {
            if (bulk_pending) {  // the last bulk store must have read the staging area
              if (lane == 0) bulk_wait_read<0>();
              __syncwarp();
              bulk_pending = false;
            }
#pragma unroll
            for (int jj = 0; jj < 7; ++jj)
              stage[stage_put<K>(lane, jj)] = make_float4(f[4 * jj], f[4 * jj + 1], f[4 * jj + 2], f[4 * jj + 3]);
            if (interior) {  // the span in one bulk (TMA) store, in output order in the staging area
              fence_proxy_async_smem();
              __syncwarp();
              if (lane == 0) {
                bulk_store(a.out + F0, stage, 128 * K * 4);
                bulk_commit();
              }
              bulk_pending = true;
              continue;
            }
          }
          __syncwarp();
#pragma unroll
          for (int jj = 0; jj < K; ++jj) {
            const float4 v = stage[stage_get<K>(32 * jj + lane)];
            const size_t fq = F0 + 4 * (32 * jj + lane);
            if (interior || (fq >= f_lo && fq + 4 <= f_hi)) {
              st_stream4(a.out + fq, v);
            } else if (fq + 4 > f_lo && fq < f_hi) {  // a float4 the neighbouring batch shares
              const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
              for (int c = 0; c < 4; ++c)
                if (fq + c >= f_lo && fq + c < f_hi) a.out[fq + c] = vv[c];
            }
          }
          __syncwarp();  // the staging area is read before the next step writes it
        }
      }
      mbar_arrive(&bars[4 + s]);  // this thread is done with the slot
    }
    if (lane == 0) bulk_wait_all<0>();  // this warp's bulk stores are complete
    if (ctid == 0 && nbatches) {
      atomicAdd(a.counters + CNT_INVOCATIONS, inv_total);
      atomicAdd(a.counters + CNT_BATCHES, nbatches);
      atomicAdd(a.counters + CNT_UNIQUE, inv_total);
    }
  }
}

// The kernel at 64 registers a thread (4 blocks of 256 threads fit an SM's
// registers) ...
template <int DEDUP, int SH, bool DYN>
__global__ void __launch_bounds__(512, 2) reuse_kernel(const __grid_constant__ DrawArgs a,
                                                       const __grid_constant__ Uniforms u) {
  reuse_body<DEDUP, SH, DYN>(a, u);
}

// ... and at up to 80 (3 blocks of 256 threads), for hash/phash draws over
// dynamic batches with the MVP or envelope shader: where shared memory already
// holds the block to 3 per SM, the extra registers cost no occupancy and spare
// the compiler's register-limited scheduling (launch_reuse picks it only then).
template <int DEDUP, int SH>
__global__ void __maxnreg__(80) reuse_kernel_wide(const __grid_constant__ DrawArgs a,
                                                  const __grid_constant__ Uniforms u) {
  reuse_body<DEDUP, SH, true>(a, u);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

template <int D, bool DYN>
static const void* reuse_fn_sh(int shader) {
  switch (shader) {
    case 0: return reinterpret_cast<const void*>(&reuse_kernel<D, 0, DYN>);
    case 1: return reinterpret_cast<const void*>(&reuse_kernel<D, 1, DYN>);
    case 2: return reinterpret_cast<const void*>(&reuse_kernel<D, 2, DYN>);
    default: return reinterpret_cast<const void*>(&reuse_kernel<D, 3, DYN>);
  }
}

static const void* reuse_kernel_ptr(int dedup, bool dyn, int shader, bool wide) {
  if (wide) {  // instantiated for hash/phash, dynamic batches, shaders 0 and 2 only
    if (dedup == DEDUP_SORT || !dyn || (shader != 0 && shader != 2)) return nullptr;
    if (dedup == DEDUP_HASH)
      return shader == 0 ? reinterpret_cast<const void*>(&reuse_kernel_wide<DEDUP_HASH, 0>)
                         : reinterpret_cast<const void*>(&reuse_kernel_wide<DEDUP_HASH, 2>);
    return shader == 0 ? reinterpret_cast<const void*>(&reuse_kernel_wide<DEDUP_PHASH, 0>)
                       : reinterpret_cast<const void*>(&reuse_kernel_wide<DEDUP_PHASH, 2>);
  }
  if (dyn) {
    switch (dedup) {
      case DEDUP_SORT: return reuse_fn_sh<DEDUP_SORT, true>(shader);
      case DEDUP_HASH: return reuse_fn_sh<DEDUP_HASH, true>(shader);
      default: return reuse_fn_sh<DEDUP_PHASH, true>(shader);
    }
  }
  switch (dedup) {
    case DEDUP_SORT: return reuse_fn_sh<DEDUP_SORT, false>(shader);
    case DEDUP_HASH: return reuse_fn_sh<DEDUP_HASH, false>(shader);
    default: return reuse_fn_sh<DEDUP_PHASH, false>(shader);
  }
}

size_t reuse_smem_bytes(int dedup, int shader, const DrawArgs& a, int threads) {
  return reuse_layout(dedup, shader, a, (uint32_t)threads).total;
}

static int blocks_per_sm(const void* fn, int threads, size_t smem) {
  if (fn == nullptr) return 0;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, smem) != cudaSuccess) return 0;
  return nb;
}

int reuse_blocks_per_sm(int dedup, bool dynamic, int shader, int threads, size_t smem, bool* wide) {
  const int nb = blocks_per_sm(reuse_kernel_ptr(dedup, dynamic, shader, false), threads, smem);
  // the 80-register kernel where it exists and fits as many blocks per SM
  *wide = nb > 0 && blocks_per_sm(reuse_kernel_ptr(dedup, dynamic, shader, true), threads, smem) == nb;
  return nb;
}

cudaError_t launch_reuse(int dedup, bool dynamic, bool wide, const DrawArgs& a, const Uniforms& u, int shader,
                         int threads, int grid, size_t smem, cudaStream_t s) {
  const void* fn = reuse_kernel_ptr(dedup, dynamic, shader, wide);
  if (fn == nullptr) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  void* args[] = {const_cast<DrawArgs*>(&a), const_cast<Uniforms*>(&u)};
  return cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, smem, s);
}

}  // namespace gp
