// The per-batch work of the reuse methods, shared by the single-draw kernel
// (one thread block per batch) and the multi-draw frame kernel (one thread
// group per batch, several groups per block):
//   * dedup           -- find the batch's unique indices (Algorithm 2 sort,
//     Algorithm 3 hash, Section 3.4 parallel hash); each warp hands its new
//     vertices to a consumer as it finds them (ShadeQueue shades them at
//     once), or (hash/phash without ranks) leaves the numbering to the caller;
//   * dedup_and_shade -- dedup with ShadeQueue;
//   * fill_stage      -- write a run of assembled triangles, in input order,
//     into a shared staging buffer.
// 'tid'/'NT' are the thread's index in and the size of its group; 'sync' is
// the group barrier (__syncthreads for a whole block, a named barrier for a
// part of one).
#pragma once

#include "gp_device.cuh"

namespace gp {

constexpr uint32_t kNewFlag = 0x8000u;  // map entry flag (hash/phash without ranks); slots < 2^15
constexpr int kIdsPerRound = 4;  // indices a thread inserts before its warp takes ranks for the new ones

struct BlockSync {
  __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

// Named barrier over the nthreads threads of one group (a multiple of 32).
struct GroupSync {
  uint32_t id, nthreads;
  __device__ __forceinline__ void operator()() const {
    if (nthreads == 32) __syncwarp();
    else asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
  }
};

// Shared-memory working set of one batch.
struct BatchSmem {
  uint16_t* map;                // corner position -> slot (hash) or rank (sort)
  unsigned long long* keys;     // sort: (id << 32 | position)
  uint32_t* table;              // hash: open-addressing table, kEmpty = free
  uint16_t* dense;              // hash: slot -> rank
  uint32_t* uniq;               // rank -> vertex id
  float* vsh;                   // rank -> shaded vertex (KS floats)
  uint32_t* ucount;             // unique count of the batch
  uint32_t* wsum;               // per-warp totals for the sort's scan (>= NT/32 words)
};

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

// Shades the new vertices of ranks [rb, re) (ids in uniq; ranks >= ucap
// were not stored) in full-warp passes: two vertices per lane per pass, both
// loads issued before the math.
template <int SH>
__device__ __forceinline__ void shade_range(const DrawArgs& a, const Uniforms& u, const float* palette, float* vsh,
                                            const uint32_t* uniq, uint32_t rb, uint32_t re, uint32_t lane) {
  re = min(re, a.ucap);
  for (uint32_t r0 = rb + lane; r0 < re; r0 += 64) {
    const uint32_t r1 = r0 + 32;
    const bool has1 = r1 < re;
    const uint32_t id0 = uniq[r0];
    const uint32_t id1 = has1 ? uniq[r1] : kInvalidId;
    VertexIn v0, v1;
    const bool ok0 = id0 < a.num_verts, ok1 = id1 < a.num_verts;
    if (ok0) fetch_vertex<SH>(a.verts, a.stride, id0, v0, a.vec8 != 0);
    if (ok1) fetch_vertex<SH>(a.verts, a.stride, id1, v1, a.vec8 != 0);
    float o[ShaderTraits<SH>::K];
    if (ok0) {
      shade_vertex<SH>(u, palette, v0, o);
    } else {
#pragma unroll
      for (int c = 0; c < ShaderTraits<SH>::K; ++c) o[c] = 0.f;
      atomicOr(a.err, EBIT_INDEX_RANGE);
    }
    store_shaded<SH>(vsh, r0, o);
    if (has1) {
      if (ok1) {
        shade_vertex<SH>(u, palette, v1, o);
      } else {
#pragma unroll
        for (int c = 0; c < ShaderTraits<SH>::K; ++c) o[c] = 0.f;
        atomicOr(a.err, EBIT_INDEX_RANGE);
      }
      store_shaded<SH>(vsh, r1, o);
    }
  }
}

// Bytes of a vertex row the shaders read, copied whole into shared memory by
// the single-draw kernel (a multiple of 16: the vertex buffer's base and
// stride are 16-byte aligned).
template <int SH>
struct RawTraits {
  static constexpr uint32_t kBytes = ShaderTraits<SH>::kSkin ? 64u : 32u;
  static constexpr uint32_t kChunks = kBytes / 16u;
};

// Consumers of new vertices: called by all lanes of a warp after __syncwarp
// with the range [rb, re) of ranks this warp has just created; S.uniq[rank]
// holds the vertex id for every rank < ucap (ranks >= ucap are a flagged
// capacity error and were not stored).
template <int SH>
struct ShadeQueue {
  const DrawArgs& a;
  const Uniforms& u;
  const float* palette;
  float* vsh;
  const uint32_t* uniq;
  __device__ __forceinline__ void operator()(uint32_t rb, uint32_t re, uint32_t lane) const {
    shade_range<SH>(a, u, palette, vsh, uniq, rb, re, lane);
  }
};

// For a caller that consumes the new vertices after dedup returns.
struct NoConsume {
  __device__ __forceinline__ void operator()(uint32_t, uint32_t, uint32_t) const {}
};

// Reads a vertex row copied into shared memory (16-byte aligned).
template <int SH>
__device__ __forceinline__ void load_raw(const unsigned char* row, VertexIn& v) {
  const float4* p = reinterpret_cast<const float4*>(row);
  const float4 x = p[0], y = p[1];
  v.px = x.x; v.py = x.y; v.pz = x.z;
  v.nx = x.w; v.ny = y.x; v.nz = y.y;
  if (ShaderTraits<SH>::kSkin) {
    const float4 z = p[2], w = p[3];
    v.bones = __float_as_uint(z.x);
    v.w0 = z.y; v.w1 = z.z; v.w2 = z.w; v.w3 = w.x;
  } else {
    v.bones = 0; v.w0 = v.w1 = v.w2 = v.w3 = 0.f;
  }
}

// Bitonic network over N = E * NT keys with E consecutive keys per thread
// in registers: stages with j < E stay in the thread, E <= j < 32 E exchange
// within the warp by shuffles (partner lane = lane ^ j/E), and only
// j >= 32 E goes through shared memory.  For k >= E a thread's E keys all
// lie in one run (ascending where (E tid) & k == 0), and for j >= E they are
// all on the same side of their pairs, so direction and side are worked out
// once per stage; each exchange is then a min or a max.
// The network on keys already in registers (r: keys E tid .. E tid + E - 1);
// the shared-memory stages use keys[0..N) as their exchange buffer.  Leaves
// the sorted keys in r.
template <int E, class T, class Sync>
__device__ __forceinline__ void bitonic_network_regs(T (&r)[E], T* keys, uint32_t N, uint32_t tid, Sync sync) {
  const uint32_t i0 = E * tid;  // this thread's first key
  for (uint32_t k = 2; k <= N; k <<= 1) {
    const bool asc = (i0 & k) == 0;  // the thread's run (k >= E)
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      if (j >= (uint32_t)E) {
        const bool take_min = ((i0 & j) == 0) == asc;  // lower side of an ascending pair, or upper of a descending
        if (j >= 32u * E) {
          sync();  // every thread has read the previous contents
#pragma unroll
          for (int e = 0; e < E; ++e) keys[i0 + e] = r[e];
          sync();
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const T y = keys[(i0 + e) ^ j];
            r[e] = take_min ? (r[e] < y ? r[e] : y) : (r[e] < y ? y : r[e]);
          }
        } else {
          const uint32_t lm = j / E;
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const T y = __shfl_xor_sync(kFull, r[e], lm);
            r[e] = take_min ? (r[e] < y ? r[e] : y) : (r[e] < y ? y : r[e]);
          }
        }
      } else {
        // j < E: both keys of a pair are in this thread (j is 1, 2 or 4, each
        // with compile-time register indices); the lower one keeps the
        // smaller key in an ascending run
        auto exch = [&](int lo, int hi) {
          const bool up = k >= (uint32_t)E ? asc : ((i0 + lo) & k) == 0;
          const T a = r[lo], b = r[hi];
          const T mn = a < b ? a : b, mx = a < b ? b : a;
          r[lo] = up ? mn : mx;
          r[hi] = up ? mx : mn;
        };
        if (j == 1) {
#pragma unroll
          for (int e = 0; e < E; e += 2) exch(e, e + 1);
        } else if (j == 2) {
#pragma unroll
          for (int e = 0; e < E; ++e)
            if ((e & 2) == 0) exch(e, e + 2);
        } else {
#pragma unroll
          for (int e = 0; e < E; ++e)
            if ((e & 4) == 0 && e + 4 < E) exch(e, e + 4);
        }
      }
    }
  }
}

// The register network on keys[0..N), N = E NT: loads each thread's E keys,
// sorts, and stores them back.
template <int E, class T, class Sync>
__device__ __forceinline__ void bitonic_sort_regs(T* keys, uint32_t N, uint32_t tid, Sync sync) {
  T r[E];
#pragma unroll
  for (int e = 0; e < E; ++e) r[e] = keys[E * tid + e];
  bitonic_network_regs<E>(r, keys, N, tid, sync);
  sync();
#pragma unroll
  for (int e = 0; e < E; ++e) keys[E * tid + e] = r[e];
  sync();
}

// Bitonic sort of keys[0..N), N a power of two.  With N = 4 NT or 8 NT the
// keys stay in registers (bitonic_sort_regs).  Otherwise the network runs
// in shared memory; for j <= 32 the pairs touched by one warp stay inside
// that warp's 64-key blocks (i = 2t - (t mod j), t = 32q + r), so those
// stages need only a warp barrier.  Leaves the sorted keys in keys[].
template <class T, class Sync>
__device__ __forceinline__ void bitonic_sort(T* keys, uint32_t N, uint32_t tid, uint32_t NT, Sync sync) {
  if (N == 4 * NT) {
    bitonic_sort_regs<4>(keys, N, tid, sync);
    return;
  }
  if (N == 8 * NT) {
    bitonic_sort_regs<8>(keys, N, tid, sync);
    return;
  }
  for (uint32_t k = 2; k <= N; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t t = tid; t < N / 2; t += NT) {
        const uint32_t i = 2 * t - (t & (j - 1));
        const uint32_t l = i + j;
        const bool up = (i & k) == 0;
        const T x = keys[i], y = keys[l];
        if ((x > y) == up) {
          keys[i] = y;
          keys[l] = x;
        }
      }
      const uint32_t nj = j > 1 ? (j >> 1) : k;  // j of the next stage
      if (j >= 64 || nj >= 64) sync();
      else __syncwarp();
    }
  }
  sync();
}

// Algorithm 2 on keys of type T = (id << pb) | position: sort, tail flags,
// exclusive prefix sum.  pb = 32 with 64-bit keys; with 32-bit keys ids must
// stay below 2^(32 - pb) - 1, the id field's largest value standing for an
// id out of range (the host picks 32-bit keys when the vertex count allows
// it: half the registers and shuffles of the sorting network).
// With N = E NT (E = 4 or 8) every step runs on registers: each thread
// builds its E consecutive keys, the network sorts them in place, and the
// thread flags, ranks and scatters the same E keys -- no pass of the keys
// through shared memory but the network's own exchange stages.
template <int E, class T, class Sync, class Consume>
__device__ __forceinline__ void sort_dedup_regs(const DrawArgs& a, const BatchSmem& S, const uint32_t* ids,
                                                uint32_t n, uint32_t tid, uint32_t NT, Sync sync,
                                                const Consume& consume, uint32_t pb) {
  const uint32_t lane = lane_id(), warp = tid >> 5, i0 = E * tid;
  T* keys = reinterpret_cast<T*>(S.keys);
  const T invalid = (T)((sizeof(T) == 4 ? (1ull << (32 - pb)) - 1 : (unsigned long long)kInvalidId));
  auto id_of = [&](T key) { return (uint32_t)(key >> pb); };
  T r[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const uint32_t i = i0 + e;
    const uint32_t id = i < n ? ids[i] : 0u;
    r[e] = i < n ? (((id < a.num_verts ? (T)id : invalid) << pb) | (T)i) : ~(T)0;
  }
  bitonic_network_regs<E>(r, keys, E * NT, tid, sync);
  // the key after this thread's last one: the next lane's first, or for
  // lane 31 the next warp's first, passed through shared memory
  sync();  // every thread has read the network's last shared-memory stage
  if (lane == 0) keys[i0] = r[0];
  sync();
  T after = __shfl_down_sync(kFull, r[0], 1);
  if (lane == 31) after = tid + 1 < NT ? keys[i0 + E] : ~(T)0;
  // tail flags (the last key of each id's group), then a group scan
  uint32_t tails = 0;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const T next = e + 1 < E ? r[e + 1 < E ? e + 1 : e] : after;
    const uint32_t i = i0 + e;
    if (i < n && (i == n - 1 || id_of(r[e]) != id_of(next))) tails |= 1u << e;
  }
  const uint32_t cnt = __popc(tails);
  const uint32_t inc = warp_inclusive_scan(cnt);
  if (lane == 31) S.wsum[warp] = inc;
  sync();
  uint32_t rk = inc - cnt;
  for (uint32_t w = 0; w < warp; ++w) rk += S.wsum[w];
  if (tid == NT - 1) *S.ucount = rk + cnt;
  const uint32_t rb = __shfl_sync(kFull, rk, 0), re = __shfl_sync(kFull, rk + cnt, 31);
  const T pmask = (T)((1ull << (sizeof(T) == 4 ? pb : 16)) - 1);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    if (i0 + e < n) {
      S.map[(uint32_t)(r[e] & pmask)] = (uint16_t)rk;
      if ((tails >> e) & 1u) {
        const uint32_t id = id_of(r[e]);
        if (rk < a.ucap) S.uniq[rk] = (T)id == invalid ? kInvalidId : id;
        else atomicOr(a.err, EBIT_CAPACITY);
        ++rk;
      }
    }
  }
  __syncwarp();
  consume(rb, re, lane);
  __syncwarp();
}

template <class T, class Sync, class Consume>
__device__ __forceinline__ void sort_dedup(const DrawArgs& a, const BatchSmem& S, const uint32_t* ids, uint32_t n,
                                           uint32_t tid, uint32_t NT, Sync sync, const Consume& consume,
                                           uint32_t pb) {
  if (a.sort_n == 8 * NT) {
    sort_dedup_regs<8, T>(a, S, ids, n, tid, NT, sync, consume, pb);
    return;
  }
  if (a.sort_n == 4 * NT) {
    sort_dedup_regs<4, T>(a, S, ids, n, tid, NT, sync, consume, pb);
    return;
  }
  const uint32_t lane = lane_id(), warp = tid >> 5;
  T* keys = reinterpret_cast<T*>(S.keys);
  const T invalid = (T)((sizeof(T) == 4 ? (1ull << (32 - pb)) - 1 : (unsigned long long)kInvalidId));
  auto id_of = [&](T key) { return (uint32_t)(key >> pb); };
  for (uint32_t i = tid; i < a.sort_n; i += NT) {
    if (i < n) {
      const uint32_t id = ids[i];
      keys[i] = ((id < a.num_verts ? (T)id : invalid) << pb) | (T)i;
    } else {
      keys[i] = ~(T)0;
    }
  }
  sync();
  bitonic_sort(keys, a.sort_n, tid, NT, sync);
  // tail flags over each thread's contiguous run, then a group scan with one
  // barrier: every thread adds up the totals of the warps before its own
  const uint32_t ipt = (n + NT - 1) / NT;
  const uint32_t lo = min(tid * ipt, n), hi = min(lo + ipt, n);
  uint32_t cnt = 0;
  for (uint32_t i = lo; i < hi; ++i) cnt += (i == n - 1 || id_of(keys[i]) != id_of(keys[i + 1])) ? 1u : 0u;
  const uint32_t inc = warp_inclusive_scan(cnt);
  if (lane == 31) S.wsum[warp] = inc;
  sync();
  uint32_t r = inc - cnt;
  for (uint32_t w = 0; w < warp; ++w) r += S.wsum[w];
  if (tid == NT - 1) *S.ucount = r + cnt;
  // the warp's ranks are contiguous: lane 0's first to lane 31's last
  const uint32_t rb = __shfl_sync(kFull, r, 0), re = __shfl_sync(kFull, r + cnt, 31);
  const T pmask = (T)((1ull << (sizeof(T) == 4 ? pb : 16)) - 1);
  for (uint32_t i = lo; i < hi; ++i) {
    const T key = keys[i];
    const uint32_t id = id_of(key);
    S.map[(uint32_t)(key & pmask)] = (uint16_t)r;
    if (i == n - 1 || id != id_of(keys[i + 1])) {  // tail of an id's group
      if (r < a.ucap) S.uniq[r] = (T)id == invalid ? kInvalidId : id;
      else atomicOr(a.err, EBIT_CAPACITY);
      ++r;
    }
  }
  __syncwarp();
  consume(rb, re, lane);
  __syncwarp();
}

// Finds the unique indices of ids[0..n) and passes each new one, once, to
// 'consume' (see ShadeQueue).  On return (after a group barrier
// the caller issues) *S.ucount holds the unique count U, S.uniq[0..U) the
// ids, and S.map each corner's rank (sort) or hash slot (hash/phash; the
// rank is S.dense[slot]).  The hash table must be empty on entry; it is left
// filled (the caller clears it after the barrier).  *S.ucount must be 0 on
// entry for hash/phash.
// RANKS == false (hash/phash only): the table and S.map (slot, with kNewFlag
// at the one position per id whose CAS stored it) are all it produces -- no
// ranks, no uniq, no consume; the caller numbers the vertices itself.
template <int DEDUP, bool RANKS, class Sync, class Consume>
__device__ __forceinline__ void dedup(const DrawArgs& a, const BatchSmem& S, const uint32_t* ids, uint32_t n,
                                      uint32_t tid, uint32_t NT, Sync sync, const Consume& consume) {
  const uint32_t lane = lane_id(), warp = tid >> 5;
  if (DEDUP == DEDUP_SORT) {
    // --- Algorithm 2: sort (id, position), tail flags, exclusive prefix sum
    if (a.sort_pos_bits) sort_dedup<uint32_t>(a, S, ids, n, tid, NT, sync, consume, a.sort_pos_bits);
    else sort_dedup<unsigned long long>(a, S, ids, n, tid, NT, sync, consume, 32);
  } else {
    // --- Algorithm 3 / Section 3.4: every index tries to store its id in its
    // home slot with atomicCAS and probes on after a collision (hash: linear,
    // one slot at a time; phash: up to probe_k slots alone, then 32
    // consecutive slots at a time with the whole warp).  A thread handles
    // kIdsPerRound indices one after another; the other warps of the SM hide
    // the atomics' latency.
    const uint32_t mask = a.hash_slots - 1;
    for (uint32_t rbase = 0; rbase < n; rbase += kIdsPerRound * NT) {
      uint32_t idq[kIdsPerRound], hq[kIdsPerRound], prevq[kIdsPerRound];
      uint32_t newbits = 0;  // bit q: this thread stored idq[q]
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
            uint32_t prev = atomicCAS(&S.table[h], kEmpty, id);
            for (uint32_t probes = 1; prev != kEmpty && prev != id; ++probes) {
              if (probes >= a.hash_slots) {  // table full: cannot happen within capacity
                atomicOr(a.err, EBIT_CAPACITY);
                h = 0;
                break;
              }
              h = (h + 1) & mask;
              prev = atomicCAS(&S.table[h], kEmpty, id);
            }
            is_new = prev == kEmpty;
          }
        } else {
          bool pending = active;
          for (uint32_t p = 0; p < a.probe_k && pending; ++p) {
            const uint32_t prev = atomicCAS(&S.table[h], kEmpty, id);
            if (prev == kEmpty || prev == id) {
              pending = false;
              is_new = prev == kEmpty;
            } else {
              h = (h + 1) & mask;
            }
          }
          uint32_t left = __ballot_sync(kFull, pending);
          while (left) {
            const uint32_t leader = __ffs(left) - 1;
            const uint32_t lid = __shfl_sync(kFull, id, leader);
            uint32_t lh = __shfl_sync(kFull, h, leader);  // the next slot to probe
            uint32_t found = kEmpty;
            bool fresh = false;
            for (uint32_t guard = 0; found == kEmpty; ++guard) {
              if (guard > a.hash_slots / 16 + 64) {  // table full: cannot happen within capacity
                if (lane == 0) atomicOr(a.err, EBIT_CAPACITY);
                found = 0;
                break;
              }
              const uint32_t s = (lh + lane) & mask;
              const uint32_t val = S.table[s];
              const uint32_t hit = __ballot_sync(kFull, val == lid);
              if (hit) {
                found = (lh + __ffs(hit) - 1) & mask;
                break;
              }
              const uint32_t emp = __ballot_sync(kFull, val == kEmpty);
              if (emp) {
                const uint32_t fl = __ffs(emp) - 1;
                const uint32_t cs = (lh + fl) & mask;
                uint32_t pv = 0;
                if (lane == fl) pv = atomicCAS(&S.table[cs], kEmpty, lid);
                pv = __shfl_sync(kFull, pv, fl);
                if (pv == kEmpty || pv == lid) {
                  found = cs;
                  fresh = pv == kEmpty;
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
            left &= left - 1;
          }
        }
        // without ranks, bit 15 marks the position whose CAS stored the id
        // (the caller numbers the vertices in the order of these positions)
        if (active && !RANKS) S.map[i] = (uint16_t)(h | (is_new ? kNewFlag : 0u));
        idq[q] = id;
        hq[q] = h;
        newbits |= is_new ? (1u << q) : 0u;
      }
      if (RANKS) {
        // dense ranks: one atomicAdd per warp for the round (lane order
        // within each q, q after q), so the warp's new ranks are contiguous
        uint32_t total = 0;
#pragma unroll
        for (int q = 0; q < kIdsPerRound; ++q) {
          const uint32_t m = __ballot_sync(kFull, (newbits >> q) & 1u);
          prevq[q] = total + __popc(m & lanemask_lt());  // rank offset of this lane's q-th new id
          total += __popc(m);
        }
        uint32_t wbase = 0;
        if (lane == 0 && total) wbase = atomicAdd(S.ucount, total);
        wbase = __shfl_sync(kFull, wbase, 0);
#pragma unroll
        for (int q = 0; q < kIdsPerRound; ++q)
          if ((newbits >> q) & 1u) {
            const uint32_t rk = wbase + prevq[q];
            if (rk < a.ucap) {
              S.dense[hq[q]] = (uint16_t)rk;
              S.uniq[rk] = idq[q];
            } else {
              atomicOr(a.err, EBIT_CAPACITY);
            }
          }
#pragma unroll
        for (int q = 0; q < kIdsPerRound; ++q) {
          const uint32_t i = rbase + q * NT + tid;
          if (i < n) S.map[i] = (uint16_t)hq[q];
        }
        __syncwarp();
        consume(wbase, wbase + total, lane);
        __syncwarp();
      }
    }
  }
}

// dedup, shading each new vertex as soon as its warp finds it: on return
// S.vsh holds every unique vertex shaded.
template <int DEDUP, int SH, class Sync>
__device__ __forceinline__ void dedup_and_shade(const DrawArgs& a, const Uniforms& u, const float* palette,
                                                const BatchSmem& S, const uint32_t* ids, uint32_t n, uint32_t tid,
                                                uint32_t NT, Sync sync) {
  dedup<DEDUP, true>(a, S, ids, n, tid, NT, sync, ShadeQueue<SH>{a, u, palette, S.vsh, S.uniq});
}

// Writes corners [cbase, cbase + nc) of the batch (local corner numbering)
// to st[0..nc*K): the shaded result of each corner's vertex, in input order.
// Also records each corner's source vertex in a.corner_ids[gcorner0 + ...].
template <int DEDUP, int SH>
__device__ __forceinline__ void fill_stage(const DrawArgs& a, const BatchSmem& S, float* st, uint32_t cbase,
                                           uint32_t nc, uint32_t U, uint64_t gcorner0, uint32_t tid, uint32_t NT,
                                           bool aligned16) {
  constexpr int K = ShaderTraits<SH>::K;
  constexpr int KS = ShaderTraits<SH>::KS;
  for (uint32_t lc = tid; lc < nc; lc += NT) {
    const uint32_t m = S.map[cbase + lc];
    uint32_t s = (DEDUP == DEDUP_SORT) ? m : S.dense[m];
    s = s < U ? s : 0u;  // only reachable after a flagged capacity error; keeps reads in bounds
    if (K == 8 && aligned16) {
      const float4* sv = reinterpret_cast<const float4*>(S.vsh + s * KS);
      float4* dv = reinterpret_cast<float4*>(st + lc * K);
      dv[0] = sv[0];
      dv[1] = sv[1];
    } else {
#pragma unroll
      for (int c = 0; c < K; ++c) st[lc * K + c] = S.vsh[s * KS + c];
    }
    if (a.corner_ids != nullptr) a.corner_ids[gcorner0 + lc] = S.uniq[s];
  }
}

}  // namespace gp
