// Parallel random walk with on-the-fly reuse (Section 5.4).
//
// Agents live on a toroidal W x H grid; each is the packed key (x << 16) | y.
// Per step an agent evaluates every move (dx, dy) with 1 <= dx^2 + dy^2 <=
// 16^2 -- likelihood A[target] * (65536 / r^2), integers, so comparisons are
// exact -- keeps the 8 largest (earlier candidates first on ties) and draws
// one with probability proportional to its likelihood from a SplitMix64
// number of (seed, step, agent).  The 8 kept moves depend only on the cell,
// so the key is the "index" of the reuse methods:
//   naive  -- every agent evaluates its own cell;
//   warp   -- each warp takes 32 agents; __match_any_sync groups equal keys
//             and the lowest lane of a group evaluates the cell for all;
//   sort / hash / phash -- one thread block per static batch of agents runs
//             the shared dedup body (Algorithm 2 / Algorithm 3 / Section 3.4)
//             on the batch's keys; each unique cell is evaluated once into
//             shared memory, then every agent draws from its cell's row.
//
// The candidate moves sit in constant memory in tie-breaking order (dy, then
// dx, each from -16 to 16); all lanes of a warp walk them in step, so each
// constant read is a broadcast.
#include <algorithm>
#include <mutex>

#include "gp.h"
#include "gp_batch_body.cuh"

namespace gp {

constexpr int kWalkRadius = 16;
constexpr int kWalkKeep = 8;
constexpr int kWalkCand = 796;  // offsets with 1 <= dx^2 + dy^2 <= 256

__constant__ int32_t c_walk_off[kWalkCand];  // (dx + 16) | (dy + 16) << 8
__constant__ uint32_t c_walk_w[kWalkCand];   // 65536 / r^2

struct WalkArgs {
  const uint32_t* act;  // [h][w]
  uint32_t w, h;
  const uint32_t* pin;
  uint32_t* pout;
  uint32_t n;
  uint64_t seed;
  uint32_t step;
  uint32_t batch;                  // agents per batch (counts; sort/hash/phash block size unit)
  unsigned long long* counters;    // [0] evaluations, [1] batches, [2] error bits
};

// One step of SplitMix64 from state x: the increment, then the mix.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// The 8 kept moves of cell (x, y): running sums of their likelihoods
// (cum[7] = total) and the moves, packed as in c_walk_off.
struct CellMoves {
  uint64_t cum[kWalkKeep];
  uint32_t mv[kWalkKeep];
};

__device__ __forceinline__ void eval_cell(const WalkArgs& a, uint32_t key, CellMoves& out) {
  const int x = (int)(key >> 16), y = (int)(key & 0xFFFFu);
  uint64_t lik[kWalkKeep];
  uint32_t mv[kWalkKeep];
#pragma unroll
  for (int k = 0; k < kWalkKeep; ++k) {
    lik[k] = 0;
    mv[k] = 0;
  }
  static_assert(kWalkCand % 4 == 0, "candidates are read four at a time");
  for (int j = 0; j < kWalkCand; j += 4) {
    // four independent activity reads in flight, then the four insertions
    uint32_t av[4];
    int32_t oo[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int32_t o = c_walk_off[j + q];
      int tx = x + (o & 0xFF) - kWalkRadius, ty = y + (o >> 8) - kWalkRadius;
      tx += tx < 0 ? (int)a.w : 0;
      tx -= tx >= (int)a.w ? (int)a.w : 0;
      ty += ty < 0 ? (int)a.h : 0;
      ty -= ty >= (int)a.h ? (int)a.h : 0;
      oo[q] = o;
      av[q] = __ldg(a.act + (uint32_t)ty * a.w + (uint32_t)tx);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint64_t cur = (uint64_t)av[q] * c_walk_w[j + q];
      if (cur > lik[kWalkKeep - 1]) {
        // insertion; order: likelihood descending, then candidate order (the
        // packed offset grows with it), which also places an element pushed
        // down correctly among equal ones
        uint32_t cm = (uint32_t)oo[q];
#pragma unroll
        for (int k = 0; k < kWalkKeep; ++k) {
          if (cur > lik[k] || (cur == lik[k] && cm < mv[k])) {
            const uint64_t t = lik[k];
            lik[k] = cur;
            cur = t;
            const uint32_t tm = mv[k];
            mv[k] = cm;
            cm = tm;
          }
        }
      }
    }
  }
  uint64_t acc = 0;
#pragma unroll
  for (int k = 0; k < kWalkKeep; ++k) {
    acc += lik[k];
    out.cum[k] = acc;
    out.mv[k] = mv[k];
  }
}

__device__ __forceinline__ uint32_t take_move(const WalkArgs& a, uint32_t key, uint32_t agent, const uint64_t* cum,
                                              const uint32_t* mv) {
  if (cum[kWalkKeep - 1] == 0) return key;  // no move has a positive likelihood: stay
  const uint64_t u = splitmix64(a.seed ^ (((uint64_t)a.step << 32) | agent));
  const uint64_t r = u % cum[kWalkKeep - 1];
  uint32_t m = mv[kWalkKeep - 1];
#pragma unroll
  for (int k = kWalkKeep - 2; k >= 0; --k) m = cum[k] > r ? mv[k] : m;
  int x = (int)(key >> 16) + (int)(m & 0xFF) - kWalkRadius;
  int y = (int)(key & 0xFFFFu) + (int)(m >> 8) - kWalkRadius;
  x += x < 0 ? (int)a.w : 0;
  x -= x >= (int)a.w ? (int)a.w : 0;
  y += y < 0 ? (int)a.h : 0;
  y -= y >= (int)a.h ? (int)a.h : 0;
  return ((uint32_t)x << 16) | (uint32_t)y;
}

__global__ void __launch_bounds__(256) walk_naive_kernel(const __grid_constant__ WalkArgs a) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const uint32_t key = a.pin[i];
  CellMoves cm;
  eval_cell(a, key, cm);
  a.pout[i] = take_move(a, key, i, cm.cum, cm.mv);
  if (threadIdx.x == 0) {
    atomicAdd(a.counters + 0, (unsigned long long)min(blockDim.x, a.n - blockIdx.x * blockDim.x));
    atomicAdd(a.counters + 1, 1ull);
  }
}

// One warp per 32 agents; the group leader's row goes through shared memory.
__global__ void __launch_bounds__(256) walk_warp_kernel(const __grid_constant__ WalkArgs a) {
  __shared__ CellMoves rows[256];
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t lane = lane_id(), wbase = threadIdx.x & ~31u;
  if ((i & ~31u) >= a.n) return;  // warp-uniform
  const bool active = i < a.n;
  const uint32_t key = active ? a.pin[i] : 0xFFFFFFFFu;
  const uint32_t grp = __match_any_sync(kFull, key);
  const uint32_t leader = __ffs(grp) - 1;
  if (active && lane == leader) eval_cell(a, key, rows[threadIdx.x]);
  __syncwarp();
  if (active) {
    const CellMoves& r = rows[wbase + leader];
    a.pout[i] = take_move(a, key, i, r.cum, r.mv);
  }
  const uint32_t leaders = __ballot_sync(kFull, active && lane == leader);
  if (lane == 0) atomicAdd(a.counters + 0, (unsigned long long)__popc(leaders));
  if (threadIdx.x == 0) atomicAdd(a.counters + 1, 1ull);
}

// One block per batch of a.batch agents: dedup of the keys, one evaluation
// per unique cell into shared memory, then every agent's draw.
struct WalkShade {
  const WalkArgs& wa;
  const uint32_t* uniq;
  CellMoves* rows;
  uint32_t ucap;
  __device__ __forceinline__ void operator()(uint32_t rb, uint32_t re, uint32_t lane) const {
    re = min(re, ucap);  // ranks >= ucap (a flagged capacity error) were not stored
    for (uint32_t r = rb + lane; r < re; r += 32) eval_cell(wa, uniq[r], rows[r]);
  }
};

template <int DEDUP>
__global__ void __launch_bounds__(512) walk_batched_kernel(const __grid_constant__ WalkArgs wa,
                                                           const __grid_constant__ DrawArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t S = wa.batch, tid = threadIdx.x, NT = blockDim.x;
  const uint32_t i0 = blockIdx.x * S, n = min(S, wa.n - i0);
  // layout: rows [S] | keys [S] | map [S] u16 | uniq [S] | table [slots] + dense [slots] u16 or sort keys | misc
  CellMoves* rows = reinterpret_cast<CellMoves*>(smem);
  uint32_t* keys = reinterpret_cast<uint32_t*>(rows + S);
  uint16_t* map = reinterpret_cast<uint16_t*>(keys + S);
  uint32_t* uniq = reinterpret_cast<uint32_t*>(map + ((S + 1) & ~1u));
  unsigned char* tail = reinterpret_cast<unsigned char*>(uniq + S);
  BatchSmem B;
  B.map = map;
  B.uniq = uniq;
  if (DEDUP == DEDUP_SORT) {
    B.keys = reinterpret_cast<unsigned long long*>(tail);
    tail += (size_t)a.sort_n * 8;
  } else {
    B.table = reinterpret_cast<uint32_t*>(tail);
    B.dense = reinterpret_cast<uint16_t*>(tail + (size_t)a.hash_slots * 4);
    tail += (size_t)a.hash_slots * 6;
  }
  uint32_t* misc = reinterpret_cast<uint32_t*>(tail);
  B.ucount = misc;
  B.wsum = misc + 8;
  B.vsh = nullptr;
  for (uint32_t k = tid; k < n; k += NT) keys[k] = wa.pin[i0 + k];
  if (DEDUP != DEDUP_SORT)
    for (uint32_t s = tid; s < a.hash_slots; s += NT) B.table[s] = kEmpty;
  if (tid == 0) *B.ucount = 0;
  __syncthreads();
  dedup<DEDUP, true>(a, B, keys, n, tid, NT, BlockSync(), WalkShade{wa, uniq, rows, a.ucap});
  __syncthreads();
  const uint32_t U = min(*B.ucount, a.ucap);
  for (uint32_t k = tid; k < n; k += NT) {
    uint32_t r = map[k];
    if (DEDUP != DEDUP_SORT) r = B.dense[r];
    r = r < U ? r : 0u;  // only after a flagged capacity error
    wa.pout[i0 + k] = take_move(wa, keys[k], i0 + k, rows[r].cum, rows[r].mv);
  }
  if (tid == 0) {
    atomicAdd(wa.counters + 0, (unsigned long long)U);
    atomicAdd(wa.counters + 1, 1ull);
  }
}

size_t walk_batched_smem(int dedup, uint32_t S, uint32_t slots, uint32_t sort_n) {
  size_t o = (size_t)S * sizeof(CellMoves) + (size_t)S * 4 + (size_t)((S + 1) & ~1u) * 2 + (size_t)S * 4;
  o += dedup == DEDUP_SORT ? (size_t)sort_n * 8 : (size_t)slots * 6;
  return o + 64 * 4;
}

}  // namespace gp

using namespace gp;

namespace {

std::mutex g_walk_mu;
uint64_t g_walk_ready = 0;  // bit d: the candidate table is in device d's constant memory

gp_status walk_tables(int device) {
  std::lock_guard<std::mutex> lk(g_walk_mu);
  if (device < 64 && (g_walk_ready >> device) & 1) return GP_OK;
  int32_t off[kWalkCand];
  uint32_t w[kWalkCand];
  int k = 0;
  for (int dy = -kWalkRadius; dy <= kWalkRadius; ++dy)
    for (int dx = -kWalkRadius; dx <= kWalkRadius; ++dx) {
      const int r2 = dx * dx + dy * dy;
      if (r2 < 1 || r2 > kWalkRadius * kWalkRadius) continue;
      off[k] = (dx + kWalkRadius) | ((dy + kWalkRadius) << 8);
      w[k] = 65536u / (uint32_t)r2;
      ++k;
    }
  if (k != kWalkCand) return GP_ERR_UNSUPPORTED;
  if (cudaMemcpyToSymbol(c_walk_off, off, sizeof(off)) != cudaSuccess ||
      cudaMemcpyToSymbol(c_walk_w, w, sizeof(w)) != cudaSuccess)
    return GP_ERR_CUDA;
  if (device < 64) g_walk_ready |= 1ull << device;
  return GP_OK;
}

uint32_t pow2_at_least(uint32_t x) {
  uint32_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

}  // namespace

extern "C" gp_status gp_random_walk(const gp_walk_desc* d) {
  // Section 5.4; see include/gp.h
  if (!d) return GP_ERR_INVALID;
  if (d->width < 17 || d->height < 17 || d->width > 32768 || d->height > 32768 || !d->d_activity ||
      !d->d_counters)
    return GP_ERR_INVALID;
  if (d->num_agents && (!d->d_pos || !d->d_scratch)) return GP_ERR_INVALID;
  const int32_t v = d->variant;
  if (v != GP_NAIVE && v != GP_WARP && v != GP_SORT && v != GP_HASH && v != GP_PHASH) return GP_ERR_INVALID;
  const uint32_t S = d->batch_agents ? d->batch_agents : 576;
  const uint32_t threads = d->threads ? d->threads : 256;
  if (S % 32 || S == 0) return GP_ERR_INVALID;
  if (v >= GP_SORT && (S > 1024 || threads % 32 || (threads & (threads - 1)) || threads > 512))
    return GP_ERR_INVALID;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return GP_ERR_CUDA;
  gp_status st = walk_tables(device);
  if (st != GP_OK) return st;
  if (d->num_agents == 0 || d->steps == 0) return GP_OK;
  cudaStream_t s = static_cast<cudaStream_t>(d->stream);
  WalkArgs wa{};
  wa.act = d->d_activity;
  wa.w = d->width;
  wa.h = d->height;
  wa.n = d->num_agents;
  wa.seed = d->seed;
  wa.batch = S;
  wa.counters = d->d_counters;
  DrawArgs a{};
  size_t smem = 0;
  int dedup = DEDUP_HASH;
  if (v >= GP_SORT) {
    dedup = v == GP_SORT ? DEDUP_SORT : (v == GP_HASH ? DEDUP_HASH : DEDUP_PHASH);
    a.num_verts = 0xFFFFFFF0u;  // every key (< 2^31) is a valid "vertex"
    a.ucap = S;
    a.max_batch_idx = S;
    a.hash_slots = std::max(pow2_at_least(2 * S), pow2_at_least(threads));
    uint32_t bits = 0;
    while ((1u << bits) < a.hash_slots) ++bits;
    a.hash_bits = bits;
    a.sort_n = pow2_at_least(S);
    a.probe_k = 4;
    a.err = reinterpret_cast<uint32_t*>(d->d_counters + 2);
    smem = walk_batched_smem(dedup, S, a.hash_slots, a.sort_n);
    const void* fn = dedup == DEDUP_SORT ? (const void*)walk_batched_kernel<DEDUP_SORT>
                     : dedup == DEDUP_HASH ? (const void*)walk_batched_kernel<DEDUP_HASH>
                                           : (const void*)walk_batched_kernel<DEDUP_PHASH>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return GP_ERR_UNSUPPORTED;
  }
  for (uint32_t k = 0; k < d->steps; ++k) {
    wa.step = d->first_step + k;
    wa.pin = (k & 1) ? d->d_scratch : d->d_pos;
    wa.pout = (k & 1) ? d->d_pos : d->d_scratch;
    if (v == GP_NAIVE) {
      walk_naive_kernel<<<(d->num_agents + 255) / 256, 256, 0, s>>>(wa);
    } else if (v == GP_WARP) {
      walk_warp_kernel<<<(d->num_agents + 255) / 256, 256, 0, s>>>(wa);
    } else {
      const uint32_t grid = (d->num_agents + S - 1) / S;
      if (dedup == DEDUP_SORT) walk_batched_kernel<DEDUP_SORT><<<grid, threads, smem, s>>>(wa, a);
      else if (dedup == DEDUP_HASH) walk_batched_kernel<DEDUP_HASH><<<grid, threads, smem, s>>>(wa, a);
      else walk_batched_kernel<DEDUP_PHASH><<<grid, threads, smem, s>>>(wa, a);
    }
    if (cudaGetLastError() != cudaSuccess) return GP_ERR_CUDA;
  }
  if (d->steps & 1) {  // the last step wrote the scratch buffer
    if (cudaMemcpyAsync(d->d_pos, d->d_scratch, (size_t)d->num_agents * 4, cudaMemcpyDeviceToDevice, s) !=
        cudaSuccess)
      return GP_ERR_CUDA;
  }
  return GP_OK;
}
