// Loop subdivision with on-the-fly reuse (Section 5.2): one subdivision step
// of a triangle mesh, streamed triangle by triangle.  Each input triangle
// (v0, v1, v2) yields four output triangles
//   (E0, M0, M2), (E1, M1, M0), (E2, M2, M1), (M0, M1, M2)
// where E_k is vertex k moved by Loop's vertex rule (its 1-ring, weight beta
// of Loop's thesis; boundary vertices: 3/4 v + 1/8 of their two boundary
// neighbours) and M_k is the new vertex on edge (v_k, v_k+1) (3/8 of the
// edge's ends plus 1/8 of the two opposite vertices; boundary edges: the
// midpoint).  The vertex rule reads a whole 1-ring, so it is the "vertex
// shader" the reuse methods share:
//   naive            -- every triangle evaluates its three vertices itself;
//   warp             -- Algorithm 1's rounds on static batches, one warp per
//                       batch: the lanes holding a round's vertices evaluate
//                       the rule, the round's triangles gather it by shuffles;
//   sort/hash/phash  -- one thread block per batch (static, or the dynamic
//                       batches of the partition) runs the shared dedup body;
//                       each unique vertex's rule is evaluated once into
//                       shared memory together with its position, then one
//                       thread per triangle builds the edge vertices and
//                       writes the four triangles.
// Output: 4 triangles x 3 corners x 3 floats = 144 bytes (9 aligned 16-byte
// words) per input triangle, in input order.
#include <algorithm>

#include "gp.h"
#include "gp_batch_body.cuh"
#include "gp_warp_body.cuh"

namespace gp {

struct LoopArgs {
  const uint32_t* idx;
  uint32_t num_tris;
  const unsigned char* verts;
  uint32_t stride, num_verts;
  const uint32_t* ring_off;
  const uint32_t* ring;
  uint32_t ring_count;
  const uint32_t* vflags;
  const uint32_t* opp;
  float* out;
  const uint32_t* starts;         // dynamic batches (triangles), or nullptr for static
  uint32_t static_tris;           // static: triangles per batch
  uint32_t num_batches;           // static
  const uint32_t* num_batches_dev;  // dynamic
  unsigned long long* counters;   // [0] vertex-rule evaluations, [1] batches, [2] error bits
};

// Position of vertex v; an id out of range (a bad index or adjacency entry)
// reads as the origin and flags GP_ERR_INDEX_RANGE.
__device__ __forceinline__ float3 loop_pos(const LoopArgs& a, uint32_t v) {
  if (v >= a.num_verts) {
    atomicOr(a.counters + 2, (unsigned long long)EBIT_INDEX_RANGE);
    return make_float3(0.f, 0.f, 0.f);
  }
  const float* p = reinterpret_cast<const float*>(a.verts + (size_t)v * a.stride);
  return make_float3(__ldg(p), __ldg(p + 1), __ldg(p + 2));
}

// Loop's vertex rule for vertex v.
__device__ __forceinline__ float3 loop_even(const LoopArgs& a, uint32_t v) {
  const float3 p = loop_pos(a, v);
  if (v >= a.num_verts) return p;
  // ring entries past the ring array (inconsistent adjacency) are not read
  const uint32_t o0 = min(__ldg(a.ring_off + v), a.ring_count);
  const uint32_t o1 = max(o0, min(__ldg(a.ring_off + v + 1), a.ring_count));
  if ((__ldg(a.vflags + v) & 1u) && o1 - o0 >= 2) {
    const float3 b0 = loop_pos(a, __ldg(a.ring + o0)), b1 = loop_pos(a, __ldg(a.ring + o0 + 1));
    return make_float3(__fmaf_rn(0.75f, p.x, __fmul_rn(0.125f, __fadd_rn(b0.x, b1.x))),
                       __fmaf_rn(0.75f, p.y, __fmul_rn(0.125f, __fadd_rn(b0.y, b1.y))),
                       __fmaf_rn(0.75f, p.z, __fmul_rn(0.125f, __fadd_rn(b0.z, b1.z))));
  }
  const uint32_t n = o1 - o0;
  if (n == 0) return p;
  float sx = 0.f, sy = 0.f, sz = 0.f;
  for (uint32_t k = o0; k < o1; ++k) {
    const float3 q = loop_pos(a, __ldg(a.ring + k));
    sx = __fadd_rn(sx, q.x);
    sy = __fadd_rn(sy, q.y);
    sz = __fadd_rn(sz, q.z);
  }
  const float c = __fmaf_rn(0.25f, cosf(6.283185307179586f / (float)n), 0.375f);
  const float beta = __fdiv_rn(__fmaf_rn(-c, c, 0.625f), (float)n);
  const float w = __fmaf_rn(-(float)n, beta, 1.0f);
  return make_float3(__fmaf_rn(w, p.x, __fmul_rn(beta, sx)), __fmaf_rn(w, p.y, __fmul_rn(beta, sy)),
                     __fmaf_rn(w, p.z, __fmul_rn(beta, sz)));
}

// Loop's edge rule for edge (pa, pb) with opposite vertices pc (this
// triangle) and d (the neighbour; kEmpty on a boundary).
__device__ __forceinline__ float3 loop_odd(const LoopArgs& a, float3 pa, float3 pb, float3 pc, uint32_t d) {
  if (d == kEmpty)
    return make_float3(__fmul_rn(0.5f, __fadd_rn(pa.x, pb.x)), __fmul_rn(0.5f, __fadd_rn(pa.y, pb.y)),
                       __fmul_rn(0.5f, __fadd_rn(pa.z, pb.z)));
  const float3 pd = loop_pos(a, d);
  return make_float3(__fmaf_rn(0.375f, __fadd_rn(pa.x, pb.x), __fmul_rn(0.125f, __fadd_rn(pc.x, pd.x))),
                     __fmaf_rn(0.375f, __fadd_rn(pa.y, pb.y), __fmul_rn(0.125f, __fadd_rn(pc.y, pd.y))),
                     __fmaf_rn(0.375f, __fadd_rn(pa.z, pb.z), __fmul_rn(0.125f, __fadd_rn(pc.z, pd.z))));
}

// Writes triangle t's four output triangles from its moved vertices E and
// positions P (corner order).
__device__ __forceinline__ void loop_emit(const LoopArgs& a, uint32_t t, const float3* E, const float3* P) {
  float3 M[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) M[k] = loop_odd(a, P[k], P[(k + 1) % 3], P[(k + 2) % 3], __ldg(a.opp + 3 * t + k));
  const float3 c[12] = {E[0], M[0], M[2], E[1], M[1], M[0], E[2], M[2], M[1], M[0], M[1], M[2]};
  const float f[36] = {c[0].x, c[0].y, c[0].z, c[1].x, c[1].y, c[1].z, c[2].x, c[2].y, c[2].z,
                       c[3].x, c[3].y, c[3].z, c[4].x, c[4].y, c[4].z, c[5].x, c[5].y, c[5].z,
                       c[6].x, c[6].y, c[6].z, c[7].x, c[7].y, c[7].z, c[8].x, c[8].y, c[8].z,
                       c[9].x, c[9].y, c[9].z, c[10].x, c[10].y, c[10].z, c[11].x, c[11].y, c[11].z};
  float4* o = reinterpret_cast<float4*>(a.out + (size_t)t * 36);
#pragma unroll
  for (int w = 0; w < 9; ++w) __stcs(o + w, make_float4(f[4 * w], f[4 * w + 1], f[4 * w + 2], f[4 * w + 3]));
}

__global__ void __launch_bounds__(256) loop_naive_kernel(const __grid_constant__ LoopArgs a) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (threadIdx.x == 0) {
    atomicAdd(a.counters + 0, 3ull * min(blockDim.x, a.num_tris - blockIdx.x * blockDim.x));
    atomicAdd(a.counters + 1, 1ull);
  }
  if (t >= a.num_tris) return;
  float3 E[3], P[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const uint32_t v = __ldg(a.idx + 3 * t + k);
    E[k] = loop_even(a, v);
    P[k] = loop_pos(a, v);
  }
  loop_emit(a, t, E, P);
}

// Evaluates the vertex rule of the warp's new ranks into shared memory.
struct LoopEven {
  const LoopArgs& la;
  const uint32_t* uniq;
  float* esh;  // rank -> moved position (3 floats)
  float* psh;  // rank -> position (3 floats)
  uint32_t ucap;
  __device__ __forceinline__ void operator()(uint32_t rb, uint32_t re, uint32_t lane) const {
    re = min(re, ucap);  // ranks >= ucap (a flagged capacity error) were not stored
    for (uint32_t r = rb + lane; r < re; r += 32) {
      const uint32_t v = uniq[r];
      const float3 e = loop_even(la, v), p = loop_pos(la, v);
      esh[3 * r] = e.x; esh[3 * r + 1] = e.y; esh[3 * r + 2] = e.z;
      psh[3 * r] = p.x; psh[3 * r + 1] = p.y; psh[3 * r + 2] = p.z;
    }
  }
};

template <int DEDUP>
__global__ void __launch_bounds__(512) loop_batched_kernel(const __grid_constant__ LoopArgs la,
                                                           const __grid_constant__ DrawArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t b = blockIdx.x, tid = threadIdx.x, NT = blockDim.x;
  const uint32_t nb = la.starts ? *la.num_batches_dev : la.num_batches;
  if (b >= nb) return;
  uint32_t t0, t1;
  if (la.starts) {
    t0 = __ldg(la.starts + b);
    t1 = __ldg(la.starts + b + 1);
  } else {
    t0 = b * la.static_tris;
    t1 = min(t0 + la.static_tris, la.num_tris);
  }
  const uint32_t n = 3 * (t1 - t0), cap = a.max_batch_idx, ucap = a.ucap;
  if (n > cap) {  // cannot happen with a consistent partition
    if (tid == 0) atomicOr(a.err, EBIT_CAPACITY);
    return;
  }
  uint32_t* win = reinterpret_cast<uint32_t*>(smem);
  uint16_t* map = reinterpret_cast<uint16_t*>(win + cap);
  uint32_t* uniq = reinterpret_cast<uint32_t*>(map + ((cap + 1) & ~1u));
  float* esh = reinterpret_cast<float*>(uniq + ucap);
  float* psh = esh + 3 * ucap;
  unsigned char* tail = reinterpret_cast<unsigned char*>(psh + 3 * ucap);
  tail = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tail) + 15) & ~(uintptr_t)15);
  BatchSmem B;
  B.map = map;
  B.uniq = uniq;
  B.vsh = nullptr;
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
  for (uint32_t i = tid; i < n; i += NT) win[i] = __ldg(la.idx + 3 * t0 + i);
  if (DEDUP != DEDUP_SORT)
    for (uint32_t s = tid; s < a.hash_slots; s += NT) B.table[s] = kEmpty;
  if (tid == 0) *B.ucount = 0;
  __syncthreads();
  dedup<DEDUP, true>(a, B, win, n, tid, NT, BlockSync(), LoopEven{la, uniq, esh, psh, ucap});
  __syncthreads();
  const uint32_t U = min(*B.ucount, ucap);
  for (uint32_t j = tid; j < t1 - t0; j += NT) {
    float3 E[3], P[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint32_t r = map[3 * j + k];
      if (DEDUP != DEDUP_SORT) r = B.dense[r];
      r = r < U ? r : 0u;  // only after a flagged capacity or index-range error
      E[k] = make_float3(esh[3 * r], esh[3 * r + 1], esh[3 * r + 2]);
      P[k] = make_float3(psh[3 * r], psh[3 * r + 1], psh[3 * r + 2]);
    }
    loop_emit(la, t0 + j, E, P);
  }
  if (tid == 0) {
    atomicAdd(la.counters + 0, (unsigned long long)U);
    atomicAdd(la.counters + 1, 1ull);
  }
}

// Algorithm 1 per warp: per-warp shared memory held[32] | ids[S] | map[S].
__host__ __device__ inline uint32_t loop_warp_bytes(uint32_t S) { return 128 + ((S + 3) & ~3u) * 4 + ((S + 15) & ~15u); }

__global__ void __launch_bounds__(256) loop_warp_kernel(const __grid_constant__ LoopArgs la, uint32_t S,
                                                        uint32_t nbatches) {
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  unsigned char* wp = smem + warp * loop_warp_bytes(S);
  uint32_t* held = reinterpret_cast<uint32_t*>(wp);
  uint32_t* widx = held + 32;
  unsigned char* map = reinterpret_cast<unsigned char*>(widx + ((S + 3) & ~3u));
  unsigned long long inv = 0, nb = 0;
  for (uint32_t b = blockIdx.x * wpb + warp; b < nbatches; b += gridDim.x * wpb) {
    const uint32_t B0 = b * S, n = min(B0 + S, 3 * la.num_tris) - B0;
    for (uint32_t i = lane; i < n; i += 32) {
      const uint32_t id = __ldg(la.idx + B0 + i);
      widx[i] = id < la.num_verts ? id : kInvalidId;
    }
    __syncwarp();
    for (uint32_t c = 0; c < n;) {
      uint32_t fill, done;
      warp_vote_round(widx, n, c, held, map, lane, fill, done);
      const uint32_t tris = done / 3;
      if (tris == 0) {  // cannot happen: a round's first chunk always places its lanes
        if (lane == 0) atomicOr(la.counters + 2, (unsigned long long)EBIT_CAPACITY);
        break;
      }
      float3 E = make_float3(0.f, 0.f, 0.f), P = E;
      if (lane < fill) {
        E = loop_even(la, held[lane]);
        P = loop_pos(la, held[lane]);
      }
      inv += fill;
      const uint32_t tfirst = (B0 + c) / 3;
      for (uint32_t p = 0; p < tris; p += 32) {
        const uint32_t j = p + lane;
        const bool live = j < tris;
        float3 Ec[3], Pc[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const uint32_t sl = live ? map[3 * j + k] : 0u;
          Ec[k] = make_float3(__shfl_sync(kFull, E.x, sl), __shfl_sync(kFull, E.y, sl), __shfl_sync(kFull, E.z, sl));
          Pc[k] = make_float3(__shfl_sync(kFull, P.x, sl), __shfl_sync(kFull, P.y, sl), __shfl_sync(kFull, P.z, sl));
        }
        if (live) loop_emit(la, tfirst + j, Ec, Pc);
      }
      __syncwarp();  // the next round overwrites held/map
      c += 3 * tris;
    }
    ++nb;
  }
  if (lane == 0 && nb) {
    atomicAdd(la.counters + 0, inv);
    atomicAdd(la.counters + 1, nb);
  }
}

size_t loop_batched_smem(int dedup, uint32_t cap, uint32_t ucap, uint32_t slots, uint32_t sort_n) {
  size_t o = (size_t)cap * 4 + (size_t)((cap + 1) & ~1u) * 2 + (size_t)ucap * 4 + (size_t)ucap * 24;
  o = (o + 15) & ~(size_t)15;
  o += dedup == DEDUP_SORT ? (size_t)sort_n * 8 : (size_t)slots * 6;
  return o + 64 * 4;
}

}  // namespace gp

using namespace gp;

namespace {
uint32_t loop_pow2(uint32_t x) {
  uint32_t p = 1;
  while (p < x) p <<= 1;
  return p;
}
}  // namespace

extern "C" gp_status gp_loop_subdivide(const gp_loop_desc* d) {
  // Section 5.2; see include/gp.h
  if (!d || !d->d_counters) return GP_ERR_INVALID;
  const int32_t v = d->variant;
  if (v != GP_NAIVE && v != GP_WARP && v != GP_SORT && v != GP_HASH && v != GP_PHASH) return GP_ERR_INVALID;
  if (d->num_indices % 3) return GP_ERR_INVALID;
  const uint32_t T = (uint32_t)(d->num_indices / 3);
  if (d->num_indices >= 0xFFFFFFF0ull) return GP_ERR_INVALID;
  if (T && (!d->d_indices || !d->d_vertices || !d->d_ring_offsets || !d->d_vertex_flags || !d->d_opposite ||
            !d->d_out))
    return GP_ERR_INVALID;
  if (reinterpret_cast<uintptr_t>(d->d_out) % 16 || d->stride_bytes < 12 || d->stride_bytes % 4)
    return GP_ERR_INVALID;
  const bool dyn = d->d_starts != nullptr;
  if ((v == GP_NAIVE || v == GP_WARP) && dyn) return GP_ERR_INVALID;
  if (dyn && (!d->d_num_batches || d->max_batch_indices == 0 || d->max_batch_indices % 3 || d->max_batches == 0))
    return GP_ERR_INVALID;
  const uint32_t S = dyn ? d->max_batch_indices : (d->batch_indices ? d->batch_indices : (v == GP_WARP ? 96 : 768));
  if (S % 3 || S > 4095 || (v == GP_WARP && S > kWarpMaxBatch)) return GP_ERR_INVALID;
  const uint32_t threads = d->threads ? d->threads : (v == GP_WARP ? 64 : 256);
  if (v == GP_WARP && (threads % 32 || threads > 256)) return GP_ERR_INVALID;
  if (v != GP_NAIVE && v != GP_WARP && (threads % 32 || (threads & (threads - 1)) || threads > 512))
    return GP_ERR_INVALID;
  if (T == 0) return GP_OK;
  cudaStream_t s = static_cast<cudaStream_t>(d->stream);
  LoopArgs la{};
  la.idx = d->d_indices;
  la.num_tris = T;
  la.verts = static_cast<const unsigned char*>(d->d_vertices);
  la.stride = d->stride_bytes;
  la.num_verts = (uint32_t)d->num_vertices;
  la.ring_off = d->d_ring_offsets;
  la.ring = d->d_ring;
  la.ring_count = (uint32_t)std::min<uint64_t>(d->ring_count, 0xFFFFFFFFu);
  la.vflags = d->d_vertex_flags;
  la.opp = d->d_opposite;
  la.out = d->d_out;
  la.counters = d->d_counters;
  if (v == GP_NAIVE) {
    loop_naive_kernel<<<(T + 255) / 256, 256, 0, s>>>(la);
    return cudaGetLastError() == cudaSuccess ? GP_OK : GP_ERR_CUDA;
  }
  if (v == GP_WARP) {
    const uint32_t nbatches = (3 * T + S - 1) / S, wpb = threads / 32;
    const size_t smem = (size_t)wpb * loop_warp_bytes(S);
    loop_warp_kernel<<<(nbatches + wpb - 1) / wpb, threads, smem, s>>>(la, S, nbatches);
    return cudaGetLastError() == cudaSuccess ? GP_OK : GP_ERR_CUDA;
  }
  DrawArgs a{};
  const int dedup = v == GP_SORT ? DEDUP_SORT : (v == GP_HASH ? DEDUP_HASH : DEDUP_PHASH);
  const uint32_t ucap = dyn ? std::min(d->max_unique ? d->max_unique : S, S) : S;
  a.num_verts = la.num_verts;
  a.ucap = ucap;
  a.max_batch_idx = S;
  a.hash_slots = std::max(loop_pow2(2 * ucap), loop_pow2(threads));
  uint32_t bits = 0;
  while ((1u << bits) < a.hash_slots) ++bits;
  a.hash_bits = bits;
  a.sort_n = loop_pow2(S);
  a.probe_k = 4;
  a.err = reinterpret_cast<uint32_t*>(d->d_counters + 2);
  uint32_t grid;
  if (dyn) {
    la.starts = d->d_starts;
    la.num_batches_dev = d->d_num_batches;
    grid = d->max_batches;  // blocks past the device count return at once
  } else {
    la.static_tris = S / 3;
    la.num_batches = (T + la.static_tris - 1) / la.static_tris;
    grid = la.num_batches;
  }
  const size_t smem = loop_batched_smem(dedup, S, ucap, a.hash_slots, a.sort_n);
  const void* fn = dedup == DEDUP_SORT ? (const void*)loop_batched_kernel<DEDUP_SORT>
                   : dedup == DEDUP_HASH ? (const void*)loop_batched_kernel<DEDUP_HASH>
                                         : (const void*)loop_batched_kernel<DEDUP_PHASH>;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return GP_ERR_UNSUPPORTED;
  if (dedup == DEDUP_SORT) loop_batched_kernel<DEDUP_SORT><<<grid, threads, smem, s>>>(la, a);
  else if (dedup == DEDUP_HASH) loop_batched_kernel<DEDUP_HASH><<<grid, threads, smem, s>>>(la, a);
  else loop_batched_kernel<DEDUP_PHASH><<<grid, threads, smem, s>>>(la, a);
  return cudaGetLastError() == cudaSuccess ? GP_OK : GP_ERR_CUDA;
}
