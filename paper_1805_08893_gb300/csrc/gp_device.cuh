// Device-side building blocks shared by the draw kernels: vertex fetch and
// the vertex shaders, bulk-copy (TMA) and mbarrier wrappers, block scans.
//
// The shaders use explicit fused multiply-adds and the file is compiled
// with --fmad=false, so every kernel that calls them produces bit-identical
// results for the same vertex (naive and reuse outputs compare exactly).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gp_internal.h"

namespace gp {

constexpr int kWarp = 32;
constexpr unsigned kFull = 0xFFFFFFFFu;

template <int SH>
struct ShaderTraits {
  static constexpr int K = (SH == 2) ? 8 : 7;         // floats per output corner
  static constexpr int KS = (SH == 2) ? 8 : 7;        // smem stride of a shaded vertex
  static constexpr bool kSkin = (SH == 1);
};

// ---------------------------------------------------------------------------
// vertex fetch + shade
// ---------------------------------------------------------------------------

struct VertexIn {
  float px, py, pz, nx, ny, nz;
  uint32_t bones;
  float w0, w1, w2, w3;
};

// 32 bytes from a 32-byte-aligned global address in one 256-bit load
// (read-only path).
__device__ __forceinline__ void ldg_v8(const void* p, float* r) {
  asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7])
               : "l"(p));
}

// Reads the attributes the shader needs.  vec8: the row is 32-byte aligned,
// so one 256-bit load per 32 bytes; otherwise 16-byte loads.
template <int SH>
__device__ __forceinline__ void fetch_vertex(const unsigned char* verts, uint32_t stride, uint32_t id,
                                             VertexIn& v, bool vec8 = false) {
  const unsigned char* row = verts + (size_t)id * stride;
  float r[16];
  if (vec8) {
    ldg_v8(row, r);
    if (ShaderTraits<SH>::kSkin) ldg_v8(row + 32, r + 8);
  } else {
    const float4* p = reinterpret_cast<const float4*>(row);
    float4 a = __ldg(p), b = __ldg(p + 1);
    r[0] = a.x; r[1] = a.y; r[2] = a.z; r[3] = a.w; r[4] = b.x; r[5] = b.y; r[6] = b.z; r[7] = b.w;
    if (ShaderTraits<SH>::kSkin) {
      float4 c = __ldg(p + 2), d = __ldg(p + 3);
      r[8] = c.x; r[9] = c.y; r[10] = c.z; r[11] = c.w; r[12] = d.x; r[13] = d.y; r[14] = d.z; r[15] = d.w;
    }
  }
  v.px = r[0]; v.py = r[1]; v.pz = r[2];
  v.nx = r[3]; v.ny = r[4]; v.nz = r[5];
  if (ShaderTraits<SH>::kSkin) {
    v.bones = __float_as_uint(r[8]);
    v.w0 = r[9]; v.w1 = r[10]; v.w2 = r[11]; v.w3 = r[12];
  } else {
    v.bones = 0; v.w0 = v.w1 = v.w2 = v.w3 = 0.f;
  }
}

// clip = M (p, 1), n' = N n
__device__ __forceinline__ void mvp_transform(const Uniforms& u, float px, float py, float pz, float nx,
                                              float ny, float nz, float* o) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
    o[i] = __fmaf_rn(u.mvp[4 * i + 0], px,
                     __fmaf_rn(u.mvp[4 * i + 1], py, __fmaf_rn(u.mvp[4 * i + 2], pz, u.mvp[4 * i + 3])));
#pragma unroll
  for (int i = 0; i < 3; ++i)
    o[4 + i] = __fmaf_rn(u.nrm[3 * i + 0], nx, __fmaf_rn(u.nrm[3 * i + 1], ny, __fmul_rn(u.nrm[3 * i + 2], nz)));
}

// Shades one vertex into o[0..K).  'palette' is the skinning palette in
// shared memory (64 x 12 floats) for SH == 1, unused otherwise.
template <int SH>
__device__ __forceinline__ void shade_vertex(const Uniforms& u, const float* palette, const VertexIn& v,
                                             float* o) {
  if (SH == 0) {
    mvp_transform(u, v.px, v.py, v.pz, v.nx, v.ny, v.nz, o);
  } else if (SH == 1) {
    float ps0 = 0.f, ps1 = 0.f, ps2 = 0.f, ns0 = 0.f, ns1 = 0.f, ns2 = 0.f;
    const float w[4] = {v.w0, v.w1, v.w2, v.w3};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float* B = palette + 12 * ((v.bones >> (8 * i)) & 0xFFu);
      float t0 = __fmaf_rn(B[0], v.px, __fmaf_rn(B[1], v.py, __fmaf_rn(B[2], v.pz, B[3])));
      float t1 = __fmaf_rn(B[4], v.px, __fmaf_rn(B[5], v.py, __fmaf_rn(B[6], v.pz, B[7])));
      float t2 = __fmaf_rn(B[8], v.px, __fmaf_rn(B[9], v.py, __fmaf_rn(B[10], v.pz, B[11])));
      float m0 = __fmaf_rn(B[0], v.nx, __fmaf_rn(B[1], v.ny, __fmul_rn(B[2], v.nz)));
      float m1 = __fmaf_rn(B[4], v.nx, __fmaf_rn(B[5], v.ny, __fmul_rn(B[6], v.nz)));
      float m2 = __fmaf_rn(B[8], v.nx, __fmaf_rn(B[9], v.ny, __fmul_rn(B[10], v.nz)));
      ps0 = __fmaf_rn(w[i], t0, ps0); ps1 = __fmaf_rn(w[i], t1, ps1); ps2 = __fmaf_rn(w[i], t2, ps2);
      ns0 = __fmaf_rn(w[i], m0, ns0); ns1 = __fmaf_rn(w[i], m1, ns1); ns2 = __fmaf_rn(w[i], m2, ns2);
    }
    mvp_transform(u, ps0, ps1, ps2, ns0, ns1, ns2, o);
  } else if (SH == 2) {
    // four directions' Horner chains at a time (independent, so their
    // latencies overlap); the terms are still summed in direction order
    float hsum = 0.f;
    uint32_t j = 0;
    for (; j + 4 <= u.num_dirs; j += 4) {
      float s[4], h[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float* dq = u.dirs + 3 * (j + q);
        s[q] = __fmul_rn(0.5f, __fmaf_rn(dq[0], v.px, __fmaf_rn(dq[1], v.py, __fmul_rn(dq[2], v.pz))));
        h[q] = u.coef[kEnvelopeTerms - 1];
      }
#pragma unroll
      for (int k = kEnvelopeTerms - 2; k >= 0; --k)
#pragma unroll
        for (int q = 0; q < 4; ++q) h[q] = __fmaf_rn(h[q], s[q], u.coef[k]);
#pragma unroll
      for (int q = 0; q < 4; ++q) hsum = __fadd_rn(hsum, h[q]);
    }
    for (; j < u.num_dirs; ++j) {
      float s = __fmul_rn(0.5f, __fmaf_rn(u.dirs[3 * j], v.px,
                                          __fmaf_rn(u.dirs[3 * j + 1], v.py, __fmul_rn(u.dirs[3 * j + 2], v.pz))));
      float h = u.coef[kEnvelopeTerms - 1];
#pragma unroll
      for (int k = kEnvelopeTerms - 2; k >= 0; --k) h = __fmaf_rn(h, s, u.coef[k]);
      hsum = __fadd_rn(hsum, h);
    }
    const float off = __fmul_rn(u.d, __fmul_rn(hsum, u.inv_dirs));
    o[0] = __fmaf_rn(-off, v.nx, v.px); o[1] = __fmaf_rn(-off, v.ny, v.py); o[2] = __fmaf_rn(-off, v.nz, v.pz);
    o[3] = 1.f;
    o[4] = __fmaf_rn(off, v.nx, v.px); o[5] = __fmaf_rn(off, v.ny, v.py); o[6] = __fmaf_rn(off, v.nz, v.pz);
    o[7] = 1.f;
  } else {
    mvp_transform(u, v.px, v.py, v.pz, v.nx, v.ny, v.nz, o);
    const float c = __fmaf_rn(1e-3f, v.px, 0.5f);
    float sig = 1.f;
    for (uint32_t k = 0; k < u.steps; ++k) sig = __fmaf_rn(sig, 0.5f, c);
    o[4] = __fmul_rn(o[4], sig); o[5] = __fmul_rn(o[5], sig); o[6] = __fmul_rn(o[6], sig);
  }
}

// Fetches and shades vertex 'id', or writes zeros and flags an index-range
// error when id >= num_verts.
template <int SH>
__device__ __forceinline__ void fetch_and_shade(const DrawArgs& a, const Uniforms& u, const float* palette,
                                                uint32_t id, float* o) {
  if (id < a.num_verts) {
    VertexIn v;
    fetch_vertex<SH>(a.verts, a.stride, id, v, a.vec8 != 0);
    shade_vertex<SH>(u, palette, v, o);
  } else {
#pragma unroll
    for (int k = 0; k < ShaderTraits<SH>::K; ++k) o[k] = 0.f;
    atomicOr(a.err, EBIT_INDEX_RANGE);
  }
}

// ---------------------------------------------------------------------------
// PTX wrappers: mbarrier, bulk copies (TMA, non-tensor), proxy fences
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

// Plain arrival (release semantics for this thread's earlier shared-memory
// writes).
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// The mbarrier's current phase cannot complete before this thread's earlier
// cp.async copies have landed (its pending count is raised now and lowered
// when they complete).
__device__ __forceinline__ void cp_async_mbar_arrive(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// As mbar_try_wait, but the thread sleeps until the phase completes or up
// to hint_ns nanoseconds have passed (it issues nothing meanwhile).
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, uint32_t parity, uint32_t hint_ns) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok != 0;
}

// Bounded wait: gives up after ~2^22 polls (each try_wait itself suspends
// for a hardware-defined interval), sets EBIT_TIMEOUT and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t* err) {
  for (uint32_t it = 0; it < (1u << 22); ++it)
    if (mbar_try_wait(bar, parity)) return true;
  atomicOr(err, EBIT_TIMEOUT);
  return false;
}

// global -> shared bulk copy completing on an mbarrier (16-byte aligned
// addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_load(void* dst_smem, const void* src_gmem, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// shared -> global bulk copy in a bulk async-group.
__device__ __forceinline__ void bulk_store(void* dst_gmem, const void* src_smem, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst_gmem),
               "r"(smem_addr(src_smem)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}

template <int N>
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group %0;" ::"n"(N) : "memory");
}

// Makes this thread's generic-proxy shared-memory writes visible to the
// async proxy (a following bulk store reads them).
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// global -> shared 16-byte asynchronous copy (L2 only), tracked per thread
// in cp.async groups; both addresses 16-byte aligned.
__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src_gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst_smem)), "l"(src_gmem) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

// Waits until at most N of this thread's most recent cp.async groups are pending.
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// ---------------------------------------------------------------------------
// scans
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t warp_inclusive_scan(uint32_t x) {
  const uint32_t lane = lane_id();
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(kFull, x, o);
    if (lane >= (uint32_t)o) x += y;
  }
  return x;
}

// Block-wide exclusive scan of one value per thread.  'warp_sums' holds
// >= blockDim.x/32 + 1 words of shared memory.  Returns the exclusive prefix;
// *total receives the block total.  Contains __syncthreads().
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t* warp_sums, uint32_t* total) {
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  uint32_t inc = warp_inclusive_scan(x);
  if (lane == 31) warp_sums[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint32_t s = lane < nwarps ? warp_sums[lane] : 0u;
    uint32_t si = warp_inclusive_scan(s);
    if (lane < nwarps) warp_sums[lane] = si - s;
    if (lane == 31) warp_sums[nwarps] = si;
  }
  __syncthreads();
  uint32_t r = warp_sums[warp] + inc - x;
  *total = warp_sums[nwarps];
  return r;
}

}  // namespace gp
