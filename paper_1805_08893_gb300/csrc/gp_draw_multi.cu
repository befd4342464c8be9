// Multi-kernel (non-streaming) geometry stage, the paper's comparator for
// the reuse methods (Section 5, "multi" in Table 2): one kernel shades every
// vertex of the vertex buffer exactly once into a buffer in global memory,
// a second kernel assembles each triangle's corners from it.  Every vertex
// is shaded once whether or not an index refers to it.
//
// GB300 layout: shaded vertices are 32-byte rows (K floats, zero-padded to
// 8), one aligned 32-byte sector each; the buffer of the 3.6M-vertex mesh
// (115 MB) fits in the 126 MB L2, so the assembly's random row reads mostly
// hit L2.  The assembly stages each warp's 32 triangles in shared memory and
// writes them with 16-byte streaming stores, like the naive kernel.
#include "gp_device.cuh"

namespace gp {

template <int SH>
__global__ void __launch_bounds__(256) shade_all_kernel(const __grid_constant__ DrawArgs a,
                                                        const __grid_constant__ Uniforms u, float4* rows) {
  constexpr int K = ShaderTraits<SH>::K;
  __shared__ float palette[ShaderTraits<SH>::kSkin ? 768 : 1];
  if (ShaderTraits<SH>::kSkin) {
    for (int i = threadIdx.x; i < 768; i += blockDim.x) palette[i] = u.palette[i];
    __syncthreads();
  }
  const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= a.num_verts) return;
  VertexIn in;
  fetch_vertex<SH>(a.verts, a.stride, v, in, a.vec8 != 0);
  float o[8];
  shade_vertex<SH>(u, palette, in, o);
#pragma unroll
  for (int c = K; c < 8; ++c) o[c] = 0.f;
  rows[2 * (size_t)v] = make_float4(o[0], o[1], o[2], o[3]);
  rows[2 * (size_t)v + 1] = make_float4(o[4], o[5], o[6], o[7]);
}

template <int SH>
__global__ void __launch_bounds__(256) assemble_kernel(const __grid_constant__ DrawArgs a,
                                                       const float4* __restrict__ rows) {
  constexpr int K = ShaderTraits<SH>::K;
  constexpr int F = 3 * K;
  extern __shared__ __align__(16) float stage_all[];
  const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
  // the whole draw is one "batch" whose invocations are all vertices
  if (a.batch_inv != nullptr && a.batch_cap > 0 && blockIdx.x == 0 && threadIdx.x == 0) a.batch_inv[0] = a.num_verts;
  float* stage = stage_all + warp * (32 * F);
  const uint32_t tw0 = blockIdx.x * blockDim.x + warp * 32;  // first triangle of the warp
  if (tw0 >= a.num_tris) return;                              // warp-uniform; no block barrier follows
  const uint32_t ntw = min(32u, a.num_tris - tw0);
  const uint32_t t = tw0 + lane;
  if (lane < ntw) {
    uint32_t id[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) id[k] = __ldg(a.idx + 3u * t + k);
    float4 r[6];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (id[k] < a.num_verts) {
        r[2 * k] = __ldg(rows + 2 * (size_t)id[k]);
        r[2 * k + 1] = __ldg(rows + 2 * (size_t)id[k] + 1);
      } else {
        r[2 * k] = r[2 * k + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    bool bad = false;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      bad |= id[k] >= a.num_verts;
      const float o[8] = {r[2 * k].x, r[2 * k].y, r[2 * k].z, r[2 * k].w,
                          r[2 * k + 1].x, r[2 * k + 1].y, r[2 * k + 1].z, r[2 * k + 1].w};
#pragma unroll
      for (int c = 0; c < K; ++c) stage[lane * F + k * K + c] = o[c];
      if (a.corner_ids != nullptr) a.corner_ids[3u * t + k] = id[k];
    }
    if (bad) atomicOr(a.err, EBIT_INDEX_RANGE);
  }
  __syncwarp();
  const uint32_t nfl = ntw * F;
  float* dst = a.out + (size_t)tw0 * F;
  const uint32_t n4 = nfl >> 2;
  float4* d4 = reinterpret_cast<float4*>(dst);
  const float4* s4 = reinterpret_cast<const float4*>(stage);
  for (uint32_t i = lane; i < n4; i += 32) __stcs(d4 + i, s4[i]);
  for (uint32_t i = (n4 << 2) + lane; i < nfl; i += 32) dst[i] = stage[i];
}

template <int SH>
static cudaError_t launch_multi_t(const DrawArgs& a, const Uniforms& u, float4* rows, int block, cudaStream_t s) {
  constexpr int F = 3 * ShaderTraits<SH>::K;
  if (a.num_verts) {
    shade_all_kernel<SH><<<(a.num_verts + 255) / 256, 256, 0, s>>>(a, u, rows);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const uint32_t grid = (a.num_tris + block - 1) / block;
  if (grid == 0) return cudaSuccess;
  assemble_kernel<SH><<<grid, block, (size_t)(block / 32) * 32 * F * 4, s>>>(a, rows);
  return cudaGetLastError();
}

cudaError_t launch_multi(const DrawArgs& a, const Uniforms& u, int shader, float4* rows, int block,
                         cudaStream_t s) {
  switch (shader) {
    case 0: return launch_multi_t<0>(a, u, rows, block, s);
    case 1: return launch_multi_t<1>(a, u, rows, block, s);
    case 2: return launch_multi_t<2>(a, u, rows, block, s);
    case 3: return launch_multi_t<3>(a, u, rows, block, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace gp
