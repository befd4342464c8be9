// Statically batched naive geometry stage (Section 3.3): one thread per
// triangle shades all three of its corners, with no communication about
// reuse.  This is the baseline the reuse methods are measured against.
//
// GB300 layout: each warp owns 32 consecutive triangles.  Shaded corners are
// staged in the warp's slice of shared memory and written back with 16-byte
// streaming stores, so the output (the dominant HBM traffic) is fully
// coalesced; 32 triangles of K-float corners always start on a 16-byte
// boundary (32 * 3 * K floats is a multiple of 4).
#include "gp_device.cuh"

namespace gp {

template <int SH>
__global__ void __launch_bounds__(256) naive_kernel(const __grid_constant__ DrawArgs a,
                                                    const __grid_constant__ Uniforms u) {
  constexpr int K = ShaderTraits<SH>::K;
  constexpr int F = 3 * K;
  extern __shared__ __align__(16) float smem_f[];
  float* palette = smem_f;
  float* stage_all = smem_f + (ShaderTraits<SH>::kSkin ? 768 : 0);
  if (ShaderTraits<SH>::kSkin) {
    for (int i = threadIdx.x; i < 768; i += blockDim.x) palette[i] = u.palette[i];
    __syncthreads();
  }
  const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
  float* stage = stage_all + warp * (32 * F);

  const uint32_t tb0 = blockIdx.x * blockDim.x;  // first triangle of the block
  if (a.batch_inv != nullptr && threadIdx.x == 0 && blockIdx.x < a.batch_cap) {
    const uint32_t nt = min((uint32_t)blockDim.x, a.num_tris - tb0);
    a.batch_inv[blockIdx.x] = 3u * nt;
  }
  const uint32_t tw0 = tb0 + warp * 32;  // first triangle of the warp
  if (tw0 >= a.num_tris) return;         // warp-uniform; no block barrier follows
  const uint32_t ntw = min(32u, a.num_tris - tw0);
  const uint32_t t = tw0 + lane;
  if (lane < ntw) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint32_t id = __ldg(a.idx + 3u * t + k);
      float o[K];
      fetch_and_shade<SH>(a, u, palette, id, o);
#pragma unroll
      for (int c = 0; c < K; ++c) stage[lane * F + k * K + c] = o[c];
      if (a.corner_ids != nullptr) a.corner_ids[3u * t + k] = id;
    }
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
static cudaError_t launch_naive_t(const DrawArgs& a, const Uniforms& u, int block, cudaStream_t s) {
  constexpr int F = 3 * ShaderTraits<SH>::K;
  const size_t smem = (ShaderTraits<SH>::kSkin ? 768 * 4 : 0) + (size_t)(block / 32) * 32 * F * 4;
  const uint32_t grid = (a.num_tris + block - 1) / block;
  if (grid == 0) return cudaSuccess;
  naive_kernel<SH><<<grid, block, smem, s>>>(a, u);
  return cudaGetLastError();
}

cudaError_t launch_naive(const DrawArgs& a, const Uniforms& u, int shader, int block, cudaStream_t s) {
  switch (shader) {
    case 0: return launch_naive_t<0>(a, u, block, s);
    case 1: return launch_naive_t<1>(a, u, block, s);
    case 2: return launch_naive_t<2>(a, u, block, s);
    case 3: return launch_naive_t<3>(a, u, block, s);
  }
  return cudaErrorInvalidValue;
}

int out_floats(int shader) { return shader == 2 ? 8 : 7; }

}  // namespace gp
