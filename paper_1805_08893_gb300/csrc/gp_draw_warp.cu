// Statically batched warp voting (Algorithm 1, Section 3.3): one warp per
// static batch, persistent warps walking the batches with a grid stride.  The
// per-batch work is warp_vote_batch (gp_warp_body.cuh).
#include "gp_warp_body.cuh"

namespace gp {

template <int SH>
__global__ void __launch_bounds__(256) warp_kernel(const __grid_constant__ DrawArgs a,
                                                   const __grid_constant__ Uniforms u) {
  using L = WarpSmem<SH>;
  constexpr int K = L::K;
  constexpr int F = L::F;
  extern __shared__ __align__(16) unsigned char smem[];
  float* palette = reinterpret_cast<float*>(smem);
  unsigned char* wbase = smem + (ShaderTraits<SH>::kSkin ? 768 * 4 : 0);
  if (ShaderTraits<SH>::kSkin) {
    for (int i = threadIdx.x; i < 768; i += blockDim.x) palette[i] = u.palette[i];
    __syncthreads();
  }
  const uint32_t S = 3u * a.static_batch_tris;
  const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
  unsigned char* wp = wbase + warp * L::per_warp_bytes(S);

  const uint32_t warps_total = gridDim.x * (blockDim.x >> 5);
  unsigned long long inv_total = 0, batches = 0;
  for (uint32_t b = blockIdx.x * (blockDim.x >> 5) + warp; b < a.num_batches; b += warps_total) {
    const uint32_t inv = warp_vote_batch<SH>(a, u, palette, b, wp, lane);
    if (lane == 0 && a.batch_inv != nullptr && b < a.batch_cap) a.batch_inv[b] = inv;
    inv_total += inv;
    batches += 1;
    __syncwarp();
  }
  if (lane == 0 && batches) {
    atomicAdd(a.counters + CNT_INVOCATIONS, inv_total);
    atomicAdd(a.counters + CNT_BATCHES, batches);
  }
}

size_t warp_kernel_smem(int shader, int warps_per_block, uint32_t batch_idx) {
  uint32_t per;
  switch (shader) {
    case 0: per = WarpSmem<0>::per_warp_bytes(batch_idx); break;
    case 1: per = WarpSmem<1>::per_warp_bytes(batch_idx); break;
    case 2: per = WarpSmem<2>::per_warp_bytes(batch_idx); break;
    default: per = WarpSmem<3>::per_warp_bytes(batch_idx); break;
  }
  return (shader == 1 ? 768 * 4 : 0) + (size_t)warps_per_block * per;
}

template <int SH>
static const void* warp_fn() {
  return reinterpret_cast<const void*>(&warp_kernel<SH>);
}

static const void* warp_kernel_ptr(int shader) {
  switch (shader) {
    case 0: return warp_fn<0>();
    case 1: return warp_fn<1>();
    case 2: return warp_fn<2>();
    default: return warp_fn<3>();
  }
}

int warp_kernel_blocks_per_sm(int shader, int warps_per_block) {
  const void* fn = warp_kernel_ptr(shader);
  const size_t smem = warp_kernel_smem(shader, warps_per_block, 96);
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, warps_per_block * 32, smem) != cudaSuccess) return 1;
  return nb > 0 ? nb : 1;
}

cudaError_t launch_warp(const DrawArgs& a, const Uniforms& u, int shader, int warps_per_block, int grid,
                        cudaStream_t s) {
  if (3u * a.static_batch_tris > kWarpMaxBatch) return cudaErrorInvalidValue;
  if (a.num_batches == 0) return cudaSuccess;
  const size_t smem = warp_kernel_smem(shader, warps_per_block, 3u * a.static_batch_tris);
  const void* fn = warp_kernel_ptr(shader);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int threads = warps_per_block * 32;
  switch (shader) {
    case 0: warp_kernel<0><<<grid, threads, smem, s>>>(a, u); break;
    case 1: warp_kernel<1><<<grid, threads, smem, s>>>(a, u); break;
    case 2: warp_kernel<2><<<grid, threads, smem, s>>>(a, u); break;
    default: warp_kernel<3><<<grid, threads, smem, s>>>(a, u); break;
  }
  return cudaGetLastError();
}

}  // namespace gp
