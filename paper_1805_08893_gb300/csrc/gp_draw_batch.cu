// Single-draw kernels over the pipeline of gp_batch_pipeline.cuh: each block
// is persistent (grid = SMs x resident blocks) and runs the batches
// blockIdx.x, blockIdx.x + gridDim.x, ... of the draw.
#include "gp_batch_pipeline.cuh"

namespace gp {

template <int DEDUP, int SH, bool DYN>
__global__ void __launch_bounds__(512, 2) batched_kernel(const __grid_constant__ DrawArgs a,
                                                         const __grid_constant__ Uniforms u) {
  extern __shared__ __align__(128) unsigned char smem[];
  const BatchLayout L = batch_layout(DEDUP, ShaderTraits<SH>::K, ShaderTraits<SH>::K | 1, RawTraits<SH>::kBytes,
                                     ShaderTraits<SH>::kSkin, a.max_batch_idx, a.ucap, a.hash_slots, a.sort_n,
                                     a.out_chunk);
  const uint32_t nb = DYN ? *a.num_batches_dev : a.num_batches;
  if (blockIdx.x >= nb) return;
  const uint32_t tid = threadIdx.x;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.off_bars);
  float* palette = reinterpret_cast<float*>(smem + L.off_pal);
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
  }
  if (ShaderTraits<SH>::kSkin)
    for (uint32_t i = tid; i < 768; i += blockDim.x) palette[i] = u.palette[i];
  PipeBars pb{bars, 0u, 0u};
  unsigned long long inv_total = 0, nbatches = 0;
  pipeline_run<DEDUP, SH, DYN>(a, u, palette, smem, L, pb, blockIdx.x, gridDim.x, nb, inv_total, nbatches);
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
  (void)threads;
  const uint32_t K = shader == 2 ? 8 : 7;
  const uint32_t KV = K | 1u;
  const uint32_t RB = shader == 1 ? 64 : 32;
  const BatchLayout L = batch_layout(dedup, K, KV, RB, shader == 1, a.max_batch_idx, a.ucap, a.hash_slots, a.sort_n,
                                     a.out_chunk);
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
