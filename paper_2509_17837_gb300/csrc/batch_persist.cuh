// Persistent multi-distance annealing kernel of the batch for distances up to
// DMAX, one (chains per CTA, sweep unroll) variant.  Each batch_persist*.cu
// instantiates some of the variants, so they compile in parallel.
#pragma once

#include "batch_anneal.cuh"

namespace xzzx {
namespace batch {

template <int DMAX, int NT, int U>
xzzx_status launch_persistent_v(const AnnealLaunch& L, int grid, cudaStream_t stream) {
  constexpr size_t smem = persistent_smem<DMAX, NT>();
  persistent_kernel_of<DMAX, NT, U>()<<<(unsigned)grid, NT, smem, stream>>>(L);
  XZZX_CUDA_TRY(cudaGetLastError());
  return XZZX_OK;
}

template <int DMAX, int NT, int U>
xzzx_status configure_persistent_v(int* ctas_per_sm) {
  constexpr size_t smem = persistent_smem<DMAX, NT>();
  XZZX_CUDA_TRY(cudaFuncSetAttribute(persistent_kernel_of<DMAX, NT, U>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
  XZZX_CUDA_TRY(
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, persistent_kernel_of<DMAX, NT, U>(), NT, smem));
  return XZZX_OK;
}

#define XZZX_PERSIST_VARIANT(DMAX, NT, U)                                                             \
  template xzzx_status launch_persistent_v<DMAX, NT, U>(const AnnealLaunch&, int, cudaStream_t);     \
  template xzzx_status configure_persistent_v<DMAX, NT, U>(int*);

}  // namespace batch
}  // namespace xzzx
