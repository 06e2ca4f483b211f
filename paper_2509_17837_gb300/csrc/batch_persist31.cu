// Persistent multi-distance annealing kernel for distances up to 31.
#include "batch_anneal.cuh"

namespace xzzx {
namespace batch {

xzzx_status launch_persistent_31(const AnnealLaunch& L, int grid, cudaStream_t stream) {
  constexpr size_t smem = persistent_smem<31>();
  anneal_persistent_kernel<31><<<(unsigned)grid, kNT, smem, stream>>>(L);
  XZZX_CUDA_TRY(cudaGetLastError());
  return XZZX_OK;
}

xzzx_status configure_persistent_31() {
  constexpr size_t smem = persistent_smem<31>();
  XZZX_CUDA_TRY(
      cudaFuncSetAttribute(anneal_persistent_kernel<31>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  return XZZX_OK;
}

xzzx_status occupancy_persistent_31(int* ctas_per_sm) {
  constexpr size_t smem = persistent_smem<31>();
  XZZX_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, anneal_persistent_kernel<31>, kNT, smem));
  return XZZX_OK;
}

}  // namespace batch
}  // namespace xzzx
