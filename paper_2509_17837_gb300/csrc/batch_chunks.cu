// Per-distance chunk kernels of the batch (the plain one-launch-per-distance form).
#include "batch_anneal.cuh"

namespace xzzx {
namespace batch {

template <int D>
static xzzx_status chunks_d(const AnnealLaunch& L, cudaStream_t stream) {
  constexpr size_t smem = core::smem_bytes<D, kNT>();
  if (L.n_chunks == 0) return XZZX_OK;
  anneal_chunks_kernel<D><<<(unsigned)L.n_chunks, kNT, smem, stream>>>(L);
  XZZX_CUDA_TRY(cudaGetLastError());
  return XZZX_OK;
}

template <int D>
static xzzx_status configure_chunks_d() {
  constexpr size_t smem = core::smem_bytes<D, kNT>();
  XZZX_CUDA_TRY(cudaFuncSetAttribute(anneal_chunks_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  return XZZX_OK;
}

template <int D>
static xzzx_status occupancy_chunks_d(int* ctas_per_sm) {
  constexpr size_t smem = core::smem_bytes<D, kNT>();
  XZZX_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, anneal_chunks_kernel<D>, kNT, smem));
  return XZZX_OK;
}

xzzx_status occupancy_chunks(int d, int* ctas_per_sm) {
  switch (d) {
#define XZZX_CASE(DD) \
  case DD:            \
    return occupancy_chunks_d<DD>(ctas_per_sm);
    XZZX_CASE(3) XZZX_CASE(5) XZZX_CASE(7) XZZX_CASE(9) XZZX_CASE(11) XZZX_CASE(13) XZZX_CASE(15)
    XZZX_CASE(17) XZZX_CASE(19) XZZX_CASE(21) XZZX_CASE(23) XZZX_CASE(25) XZZX_CASE(27) XZZX_CASE(29)
    XZZX_CASE(31)
#undef XZZX_CASE
    default:
      return fail(XZZX_EUNSUPPORTED, "no annealing kernel for this distance");
  }
}

xzzx_status launch_chunks(int d, const AnnealLaunch& L, cudaStream_t stream) {
  switch (d) {
#define XZZX_CASE(DD) \
  case DD:            \
    return chunks_d<DD>(L, stream);
    XZZX_CASE(3) XZZX_CASE(5) XZZX_CASE(7) XZZX_CASE(9) XZZX_CASE(11) XZZX_CASE(13) XZZX_CASE(15)
    XZZX_CASE(17) XZZX_CASE(19) XZZX_CASE(21) XZZX_CASE(23) XZZX_CASE(25) XZZX_CASE(27) XZZX_CASE(29)
    XZZX_CASE(31)
#undef XZZX_CASE
    default:
      return fail(XZZX_EUNSUPPORTED, "no annealing kernel for this distance");
  }
}

xzzx_status configure_chunk_kernels() {
  xzzx_status st;
#define XZZX_CFG(DD) \
  if ((st = configure_chunks_d<DD>())) return st;
  XZZX_CFG(3) XZZX_CFG(5) XZZX_CFG(7) XZZX_CFG(9) XZZX_CFG(11) XZZX_CFG(13) XZZX_CFG(15) XZZX_CFG(17) XZZX_CFG(19)
  XZZX_CFG(21) XZZX_CFG(23) XZZX_CFG(25) XZZX_CFG(27) XZZX_CFG(29) XZZX_CFG(31)
#undef XZZX_CFG
  return XZZX_OK;
}

}  // namespace batch
}  // namespace xzzx
