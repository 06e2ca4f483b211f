// Per-distance chunk kernels of the batch (the plain one-launch-per-distance
// form), for one (chains per CTA, sweep unroll) variant.  Each
// batch_chunks_nt*_u*.cu instantiates one variant, so the variants compile in
// parallel.
#pragma once

#include "batch_anneal.cuh"

namespace xzzx {
namespace batch {

template <int D, int NT, int U>
static xzzx_status chunks_d(const AnnealLaunch& L, cudaStream_t stream) {
  constexpr size_t smem = core::smem_bytes<D, NT>();
  if (L.n_chunks == 0) return XZZX_OK;
  chunks_kernel_of<D, NT, U>()<<<(unsigned)L.n_chunks, NT, smem, stream>>>(L);
  XZZX_CUDA_TRY(cudaGetLastError());
  return XZZX_OK;
}

template <int D, int NT, int U>
static xzzx_status configure_chunks_d() {
  constexpr size_t smem = core::smem_bytes<D, NT>();
  XZZX_CUDA_TRY(
      cudaFuncSetAttribute(chunks_kernel_of<D, NT, U>(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  return XZZX_OK;
}

template <int D, int NT, int U>
static xzzx_status occupancy_chunks_d(int* ctas_per_sm) {
  constexpr size_t smem = core::smem_bytes<D, NT>();
  XZZX_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, chunks_kernel_of<D, NT, U>(), NT, smem));
  return XZZX_OK;
}

#define XZZX_ALL_D(M) M(3) M(5) M(7) M(9) M(11) M(13) M(15) M(17) M(19) M(21) M(23) M(25) M(27) M(29) M(31)

template <int NT, int U>
xzzx_status occupancy_chunks_v(int d, int* ctas_per_sm) {
  switch (d) {
#define XZZX_CASE(DD) \
  case DD:            \
    return occupancy_chunks_d<DD, NT, U>(ctas_per_sm);
    XZZX_ALL_D(XZZX_CASE)
#undef XZZX_CASE
    default:
      return fail(XZZX_EUNSUPPORTED, "no annealing kernel for this distance");
  }
}

template <int NT, int U>
xzzx_status launch_chunks_v(int d, const AnnealLaunch& L, cudaStream_t stream) {
  switch (d) {
#define XZZX_CASE(DD) \
  case DD:            \
    return chunks_d<DD, NT, U>(L, stream);
    XZZX_ALL_D(XZZX_CASE)
#undef XZZX_CASE
    default:
      return fail(XZZX_EUNSUPPORTED, "no annealing kernel for this distance");
  }
}

template <int NT, int U>
xzzx_status configure_chunks_v() {
  xzzx_status st;
#define XZZX_CFG(DD) \
  if ((st = configure_chunks_d<DD, NT, U>())) return st;
  XZZX_ALL_D(XZZX_CFG)
#undef XZZX_CFG
  return XZZX_OK;
}

#undef XZZX_ALL_D

// Explicit instantiation of one variant.
#define XZZX_CHUNK_VARIANT(NT, U)                                                                      \
  template xzzx_status occupancy_chunks_v<NT, U>(int, int*);                                          \
  template xzzx_status launch_chunks_v<NT, U>(int, const AnnealLaunch&, cudaStream_t);                \
  template xzzx_status configure_chunks_v<NT, U>();

}  // namespace batch
}  // namespace xzzx
