// Batched annealing kernels: a chunk of NT chains of one segment per CTA.
//
// anneal_chunks_kernel<D, NT, U>: one CTA per chunk of distance D (the plain,
// one-launch-per-distance form).  anneal_persistent_kernel<DMAX, NT, U>: a
// grid sized to the GPU whose CTAs pull chunk indices from a global atomic
// counter and run each chunk with the distance-templated core, so distances
// up to DMAX share one launch.  NT (chains per CTA) and U (sweep-loop unroll)
// are tuning knobs.  Every form calls core::anneal_cta with the same chain ids
// as xzzx_anneal, so results are identical to per-segment calls.
#pragma once

#include "anneal_core.cuh"
#include "batch_internal.h"

namespace xzzx {
namespace batch {

template <int D, int NT, int U>
__device__ __forceinline__ void run_chunk(const ChunkDev& ch, const SegDev& sg, const PhiloxKeys& K, uint8_t* smem) {
  constexpr int W = core::Shape<D>::kW;
  const int tid = threadIdx.x;
  const bool active = tid < ch.n_chains;
  const int64_t c = (int64_t)ch.first_chain + (active ? tid : ch.n_chains - 1);  // chain index in the segment
  const uint64_t chain = sg.shot0 * (uint64_t)sg.restarts * 4u + (uint64_t)c;
  core::SweepTables tab;
  tab.T = ch.T;
  tab.sig = ch.sig;
  tab.n_sweeps = ch.n_sweeps;
  tab.n_classes = ch.n_classes;
  for (int k = 0; k < 4; ++k) tab.W[k] = ch.W[k];
  tab.err = sg.code.err;
  core::ChainOut out;
  out.best_E = sg.chain_E + c;
  out.best_cfg = nullptr;
  out.final_E = nullptr;
  out.final_cfg = nullptr;
  core::anneal_cta<D, NT, U>(sg.init + (size_t)(c >> 2) * 2 * W, chain, (int)(c & 3), active, out, tab, K, smem);
}

// Register bounds: kernels on the pair path (d <= 15) are held to 1024
// threads per SM (64 registers); kernels on the row path keep the compiler's
// choice for their CTA size.
template <int D, int NT, int U>
__global__ void __launch_bounds__(NT, (1024 / NT)) anneal_chunks_kernel(const __grid_constant__ AnnealLaunch L) {
  extern __shared__ __align__(16) uint8_t smem[];
  const ChunkDev ch = L.chunks[L.chunk0 + blockIdx.x];
  run_chunk<D, NT, U>(ch, L.segs[ch.seg], L.keys, smem);
}
template <int D, int NT, int U>
__global__ void __launch_bounds__(NT) anneal_chunks_kernel_rows(const __grid_constant__ AnnealLaunch L) {
  extern __shared__ __align__(16) uint8_t smem[];
  const ChunkDev ch = L.chunks[L.chunk0 + blockIdx.x];
  run_chunk<D, NT, U>(ch, L.segs[ch.seg], L.keys, smem);
}
template <int D, int NT, int U>
constexpr auto chunks_kernel_of() {
  if constexpr (D <= core::kPairMaxD) return &anneal_chunks_kernel<D, NT, U>;
  else return &anneal_chunks_kernel_rows<D, NT, U>;
}

template <int D, int DMAX, int NT, int U>
__device__ __forceinline__ void dispatch_chunk(const ChunkDev& ch, const SegDev& sg, const PhiloxKeys& K,
                                               uint8_t* smem) {
  if constexpr (D <= DMAX) {
    if (ch.d == D) {
      run_chunk<D, NT, U>(ch, sg, K, smem);
      return;
    }
    dispatch_chunk<D + 2, DMAX, NT, U>(ch, sg, K, smem);
  }
}

template <int DMAX, int NT, int U>
__device__ __forceinline__ void persistent_body(const AnnealLaunch& L) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ int s_next;
  for (;;) {
    if (threadIdx.x == 0) s_next = atomicAdd(L.head, 1);
    __syncthreads();
    const int k = s_next;
    __syncthreads();
    if (k >= L.n_chunks) break;
    const ChunkDev ch = L.chunks[L.chunk0 + k];
    dispatch_chunk<3, DMAX, NT, U>(ch, L.segs[ch.seg], L.keys, smem);
  }
}
template <int DMAX, int NT, int U>
__global__ void __launch_bounds__(NT, (1024 / NT)) anneal_persistent_kernel(const __grid_constant__ AnnealLaunch L) {
  persistent_body<DMAX, NT, U>(L);
}
template <int DMAX, int NT, int U>
__global__ void __launch_bounds__(NT) anneal_persistent_kernel_rows(const __grid_constant__ AnnealLaunch L) {
  persistent_body<DMAX, NT, U>(L);
}
template <int DMAX, int NT, int U>
constexpr auto persistent_kernel_of() {
  if constexpr (DMAX <= core::kPairMaxD) return &anneal_persistent_kernel<DMAX, NT, U>;
  else return &anneal_persistent_kernel_rows<DMAX, NT, U>;
}

// The largest shared memory of any distance the persistent kernel runs.
template <int DMAX, int NT, int D = 3>
constexpr size_t persistent_smem() {
  if constexpr (D > DMAX) {
    return 0;
  } else {
    constexpr size_t here = core::smem_bytes<D, NT>();
    constexpr size_t rest = persistent_smem<DMAX, NT, D + 2>();
    return here > rest ? here : rest;
  }
}

}  // namespace batch
}  // namespace xzzx
