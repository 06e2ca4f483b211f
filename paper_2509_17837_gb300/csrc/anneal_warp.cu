// Launch of the warp-per-chain annealing kernel (anneal_warp.cuh).
#include "anneal_warp.cuh"

namespace xzzx {

xzzx_status check_anneal_args(const xzzx_code*, const xzzx_schedule*, int, int);

namespace warpchain {
namespace {

constexpr int kWPC = 4;  // chains (warps) per CTA

struct Args {
  PhiloxKeys keys;
  uint64_t chain0;
  int64_t n_chains;
  core::SweepTables tab;
  const uint32_t* init;
  int32_t* best_E;
  uint32_t* best_cfg;
  int32_t* final_E;
  uint32_t* final_cfg;
};

template <int D>
__global__ void __launch_bounds__(kWPC * 32) anneal_warp_kernel(const __grid_constant__ Args A) {
  constexpr int W = core::Shape<D>::kW;
  extern __shared__ __align__(16) uint8_t smem[];
  const int64_t c_raw = (int64_t)blockIdx.x * kWPC + (threadIdx.x >> 5);
  const bool active = c_raw < A.n_chains;
  const int64_t c = active ? c_raw : A.n_chains - 1;
  core::ChainOut out;
  out.best_E = A.best_E + c;
  out.best_cfg = A.best_cfg ? A.best_cfg + (size_t)c * 2 * W : nullptr;
  out.final_E = A.final_E ? A.final_E + c : nullptr;
  out.final_cfg = A.final_cfg ? A.final_cfg + (size_t)c * 2 * W : nullptr;
  anneal_warp_cta<D, kWPC>(A.init + (size_t)(c >> 2) * 2 * W, A.chain0 + (uint64_t)c, (int)(c & 3), active, out,
                           A.tab, A.keys, smem);
}

template <int D>
xzzx_status launch_d(const Args& A, cudaStream_t stream) {
  constexpr size_t smem = smem_bytes<D, kWPC>();
  const int64_t grid = (A.n_chains + kWPC - 1) / kWPC;
  if (grid > 0x7FFFFFFF) return fail(XZZX_EINVAL, "too many chains for one launch");
  anneal_warp_kernel<D><<<(unsigned)grid, kWPC * 32, smem, stream>>>(A);
  XZZX_CUDA_TRY(cudaGetLastError());
  return XZZX_OK;
}

}  // namespace
}  // namespace warpchain

xzzx_status launch_anneal_warp(const xzzx_code* code, const xzzx_schedule* sched, uint64_t seed, uint64_t shot0,
                               int n_shots, int restarts, const uint32_t* init, int32_t* best_E, uint32_t* best_cfg,
                               int32_t* final_E, uint32_t* final_cfg, cudaStream_t stream) {
  warpchain::Args A;
  A.keys = philox_keys(seed);
  A.chain0 = shot0 * (uint64_t)restarts * 4u;
  A.n_chains = (int64_t)n_shots * restarts * 4;
  A.tab.T = sched->d_T;
  A.tab.sig = sched->d_sig;
  A.tab.n_sweeps = sched->n_sweeps;
  A.tab.n_classes = sched->n_classes;
  for (int k = 0; k < 4; ++k) A.tab.W[k] = sched->noise.W[k];
  A.tab.err = code->dev.err;
  A.init = init;
  A.best_E = best_E;
  A.best_cfg = best_cfg;
  A.final_E = final_E;
  A.final_cfg = final_cfg;
  switch (code->d) {
#define XZZX_CASE(DD) \
  case DD:            \
    return warpchain::launch_d<DD>(A, stream);
    XZZX_CASE(3) XZZX_CASE(5) XZZX_CASE(7) XZZX_CASE(9) XZZX_CASE(11) XZZX_CASE(13) XZZX_CASE(15)
    XZZX_CASE(17) XZZX_CASE(19) XZZX_CASE(21) XZZX_CASE(23) XZZX_CASE(25) XZZX_CASE(27) XZZX_CASE(29)
    XZZX_CASE(31)
#undef XZZX_CASE
    default:
      return fail(XZZX_EUNSUPPORTED, "no annealing kernel for this distance");
  }
}

}  // namespace xzzx

using namespace xzzx;

extern "C" xzzx_status xzzx_anneal_warp(const xzzx_code* code, const xzzx_schedule* sched, uint64_t seed,
                                        uint64_t shot0, int n_shots, int restarts, const uint32_t* init,
                                        int32_t* best_E, uint32_t* best_cfg, int32_t* final_E, uint32_t* final_cfg,
                                        void* stream) {
  xzzx_status st = check_anneal_args(code, sched, n_shots, restarts);
  if (st) return st;
  if (code->layout != kLayoutRotated) return fail(XZZX_EUNSUPPORTED, "the warp-per-chain kernel takes rotated codes");
  if (n_shots == 0) return XZZX_OK;
  if ((st = check_ptr(init, "init")) || (st = check_ptr(best_E, "best_E"))) return st;
  return launch_anneal_warp(code, sched, seed, shot0, n_shots, restarts, init, best_E, best_cfg, final_E, final_cfg,
                            (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// Batched form: one warp per chain over the chains of several segments of one
// distance (batch plan mode 2).
// ---------------------------------------------------------------------------
#include "batch_internal.h"

#include <algorithm>

namespace xzzx {
namespace batch {
namespace {

__device__ __forceinline__ int find_segment_w(const int64_t* __restrict__ prefix, int n_segs, int64_t x) {
  int lo = 0, hi = n_segs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

constexpr int kWPC = 4;

template <int D>
__global__ void __launch_bounds__(kWPC * 32) warp_chains_kernel(const __grid_constant__ WarpLaunch L) {
  constexpr int W = core::Shape<D>::kW;
  extern __shared__ __align__(16) uint8_t smem[];
  const int64_t g_raw = (int64_t)blockIdx.x * kWPC + (threadIdx.x >> 5);
  const bool active = g_raw < L.n_chains;
  const int64_t x = L.chain0 + (active ? g_raw : L.n_chains - 1);
  const int s = find_segment_w(L.chain_prefix, L.n_segs, x);
  const SegDev& sg = L.segs[s];
  const int64_t c = x - L.chain_prefix[s];
  core::SweepTables tab;
  tab.T = sg.T;
  tab.sig = sg.sig;
  tab.n_sweeps = sg.n_sweeps;
  tab.n_classes = sg.n_classes;
  for (int k = 0; k < 4; ++k) tab.W[k] = sg.W[k];
  tab.err = sg.code.err;
  core::ChainOut out;
  out.best_E = sg.chain_E + c;
  out.best_cfg = nullptr;
  out.final_E = nullptr;
  out.final_cfg = nullptr;
  warpchain::anneal_warp_cta<D, kWPC>(sg.init + (size_t)(c >> 2) * 2 * W,
                                      sg.shot0 * (uint64_t)sg.restarts * 4u + (uint64_t)c, (int)(c & 3), active, out,
                                      tab, L.keys, smem);
}

template <int D>
xzzx_status warp_chains_d(const WarpLaunch& L, cudaStream_t stream) {
  const size_t smem = std::max(warpchain::smem_bytes<D, kWPC>(), (size_t)std::max(L.smem, 0));
  if (L.n_chains <= 0) return XZZX_OK;
  const int64_t grid = (L.n_chains + kWPC - 1) / kWPC;
  if (grid > 0x7FFFFFFF) return fail(XZZX_EINVAL, "too many chains for one launch");
  warp_chains_kernel<D><<<(unsigned)grid, kWPC * 32, smem, stream>>>(L);
  XZZX_CUDA_TRY(cudaGetLastError());
  return XZZX_OK;
}

// Shared memory per CTA that holds the kernel at no more than cap resident
// CTAs per SM (cap 0: its own need, no cap); the kernel is set to prefer the
// largest shared-memory carveout so the cap is what decides.
template <int D>
xzzx_status warp_chains_configure_d(int cap, int* smem_out, int* ctas_per_sm) {
  size_t smem = warpchain::smem_bytes<D, kWPC>();
  int dev = 0, per_sm_bytes = 0, reserved = 0, optin = 0;
  XZZX_CUDA_TRY(cudaGetDevice(&dev));
  XZZX_CUDA_TRY(cudaDeviceGetAttribute(&per_sm_bytes, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  XZZX_CUDA_TRY(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev));
  XZZX_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (cap > 0) {
    const long pad = ((long)per_sm_bytes / cap - reserved) & ~15L;
    smem = std::max(smem, (size_t)std::min<long>(pad, optin));
  }
  XZZX_CUDA_TRY(cudaFuncSetAttribute(warp_chains_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  XZZX_CUDA_TRY(cudaFuncSetAttribute(warp_chains_kernel<D>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared));
  XZZX_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, warp_chains_kernel<D>, kWPC * 32, smem));
  *smem_out = (int)smem;
  return XZZX_OK;
}

}  // namespace

xzzx_status configure_warp_chains(int d, int cap, int* smem, int* ctas_per_sm) {
  switch (d) {
#define XZZX_CASE(DD) \
  case DD:            \
    return warp_chains_configure_d<DD>(cap, smem, ctas_per_sm);
    XZZX_CASE(3) XZZX_CASE(5) XZZX_CASE(7) XZZX_CASE(9) XZZX_CASE(11) XZZX_CASE(13) XZZX_CASE(15)
    XZZX_CASE(17) XZZX_CASE(19) XZZX_CASE(21) XZZX_CASE(23) XZZX_CASE(25) XZZX_CASE(27) XZZX_CASE(29)
    XZZX_CASE(31)
#undef XZZX_CASE
    default:
      return fail(XZZX_EUNSUPPORTED, "no annealing kernel for this distance");
  }
}

xzzx_status launch_warp_chains(int d, const WarpLaunch& L, cudaStream_t stream) {
  switch (d) {
#define XZZX_CASE(DD) \
  case DD:            \
    return warp_chains_d<DD>(L, stream);
    XZZX_CASE(3) XZZX_CASE(5) XZZX_CASE(7) XZZX_CASE(9) XZZX_CASE(11) XZZX_CASE(13) XZZX_CASE(15)
    XZZX_CASE(17) XZZX_CASE(19) XZZX_CASE(21) XZZX_CASE(23) XZZX_CASE(25) XZZX_CASE(27) XZZX_CASE(29)
    XZZX_CASE(31)
#undef XZZX_CASE
    default:
      return fail(XZZX_EUNSUPPORTED, "no annealing kernel for this distance");
  }
}

}  // namespace batch
}  // namespace xzzx
