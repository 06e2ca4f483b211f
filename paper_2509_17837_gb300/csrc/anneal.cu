// The plain annealing launch (Alg. 2 with the Metropolis step of Alg. 3):
// one launch per distance, one chain per thread, chains of consecutive
// (shot, restart, coset) indices.  The per-CTA work is core::anneal_cta.
#include "anneal_core.cuh"

namespace xzzx {
namespace {

using namespace core;

struct AnnealArgs {
  PhiloxKeys keys;
  uint64_t chain0;  // global id of local chain 0
  int64_t n_chains;
  int restarts;
  int n_sweeps, n_classes;
  int32_t W[4];
  const uint32_t* T;
  const int2* sig;
  const uint32_t* init;
  int32_t* best_E;
  uint32_t* best_cfg;
  int32_t* final_E;
  uint32_t* final_cfg;
  uint32_t* err;
};

// One chain per thread.  The pair path (d <= 15) is bounded to four 256-thread
// CTAs per SM (64 registers); the row path keeps the compiler's choice for
// 128-thread CTAs (about 120 registers up to d = 29, 160 at d = 31).
template <int D>
__device__ __forceinline__ void anneal_body(const AnnealArgs& A) {
  constexpr int NT = Shape<D>::kThreads;
  constexpr int W = Shape<D>::kW;
  extern __shared__ __align__(16) uint8_t smem[];
  const int64_t c_raw = (int64_t)blockIdx.x * NT + threadIdx.x;
  const bool active = c_raw < A.n_chains;
  const int64_t c = active ? c_raw : A.n_chains - 1;
  SweepTables tab;
  tab.T = A.T;
  tab.sig = A.sig;
  tab.n_sweeps = A.n_sweeps;
  tab.n_classes = A.n_classes;
  for (int k = 0; k < 4; ++k) tab.W[k] = A.W[k];
  tab.err = A.err;
  ChainOut out;
  out.best_E = A.best_E + c;
  out.best_cfg = A.best_cfg ? A.best_cfg + (size_t)c * 2 * W : nullptr;
  out.final_E = A.final_E ? A.final_E + c : nullptr;
  out.final_cfg = A.final_cfg ? A.final_cfg + (size_t)c * 2 * W : nullptr;
  anneal_cta<D, NT>(A.init + (size_t)(c >> 2) * 2 * W, A.chain0 + (uint64_t)c, (int)(c & 3), active, out, tab,
                    A.keys, smem);
}

template <int D>
__global__ void __launch_bounds__(Shape<D>::kThreads, 4) anneal_kernel(const __grid_constant__ AnnealArgs A) {
  anneal_body<D>(A);
}
template <int D>
__global__ void __launch_bounds__(Shape<D>::kThreads) anneal_kernel_rows(const __grid_constant__ AnnealArgs A) {
  anneal_body<D>(A);
}
// d >= 29: held to 128 registers, four CTAs per SM instead of three (the
// compiler's own choice is about 158); more chains in flight hide the sweep's
// dependent integer chain better than the extra registers do.
template <int D>
__global__ void __launch_bounds__(Shape<D>::kThreads, 4) anneal_kernel_rows4(const __grid_constant__ AnnealArgs A) {
  anneal_body<D>(A);
}
template <int D>
constexpr auto anneal_kernel_of() {
  if constexpr (D <= kPairMaxD) return &anneal_kernel<D>;
  else if constexpr (D >= 29) return &anneal_kernel_rows4<D>;
  else return &anneal_kernel_rows<D>;
}

template <int D>
xzzx_status launch_d(const AnnealArgs& A, cudaStream_t stream) {
  constexpr int NT = Shape<D>::kThreads;
  const size_t smem = smem_bytes<D, NT>();
  static DeviceOnce once;
  xzzx_status st = once.run([&]() -> xzzx_status {
    XZZX_CUDA_TRY(cudaFuncSetAttribute(anneal_kernel_of<D>(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return XZZX_OK;
  });
  if (st) return st;
  const int64_t grid = (A.n_chains + NT - 1) / NT;
  if (grid > 0x7FFFFFFF) return fail(XZZX_EINVAL, "too many chains for one launch");
  anneal_kernel_of<D>()<<<(unsigned)grid, NT, smem, stream>>>(A);
  XZZX_CUDA_TRY(cudaGetLastError());
  return XZZX_OK;
}

}  // namespace

xzzx_status launch_anneal_planar(const xzzx_code* code, const xzzx_schedule* sched, uint64_t seed, uint64_t shot0,
                                 int n_shots, int restarts, int order, int emin, const uint32_t* init, int32_t* best_E,
                                 uint32_t* best_cfg, int32_t* final_E, uint32_t* final_cfg, cudaStream_t stream);

xzzx_status launch_anneal(const xzzx_code* code, const xzzx_schedule* sched, uint64_t seed, uint64_t shot0,
                          int n_shots, int restarts, const uint32_t* init, int32_t* best_E, uint32_t* best_cfg,
                          int32_t* final_E, uint32_t* final_cfg, cudaStream_t stream) {
  NvtxRange nvtx_range("xzzx K2 anneal");
  if (code->layout == kLayoutPlanar)  // colour sweep, minimum per colour phase
    return launch_anneal_planar(code, sched, seed, shot0, n_shots, restarts, 0, 0, init, best_E, best_cfg, final_E,
                                final_cfg, stream);
  AnnealArgs A;
  A.keys = philox_keys(seed);
  A.chain0 = shot0 * (uint64_t)restarts * 4u;
  A.n_chains = (int64_t)n_shots * restarts * 4;
  A.restarts = restarts;
  A.n_sweeps = sched->n_sweeps;
  A.n_classes = sched->n_classes;
  for (int k = 0; k < 4; ++k) A.W[k] = sched->noise.W[k];
  A.T = sched->d_T;
  A.sig = sched->d_sig;
  A.init = init;
  A.best_E = best_E;
  A.best_cfg = best_cfg;
  A.final_E = final_E;
  A.final_cfg = final_cfg;
  A.err = code->dev.err;
  switch (code->d) {
#define XZZX_CASE(DD) \
  case DD:            \
    return launch_d<DD>(A, stream);
    XZZX_CASE(3) XZZX_CASE(5) XZZX_CASE(7) XZZX_CASE(9) XZZX_CASE(11) XZZX_CASE(13) XZZX_CASE(15)
    XZZX_CASE(17) XZZX_CASE(19) XZZX_CASE(21) XZZX_CASE(23) XZZX_CASE(25) XZZX_CASE(27) XZZX_CASE(29)
    XZZX_CASE(31)
#undef XZZX_CASE
    default:
      return fail(XZZX_EUNSUPPORTED, "no annealing kernel for this distance");
  }
}

xzzx_status check_anneal_args(const xzzx_code* code, const xzzx_schedule* sched, int n_shots, int restarts) {
  xzzx_status st = check_code(code);
  if (st) return st;
  if (!sched) return fail(XZZX_EINVAL, "schedule is NULL");
  if (!sched->d_sig) return fail(XZZX_EINVAL, "schedule has no device tables (created without a GPU)");
  if ((st = check_device(sched->device))) return st;
  if (n_shots < 0) return fail(XZZX_EINVAL, "n_shots < 0");
  if (restarts < 1 || restarts > 65535) return fail(XZZX_EINVAL, "restarts must be in [1, 65535]");
  int32_t wmax = 0;
  for (int k = 0; k < 4; ++k) wmax = wmax > sched->noise.W[k] ? wmax : sched->noise.W[k];
  if ((int64_t)wmax * code->nq * 2 > 0x7FFFFFFFll) return fail(XZZX_EINVAL, "energies would overflow int32");
  return XZZX_OK;
}

}  // namespace xzzx

using namespace xzzx;

extern "C" xzzx_status xzzx_anneal(const xzzx_code* code, const xzzx_schedule* sched, uint64_t seed, uint64_t shot0,
                                   int n_shots, int restarts, const uint32_t* init, int32_t* best_E,
                                   uint32_t* best_cfg, int32_t* final_E, uint32_t* final_cfg, void* stream) {
  xzzx_status st = check_anneal_args(code, sched, n_shots, restarts);
  if (st) return st;
  if (n_shots == 0) return XZZX_OK;
  if ((st = check_ptr(init, "init")) || (st = check_ptr(best_E, "best_E"))) return st;
  return launch_anneal(code, sched, seed, shot0, n_shots, restarts, init, best_E, best_cfg, final_E, final_cfg,
                       (cudaStream_t)stream);
}
