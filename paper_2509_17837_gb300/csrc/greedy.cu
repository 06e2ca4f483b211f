// Randomised greedy matching (Algs. 5 and 6): the per-launch entry point.
// The per-CTA work is greedy::greedy_cta (greedy_core.cuh).
#include "greedy_core.cuh"

namespace xzzx {
namespace {

using namespace greedy;

struct GreedyArgs {
  DevCode code;
  PhiloxKeys keys;
  uint64_t shot0;
  int n_shots, restarts, randomised, groups, rpw;
  int32_t Wt_x, Wt_z;
  const uint32_t* syndromes;
  uint32_t* init;
  uint8_t* cbits;
};

template <class G, bool L>
__global__ void __launch_bounds__(kWarps * 32, L ? G::kMinCtasLists : 1)
    greedy_kernel(const __grid_constant__ GreedyArgs A) {
  __shared__ SharedT<G, L> S;
  const int k = blockIdx.x / A.groups;
  greedy_cta<G, L>(A.code, A.keys, A.shot0 + (uint64_t)k, blockIdx.x % A.groups, A.restarts, A.rpw, A.randomised,
                   A.Wt_x, A.Wt_z, A.syndromes + (size_t)k * A.code.sw,
                   A.init + (size_t)k * A.restarts * 2 * A.code.w, A.cbits + (size_t)k * A.restarts, S);
}

}  // namespace

xzzx_status launch_greedy(const xzzx_code* code, const xzzx_noise* noise, uint64_t seed, uint64_t shot0, int n_shots,
                          int restarts, int randomised, const uint32_t* syndromes, uint32_t* init, uint8_t* cbits,
                          cudaStream_t stream) {
  NvtxRange nvtx_range("xzzx K1 greedy");
  GreedyArgs A;
  A.code = code->dev;
  A.keys = philox_keys(seed);
  A.shot0 = shot0;
  A.n_shots = n_shots;
  A.restarts = restarts;
  A.randomised = randomised;
  A.rpw = 1;  // several restarts per warp only with candidate lists (d <= 17)
  for (int r = kMaxRestartsPerWarp; r > 1 && code->layout != kLayoutPlanar && code->d <= kListMaxD; r >>= 1)
    if ((int64_t)n_shots * greedy_groups(restarts, r) >= kMinGreedyCtas) {
      A.rpw = r;
      break;
    }
  A.groups = greedy_groups(restarts, A.rpw);
  A.Wt_x = noise->Wt_x;
  A.Wt_z = noise->Wt_z;
  A.syndromes = syndromes;
  A.init = init;
  A.cbits = cbits;
  const uint64_t grid = (uint64_t)n_shots * A.groups;
  if (grid > 0x7FFFFFFFull) return fail(XZZX_EINVAL, "too many shots x restarts for one launch");
  if (code->layout == kLayoutPlanar)
    greedy_kernel<PlanarGeo, false><<<(unsigned)grid, kWarps * 32, 0, stream>>>(A);
  else if (code->d <= kListMaxD)
    greedy_kernel<RotGeo, true><<<(unsigned)grid, kWarps * 32, 0, stream>>>(A);
  else
    greedy_kernel<RotGeo, false><<<(unsigned)grid, kWarps * 32, 0, stream>>>(A);
  XZZX_CUDA_TRY(cudaGetLastError());
  return XZZX_OK;
}

}  // namespace xzzx

using namespace xzzx;

extern "C" xzzx_status xzzx_greedy_init(const xzzx_code* code, const xzzx_noise* noise, uint64_t seed, uint64_t shot0,
                                        int n_shots, int restarts, int randomised, const uint32_t* syndromes,
                                        uint32_t* init, uint8_t* cbits, void* stream) {
  xzzx_status st = check_code(code);
  if (st) return st;
  if (!noise) return fail(XZZX_EINVAL, "noise is NULL");
  if (n_shots < 0) return fail(XZZX_EINVAL, "n_shots < 0");
  if (restarts < 1 || restarts > 65535) return fail(XZZX_EINVAL, "restarts must be in [1, 65535]");
  if (randomised < 0 || randomised > 2) return fail(XZZX_EINVAL, "init mode must be 0, 1 or 2");
  if (noise->Wt_x <= 0 || noise->Wt_z <= 0) return fail(XZZX_EINVAL, "matching weights must be positive");
  if ((int64_t)noise->Wt_x * 4 * code->nq > kInf || (int64_t)noise->Wt_z * 4 * code->nq > kInf)
    return fail(XZZX_EINVAL, "matching weights too large for int32 path lengths");
  if (n_shots == 0) return XZZX_OK;
  if ((st = check_ptr(syndromes, "syndromes")) || (st = check_ptr(init, "init")) || (st = check_ptr(cbits, "cbits")))
    return st;
  return launch_greedy(code, noise, seed, shot0, n_shots, restarts, randomised, syndromes, init, cbits,
                       (cudaStream_t)stream);
}
