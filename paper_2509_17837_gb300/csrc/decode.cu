// The coset decision launch and the fused decoder entry point (Alg. 7).
// The per-shot work is reduce::reduce_warp (reduce_core.cuh).
#include "internal.h"
#include "reduce_core.cuh"

namespace xzzx {

xzzx_status launch_greedy(const xzzx_code*, const xzzx_noise*, uint64_t, uint64_t, int, int, int, const uint32_t*,
                          uint32_t*, uint8_t*, cudaStream_t);
xzzx_status launch_anneal(const xzzx_code*, const xzzx_schedule*, uint64_t, uint64_t, int, int, const uint32_t*,
                          int32_t*, uint32_t*, int32_t*, uint32_t*, cudaStream_t);
xzzx_status check_anneal_args(const xzzx_code*, const xzzx_schedule*, int, int);

namespace {

constexpr int kWarps = 4;

struct ReduceArgs {
  DevCode code;
  int n_shots, restarts;
  const uint32_t* init;
  const uint8_t* cbits;
  const int32_t* chain_E;
  const uint32_t* chain_cfg;
  const uint32_t* true_errors;
  uint8_t* cls;
  int32_t* E4;
  uint32_t* recovery;
  uint32_t* best_cfg_out;
  uint8_t* fail;
};

__global__ void __launch_bounds__(kWarps * 32) reduce_kernel(const __grid_constant__ ReduceArgs A) {
  const int warp = threadIdx.x >> 5;
  const int64_t k = (int64_t)blockIdx.x * kWarps + warp;
  if (k >= A.n_shots) return;
  const int R = A.restarts, w = A.code.w;
  reduce::reduce_warp(A.code, R, A.init + (size_t)k * R * 2 * w, A.cbits + (size_t)k * R, A.chain_E + (size_t)k * 4 * R,
                      A.chain_cfg ? A.chain_cfg + (size_t)k * 4 * R * 2 * w : nullptr,
                      A.true_errors ? A.true_errors + (size_t)k * 2 * w : nullptr, A.cls + k, A.E4 + 4 * k,
                      A.recovery + (size_t)k * 2 * w, A.best_cfg_out ? A.best_cfg_out + (size_t)k * 2 * w : nullptr,
                      A.fail ? A.fail + k : nullptr);
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Workspace {
  size_t o_init, o_cbits, o_E, o_cfg, total;
};

Workspace layout(const xzzx_code* code, int n_shots, int restarts, int want_cfg) {
  Workspace L;
  const size_t chains = (size_t)n_shots * restarts * 4;
  L.o_init = 0;
  L.o_cbits = align256(L.o_init + sizeof(uint32_t) * (size_t)n_shots * restarts * 2 * code->w);
  L.o_E = align256(L.o_cbits + (size_t)n_shots * restarts);
  L.o_cfg = align256(L.o_E + sizeof(int32_t) * chains);
  L.total = align256(L.o_cfg + (want_cfg ? sizeof(uint32_t) * chains * 2 * code->w : 0));
  return L;
}

}  // namespace

xzzx_status launch_reduce(const xzzx_code* code, int n_shots, int restarts, const uint32_t* init, const uint8_t* cbits,
                          const int32_t* chain_E, const uint32_t* chain_cfg, const uint32_t* true_errors, uint8_t* cls,
                          int32_t* E4, uint32_t* recovery, uint32_t* best_cfg_out, uint8_t* fail_out,
                          cudaStream_t stream) {
  NvtxRange nvtx_range("xzzx K3 reduce");
  ReduceArgs A;
  A.code = code->dev;
  A.n_shots = n_shots;
  A.restarts = restarts;
  A.init = init;
  A.cbits = cbits;
  A.chain_E = chain_E;
  A.chain_cfg = chain_cfg;
  A.true_errors = true_errors;
  A.cls = cls;
  A.E4 = E4;
  A.recovery = recovery;
  A.best_cfg_out = best_cfg_out;
  A.fail = fail_out;
  const unsigned grid = (unsigned)((n_shots + kWarps - 1) / kWarps);
  reduce_kernel<<<grid, kWarps * 32, 0, stream>>>(A);
  XZZX_CUDA_TRY(cudaGetLastError());
  return XZZX_OK;
}

}  // namespace xzzx

using namespace xzzx;

extern "C" {

xzzx_status xzzx_decode_reduce(const xzzx_code* code, int n_shots, int restarts, const uint32_t* init,
                               const uint8_t* cbits, const int32_t* chain_E, const uint32_t* chain_cfg,
                               const uint32_t* true_errors, uint8_t* cls, int32_t* E4, uint32_t* recovery,
                               uint32_t* best_cfg_out, uint8_t* fail_out, void* stream) {
  xzzx_status st = check_code(code);
  if (st) return st;
  if (n_shots < 0 || restarts < 1 || restarts > 65535) return fail(XZZX_EINVAL, "bad n_shots or restarts");
  if (n_shots == 0) return XZZX_OK;
  if ((st = check_ptr(init, "init")) || (st = check_ptr(cbits, "cbits")) || (st = check_ptr(chain_E, "chain_E")) ||
      (st = check_ptr(cls, "cls")) || (st = check_ptr(E4, "E4")) || (st = check_ptr(recovery, "recovery")))
    return st;
  if (best_cfg_out && !chain_cfg) return fail(XZZX_EINVAL, "best_cfg_out needs chain_cfg");
  if (fail_out && !true_errors) return fail(XZZX_EINVAL, "fail needs true_errors");
  return launch_reduce(code, n_shots, restarts, init, cbits, chain_E, chain_cfg, true_errors, cls, E4, recovery,
                       best_cfg_out, fail_out, (cudaStream_t)stream);
}

xzzx_status xzzx_decode_workspace_size(const xzzx_code* code, int n_shots, int restarts, int want_best_cfg,
                                       size_t* bytes) {
  if (!code || !bytes) return fail(XZZX_EINVAL, "NULL argument");
  if (n_shots < 0 || restarts < 1 || restarts > 65535) return fail(XZZX_EINVAL, "bad n_shots or restarts");
  *bytes = layout(code, n_shots, restarts, want_best_cfg).total;
  return XZZX_OK;
}

xzzx_status xzzx_decode_batch(const xzzx_code* code, const xzzx_noise* noise, const xzzx_schedule* sched,
                              uint64_t seed, uint64_t shot0, int n_shots, int restarts, int randomised,
                              const uint32_t* syndromes, const uint32_t* true_errors, uint8_t* cls, int32_t* E4,
                              uint32_t* recovery, uint32_t* best_cfg_out, uint8_t* fail_out, void* workspace,
                              size_t workspace_bytes, void* stream) {
  xzzx_status st = check_anneal_args(code, sched, n_shots, restarts);
  if (st) return st;
  if (!noise) return fail(XZZX_EINVAL, "noise is NULL");
  if (noise->Wt_x <= 0 || noise->Wt_z <= 0) return fail(XZZX_EINVAL, "matching weights must be positive");
  if (n_shots == 0) return XZZX_OK;
  if ((st = check_ptr(syndromes, "syndromes")) || (st = check_ptr(cls, "cls")) || (st = check_ptr(E4, "E4")) ||
      (st = check_ptr(recovery, "recovery")) || (st = check_ptr(workspace, "workspace")))
    return st;
  if (fail_out && !true_errors) return fail(XZZX_EINVAL, "fail needs true_errors");
  if (randomised < 0 || randomised > 2) return fail(XZZX_EINVAL, "init mode must be 0, 1 or 2");
  if (((uintptr_t)workspace & 255u) != 0) return fail(XZZX_EINVAL, "workspace must be 256-byte aligned");
  const Workspace L = layout(code, n_shots, restarts, best_cfg_out != nullptr);
  if (workspace_bytes < L.total)
    return fail(XZZX_EINVAL, "workspace too small: need " + std::to_string(L.total) + " bytes");
  NvtxRange nvtx_range("xzzx decode_batch");
  char* ws = (char*)workspace;
  uint32_t* init = (uint32_t*)(ws + L.o_init);
  uint8_t* cbits = (uint8_t*)(ws + L.o_cbits);
  int32_t* chain_E = (int32_t*)(ws + L.o_E);
  uint32_t* chain_cfg = best_cfg_out ? (uint32_t*)(ws + L.o_cfg) : nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = launch_greedy(code, noise, seed, shot0, n_shots, restarts, randomised, syndromes, init, cbits, s)))
    return st;
  if ((st = launch_anneal(code, sched, seed, shot0, n_shots, restarts, init, chain_E, chain_cfg, nullptr, nullptr, s)))
    return st;
  return launch_reduce(code, n_shots, restarts, init, cbits, chain_E, chain_cfg, true_errors, cls, E4, recovery,
                       best_cfg_out, fail_out, s);
}

}  // extern "C"
