// Coset relabelling and decision (Alg. 7; Eqs. coset_correspondence,
// determine_P_from_E) and the fused decoder entry point.
//
// One warp per shot.  Chain (i, P) belongs to coset Q_i P, where the class bits
// of Q_i are those of R_i xor those of R_1 (commutation with L_Z and L_X is
// linear).  Each lane folds its chains into per-coset minima of the key
// (energy, chain index), so ties keep the lowest chain; a warp butterfly
// reduces the four keys.
#include "internal.h"

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

// Pauli index (I, X, Y, Z) <-> class bits (bit 0: anticommutes with L_Z, bit 1: with L_X).
__device__ __forceinline__ uint32_t index_to_bits(uint32_t p) { return (0x2310u >> (4 * p)) & 3u; }
__device__ __forceinline__ uint32_t bits_to_index(uint32_t b) { return (0x2310u >> (4 * b)) & 3u; }

__global__ void __launch_bounds__(kWarps * 32) reduce_kernel(const __grid_constant__ ReduceArgs A) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t k = (int64_t)blockIdx.x * kWarps + warp;
  if (k >= A.n_shots) return;
  const int R = A.restarts, w = A.code.w;
  const uint8_t* cb = A.cbits + (size_t)k * R;
  const uint32_t q0 = cb[0] & 3u;
  uint64_t best[4] = {~0ull, ~0ull, ~0ull, ~0ull};
  for (int c = lane; c < 4 * R; c += 32) {
    const uint32_t q = (cb[c >> 2] & 3u) ^ q0;
    const uint32_t coset = bits_to_index(q ^ index_to_bits((uint32_t)(c & 3)));
    const uint32_t e = (uint32_t)A.chain_E[(size_t)k * 4 * R + c] ^ 0x80000000u;  // order-preserving
    const uint64_t key = ((uint64_t)e << 32) | (uint32_t)c;
#pragma unroll
    for (int p = 0; p < 4; ++p)
      if (coset == (uint32_t)p && key < best[p]) best[p] = key;
  }
#pragma unroll
  for (int p = 0; p < 4; ++p)
    for (int off = 16; off > 0; off >>= 1) {
      const uint64_t o = __shfl_xor_sync(0xFFFFFFFFu, best[p], off);
      best[p] = o < best[p] ? o : best[p];
    }
  int pstar = 0;
#pragma unroll
  for (int p = 1; p < 4; ++p)
    if ((best[p] >> 32) < (best[pstar] >> 32)) pstar = p;
  if (lane == 0) {
    A.cls[k] = (uint8_t)pstar;
#pragma unroll
    for (int p = 0; p < 4; ++p) A.E4[4 * k + p] = (int32_t)((uint32_t)(best[p] >> 32) ^ 0x80000000u);
  }
  // recovery = R_1 L_{P*}
  const uint32_t pbits = index_to_bits((uint32_t)pstar);
  const uint32_t* R1 = A.init + (size_t)k * R * 2 * w;
  const uint32_t* LX = A.code.logical;
  const uint32_t* LZ = A.code.logical + 2 * w;
  int par_z = 0, par_x = 0;
  for (int j = lane; j < 2 * w; j += 32) {
    uint32_t v = R1[j];
    if (pbits & 1u) v ^= LX[j];
    if (pbits & 2u) v ^= LZ[j];
    A.recovery[(size_t)k * 2 * w + j] = v;
    if (A.true_errors) {
      const uint32_t e = v ^ A.true_errors[(size_t)k * 2 * w + j];
      // symplectic product with L_Z and L_X: x part meets the z part and vice versa
      const int jj = j < w ? j + w : j - w;
      par_z ^= __popc(e & LZ[jj]) & 1;
      par_x ^= __popc(e & LX[jj]) & 1;
    }
  }
  if (A.true_errors) {
    for (int off = 16; off > 0; off >>= 1) {
      par_z ^= __shfl_xor_sync(0xFFFFFFFFu, par_z, off);
      par_x ^= __shfl_xor_sync(0xFFFFFFFFu, par_x, off);
    }
    if (lane == 0 && A.fail) A.fail[k] = (uint8_t)((par_z | par_x) != 0);
  }
  if (A.best_cfg_out && A.chain_cfg) {
    const uint32_t bc = (uint32_t)best[pstar];
    const uint32_t* src = A.chain_cfg + ((size_t)k * 4 * R + bc) * 2 * w;
    for (int j = lane; j < 2 * w; j += 32) A.best_cfg_out[(size_t)k * 2 * w + j] = src[j];
  }
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
  if (((uintptr_t)workspace & 255u) != 0) return fail(XZZX_EINVAL, "workspace must be 256-byte aligned");
  const Workspace L = layout(code, n_shots, restarts, best_cfg_out != nullptr);
  if (workspace_bytes < L.total)
    return fail(XZZX_EINVAL, "workspace too small: need " + std::to_string(L.total) + " bytes");
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
