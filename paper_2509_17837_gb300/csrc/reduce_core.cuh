// Coset relabelling and decision for one shot, one warp (Alg. 7; Eqs.
// coset_correspondence, determine_P_from_E).
//
// Chain (i, P) belongs to coset Q_i P, where the class bits of Q_i are those
// of R_i xor those of R_1 (commutation with L_Z and L_X is linear).  Each lane
// folds its chains into per-coset minima of the key (energy, chain index), so
// ties keep the lowest chain; a warp butterfly reduces the four keys.
#pragma once

#include "internal.h"

namespace xzzx {
namespace reduce {

// Pauli index (I, X, Y, Z) <-> class bits (bit 0: anticommutes with L_Z, bit 1: with L_X).
__device__ __forceinline__ uint32_t index_to_bits(uint32_t p) { return (0x2310u >> (4 * p)) & 3u; }
__device__ __forceinline__ uint32_t bits_to_index(uint32_t b) { return (0x2310u >> (4 * b)) & 3u; }

// All pointers are already offset to the shot: init (R x 2w words, R_1 first),
// cb (R class bytes), chain_E (4R), chain_cfg (4R x 2w or null), true_err
// (2w or null); outputs cls (1), E4 (4), recovery (2w), best_cfg_out (2w or
// null), fail (1 or null).
__device__ __forceinline__ void reduce_warp(const DevCode& C, int R, const uint32_t* __restrict__ init,
                                            const uint8_t* __restrict__ cb, const int32_t* __restrict__ chain_E,
                                            const uint32_t* __restrict__ chain_cfg,
                                            const uint32_t* __restrict__ true_err, uint8_t* cls, int32_t* E4,
                                            uint32_t* recovery, uint32_t* best_cfg_out, uint8_t* fail) {
  const int lane = threadIdx.x & 31, w = C.w;
  const uint32_t q0 = cb[0] & 3u;
  uint64_t best[4] = {~0ull, ~0ull, ~0ull, ~0ull};
  for (int c = lane; c < 4 * R; c += 32) {
    const uint32_t q = (cb[c >> 2] & 3u) ^ q0;
    const uint32_t coset = bits_to_index(q ^ index_to_bits((uint32_t)(c & 3)));
    const uint32_t e = (uint32_t)chain_E[c] ^ 0x80000000u;  // order-preserving
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
  uint64_t bstar = best[0];
#pragma unroll
  for (int p = 1; p < 4; ++p)
    if (p == pstar) bstar = best[p];
  if (lane == 0) {
    *cls = (uint8_t)pstar;
#pragma unroll
    for (int p = 0; p < 4; ++p) E4[p] = (int32_t)((uint32_t)(best[p] >> 32) ^ 0x80000000u);
  }
  // recovery = R_1 L_{P*}
  const uint32_t pbits = index_to_bits((uint32_t)pstar);
  const uint32_t* LX = C.logical;
  const uint32_t* LZ = C.logical + 2 * w;
  int par_z = 0, par_x = 0;
  for (int j = lane; j < 2 * w; j += 32) {
    uint32_t v = init[j];
    if (pbits & 1u) v ^= LX[j];
    if (pbits & 2u) v ^= LZ[j];
    recovery[j] = v;
    if (true_err) {
      const uint32_t e = v ^ true_err[j];
      // symplectic product with L_Z and L_X: the x part meets the z part and vice versa
      const int jj = j < w ? j + w : j - w;
      par_z ^= __popc(e & LZ[jj]) & 1;
      par_x ^= __popc(e & LX[jj]) & 1;
    }
  }
  if (true_err) {
    for (int off = 16; off > 0; off >>= 1) {
      par_z ^= __shfl_xor_sync(0xFFFFFFFFu, par_z, off);
      par_x ^= __shfl_xor_sync(0xFFFFFFFFu, par_x, off);
    }
    if (lane == 0 && fail) *fail = (uint8_t)((par_z | par_x) != 0);
  }
  if (best_cfg_out && chain_cfg && XZZX_CHECK(C.err, (uint32_t)bstar < 4u * (uint32_t)R)) {
    const uint32_t* src = chain_cfg + (size_t)(uint32_t)bstar * 2 * w;
    for (int j = lane; j < 2 * w; j += 32) best_cfg_out[j] = src[j];
  }
}

}  // namespace reduce
}  // namespace xzzx
