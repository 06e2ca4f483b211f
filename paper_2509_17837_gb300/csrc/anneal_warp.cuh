// Warp-per-chain annealing (the colour-parallel form of Alg. 2 / Alg. 3).
//
// One warp anneals one chain.  The chain's rows (two bits per qubit, one
// 64-bit word per lattice row) live in shared memory.  Inside a colour phase
// the faces are disjoint, so the lanes take them in parallel: lane L handles
// the groups L, L+32, ... of the phase, a group being the (up to) four faces
// of one column and one row group -- exactly the faces one Philox block
// serves.  A lane reads the two rows of each face, looks the move up in the
// warp's per-sweep table, draws if needed, and applies an accepted move with
// shared-memory atomic XORs (faces of other columns in the same rows change
// other bits of the same words).  Per-lane energy changes are summed with warp
// shuffles at the end of each phase, where the minimum is tracked as in the
// one-chain-per-thread kernel.  Chain ids, counters, sweep order and the
// per-phase minimum are identical to that kernel, so results are identical;
// the chain's sequential work is up to 32 times shorter, which is what a
// latency-bound caller (a lightly loaded server) needs.
#pragma once

#include "anneal_core.cuh"

namespace xzzx {
namespace warpchain {

using core::kLutN;

// Shared memory per CTA: static (dE, class) table, then per warp its table,
// its rows and its minimum-energy rows, and a staging area for the output.
template <int D, int WPC>
__host__ __device__ constexpr size_t smem_bytes() {
  return kLutN * sizeof(int2) +
         (size_t)WPC * (kLutN * sizeof(uint2) + 2 * D * sizeof(unsigned long long) + 2 * 32 * sizeof(uint32_t));
}

// One colour phase, lanes in parallel; returns this lane's energy change.
template <int D, int C>
__device__ __forceinline__ int32_t warp_phase(unsigned long long* rows, const uint2* __restrict__ L, uint32_t t,
                                              uint32_t c2, uint32_t c3, const PhiloxKeys& K, int lane) {
  constexpr int NR = (C == 0 || C == 3) ? (D + 1) / 2 : (D - 1) / 2;
  constexpr int AOFF = (C == 1) ? 1 : (C == 3) ? -1 : 0;
  constexpr int IAOFF = (C == 1) ? 1 : 0;
  constexpr int NG = (NR - 1 + IAOFF) / 4 + 1;
  constexpr int PB = C >> 1;
  constexpr int NCB = (D - 1) / 2;
  constexpr int NCOL = NCB + ((C == 1 || C == 2) ? 1 : 0);  // bulk columns + the boundary column
  int32_t dsum = 0;
  for (int gi = lane; gi < NCOL * NG; gi += 32) {
    const int col = gi / NG, g = gi % NG;
    const bool bcol = col == NCB;  // colours 1, 2: the boundary column
    int b;
    if (bcol) b = (C == 1) ? D - 1 : -1;
    else b = 2 * col + PB;
    const uint32_t ib = (uint32_t)(b + 1) >> 1;
    const uint32_t s = bcol ? 2u * (uint32_t)(D - 1) : 2u * (uint32_t)b;  // unused for the left column
    uint2 e[4];
    int rowa[4];
    uint32_t need = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int j = 4 * g + k - IAOFF;  // row index inside the colour
      rowa[k] = -2;
      e[k] = make_uint2(0u, 0u);
      if (j < 0 || j >= NR) continue;
      const int a = 2 * j + AOFF;
      rowa[k] = a;
      uint32_t idx;
      if (bcol) {
        const unsigned long long r0 = rows[a], r1 = rows[a + 1];
        if (C == 1)
          idx = sig_base(kRight) + (((uint32_t)(r0 >> s) & 3u) | (((uint32_t)(r1 >> s) & 3u) << 2));
        else
          idx = sig_base(kLeft) + (((uint32_t)r0 & 3u) | (((uint32_t)r1 & 3u) << 2));
      } else if (a == -1) {
        idx = sig_base(kTop) + ((uint32_t)(rows[0] >> s) & 0xFu);
      } else if (a == D - 1) {
        idx = sig_base(kBottom) + ((uint32_t)(rows[D - 1] >> s) & 0xFu);
      } else {
        idx = ((uint32_t)(rows[a] >> s) & 0xFu) | (((uint32_t)(rows[a + 1] >> s) & 0xFu) << 4);
      }
      e[k] = L[idx];
      need |= e[k].y;
    }
    uint4 r = make_uint4(0u, 0u, 0u, 0u);
    if (need) r = philox4x32_10(((uint32_t)C << 16) | (ib << 8) | (uint32_t)g, t, c2, c3, K);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int a = rowa[k];
      if (a == -2) continue;
      const int ia = 4 * g + k;  // (a+1)>>1
      const uint32_t u = lane_of(r, ia & 3);
      const int32_t dE = (int32_t)e[k].x;
      if (!((dE <= 0) | (u < e[k].y))) continue;
      dsum += dE;
      if (bcol) {
        if (C == 1) {
          atomicXor(&rows[a], 2ull << s);
          atomicXor(&rows[a + 1], 1ull << s);
        } else {
          atomicXor(&rows[a], 1ull);
          atomicXor(&rows[a + 1], 2ull);
        }
      } else if (a == -1) {
        atomicXor(&rows[0], 0x9ull << s);
      } else if (a == D - 1) {
        atomicXor(&rows[D - 1], 0x6ull << s);
      } else {
        atomicXor(&rows[a], 0x6ull << s);
        atomicXor(&rows[a + 1], 0x9ull << s);
      }
    }
  }
  return dsum;
}

__device__ __forceinline__ int32_t warp_sum(int32_t v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, off);
  return v;
}

// Anneal one chain per warp.  Every thread of the CTA must call this (one
// barrier at the start).  Arguments as core::anneal_cta, per warp.
template <int D, int WPC>
__device__ __forceinline__ void anneal_warp_cta(const uint32_t* __restrict__ init, uint64_t chain, int P, bool active,
                                                const core::ChainOut& out, const core::SweepTables& tab,
                                                const PhiloxKeys& K, uint8_t* smem) {
  constexpr int W = core::Shape<D>::kW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int2* sig_static = reinterpret_cast<int2*>(smem);
  uint8_t* wbase = smem + kLutN * sizeof(int2) +
                   (size_t)warp * (kLutN * sizeof(uint2) + 2 * D * sizeof(unsigned long long) + 64 * sizeof(uint32_t));
  uint2* L = reinterpret_cast<uint2*>(wbase);
  unsigned long long* rows = reinterpret_cast<unsigned long long*>(wbase + kLutN * sizeof(uint2));
  unsigned long long* best = rows + D;
  uint32_t* stage = reinterpret_cast<uint32_t*>(best + D);  // 2w <= 62 words
  const uint32_t c2 = (uint32_t)chain;
  const uint32_t c3 = kTagSA | ((uint32_t)(chain >> 32) << 8);
  const int n_sweeps = tab.n_sweeps;

  for (int idx = threadIdx.x; idx < kLutN; idx += WPC * 32) sig_static[idx] = __ldg(&tab.sig[idx]);
  __syncthreads();
  if (n_sweeps > 0) core::build_lut_warp(L, sig_static, tab.T, lane);

  // Rows of R_i L_P, one lane per row.
  int32_t e_lane = 0;
  for (int r = lane; r < D; r += 32) {
    const uint32_t x = core::plane_field(init, W, r * D, D);
    const uint32_t z = core::plane_field(init + W, W, r * D, D);
    unsigned long long v = core::spread2(z) | (core::spread2(x) << 1);
    if (P == 1 || P == 2) v ^= (r & 1) ? 1ull : 2ull;
    if ((P == 2 || P == 3) && r == 0)
      v ^= 0x9999999999999999ull & ((2 * D >= 64) ? ~0ull : ((1ull << (2 * D)) - 1ull));
    rows[r] = v;
    best[r] = v;
    const unsigned long long zz = v & 0x5555555555555555ull, xx = (v >> 1) & 0x5555555555555555ull;
    e_lane += __popcll(xx & ~zz) * tab.W[2] + __popcll(xx & zz) * tab.W[3] + __popcll(zz & ~xx) * tab.W[1];
  }
  int32_t E = warp_sum(e_lane);
  int32_t E_best = E;
  __syncwarp();

  for (int t = 0; t < n_sweeps; ++t) {
    const uint32_t tt = (uint32_t)t;
#define XZZX_WPHASE(CC)                                               \
  {                                                                   \
    const int32_t d = warp_phase<D, CC>(rows, L, tt, c2, c3, K, lane); \
    E += warp_sum(d);                                                 \
    __syncwarp();                                                     \
    if (E < E_best) {                                                 \
      E_best = E;                                                     \
      for (int r = lane; r < D; r += 32) best[r] = rows[r];           \
    }                                                                 \
  }
    XZZX_WPHASE(0)
    XZZX_WPHASE(1)
    XZZX_WPHASE(2)
    XZZX_WPHASE(3)
#undef XZZX_WPHASE
    if (t + 1 < n_sweeps) {
      __syncwarp();
      core::build_lut_warp(L, sig_static, tab.T + (size_t)(t + 1) * tab.n_classes, lane);
    }
    __syncwarp();
  }

  if (!active) return;
  if (lane == 0) *out.best_E = E_best;
  if (lane == 0 && out.final_E) *out.final_E = E;
  // Rows -> planar words: each lane places its rows' bits, then the warp writes.
  auto emit = [&](const unsigned long long* src, uint32_t* dst) {
    for (int i = lane; i < 2 * W; i += 32) stage[i] = 0u;
    __syncwarp();
    for (int r = lane; r < D; r += 32) {
      const unsigned long long v = src[r];
      const uint64_t fz = core::gather2(v), fx = core::gather2(v >> 1);
      const int start = r * D, wi = start >> 5, off = start & 31;
      atomicOr(&stage[W + wi], (uint32_t)(fz << off));
      atomicOr(&stage[wi], (uint32_t)(fx << off));
      if (wi + 1 < W && off + D > 32) {
        atomicOr(&stage[W + wi + 1], (uint32_t)(fz >> (32 - off)));
        atomicOr(&stage[wi + 1], (uint32_t)(fx >> (32 - off)));
      }
    }
    __syncwarp();
    for (int i = lane; i < 2 * W; i += 32) dst[i] = stage[i];
    __syncwarp();
  };
  if (out.final_cfg) emit(rows, out.final_cfg);
  if (out.best_cfg) emit(best, out.best_cfg);
}

}  // namespace warpchain
}  // namespace xzzx
