// Device core of the annealing kernels: one CTA anneals NT chains.
//
// The plain per-distance kernel, the per-chunk kernels and the persistent
// multi-distance kernel all call anneal_cta<D, NT>, so every launch form runs
// the same instruction stream on the same state and gives identical results.
//
// State.  A chain lives in registers as one word per lattice row, two bits per
// qubit (bit 2c = Z bit, bit 2c+1 = X bit of column c): 32-bit rows for d <= 15,
// 64-bit rows up to d = 31.  The four corners of face (a, b) are then the
// 4-bit fields at bit 2b of rows a and a+1, and applying G_f is two XORs with
// fixed masks.
//
// Sweep.  Colours 0..3 in order (faces of one colour have disjoint supports,
// so their order inside a colour does not matter).  Inside a colour the loop
// runs over the face columns at run time and unrolls the rows, so register
// indices stay compile-time constants and the code stays small at any d.
//
// Acceptance.  An 8-bit corner signature indexes a per-sweep table of
// (dE, A): A = T[t][dE] for dE > 0 and A = 0 otherwise, so a move is accepted
// iff dE <= 0 or u < A.  Draws come four at a time from Philox blocks keyed by
// (colour, column, row group, sweep, chain); a block is computed only when some
// lane of the warp has a move with A > 0 in it, since with A = 0 the draw
// cannot change the outcome.  The table is rebuilt for the next sweep after the
// warp finishes a sweep, by the warp itself (one copy per warp), so warps
// never wait for each other.
//
// Minimum tracking.  The lowest energy and its rows are recorded at the start
// and after every colour phase (strict improvement), the rows in shared memory.
#pragma once

#include <type_traits>

#include "internal.h"
#include "philox.cuh"

namespace xzzx {
namespace core {

constexpr int kLutN = kSigRot;  // the rotated entries of the schedule's table

template <int D>
struct Shape {
  static constexpr bool kWide = 2 * D > 32;
  using Row = typename std::conditional<kWide, uint64_t, uint32_t>::type;
  static constexpr int kW = (D * D + 31) / 32;
  static constexpr int kThreads = kWide ? 128 : 256;
};

template <typename Row>
__device__ __forceinline__ uint32_t nib(Row x, uint32_t s) {
  return (uint32_t)(x >> s) & 0xFu;
}

// Bits [start, start+len) of a bit plane (len <= 31).
__device__ __forceinline__ uint32_t plane_field(const uint32_t* __restrict__ p, int words, int start, int len) {
  const int wi = start >> 5, off = start & 31;
  const uint32_t lo = p[wi];
  const uint32_t hi = (wi + 1 < words) ? p[wi + 1] : 0u;
  return __funnelshift_r(lo, hi, off) & ((1u << len) - 1u);
}

__device__ __forceinline__ uint64_t spread2(uint32_t v) {  // bit i -> bit 2i
  uint64_t x = v;
  x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
  x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
  x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
  x = (x | (x << 2)) & 0x3333333333333333ull;
  x = (x | (x << 1)) & 0x5555555555555555ull;
  return x;
}

__device__ __forceinline__ uint32_t gather2(uint64_t x) {  // bit 2i -> bit i
  x &= 0x5555555555555555ull;
  x = (x | (x >> 1)) & 0x3333333333333333ull;
  x = (x | (x >> 2)) & 0x0F0F0F0F0F0F0F0Full;
  x = (x | (x >> 4)) & 0x00FF00FF00FF00FFull;
  x = (x | (x >> 8)) & 0x0000FFFF0000FFFFull;
  x = (x | (x >> 16)) & 0x00000000FFFFFFFFull;
  return (uint32_t)x;
}

template <int D, typename Row>
__device__ __forceinline__ int32_t energy_of(const Row (&R)[D], const int32_t (&W)[4]) {
  int32_t nx = 0, ny = 0, nz = 0;
#pragma unroll
  for (int r = 0; r < D; ++r) {
    const uint64_t v = (uint64_t)R[r];
    const uint64_t z = v & 0x5555555555555555ull, x = (v >> 1) & 0x5555555555555555ull;
    ny += __popcll(x & z);
    nx += __popcll(x & ~z);
    nz += __popcll(z & ~x);
  }
  return nx * W[2] + ny * W[3] + nz * W[1];
}

// Planar configuration (x plane then z plane) -> rows.  For 5 <= d <= 15 the
// 2w words are first read with 8-byte vector loads (when the buffer allows
// it) and the row fields cut from registers.
template <int D, typename Row>
__device__ __forceinline__ void load_rows(const uint32_t* __restrict__ cfg, Row (&R)[D]) {
  constexpr int W = Shape<D>::kW;
  if constexpr (W <= 8 && D >= 5) {
    uint32_t w[2 * W];
    if ((reinterpret_cast<uintptr_t>(cfg) & 7u) == 0) {
      const uint2* v = reinterpret_cast<const uint2*>(cfg);
#pragma unroll
      for (int k = 0; k < W; ++k) {
        const uint2 t = __ldg(&v[k]);
        w[2 * k] = t.x;
        w[2 * k + 1] = t.y;
      }
    } else {
#pragma unroll
      for (int k = 0; k < 2 * W; ++k) w[k] = __ldg(&cfg[k]);
    }
#pragma unroll
    for (int r = 0; r < D; ++r) {
      const uint32_t x = plane_field(w, W, r * D, D);
      const uint32_t z = plane_field(w + W, W, r * D, D);
      R[r] = (Row)(spread2(z) | (spread2(x) << 1));
    }
  } else {
#pragma unroll
    for (int r = 0; r < D; ++r) {
      const uint32_t x = plane_field(cfg, W, r * D, D);
      const uint32_t z = plane_field(cfg + W, W, r * D, D);
      R[r] = (Row)(spread2(z) | (spread2(x) << 1));
    }
  }
}

// Rows -> planar configuration.
template <int D, typename Row>
__device__ __forceinline__ void store_rows(const Row (&R)[D], uint32_t* __restrict__ cfg) {
  constexpr int W = Shape<D>::kW;
  uint32_t px[W], pz[W];
#pragma unroll
  for (int j = 0; j < W; ++j) px[j] = pz[j] = 0u;
#pragma unroll
  for (int r = 0; r < D; ++r) {
    const uint64_t v = (uint64_t)R[r];
    const uint64_t fz = gather2(v), fx = gather2(v >> 1);
    const int start = r * D, wi = start >> 5, off = start & 31;
    pz[wi] |= (uint32_t)(fz << off);
    px[wi] |= (uint32_t)(fx << off);
    if (wi + 1 < W && off + D > 32) {
      pz[wi + 1] |= (uint32_t)(fz >> (32 - off));
      px[wi + 1] |= (uint32_t)(fx >> (32 - off));
    }
  }
#pragma unroll
  for (int j = 0; j < W; ++j) {
    cfg[j] = px[j];
    cfg[W + j] = pz[j];
  }
}

// One colour phase of one sweep.
template <int D, int C, typename Row>
__device__ __forceinline__ void colour_phase(Row (&R)[D], int32_t& E, const uint2* __restrict__ L, uint32_t t,
                                             uint32_t c2, uint32_t c3, const PhiloxKeys& K, uint32_t* err) {
  // Rows of this colour: a = 2j + AOFF; colour 0 ends with the bottom boundary
  // row a = d-1, colour 3 starts with the top boundary row a = -1.
  constexpr int NR = (C == 0 || C == 3) ? (D + 1) / 2 : (D - 1) / 2;
  constexpr int AOFF = (C == 1) ? 1 : (C == 3) ? -1 : 0;
  constexpr int IAOFF = (C == 1) ? 1 : 0;  // ia = (a+1)>>1 = j + IAOFF
  constexpr int NG = (NR - 1 + IAOFF) / 4 + 1;
  constexpr int PB = C >> 1;
  constexpr int NCB = (D - 1) / 2;

#pragma unroll 1
  for (int jb = 0; jb < NCB; ++jb) {
    const int b = 2 * jb + PB;
    const uint32_t s = 2u * (uint32_t)b;
    const uint32_t ib = (uint32_t)(b + 1) >> 1;
    const Row m_top = (Row)0x6u << s;  // X on TL, Z on TR
    const Row m_bot = (Row)0x9u << s;  // Z on BL, X on BR
    uint2 e[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      const int a = 2 * j + AOFF;
      uint32_t idx;
      if (C == 3 && j == 0) {
        idx = sig_base(kTop) + nib(R[0], s);            // BL | BR << 2
      } else if (C == 0 && j == NR - 1) {
        idx = sig_base(kBottom) + nib(R[D - 1], s);     // TL | TR << 2
      } else {
        const int a0 = a < 0 ? 0 : a;
        const int a1 = a + 1 > D - 1 ? D - 1 : a + 1;
        idx = nib(R[a0], s) | (nib(R[a1], s) << 4);     // TL | TR << 2 | BL << 4 | BR << 6
      }
      e[j] = XZZX_CHECK(err, idx < (uint32_t)kLutN && !injected(err, XZZX_DEVERR_BOUNDS)) ? L[idx] : make_uint2(0u, 0u);
    }
    uint4 r[NG];
#pragma unroll
    for (int g = 0; g < NG; ++g) {
      uint32_t need = 0;
#pragma unroll
      for (int j = 0; j < NR; ++j)
        if (((j + IAOFF) >> 2) == g) need |= e[j].y;
      r[g] = make_uint4(0u, 0u, 0u, 0u);
      if (__any_sync(0xFFFFFFFFu, need != 0u))
        r[g] = philox4x32_10(((uint32_t)C << 16) | (ib << 8) | (uint32_t)g, t, c2, c3, K);
    }
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      const int ia = j + IAOFF;
      const uint32_t u = lane_of(r[ia >> 2], ia & 3);
      const int32_t dE = (int32_t)e[j].x;
      const bool acc = (dE <= 0) | (u < e[j].y);
      if (acc) {
        E += dE;
        if (C == 3 && j == 0) {
          R[0] ^= m_bot;
        } else if (C == 0 && j == NR - 1) {
          R[D - 1] ^= m_top;
        } else {
          const int a = 2 * j + AOFF;
          const int a0 = a < 0 ? 0 : a;
          const int a1 = a + 1 > D - 1 ? D - 1 : a + 1;
          R[a0] ^= m_top;
          R[a1] ^= m_bot;
        }
      }
    }
  }

  if (C == 1 || C == 2) {
    // Boundary column: right (b = d-1: TL and BL) for colour 1, left (b = -1:
    // TR and BR) for colour 2, over the bulk rows of the colour.
    constexpr uint32_t sr = 2u * (uint32_t)(D - 1);
    constexpr uint32_t ibb = (C == 1) ? (uint32_t)(D >> 1) : 0u;
    uint2 e[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      const int a = 2 * j + AOFF;
      uint32_t idx;
      if (C == 1)  // TL | BL << 2
        idx = sig_base(kRight) + (((uint32_t)(R[a] >> sr) & 3u) | (((uint32_t)(R[a + 1] >> sr) & 3u) << 2));
      else  // TR | BR << 2
        idx = sig_base(kLeft) + (((uint32_t)R[a] & 3u) | (((uint32_t)R[a + 1] & 3u) << 2));
      e[j] = XZZX_CHECK(err, idx < (uint32_t)kLutN && !injected(err, XZZX_DEVERR_BOUNDS)) ? L[idx] : make_uint2(0u, 0u);
    }
    uint4 r[NG];
#pragma unroll
    for (int g = 0; g < NG; ++g) {
      uint32_t need = 0;
#pragma unroll
      for (int j = 0; j < NR; ++j)
        if (((j + IAOFF) >> 2) == g) need |= e[j].y;
      r[g] = make_uint4(0u, 0u, 0u, 0u);
      if (__any_sync(0xFFFFFFFFu, need != 0u))
        r[g] = philox4x32_10(((uint32_t)C << 16) | (ibb << 8) | (uint32_t)g, t, c2, c3, K);
    }
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      const int ia = j + IAOFF;
      const uint32_t u = lane_of(r[ia >> 2], ia & 3);
      const int32_t dE = (int32_t)e[j].x;
      const bool acc = (dE <= 0) | (u < e[j].y);
      if (acc) {
        E += dE;
        const int a = 2 * j + AOFF;
        if (C == 1) {
          R[a] ^= (Row)2u << sr;
          R[a + 1] ^= (Row)1u << sr;
        } else {
          R[a] ^= (Row)1u;
          R[a + 1] ^= (Row)2u;
        }
      }
    }
  }
}

// Per-sweep table: entry (dE, A) for every compact signature, built by one
// warp into its own copy from the CTA's static (dE, class) table.
__device__ __forceinline__ void build_lut_warp(uint2* __restrict__ dst, const int2* __restrict__ sig_static,
                                               const uint32_t* __restrict__ Trow, int lane) {
  for (int idx = lane; idx < kLutN; idx += 32) {
    const int2 s = sig_static[idx];
    const uint32_t A = s.y >= 0 ? __ldg(&Trow[s.y]) : 0u;
    dst[idx] = make_uint2((uint32_t)s.x, A);
  }
}

// Tables a CTA needs: per-sweep thresholds, signature table and qubit weights.
struct SweepTables {
  const uint32_t* T;
  const int2* sig;
  int n_sweeps, n_classes;
  int32_t W[4];
  uint32_t* err;  // the code's device error area (bounds checks of the checked build)
};

// Output pointers of one chain (already offset to it), or null.
struct ChainOut {
  int32_t* best_E;
  uint32_t* best_cfg;
  int32_t* final_E;
  uint32_t* final_cfg;
};

// Shared memory: the static (dE, class) table, one per-sweep table per warp,
// and the minimum-energy rows of every chain.
template <int D, int NT>
__host__ __device__ constexpr size_t smem_bytes() {
  return kLutN * sizeof(int2) + (size_t)(NT / 32) * kLutN * sizeof(uint2) +
         (size_t)D * NT * sizeof(typename Shape<D>::Row);
}

// Anneal one chain per thread; every thread of the CTA must call this (it
// contains barriers).  init: the chain's reference R_i (2w planar words);
// chain: global chain id (Philox counter); P: coset index of L_P; inactive
// threads run a copy of a real chain and write nothing.
template <int D, int NT>
__device__ __forceinline__ void anneal_cta(const uint32_t* __restrict__ init, uint64_t chain, int P, bool active,
                                           const ChainOut& out, const SweepTables& tab, const PhiloxKeys& K,
                                           uint8_t* smem) {
  using Row = typename Shape<D>::Row;
  constexpr int W = Shape<D>::kW;
  int2* sig_static = reinterpret_cast<int2*>(smem);                                     // [kLutN]
  uint2* lut_all = reinterpret_cast<uint2*>(smem + kLutN * sizeof(int2));               // [NT/32][kLutN]
  Row* best_rows = reinterpret_cast<Row*>(smem + kLutN * sizeof(int2) + (NT / 32) * kLutN * sizeof(uint2));
  const int tid = threadIdx.x, lane = tid & 31;
  uint2* L = lut_all + (tid >> 5) * kLutN;  // this warp's table
  const uint32_t c2 = (uint32_t)chain;
  const uint32_t c3 = kTagSA | ((uint32_t)(chain >> 32) << 8);
  const int n_sweeps = tab.n_sweeps;

  for (int idx = tid; idx < kLutN; idx += NT) sig_static[idx] = __ldg(&tab.sig[idx]);
  __syncthreads();  // the only CTA barrier: warps then sweep independently
  if (n_sweeps > 0) build_lut_warp(L, sig_static, tab.T, lane);

  Row R[D];
  load_rows<D, Row>(init, R);
  // Multiply by L_P: L_X = column 0 (X on even rows, Z on odd rows), L_Z = row 0
  // (Z on even columns, X on odd columns).
  if (P == 1 || P == 2) {
#pragma unroll
    for (int r = 0; r < D; ++r) R[r] ^= (Row)((r & 1) ? 1u : 2u);
  }
  if (P == 2 || P == 3) {
    const uint64_t mz = 0x9999999999999999ull & ((2 * D >= 64) ? ~0ull : ((1ull << (2 * D)) - 1ull));
    R[0] ^= (Row)mz;
  }
  int32_t W4[4] = {tab.W[0], tab.W[1], tab.W[2], tab.W[3]};
  int32_t E = energy_of<D, Row>(R, W4);
  int32_t E_best = E;
#pragma unroll
  for (int r = 0; r < D; ++r) best_rows[r * NT + tid] = R[r];
  __syncwarp();

  for (int t = 0; t < n_sweeps; ++t) {
    const uint32_t tt = (uint32_t)t;
#define XZZX_PHASE(CC)                                                              \
  colour_phase<D, CC, Row>(R, E, L, tt, c2, c3, K, tab.err);                        \
  if (E < E_best) {                                                                 \
    E_best = E;                                                                     \
    _Pragma("unroll") for (int r = 0; r < D; ++r) best_rows[r * NT + tid] = R[r];   \
  }
    XZZX_PHASE(0)
    XZZX_PHASE(1)
    XZZX_PHASE(2)
    XZZX_PHASE(3)
#undef XZZX_PHASE
    if (t + 1 < n_sweeps) {  // next sweep's thresholds, once every lane is done with these
      __syncwarp();
      build_lut_warp(L, sig_static, tab.T + (size_t)(t + 1) * tab.n_classes, lane);
      __syncwarp();
    }
  }

  if (!active) return;
  *out.best_E = E_best;
  if (out.final_E) *out.final_E = E;
  if (out.final_cfg) store_rows<D, Row>(R, out.final_cfg);
  if (out.best_cfg) {
#pragma unroll
    for (int r = 0; r < D; ++r) R[r] = best_rows[r * NT + tid];
    store_rows<D, Row>(R, out.best_cfg);
  }
}

}  // namespace core
}  // namespace xzzx
