// Device core of the annealing kernels: one CTA anneals NT chains.
//
// The plain per-distance kernel, the per-chunk kernels and the persistent
// multi-distance kernel all call anneal_cta<D, NT>, so every launch form runs
// the same instruction stream on the same state and gives identical results.
//
// State, d > 15 ("rows").  A chain lives in registers as one 64-bit word per
// lattice row, two bits per qubit (bit 2c = Z bit, bit 2c+1 = X bit of column
// c).  The four corners of face (a, b) are then the 4-bit fields at bit 2b of
// rows a and a+1, and applying G_f is two XORs with fixed masks.
//
// State, d <= 15 ("pairs").  Two lattice rows share one pair word, four bits
// per column: bits [4c, 4c+2) hold (z, x) of column c of the first row, bits
// [4c+2, 4c+4) those of the second row; a pair word takes two 32-bit registers
// for d >= 9.  The even layout pairs rows (2j, 2j+1), the odd layout rows
// (2j-1, 2j) (row -1 and row d are empty).  Faces of colours 0 and 2 sit on
// even rows a, faces of colours 1 and 3 on odd ones, so in the layout of its
// colour the 8-bit signature of face (a, b) is one byte of one pair word, at
// bit 4b, and a move is one XOR.  The layout changes at each colour boundary
// (two shifts and a masked merge per register); the minimum is snapshotted in
// the even layout.
//
// Sweep.  Colours 0..3 in order (faces of one colour have disjoint supports,
// so their order inside a colour does not matter).  Inside a colour the loop
// runs over the face columns at run time and unrolls the rows, so register
// indices stay compile-time constants and the code stays small at any d (pair
// path: one loop per 32-bit register with the register-edge columns peeled
// for d <= 11, one loop over 64-bit pair words for d = 13, 15).
//
// Acceptance.  The corner signature indexes a per-sweep table of (dE, A): A =
// T[t][dE] for dE > 0 and A = 0 otherwise, so a move is accepted iff dE <= 0
// or u < A.  Draws come four at a time from Philox blocks keyed by (colour,
// column, row group, sweep, chain); a block is computed only when some lane of
// the warp has a move with A > 0 in it, since with A = 0 the draw cannot change
// the outcome.  The parts of a block's first two rounds that depend only on the
// chain or the sweep are computed once per chain or sweep.  The table is
// rebuilt for the next sweep after the warp finishes a sweep, by the warp
// itself (one copy per warp), so warps never wait for each other.  In the pair
// path each warp's table sits in its own 4 KB-aligned slot of shared memory,
// so a table address is the slot base OR'd with the byte offset cut from the
// pair word.
//
// Minimum tracking.  The lowest energy and its configuration are recorded at
// the start and after every colour phase (strict improvement), in shared
// memory.
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

// The annealing draws of one chain: Philox4x32-10 blocks with counter
// (c0, t, c2, c3), c0 = colour<<16 | column<<8 | row group, t the sweep, (c2,
// c3) the chain.  Round 0 multiplies c2 (chain-constant) and round 1 multiplies
// round 0's first output word, which depends only on (chain, sweep); both
// products and the XORs with constants are taken once per chain or per sweep,
// leaving one wide multiply in each of the first two rounds per block.  block()
// returns exactly philox4x32_10(c0, t, c2, c3, K).
struct SaDraws {
  uint32_t lo1, B, X1, hi1k;  // per chain
  uint32_t lo0_1, Y1;         // per sweep

  __device__ __forceinline__ void init(uint32_t c2, uint32_t c3, const PhiloxKeys& K) {
    const uint64_t p = (uint64_t)c2 * 0xCD9E8D57u;
    lo1 = (uint32_t)p;
    B = c3 ^ K.k1[0];
    X1 = lo1 ^ K.k0[1];
    hi1k = (uint32_t)(p >> 32) ^ K.k0[0];
  }
  __device__ __forceinline__ void sweep(uint32_t t, const PhiloxKeys& K) {
    const uint64_t q = (uint64_t)(hi1k ^ t) * 0xD2511F53u;  // round 1: c0 = hi(c2 M1) ^ t ^ k0[0]
    lo0_1 = (uint32_t)q;
    Y1 = (uint32_t)(q >> 32) ^ K.k1[1];
  }
  __device__ __forceinline__ uint4 block(uint32_t c0, const PhiloxKeys& K) const {
    const uint64_t p0 = (uint64_t)c0 * 0xD2511F53u;        // round 0
    const uint32_t r0_2 = (uint32_t)(p0 >> 32) ^ B, r0_3 = (uint32_t)p0;
    const uint64_t p1 = (uint64_t)r0_2 * 0xCD9E8D57u;      // round 1
    uint32_t a0 = (uint32_t)(p1 >> 32) ^ X1, a1 = (uint32_t)p1, a2 = Y1 ^ r0_3, a3 = lo0_1;
#pragma unroll
    for (int r = 2; r < 10; ++r) {
      const uint64_t q0 = (uint64_t)a0 * 0xD2511F53u;
      const uint64_t q1 = (uint64_t)a2 * 0xCD9E8D57u;
      const uint32_t n0 = (uint32_t)(q1 >> 32) ^ a1 ^ K.k0[r];
      const uint32_t n2 = (uint32_t)(q0 >> 32) ^ a3 ^ K.k1[r];
      a1 = (uint32_t)q1;
      a3 = (uint32_t)q0;
      a0 = n0;
      a2 = n2;
    }
    return make_uint4(a0, a1, a2, a3);
  }
};

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

// One colour phase of one sweep (row layout, d > 15).
template <int D, int C, typename Row>
__device__ __forceinline__ void colour_phase(Row (&R)[D], int32_t& E, const uint2* __restrict__ L, const SaDraws& dr,
                                             const PhiloxKeys& K, uint32_t* err) {
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
    // Group by group (the faces that share one Philox block): a group's
    // lookups, draw and moves finish before the next group's lookups.  Against
    // loading the whole column first this is 2% faster at d = 17, 21 and lets
    // d = 29, 31 fit 128 registers without spills.
#pragma unroll
    for (int g = 0; g < NG; ++g) {
      const int j0 = g == 0 ? 0 : 4 * g - IAOFF, j1 = (4 * (g + 1) - IAOFF) < NR ? 4 * (g + 1) - IAOFF : NR;
      uint2 e[4];
      uint32_t need = 0;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = j0 + q;
        if (j >= j1) continue;
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
        e[q] = XZZX_CHECK(err, idx < (uint32_t)kLutN && !injected(err, XZZX_DEVERR_BOUNDS)) ? L[idx]
                                                                                           : make_uint2(0u, 0u);
        need |= e[q].y;
      }
      uint4 r = make_uint4(0u, 0u, 0u, 0u);
      if (__any_sync(0xFFFFFFFFu, need != 0u)) r = dr.block(((uint32_t)C << 16) | (ib << 8) | (uint32_t)g, K);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = j0 + q;
        if (j >= j1) continue;
        const int ia = j + IAOFF;
        const uint32_t u = lane_of(r, ia & 3);
        const int32_t dE = (int32_t)e[q].x;
        const bool acc = (dE <= 0) | (u < e[q].y);
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
        r[g] = dr.block(((uint32_t)C << 16) | (ibb << 8) | (uint32_t)g, K);
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

// ---------------------------------------------------------------------------
// Pair layout (d <= 15).
// ---------------------------------------------------------------------------

template <int D>
struct PairShape {
  static constexpr int H = (D + 1) / 2;          // pair words
  static constexpr int NW = (4 * D + 31) / 32;   // 32-bit registers per pair word
};

// Per-warp table of the pair path, indexed by the pair signature: 256 bulk
// entries (TL | BL << 2 | TR << 4 | BR << 6), 64 for the top boundary (BL | BR
// << 4), 64 for the bottom (TL | TR << 4), 16 for the left (TR | BR << 2), 16
// for the right (TL | BL << 2).
constexpr int kPairTop = 256, kPairBottom = 320, kPairLeft = 384, kPairRight = 400, kPairLut = 416;
constexpr uint32_t kPairSlot = 4096;  // bytes of one warp's table slot (4 KB aligned)

// Entry of the schedule's rotated signature table for pair index p.
__device__ __forceinline__ int pair_sig_source(int p) {
  if (p < kPairTop) {
    const int TL = p & 3, BL = (p >> 2) & 3, TR = (p >> 4) & 3, BR = (p >> 6) & 3;
    return TL | (TR << 2) | (BL << 4) | (BR << 6);
  }
  if (p < kPairBottom) return sig_base(kTop) + (((p - kPairTop) & 3) | ((((p - kPairTop) >> 4) & 3) << 2));
  if (p < kPairLeft) return sig_base(kBottom) + (((p - kPairBottom) & 3) | ((((p - kPairBottom) >> 4) & 3) << 2));
  if (p < kPairRight) return sig_base(kLeft) + (p - kPairLeft);
  return sig_base(kRight) + (p - kPairRight);
}

__device__ __forceinline__ uint64_t spread_pairs(uint32_t v) {  // 2-bit field i -> bits 4i, 4i+1
  uint64_t x = v;
  x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
  x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
  x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
  x = (x | (x << 2)) & 0x3333333333333333ull;
  return x;
}

__device__ __forceinline__ uint32_t gather_pairs(uint64_t x) {  // bits 4i, 4i+1 -> 2-bit field i
  x &= 0x3333333333333333ull;
  x = (x | (x >> 2)) & 0x0F0F0F0F0F0F0F0Full;
  x = (x | (x >> 4)) & 0x00FF00FF00FF00FFull;
  x = (x | (x >> 8)) & 0x0000FFFF0000FFFFull;
  x = (x | (x >> 16)) & 0x00000000FFFFFFFFull;
  return (uint32_t)x;
}

// Rows (two bits per qubit) -> even-layout pair words, and back.  Columns
// 0..15 of a row fill registers 0 and 1 of its pair word, columns 16..30
// registers 2 and 3.
template <int D, typename Row>
__device__ __forceinline__ void rows_to_pairs(const Row (&R)[D], uint32_t (&P)[PairShape<D>::H][PairShape<D>::NW]) {
  constexpr int NW = PairShape<D>::NW;
#pragma unroll
  for (int j = 0; j < PairShape<D>::H; ++j) {
    const uint64_t r0 = (uint64_t)R[2 * j], r1 = 2 * j + 1 < D ? (uint64_t)R[2 * j + 1] : 0ull;
    const uint64_t lo = spread_pairs((uint32_t)r0) | (spread_pairs((uint32_t)r1) << 2);
    const uint64_t hi = spread_pairs((uint32_t)(r0 >> 32)) | (spread_pairs((uint32_t)(r1 >> 32)) << 2);
#pragma unroll
    for (int k = 0; k < NW; ++k) P[j][k] = (uint32_t)((k < 2 ? lo : hi) >> (32 * (k & 1)));
  }
}
template <int D, typename Row>
__device__ __forceinline__ void pairs_to_rows(const uint32_t (&P)[PairShape<D>::H][PairShape<D>::NW], Row (&R)[D]) {
  constexpr int NW = PairShape<D>::NW;
#pragma unroll
  for (int j = 0; j < PairShape<D>::H; ++j) {
    const uint64_t lo = (uint64_t)P[j][0] | (NW > 1 ? (uint64_t)P[j][1] << 32 : 0ull);
    const uint64_t hi = (NW > 2 ? (uint64_t)P[j][2] : 0ull) | (NW > 3 ? (uint64_t)P[j][3] << 32 : 0ull);
    R[2 * j] = (Row)((uint64_t)gather_pairs(lo) | ((uint64_t)gather_pairs(hi) << 32));
    if (2 * j + 1 < D) R[2 * j + 1] = (Row)((uint64_t)gather_pairs(lo >> 2) | ((uint64_t)gather_pairs(hi >> 2) << 32));
  }
}

// Even layout -> odd layout: Q_j takes row 2j-1 (upper slot of P_{j-1}) as
// its first row and row 2j (lower slot of P_j) as its second.
template <int D>
__device__ __forceinline__ void even_to_odd(uint32_t (&P)[PairShape<D>::H][PairShape<D>::NW]) {
  constexpr int H = PairShape<D>::H, NW = PairShape<D>::NW;
#pragma unroll
  for (int j = H - 1; j >= 0; --j)
#pragma unroll
    for (int k = 0; k < NW; ++k) {
      const uint32_t first = j > 0 ? (P[j - 1][k] >> 2) : 0u;
      P[j][k] = (first & 0x33333333u) | ((P[j][k] << 2) & 0xCCCCCCCCu);
    }
}
// Odd layout -> even layout: P_j takes row 2j (upper slot of Q_j) and row
// 2j+1 (lower slot of Q_{j+1}).
template <int D>
__device__ __forceinline__ void odd_to_even(uint32_t (&P)[PairShape<D>::H][PairShape<D>::NW]) {
  constexpr int H = PairShape<D>::H, NW = PairShape<D>::NW;
#pragma unroll
  for (int j = 0; j < H; ++j)
#pragma unroll
    for (int k = 0; k < NW; ++k) {
      const uint32_t second = j + 1 < H ? (P[j + 1][k] << 2) : 0u;
      P[j][k] = ((P[j][k] >> 2) & 0x33333333u) | (second & 0xCCCCCCCCu);
    }
}

// Where a column's faces sit in their pair words, as kind | register << 4.
// kIn: inside the register at bit s >= 4; kAt0: at bit 0 of the register (b =
// 8r); kAcross: bits 28..35 across the register and the next (b = 8r + 7).
enum PairKind { kIn = 0, kAt0 = 1, kAcross = 2 };

// Byte offset in the warp's table of the signature at bit s (+UP) of w.
template <int NW, int MODE, int UP>
__device__ __forceinline__ uint32_t pair_offset(const uint32_t (&w)[NW], uint32_t s, uint32_t mask) {
  constexpr int KIND = MODE & 15, RG = MODE >> 4;
  if constexpr (KIND == kIn) return (w[RG] >> (s + UP - 3)) & mask;
  else if constexpr (KIND == kAt0) return (w[RG] << (3 - UP)) & mask;
  else return __funnelshift_r(w[RG], w[RG + 1 < NW ? RG + 1 : RG], 28 + UP - 3) & mask;
}

template <int NW, int MODE>
__device__ __forceinline__ void pair_flip(uint32_t (&w)[NW], uint32_t m, uint32_t s) {
  constexpr int KIND = MODE & 15, RG = MODE >> 4;
  if constexpr (KIND == kIn) {
    w[RG] ^= m << s;
  } else if constexpr (KIND == kAt0) {
    w[RG] ^= m;
  } else {
    w[RG] ^= m << 28;
    w[RG + 1 < NW ? RG + 1 : RG] ^= m >> 4;
  }
}

__device__ __forceinline__ uint2 lds_u2(uint32_t addr) {
  uint2 v;
  asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(addr));
  return v;
}
__device__ __forceinline__ void sts_u2(uint32_t addr, uint2 v) {
  asm volatile("st.shared.v2.u32 [%0], {%1, %2};" ::"r"(addr), "r"(v.x), "r"(v.y));
}

// Table entry at shared address a inside the slot starting at Lb.
__device__ __forceinline__ uint2 pair_entry(uint32_t a, uint32_t Lb, uint32_t* err) {
  return XZZX_CHECK(err, a - Lb <= kPairSlot - 8u && !injected(err, XZZX_DEVERR_BOUNDS)) ? lds_u2(a)
                                                                                         : make_uint2(0u, 0u);
}

// One column of faces of colour C at column b (bit s of its register, as MODE
// says).  Lb: the warp's table slot.
template <int D, int C, int MODE>
__device__ __forceinline__ void pair_column(uint32_t (&P)[PairShape<D>::H][PairShape<D>::NW], int32_t& E,
                                            uint32_t Lb, const SaDraws& dr, const PhiloxKeys& K, int b, uint32_t s,
                                            uint32_t* err) {
  constexpr int H = PairShape<D>::H, NW = PairShape<D>::NW;
  constexpr int NR = (C == 0 || C == 3) ? H : H - 1;
  constexpr int JOFF = (C == 1) ? 1 : 0;   // colour 1: face row a = 2j+1 is odd pair j+1
  constexpr int IAOFF = (C == 1) ? 1 : 0;  // ia = (a+1)>>1 = j + IAOFF
  constexpr int NG = (NR - 1 + IAOFF) / 4 + 1;
  const uint32_t ib = (uint32_t)(b + 1) >> 1;
  uint2 e[NR];
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    uint32_t a;
    if (C == 3 && j == 0)  // top boundary (a = -1): second-row slots of odd pair 0
      a = pair_offset<NW, MODE, 2>(P[0], s, 0x198u) | (Lb + kPairTop * 8);
    else if (C == 0 && j == NR - 1)  // bottom boundary (a = d-1): first-row slots
      a = pair_offset<NW, MODE, 0>(P[j], s, 0x198u) | (Lb + kPairBottom * 8);
    else
      a = pair_offset<NW, MODE, 0>(P[j + JOFF], s, 0x7F8u) | Lb;
    e[j] = pair_entry(a, Lb, err);
  }
  uint4 r[NG];
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    uint32_t need = 0;
#pragma unroll
    for (int j = 0; j < NR; ++j)
      if (((j + IAOFF) >> 2) == g) need |= e[j].y;
    r[g] = make_uint4(0u, 0u, 0u, 0u);
    if (__any_sync(0xFFFFFFFFu, need != 0u)) r[g] = dr.block(((uint32_t)C << 16) | (ib << 8) | (uint32_t)g, K);
  }
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    const int ia = j + IAOFF;
    const uint32_t u = lane_of(r[ia >> 2], ia & 3);
    const int32_t dE = (int32_t)e[j].x;
    if ((dE <= 0) | (u < e[j].y)) {
      E += dE;
      if (C == 3 && j == 0) pair_flip<NW, MODE>(P[0], 0x84u, s);               // Z on BL, X on BR
      else if (C == 0 && j == NR - 1) pair_flip<NW, MODE>(P[j], 0x12u, s);     // X on TL, Z on TR
      else pair_flip<NW, MODE>(P[j + JOFF], 0x96u, s);                         // X TL, Z BL, Z TR, X BR
    }
  }
}

// The columns of colour C whose bytes start in register RG of the pair
// words: b = 8RG at bit 0 (even-b colours), then the columns inside the
// register, then b = 8RG + 7 across registers RG and RG + 1 (odd-b colours).
template <int D, int C, int RG>
__device__ __forceinline__ void pair_register_columns(uint32_t (&P)[PairShape<D>::H][PairShape<D>::NW], int32_t& E,
                                                      uint32_t Lb, const SaDraws& dr, const PhiloxKeys& K,
                                                      uint32_t* err) {
  constexpr int NW = PairShape<D>::NW;
  if constexpr (RG < NW) {
    constexpr int PB = C >> 1;
    constexpr int BMAX = PB + 2 * ((D - 1) / 2 - 1);  // the colour's last bulk column
    constexpr int B0 = 8 * RG;
    if constexpr (PB == 0 && B0 <= BMAX) pair_column<D, C, kAt0 | (RG << 4)>(P, E, Lb, dr, K, B0, 0u, err);
    constexpr int LO = B0 + (PB == 0 ? 2 : 1);
    constexpr int HI = (B0 + 6 - PB) < BMAX ? (B0 + 6 - PB) : BMAX;
#pragma unroll 1
    for (int b = LO; b <= HI; b += 2)
      pair_column<D, C, kIn | (RG << 4)>(P, E, Lb, dr, K, b, 4u * (uint32_t)(b - B0), err);
    if constexpr (PB == 1 && B0 + 7 <= BMAX && RG + 1 < NW)
      pair_column<D, C, kAcross | (RG << 4)>(P, E, Lb, dr, K, B0 + 7, 28u, err);
    pair_register_columns<D, C, RG + 1>(P, E, Lb, dr, K, err);
  }
}

// Bits [sh, sh + 32) of a pair word (zeros above it), sh < 64.
template <int NW>
__device__ __forceinline__ uint32_t pair_bits(const uint32_t (&w)[NW], uint32_t sh) {
  if constexpr (NW == 1) return w[0] >> sh;
  else return (uint32_t)((((uint64_t)w[1] << 32) | w[0]) >> sh);
}

// One column of faces of colour C at column b >= 1 of the pair words (two
// registers at most), the column a run-time value.
template <int D, int C>
__device__ __forceinline__ void pair_column_rt(uint32_t (&P)[PairShape<D>::H][PairShape<D>::NW], int32_t& E,
                                               uint32_t Lb, const SaDraws& dr, const PhiloxKeys& K, int b,
                                               uint32_t* err) {
  constexpr int H = PairShape<D>::H, NW = PairShape<D>::NW;
  static_assert(NW <= 2, "pair words of at most two registers");
  constexpr int NR = (C == 0 || C == 3) ? H : H - 1;
  constexpr int JOFF = (C == 1) ? 1 : 0;
  constexpr int IAOFF = (C == 1) ? 1 : 0;
  constexpr int NG = (NR - 1 + IAOFF) / 4 + 1;
  const uint32_t ib = (uint32_t)(b + 1) >> 1;
  const uint32_t s = 4u * (uint32_t)b;
  uint2 e[NR];
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    uint32_t a;
    if (C == 3 && j == 0)
      a = (pair_bits<NW>(P[0], s - 1u) & 0x198u) | (Lb + kPairTop * 8);
    else if (C == 0 && j == NR - 1)
      a = (pair_bits<NW>(P[j], s - 3u) & 0x198u) | (Lb + kPairBottom * 8);
    else
      a = (pair_bits<NW>(P[j + JOFF], s - 3u) & 0x7F8u) | Lb;
    e[j] = pair_entry(a, Lb, err);
  }
  uint4 r[NG];
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    uint32_t need = 0;
#pragma unroll
    for (int j = 0; j < NR; ++j)
      if (((j + IAOFF) >> 2) == g) need |= e[j].y;
    r[g] = make_uint4(0u, 0u, 0u, 0u);
    if (__any_sync(0xFFFFFFFFu, need != 0u)) r[g] = dr.block(((uint32_t)C << 16) | (ib << 8) | (uint32_t)g, K);
  }
  using M = typename std::conditional<NW == 1, uint32_t, uint64_t>::type;
  const M m_bulk = (M)0x96u << s, m_top = (M)0x84u << s, m_bottom = (M)0x12u << s;
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    const int ia = j + IAOFF;
    const uint32_t u = lane_of(r[ia >> 2], ia & 3);
    const int32_t dE = (int32_t)e[j].x;
    if ((dE <= 0) | (u < e[j].y)) {
      E += dE;
      const int row = (C == 3 && j == 0) ? 0 : (C == 0 && j == NR - 1) ? j : j + JOFF;
      const M m = (C == 3 && j == 0) ? m_top : (C == 0 && j == NR - 1) ? m_bottom : m_bulk;
      P[row][0] ^= (uint32_t)m;
      if constexpr (NW == 2) P[row][1] ^= (uint32_t)((uint64_t)m >> 32);
    }
  }
}

// The bulk columns of colour C for d >= 13: b = 0 (even-b colours) with its
// bits at the bottom of register 0, then every other column in one run-time
// loop over 64-bit pair words.  Against the per-register form this costs
// about one instruction per column for the shifted masks but cuts the sweep
// body several-fold, which pays once the body outgrows instruction fetch
// (d = 13, 15); at d <= 11 the per-register form is faster.
template <int D, int C>
__device__ __forceinline__ void pair_bulk_columns(uint32_t (&P)[PairShape<D>::H][PairShape<D>::NW], int32_t& E,
                                                  uint32_t Lb, const SaDraws& dr, const PhiloxKeys& K,
                                                  uint32_t* err) {
  constexpr int PB = C >> 1;
  constexpr int BMAX = PB + 2 * ((D - 1) / 2 - 1);  // the colour's last bulk column
  if constexpr (PB == 0) pair_column<D, C, kAt0>(P, E, Lb, dr, K, 0, 0u, err);
#pragma unroll 1
  for (int b = PB == 0 ? 2 : 1; b <= BMAX; b += 2) pair_column_rt<D, C>(P, E, Lb, dr, K, b, err);
}

// One colour phase of one sweep (pair layout: even for colours 0 and 2, odd
// for 1 and 3).
template <int D, int C>
__device__ __forceinline__ void pair_phase(uint32_t (&P)[PairShape<D>::H][PairShape<D>::NW], int32_t& E, uint32_t Lb,
                                           const SaDraws& dr, const PhiloxKeys& K, uint32_t* err) {
  constexpr int H = PairShape<D>::H;
  if constexpr (D >= 13) pair_bulk_columns<D, C>(P, E, Lb, dr, K, err);
  else pair_register_columns<D, C, 0>(P, E, Lb, dr, K, err);
  if constexpr (C == 1 || C == 2) {
    // Boundary column: right (b = d-1: TL and BL) for colour 1, left (b = -1:
    // TR and BR) for colour 2, over the bulk rows of the colour.
    constexpr int NR = H - 1;
    constexpr int IAOFF = (C == 1) ? 1 : 0;
    constexpr int JOFF = (C == 1) ? 1 : 0;
    constexpr int NG = (NR - 1 + IAOFF) / 4 + 1;
    constexpr uint32_t ibb = (C == 1) ? (uint32_t)(D >> 1) : 0u;
    constexpr int RB = 4 * (D - 1);
    constexpr int RW = RB >> 5, RS = RB & 31;
    uint2 e[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      uint32_t a;
      if constexpr (C == 1) {
        if constexpr (RS >= 3) a = ((P[j + JOFF][RW] >> (RS - 3)) & 0x78u) | (Lb + kPairRight * 8);
        else a = ((P[j + JOFF][RW] << (3 - RS)) & 0x78u) | (Lb + kPairRight * 8);
      } else {
        a = ((P[j][0] << 3) & 0x78u) | (Lb + kPairLeft * 8);
      }
      e[j] = pair_entry(a, Lb, err);
    }
    uint4 r[NG];
#pragma unroll
    for (int g = 0; g < NG; ++g) {
      uint32_t need = 0;
#pragma unroll
      for (int j = 0; j < NR; ++j)
        if (((j + IAOFF) >> 2) == g) need |= e[j].y;
      r[g] = make_uint4(0u, 0u, 0u, 0u);
      if (__any_sync(0xFFFFFFFFu, need != 0u)) r[g] = dr.block(((uint32_t)C << 16) | (ibb << 8) | (uint32_t)g, K);
    }
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      const int ia = j + IAOFF;
      const uint32_t u = lane_of(r[ia >> 2], ia & 3);
      const int32_t dE = (int32_t)e[j].x;
      if ((dE <= 0) | (u < e[j].y)) {
        E += dE;
        if constexpr (C == 1) P[j + JOFF][RW] ^= 0x6u << RS;  // X on TL, Z on BL
        else P[j][0] ^= 0x9u;                                 // Z on TR, X on BR
      }
    }
  }
}

// Lists, in index order, the entries of a static (dE, class) table whose
// threshold changes from sweep to sweep (class >= 0) as index << 16 | class;
// run by one full warp.  Returns the count.
__device__ __forceinline__ int list_threshold_entries(const int2* __restrict__ sig, int n, uint32_t* __restrict__ upd,
                                                      int lane) {
  int count = 0;
  for (int base = 0; base < n; base += 32) {
    const int idx = base + lane;
    const int cls = idx < n ? sig[idx].y : -1;
    const uint32_t m = __ballot_sync(0xFFFFFFFFu, cls >= 0);
    if (cls >= 0) upd[count + __popc(m & ((1u << lane) - 1u))] = ((uint32_t)idx << 16) | (uint32_t)cls;
    count += __popc(m);
  }
  return count;
}

__device__ __forceinline__ void sts_u32(uint32_t addr, uint32_t v) {
  asm volatile("st.shared.u32 [%0], %1;" ::"r"(addr), "r"(v));
}

// Pair table of one warp (slot at shared address Lb) for the first sweep, in
// full, from the CTA's static (dE, class) table in pair order.
__device__ __forceinline__ void build_lut_pair(uint32_t Lb, const int2* __restrict__ sig_pair,
                                               const uint32_t* __restrict__ Trow, int lane) {
  for (int idx = lane; idx < kPairLut; idx += 32) {
    const int2 s = sig_pair[idx];
    const uint32_t A = s.y >= 0 ? __ldg(&Trow[s.y]) : 0u;
    sts_u2(Lb + 8u * (uint32_t)idx, make_uint2((uint32_t)s.x, A));
  }
}

// Later sweeps only change the thresholds of the entries with dE > 0: upd
// lists them as index << 16 | class (n_upd entries).
__device__ __forceinline__ void update_lut_pair(uint32_t Lb, const uint32_t* __restrict__ upd, int n_upd,
                                                const uint32_t* __restrict__ Trow, int lane) {
  for (int k = lane; k < n_upd; k += 32) {
    const uint32_t v = upd[k];
    sts_u32(Lb + 8u * (v >> 16) + 4u, __ldg(&Trow[v & 0xFFFFu]));
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

// Shared memory of the row path: the static (dE, class) table, one per-sweep
// table per warp, the list of entries whose threshold changes per sweep, and
// the minimum-energy rows of every chain.
template <int D, int NT>
__host__ __device__ constexpr size_t smem_rows() {
  return kLutN * sizeof(int2) + (size_t)(NT / 32) * kLutN * sizeof(uint2) + kLutN * sizeof(uint32_t) + 16 +
         (size_t)D * NT * sizeof(typename Shape<D>::Row);
}

// Shared memory of the pair path: 4 KB of alignment slack, one 4 KB table slot
// per warp, the static table in pair order and the minimum-energy pair words
// of every chain.
template <int D, int NT>
__host__ __device__ constexpr size_t smem_pairs() {
  return kPairSlot + (size_t)(NT / 32) * kPairSlot + kPairLut * sizeof(int2) + kPairLut * sizeof(uint32_t) + 16 +
         (size_t)PairShape<D>::H * PairShape<D>::NW * NT * sizeof(uint32_t);
}

// Largest distance annealed in the pair layout (the row layout takes the rest).
constexpr int kPairMaxD = 15;

template <int D, int NT>
__host__ __device__ constexpr size_t smem_bytes() {
  return D <= kPairMaxD ? smem_pairs<D, NT>() : smem_rows<D, NT>();
}

// Row path (d > 15).  Arguments as anneal_cta.
template <int D, int NT, int U>
__device__ __forceinline__ void anneal_cta_rows(const uint32_t* __restrict__ init, uint64_t chain, int P, bool active,
                                                const ChainOut& out, const SweepTables& tab, const PhiloxKeys& K,
                                                uint8_t* smem) {
  using Row = typename Shape<D>::Row;
  int2* sig_static = reinterpret_cast<int2*>(smem);                                     // [kLutN]
  uint2* lut_all = reinterpret_cast<uint2*>(sig_static + kLutN);                        // [NT/32][kLutN]
  uint32_t* upd = reinterpret_cast<uint32_t*>(lut_all + (NT / 32) * kLutN);             // [kLutN]
  int* n_upd_s = reinterpret_cast<int*>(upd + kLutN);                                   // [4]
  Row* best_rows = reinterpret_cast<Row*>(n_upd_s + 4);
  const int tid = threadIdx.x, lane = tid & 31;
  uint2* L = lut_all + (tid >> 5) * kLutN;  // this warp's table
  SaDraws dr;
  dr.init((uint32_t)chain, kTagSA | ((uint32_t)(chain >> 32) << 8), K);
  const int n_sweeps = tab.n_sweeps;

  for (int idx = tid; idx < kLutN; idx += NT) sig_static[idx] = __ldg(&tab.sig[idx]);
  __syncthreads();
  if (tid < 32) {  // the entries whose threshold changes from sweep to sweep
    const int n = list_threshold_entries(sig_static, kLutN, upd, tid);
    if (tid == 0) n_upd_s[0] = n;
  }
  __syncthreads();  // the last CTA barrier: warps then sweep independently
  const int n_upd = n_upd_s[0];
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

#pragma unroll U
  for (int t = 0; t < n_sweeps; ++t) {
    dr.sweep((uint32_t)t, K);
#define XZZX_PHASE(CC)                                                              \
  colour_phase<D, CC, Row>(R, E, L, dr, K, tab.err);                                \
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
      const uint32_t* Trow = tab.T + (size_t)(t + 1) * tab.n_classes;
      for (int k = lane; k < n_upd; k += 32) {  // only the thresholds of the dE > 0 entries change
        const uint32_t v = upd[k];
        L[v >> 16].y = __ldg(&Trow[v & 0xFFFFu]);
      }
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

// Pair path.  Arguments as anneal_cta.
template <int D, int NT, int U>
__device__ __forceinline__ void anneal_cta_pairs(const uint32_t* __restrict__ init, uint64_t chain, int P_coset,
                                                 bool active, const ChainOut& out, const SweepTables& tab,
                                                 const PhiloxKeys& K, uint8_t* smem) {
  using Row = typename Shape<D>::Row;
  constexpr int H = PairShape<D>::H, NW = PairShape<D>::NW;
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
  const uint32_t pad = ((sbase + kPairSlot - 1u) & ~(kPairSlot - 1u)) - sbase;
  int2* sig_pair = reinterpret_cast<int2*>(smem + pad + (NT / 32) * kPairSlot);               // [kPairLut]
  uint32_t* upd = reinterpret_cast<uint32_t*>(sig_pair + kPairLut);                            // [kPairLut]
  int* n_upd_s = reinterpret_cast<int*>(upd + kPairLut);                                       // [4]
  uint32_t* best = reinterpret_cast<uint32_t*>(n_upd_s + 4);
  const int tid = threadIdx.x, lane = tid & 31;
  const uint32_t Lb = sbase + pad + (uint32_t)(tid >> 5) * kPairSlot;  // this warp's table slot
  SaDraws dr;
  dr.init((uint32_t)chain, kTagSA | ((uint32_t)(chain >> 32) << 8), K);
  const int n_sweeps = tab.n_sweeps;

  for (int idx = tid; idx < kPairLut; idx += NT) sig_pair[idx] = __ldg(&tab.sig[pair_sig_source(idx)]);
  __syncthreads();
  if (tid < 32) {  // the entries whose threshold changes from sweep to sweep
    const int n = list_threshold_entries(sig_pair, kPairLut, upd, tid);
    if (tid == 0) n_upd_s[0] = n;
  }
  __syncthreads();  // the last CTA barrier: warps then sweep independently
  const int n_upd = n_upd_s[0];
  if (n_sweeps > 0) build_lut_pair(Lb, sig_pair, tab.T, lane);

  Row R[D];
  load_rows<D, Row>(init, R);
  // Multiply by L_P: L_X = column 0 (X on even rows, Z on odd rows), L_Z = row 0
  // (Z on even columns, X on odd columns).
  if (P_coset == 1 || P_coset == 2) {
#pragma unroll
    for (int r = 0; r < D; ++r) R[r] ^= (Row)((r & 1) ? 1u : 2u);
  }
  if (P_coset == 2 || P_coset == 3) {
    const uint64_t mz = 0x9999999999999999ull & ((2 * D >= 64) ? ~0ull : ((1ull << (2 * D)) - 1ull));
    R[0] ^= (Row)mz;
  }
  int32_t W4[4] = {tab.W[0], tab.W[1], tab.W[2], tab.W[3]};
  int32_t E = energy_of<D, Row>(R, W4);
  int32_t E_best = E;
  uint32_t P[H][NW];
  rows_to_pairs<D, Row>(R, P);
#pragma unroll
  for (int j = 0; j < H; ++j)
#pragma unroll
    for (int k = 0; k < NW; ++k) best[(j * NW + k) * NT + tid] = P[j][k];
  __syncwarp();

#pragma unroll U
  for (int t = 0; t < n_sweeps; ++t) {
    dr.sweep((uint32_t)t, K);
#define XZZX_SNAPSHOT                                                                         \
  if (E < E_best) {                                                                           \
    E_best = E;                                                                               \
    _Pragma("unroll") for (int j = 0; j < H; ++j)                                             \
    _Pragma("unroll") for (int k = 0; k < NW; ++k) best[(j * NW + k) * NT + tid] = P[j][k];   \
  }
    pair_phase<D, 0>(P, E, Lb, dr, K, tab.err);
    XZZX_SNAPSHOT
    even_to_odd<D>(P);
    pair_phase<D, 1>(P, E, Lb, dr, K, tab.err);
    odd_to_even<D>(P);
    XZZX_SNAPSHOT
    pair_phase<D, 2>(P, E, Lb, dr, K, tab.err);
    XZZX_SNAPSHOT
    even_to_odd<D>(P);
    pair_phase<D, 3>(P, E, Lb, dr, K, tab.err);
    odd_to_even<D>(P);
    XZZX_SNAPSHOT
#undef XZZX_SNAPSHOT
    if (t + 1 < n_sweeps) {  // next sweep's thresholds, once every lane is done with these
      __syncwarp();
      update_lut_pair(Lb, upd, n_upd, tab.T + (size_t)(t + 1) * tab.n_classes, lane);
      __syncwarp();
    }
  }

  if (!active) return;
  *out.best_E = E_best;
  if (out.final_E) *out.final_E = E;
  if (out.final_cfg) {
    pairs_to_rows<D, Row>(P, R);
    store_rows<D, Row>(R, out.final_cfg);
  }
  if (out.best_cfg) {
#pragma unroll
    for (int j = 0; j < H; ++j)
#pragma unroll
      for (int k = 0; k < NW; ++k) P[j][k] = best[(j * NW + k) * NT + tid];
    pairs_to_rows<D, Row>(P, R);
    store_rows<D, Row>(R, out.best_cfg);
  }
}

// Anneal one chain per thread; every thread of the CTA must call this (it
// contains barriers).  init: the chain's reference R_i (2w planar words);
// chain: global chain id (Philox counter); P: coset index of L_P; inactive
// threads run a copy of a real chain and write nothing.  smem: smem_bytes<D,
// NT>() bytes of dynamic shared memory.  U: unroll factor of the sweep loop
// (a tuning knob; results do not depend on it).
template <int D, int NT, int U = 1>
__device__ __forceinline__ void anneal_cta(const uint32_t* __restrict__ init, uint64_t chain, int P, bool active,
                                           const ChainOut& out, const SweepTables& tab, const PhiloxKeys& K,
                                           uint8_t* smem) {
  if constexpr (D <= kPairMaxD) anneal_cta_pairs<D, NT, U>(init, chain, P, active, out, tab, K, smem);
  else anneal_cta_rows<D, NT, U>(init, chain, P, active, out, tab, K, smem);
}

}  // namespace core
}  // namespace xzzx
