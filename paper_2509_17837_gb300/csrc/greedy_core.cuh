// Randomised greedy matching (Algs. 5 and 6) on the GPU.
//
// One CTA per (shot, group of kWarps*rpw restarts); each warp takes rpw
// restarts in turn (for d <= 17 rpw = 4, 2 or 1, the most that still leaves
// the launch several waves of CTAs; 1 above).  The CTA first computes, in
// shared memory, each face's shortest distance to the open boundary of its
// decoding graph (w(u,b) of Eq. distance_u_boundary) by Bellman-Ford
// relaxation, and the defect list of each decoding-graph colour; for d <= 17,
// also every vertex's candidate list (below).  All of it depends on the shot
// only, so it serves every restart of the CTA.
//
// Matching.  All candidate pairs are totally ordered by (w, key, u, v): w the
// pair weight of Eq. distance_u_v_def_new, key a Philox draw per pair (Alg. 6)
// or 0 (Alg. 5), u < v the stabilizer indices (0xFFFF for the virtual boundary
// vertex).  Scanning that order and keeping pairs whose ends are free gives
// the same matching as repeatedly matching every pair that is the best
// remaining pair of both its ends ("locally dominant" pairs), which is what
// the warp does, round by round, in parallel over vertices.  A vertex's best
// free partner is found from its candidate list when the colour has at most
// 64 vertices: the other vertices sorted by (w, index), so the first free
// entry has the lowest weight and, among equal weights, the lowest (u, v);
// with random keys only the free entries tied with it at that weight are
// compared further.  Larger colours scan all candidates.
//
// Paths.  Every kept pair is joined by a canonical shortest path (a Z step
// toward the target whenever one is needed and possible, else an X step; to
// the boundary, the first of Z(+1,+1), Z(-1,-1), X(+1,-1), X(-1,+1) that lowers
// the boundary distance by its weight), added modulo two into the warp's
// configuration.  A walk that could not complete (never expected on a valid
// code) sets bit 7 of cbits and raises XZZX_DEVERR_GREEDY_WALK in the code's
// error area.
#pragma once

#include <type_traits>

#include "internal.h"
#include "philox.cuh"

namespace xzzx {
namespace greedy {

constexpr int kWarps = 4;
// A launch with candidate lists takes the largest restarts-per-warp count (4,
// 2 or 1) that still gives it this many CTAs (several waves on a 152-SM GPU):
// large launches then share each CTA's setup across more restarts, small ones
// keep their CTAs.  Without lists (d > 17) a warp takes one restart: the scan
// dominates there, and longer CTAs only lengthen the launch's tail.
constexpr int64_t kMinGreedyCtas = 4096;
constexpr int kMaxRestartsPerWarp = 4;

// CTAs of a shot's restarts at rpw restarts per warp.
__host__ __device__ inline int greedy_groups(int restarts, int rpw) {
  return (restarts + kWarps * rpw - 1) / (kWarps * rpw);
}
// Reference modes: greedy matching with lexicographic ties (Alg. 5), with
// random ties (Alg. 6), or every defect joined to its nearer boundary.
constexpr int kInitGreedy = 0, kInitGreedyRandom = 1, kInitBoundary = 2;
constexpr int32_t kInf = 0x3FFFFFFF;

// Geometry of the rotated layout: faces (a, b), a, b in [-1, d-1]; qubit
// (r, c) = r*d + c.  The four edges of a face in walking order: Z(+1,+1),
// Z(-1,-1), X(+1,-1), X(-1,+1), crossing the qubit (max a, max b).
struct RotGeo {
  static constexpr bool kSortedLists = true;
  // Resident CTAs per SM the kernel with candidate lists is register-bounded
  // for (64 registers; its shared memory allows 7).
  static constexpr int kMinCtasLists = 8;
  static constexpr int kMaxFaces = kMaxD * kMaxD - 1;
  static constexpr int kMaxAt = (kMaxD + 1) * (kMaxD + 1);
  static constexpr int kMaxWords = (kMaxD * kMaxD + 31) / 32;
  __device__ static int at_size(int d) { return (d + 1) * (d + 1); }
  __device__ static int face(const int16_t* at, int d, int a, int b) {
    if (a < -1 || a > d - 1 || b < -1 || b > d - 1) return -1;
    return at[(a + 1) * (d + 1) + (b + 1)];
  }
  __device__ static int qubit(int d, int r, int c) { return (r >= 0 && r < d && c >= 0 && c < d) ? r * d + c : -1; }
  __device__ static void step(int a, int b, int e, int& na, int& nb, int& qr, int& qc) {
    na = a + ((e & 1) ? -1 : 1);
    nb = b + ((e == 1 || e == 2) ? -1 : 1);
    qr = max(a, na);
    qc = max(b, nb);
  }
  // Eq. distance_u_v_internal in rotated coordinates.
  __device__ static int32_t w_int(int au, int bu, int av, int bv, int32_t Wt_x, int32_t Wt_z) {
    return Wt_z * (abs((au + bu) - (av + bv)) >> 1) + Wt_x * (abs((au - bu) - (av - bv)) >> 1);
  }
};

// Geometry of the planar layout: faces (i, j), i + j odd, of the (2d-1)^2
// grid; qubits on the sites with r + c even.  Edges in walking order: Z right
// and Z left (crossing (i, j+-1)), X down and X up (crossing (i+-1, j)).
struct PlanarGeo {
  static constexpr bool kSortedLists = false;
  static constexpr int kMinCtasLists = 1;
  static constexpr int kMaxFaces = 2 * kMaxD * (kMaxD - 1);
  static constexpr int kMaxAt = (2 * kMaxD - 1) * (2 * kMaxD - 1);
  static constexpr int kMaxWords = (kMaxD * kMaxD + (kMaxD - 1) * (kMaxD - 1) + 31) / 32;
  __device__ static int at_size(int d) { return (2 * d - 1) * (2 * d - 1); }
  __device__ static int face(const int16_t* at, int d, int a, int b) {
    const int g = 2 * d - 1;
    if (a < 0 || a >= g || b < 0 || b >= g) return -1;
    return at[a * g + b];
  }
  __device__ static int qubit(int d, int r, int c) {
    const int g = 2 * d - 1;
    if (r < 0 || r >= g || c < 0 || c >= g || ((r + c) & 1)) return -1;
    return planar_qubit(d, r, c);
  }
  __device__ static void step(int a, int b, int e, int& na, int& nb, int& qr, int& qc) {
    const int di = e < 2 ? 0 : (e == 2 ? 1 : -1);
    const int dj = e < 2 ? (e == 0 ? 1 : -1) : 0;
    na = a + 2 * di;
    nb = b + 2 * dj;
    qr = a + di;
    qc = b + dj;
  }
  // Eq. distance_u_v_internal: a Z step moves j by 2, an X step moves i by 2.
  __device__ static int32_t w_int(int au, int bu, int av, int bv, int32_t Wt_x, int32_t Wt_z) {
    return Wt_z * (abs(bu - bv) >> 1) + Wt_x * (abs(au - av) >> 1);
  }
};

// Sorted candidate lists of one CTA (rotated codes): for each colour with at
// most kListMax vertices and each vertex x, the other vertices y in
// increasing (w(x, y), y), one byte each: y, plus 0x80 when w(x, y) equals the
// previous entry's weight.  cur: each warp's first possibly-free entry.
constexpr int kListMax = 64;
struct CandidateLists {
  uint8_t l[2][kListMax][kListMax];
  uint8_t cur[kWarps][kListMax];
  int usable[2];
};
struct NoLists {};

// Largest distance whose greedy launches carry candidate lists.  At d = 17
// colours still fit kListMax vertices for p up to about 0.2 (2-3x faster
// references); past it most colours hold more, and the lists' shared memory
// would only lower the occupancy of the scan that runs.
constexpr int kListMaxD = 17;

template <class G>
struct SharedBase {
  int16_t fa[G::kMaxFaces], fb[G::kMaxFaces];
  int16_t at[G::kMaxAt];
  int32_t wb[G::kMaxFaces];
  int16_t defects[2][G::kMaxFaces / 2];
  int n_def[2];
  uint32_t syn[(G::kMaxFaces + 31) / 32];
  int16_t best[kWarps][G::kMaxFaces / 2 + 1];
  int16_t partner[kWarps][G::kMaxFaces / 2 + 1];
  uint32_t cfg[kWarps][2 * G::kMaxWords];
  int walk_error[kWarps];
};

// A CTA's shared state, with candidate lists when L (rotated codes only).
template <class G, bool L>
struct SharedT : SharedBase<G> {
  static constexpr bool kLists = G::kSortedLists && L;
  typename std::conditional<kLists, CandidateLists, NoLists>::type lists;
};

template <class G>
struct Ctx {
  const SharedBase<G>& S;
  int d, w;
  int32_t Wt_x, Wt_z;
  uint32_t* err;  // the code's device error area
  int nq;
  __device__ int face(int a, int b) const { return G::face(S.at, d, a, b); }
  __device__ int qubit(int r, int c) const { return G::qubit(d, r, c); }
  __device__ int32_t w_int(int u, int v) const { return G::w_int(S.fa[u], S.fb[u], S.fa[v], S.fb[v], Wt_x, Wt_z); }
};

template <class G>
__device__ __forceinline__ void toggle(const Ctx<G>& X, uint32_t* cfg, int q, bool z_step) {
  if (!XZZX_CHECK(X.err, q >= 0 && q < X.nq)) return;
  atomicXor(&cfg[(z_step ? X.w : 0) + (q >> 5)], 1u << (q & 31));
}

// Canonical internal walk: a Z step toward v whenever one is still needed and
// both the next face and the crossed qubit exist, else an X step.
template <class G>
__device__ bool walk_internal(const Ctx<G>& X, int u, int v, uint32_t* cfg) {
  int a = X.S.fa[u], b = X.S.fb[u];
  const int ta = X.S.fa[v], tb = X.S.fb[v];
  for (int guard = 0; guard < 8 * X.d * X.d + 8; ++guard) {
    if (a == ta && b == tb) return true;
    bool moved = false;
    for (int e = 0; e < 4 && !moved; ++e) {
      int na, nb, qr, qc;
      G::step(a, b, e, na, nb, qr, qc);
      const bool z_step = e < 2;
      // the step must lower the remaining distance of its own kind
      const int32_t before = G::w_int(a, b, ta, tb, z_step ? 0 : 1, z_step ? 1 : 0);
      const int32_t after = G::w_int(na, nb, ta, tb, z_step ? 0 : 1, z_step ? 1 : 0);
      if (after != before - 1) continue;
      const int q = X.qubit(qr, qc);
      if (X.face(na, nb) < 0 || q < 0) continue;
      toggle(X, cfg, q, z_step);
      a = na;
      b = nb;
      moved = true;
    }
    if (!moved) return false;
  }
  return false;
}

// Walk to the open boundary: at each face the first edge, in walking order,
// that lowers the boundary distance by exactly its own weight.
template <class G>
__device__ bool walk_boundary(const Ctx<G>& X, int u, uint32_t* cfg) {
  int cur = u;
  for (int guard = 0; guard < 8 * X.d * X.d + 8; ++guard) {
    const int a = X.S.fa[cur], b = X.S.fb[cur];
    const int32_t here = X.S.wb[cur];
    bool moved = false;
    for (int e = 0; e < 4; ++e) {
      int na, nb, qr, qc;
      G::step(a, b, e, na, nb, qr, qc);
      const int q = X.qubit(qr, qc);
      if (q < 0) continue;
      const bool z_step = e < 2;
      const int32_t w = z_step ? X.Wt_z : X.Wt_x;
      const int nf = X.face(na, nb);
      if (nf < 0) {
        if (w == here) {
          toggle(X, cfg, q, z_step);
          return true;
        }
      } else if (X.S.wb[nf] + w == here) {
        toggle(X, cfg, q, z_step);
        cur = nf;
        moved = true;
        break;
      }
    }
    if (!moved) return false;
  }
  return false;
}

// Pair weight of vertices x != y of a colour with nd defects (vertex nd is the
// virtual boundary vertex).
template <class G>
__device__ __forceinline__ int32_t pair_weight(const Ctx<G>& X, const int16_t* D, int nd, int x, int y) {
  if (x == nd) return X.S.wb[D[y]];
  if (y == nd) return X.S.wb[D[x]];
  return min(X.w_int(D[x], D[y]), X.S.wb[D[x]] + X.S.wb[D[y]]);
}

// Keep the smaller (keep_min) or larger of v and the value of lane ^ j.
__device__ __forceinline__ uint32_t bitonic_step(uint32_t v, int j, bool keep_min) {
  const uint32_t o = __shfl_xor_sync(0xFFFFFFFFu, v, j);
  return keep_min ? min(v, o) : max(v, o);
}

// Ascending bitonic sort across the warp of the values at positions lane (a)
// and, when N64, lane + 32 (b).
template <bool N64>
__device__ __forceinline__ void warp_sort(uint32_t& a, uint32_t& b, int lane) {
#pragma unroll
  for (int k = 2; k <= (N64 ? 64 : 32); k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j == 32) {
        const uint32_t lo = min(a, b), hi = max(a, b);
        a = lo;
        b = hi;
        continue;
      }
      const bool lower = (lane & j) == 0;
      a = bitonic_step(a, j, lower == ((lane & k) == 0));
      if (N64) b = bitonic_step(b, j, lower == (((lane + 32) & k) == 0));
    }
  }
}

// Candidate list of vertex x (nv <= kListMax vertices), built by one warp.
// Returns false if a weight does not fit the 26 bits of the sort key.
template <class G, bool N64>
__device__ __forceinline__ bool build_list(const Ctx<G>& X, const int16_t* D, int nd, int nv, int x, uint8_t* out,
                                           int lane) {
  bool fits = true;
  uint32_t key[2] = {0xFFFFFFFFu, 0xFFFFFFFFu};
#pragma unroll
  for (int h = 0; h < (N64 ? 2 : 1); ++h) {
    const int y = lane + 32 * h;
    if (y < nv && y != x) {
      const int32_t w = pair_weight(X, D, nd, x, y);
      fits = fits && w >= 0 && w < (1 << 26) - 1;  // keys stay below the 0xFFFFFFFF filler
      key[h] = ((uint32_t)w << 6) | (uint32_t)y;
    }
  }
  warp_sort<N64>(key[0], key[1], lane);
  const uint32_t prev0 = __shfl_up_sync(0xFFFFFFFFu, key[0], 1);
  const uint32_t last0 = __shfl_sync(0xFFFFFFFFu, key[0], 31);
  uint32_t prev1 = 0u;
  if (N64) {
    const uint32_t up1 = __shfl_up_sync(0xFFFFFFFFu, key[1], 1);
    prev1 = lane == 0 ? last0 : up1;
  }
#pragma unroll
  for (int h = 0; h < (N64 ? 2 : 1); ++h) {
    const int pos = lane + 32 * h;
    const uint32_t k = key[h], pk = h ? prev1 : prev0;
    if (pos < nv - 1) out[pos] = (uint8_t)((k & 63u) | ((pos > 0 && (k >> 6) == (pk >> 6)) ? 0x80u : 0u));
  }
  return __all_sync(0xFFFFFFFFu, fits);
}

// The reference of restart i of the CTA's shot, by one warp, after the CTA
// has set up the boundary distances, defect lists and candidate lists.
template <class G, bool L>
__device__ __forceinline__ void greedy_restart(const Ctx<G>& X, const DevCode& C, const PhiloxKeys& K, uint64_t shot,
                                               int i, int mode, uint32_t* __restrict__ init,
                                               uint8_t* __restrict__ cbits, SharedT<G, L>& S, int warp, int lane) {
  const int w = C.w;

  uint32_t* cfg = S.cfg[warp];
  for (int j = lane; j < 2 * w; j += 32) cfg[j] = 0u;
  if (lane == 0) S.walk_error[warp] = 0;
  int16_t* best = S.best[warp];
  int16_t* partner = S.partner[warp];
  __syncwarp();

  if (mode == kInitBoundary) {
    // Each defect joined to the nearer boundary of its decoding graph.
    for (int colour = 0; colour < 2; ++colour)
      for (int x = lane; x < S.n_def[colour]; x += 32)
        if (!walk_boundary(X, S.defects[colour][x], cfg)) S.walk_error[warp] = 1;
    __syncwarp();
  }
  for (int colour = 0; colour < 2 && mode != kInitBoundary; ++colour) {
    const int nd = S.n_def[colour];
    const int nv = nd + (nd & 1);  // vertex nd is the virtual boundary vertex when nd is odd
    const int16_t* D = S.defects[colour];
    for (int x = lane; x < nv; x += 32) {
      partner[x] = -1;
      best[x] = -1;
    }
    bool listed = false;
    if constexpr (SharedT<G, L>::kLists) {
      listed = nv >= 2 && nv <= kListMax && S.lists.usable[colour];
      if (listed)
        for (int x = lane; x < nv; x += 32) S.lists.cur[warp][x] = 0;
    }
    __syncwarp();
    int unmatched = nv;
    while (unmatched > 0 && listed) {
      if constexpr (SharedT<G, L>::kLists) {
        // Each free vertex whose best partner was taken walks its sorted list
        // from its cursor to the first free entry: the lowest weight among
        // free vertices, and the lowest (u, v) at that weight.  Keys order
        // the free entries tied at that weight (Alg. 6).
        for (int x = lane; x < nv; x += 32) {
          if (partner[x] >= 0) {
            best[x] = -1;
            continue;
          }
          const int bx = best[x];
          if (bx >= 0 && partner[bx] < 0) continue;
          const uint8_t* Lx = S.lists.l[colour][x];
          int c = S.lists.cur[warp][x];
          while (c < nv - 1 && partner[Lx[c] & 63] >= 0) ++c;
          S.lists.cur[warp][x] = (uint8_t)c;
          if (c >= nv - 1) {  // no free vertex left for x: impossible with an even count
            best[x] = -1;
            S.walk_error[warp] = 1;
            continue;
          }
          int bestv = Lx[c] & 63;
          if (mode == kInitGreedyRandom) {
            const uint32_t sx = x == nd ? kBoundary : (uint32_t)D[x];
            const uint32_t s0 = bestv == nd ? kBoundary : (uint32_t)D[bestv];
            uint32_t bu = min(sx, s0), bvv = max(sx, s0), bkey = 0;
            bool bkey_ok = false;
            const uint32_t c3 = kTagGreedy | ((uint32_t)(shot >> 32) << 8);
            for (int k = c + 1; k < nv - 1; ++k) {
              const uint32_t ent = Lx[k];
              if (!(ent & 0x80u)) break;
              const int y = (int)(ent & 63u);
              if (partner[y] >= 0) continue;
              const uint32_t sy = y == nd ? kBoundary : (uint32_t)D[y];
              const uint32_t u = min(sx, sy), v = max(sx, sy);
              if (!bkey_ok) {
                bkey = philox4x32_10(bu | (bvv << 16), (uint32_t)i, (uint32_t)shot, c3, K).x;
                bkey_ok = true;
              }
              const uint32_t key = philox4x32_10(u | (v << 16), (uint32_t)i, (uint32_t)shot, c3, K).x;
              if (key < bkey || (key == bkey && (u < bu || (u == bu && v < bvv)))) {
                bestv = y;
                bkey = key;
                bu = u;
                bvv = v;
              }
            }
          }
          best[x] = (int16_t)bestv;
        }
        __syncwarp();
        int made = 0;
        for (int x = lane; x < nv; x += 32) {
          const int y = best[x];
          if (y > x && XZZX_CHECK(C.err, y < nv) && best[y] == x) {
            partner[x] = (int16_t)y;
            partner[y] = (int16_t)x;
            made += 2;
          }
        }
        __syncwarp();
        for (int off = 16; off > 0; off >>= 1) made += __shfl_xor_sync(0xFFFFFFFFu, made, off);
        if (made == 0) {
          if (lane == 0) S.walk_error[warp] = 1;
          break;
        }
        unmatched -= made;
      }
    }
    while (unmatched > 0 && !listed) {
      // Each free vertex finds its best free partner in the order (w, key, u, v),
      // in one pass: a candidate's key is drawn only when its weight ties the
      // best so far.  A best partner that is still free stays the best (removing
      // other vertices cannot put one ahead of it), so only vertices whose best
      // was matched in the last round search again.
      for (int x = lane; x < nv; x += 32) {
        if (partner[x] >= 0) {
          best[x] = -1;
          continue;
        }
        const int bx = best[x];
        if (bx >= 0 && partner[bx] < 0) continue;
        const bool xb = x == nd;
        const int fx = xb ? 0 : D[x];
        const uint32_t sx = xb ? kBoundary : (uint32_t)fx;
        int bestv = -1;
        int32_t bw = kInf;
        uint32_t bkey = 0, bu = 0, bvv = 0;
        bool bkey_ok = false;
        for (int y = 0; y < nv; ++y) {
          if (y == x || partner[y] >= 0) continue;
          int32_t wxy;
          if (xb) wxy = S.wb[D[y]];
          else if (y == nd) wxy = S.wb[fx];
          else wxy = min(X.w_int(fx, D[y]), S.wb[fx] + S.wb[D[y]]);
          if (wxy > bw) continue;
          const uint32_t sy = (y == nd) ? kBoundary : (uint32_t)D[y];
          const uint32_t u = min(sx, sy), v = max(sx, sy);
          if (wxy < bw) {
            bestv = y;
            bw = wxy;
            bu = u;
            bvv = v;
            bkey_ok = false;
            continue;
          }
          uint32_t key = 0;
          if (mode == kInitGreedyRandom) {
            const uint32_t c3 = kTagGreedy | ((uint32_t)(shot >> 32) << 8);
            if (!bkey_ok) {
              bkey = philox4x32_10(bu | (bvv << 16), (uint32_t)i, (uint32_t)shot, c3, K).x;
              bkey_ok = true;
            }
            key = philox4x32_10(u | (v << 16), (uint32_t)i, (uint32_t)shot, c3, K).x;
          }
          if (key < bkey || (key == bkey && (u < bu || (u == bu && v < bvv)))) {
            bestv = y;
            bkey = key;
            bu = u;
            bvv = v;
          }
        }
        best[x] = (int16_t)bestv;
      }
      __syncwarp();
      // Matching phase: reads only best[], writes only partner[].
      int made = 0;
      for (int x = lane; x < nv; x += 32) {
        const int y = best[x];
        if (y > x && XZZX_CHECK(C.err, y < nv) && best[y] == x) {
          partner[x] = (int16_t)y;
          partner[y] = (int16_t)x;
          made += 2;
        }
      }
      __syncwarp();
      for (int off = 16; off > 0; off >>= 1) made += __shfl_xor_sync(0xFFFFFFFFu, made, off);
      if (made == 0) {  // impossible for a strict total order; keep the warp from spinning
        if (lane == 0) S.walk_error[warp] = 1;
        break;
      }
      unmatched -= made;
    }
    // Join every kept pair.
    for (int x = lane; x < nv; x += 32) {
      const int y = partner[x];
      if (y <= x || x == nd) continue;
      bool ok;
      const int fx = D[x];
      if (y == nd) {
        ok = walk_boundary(X, fx, cfg);
      } else {
        const int fy = D[y];
        if (X.w_int(fx, fy) <= S.wb[fx] + S.wb[fy]) ok = walk_internal(X, fx, fy, cfg);
        else ok = walk_boundary(X, fx, cfg) && walk_boundary(X, fy, cfg);
      }
      if (!ok) S.walk_error[warp] = 1;
    }
    __syncwarp();
  }

  // Output R_i and its commutation bits with L_Z (bit 0) and L_X (bit 1).
  uint32_t* out = init + (size_t)i * 2 * w;
  const uint32_t* LX = C.logical;
  const uint32_t* LZ = C.logical + 2 * w;
  int par_z = 0, par_x = 0;
  for (int j = lane; j < w; j += 32) {
    const uint32_t ex = cfg[j], ez = cfg[w + j];
    out[j] = ex;
    out[w + j] = ez;
    par_z ^= __popc((ex & LZ[w + j]) ^ (ez & LZ[j])) & 1;
    par_x ^= __popc((ex & LX[w + j]) ^ (ez & LX[j])) & 1;
  }
  for (int off = 16; off > 0; off >>= 1) {
    par_z ^= __shfl_xor_sync(0xFFFFFFFFu, par_z, off);
    par_x ^= __shfl_xor_sync(0xFFFFFFFFu, par_x, off);
  }
  if (lane == 0) {
    // A walk that could not complete is recorded in the code's error area
    // (XZZX_DEVERR_GREEDY_WALK) and in bit 7 of the restart's class byte.
    const bool bad = S.walk_error[warp] != 0 || (i == 0 && injected(C.err, XZZX_DEVERR_GREEDY_WALK));
    if (bad) raise_device_error(C.err, XZZX_DEVERR_GREEDY_WALK);
    cbits[i] = (uint8_t)(par_z | (par_x << 1) | (bad ? 0x80 : 0));
  }
}

// One CTA: references of restarts [group*kWarps*rpw, (group+1)*kWarps*rpw)
// of one shot, each warp taking rpw of them in turn, so the CTA's setup serves
// kWarps*rpw restarts.  syn: the shot's syndrome words; init / cbits: the
// shot's rows (restarts x 2w words, restarts bytes).
template <class G, bool L>
__device__ __forceinline__ void greedy_cta(const DevCode& C, const PhiloxKeys& K, uint64_t shot, int group, int restarts,
                                           int rpw, int mode, int32_t Wt_x, int32_t Wt_z, const uint32_t* __restrict__ syn,
                                           uint32_t* __restrict__ init, uint8_t* __restrict__ cbits, SharedT<G, L>& S) {
  const int d = C.d, ns = C.ns, w = C.w;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  for (int f = tid; f < ns; f += blockDim.x) {
    S.fa[f] = C.face_a[f];
    S.fb[f] = C.face_b[f];
  }
  for (int j = tid; j < G::at_size(d); j += blockDim.x) S.at[j] = C.face_at[j];
  for (int j = tid; j < C.sw; j += blockDim.x) S.syn[j] = syn[j];
  if constexpr (SharedT<G, L>::kLists) {
    if (tid < 2) S.lists.usable[tid] = 1;
  }
  __syncthreads();
  Ctx<G> X{S, d, w, Wt_x, Wt_z, C.err, C.nq};

  // Boundary distances: start from the boundary edges, relax until stable.
  for (int f = tid; f < ns; f += blockDim.x) {
    const int a = S.fa[f], b = S.fb[f];
    int32_t best = kInf;
    for (int e = 0; e < 4; ++e) {
      int na, nb, qr, qc;
      G::step(a, b, e, na, nb, qr, qc);
      if (X.qubit(qr, qc) < 0 || X.face(na, nb) >= 0) continue;
      best = min(best, e < 2 ? Wt_z : Wt_x);
    }
    S.wb[f] = best;
  }
  __syncthreads();
  for (int iter = 0; iter < ns + 1; ++iter) {
    int changed = 0;
    for (int f = tid; f < ns; f += blockDim.x) {
      const int a = S.fa[f], b = S.fb[f];
      int32_t cur = S.wb[f];
      for (int e = 0; e < 4; ++e) {
        int na, nb, qr, qc;
        G::step(a, b, e, na, nb, qr, qc);
        if (X.qubit(qr, qc) < 0) continue;
        const int nf = X.face(na, nb);
        if (nf < 0) continue;
        const int32_t cand = S.wb[nf] + (e < 2 ? Wt_z : Wt_x);
        if (cand < cur) {
          cur = cand;
          changed = 1;
        }
      }
      S.wb[f] = cur;
    }
    if (!__syncthreads_or(changed)) break;
  }

  // Defect lists of both colours, in stabilizer-index order.
  if (warp == 0) {
    int cnt[2] = {0, 0};
    for (int base = 0; base < ns; base += 32) {
      const int f = base + lane;
      const bool on = f < ns && ((S.syn[f >> 5] >> (f & 31)) & 1);
      const int c2 = f < ns ? C.face_c2[f] : 0;
      for (int c = 0; c < 2; ++c) {
        const uint32_t m = __ballot_sync(0xFFFFFFFFu, on && c2 == c);
        const int slot = cnt[c] + __popc(m & ((1u << lane) - 1));
        if (on && c2 == c && XZZX_CHECK(C.err, slot < G::kMaxFaces / 2)) S.defects[c][slot] = (int16_t)f;
        cnt[c] += __popc(m);
      }
    }
    if (lane == 0) {
      S.n_def[0] = cnt[0];
      S.n_def[1] = cnt[1];
    }
  }
  __syncthreads();
  if constexpr (SharedT<G, L>::kLists) {
    // Candidate lists of both colours, every warp of the CTA building some.
    if (mode != kInitBoundary) {
      for (int colour = 0; colour < 2; ++colour) {
        const int nd = S.n_def[colour], nv = nd + (nd & 1);
        if (nv < 2 || nv > kListMax) continue;
        bool fits = true;
        for (int x = warp; x < nv; x += kWarps)
          fits = (nv > 32 ? build_list<G, true>(X, S.defects[colour], nd, nv, x, S.lists.l[colour][x], lane)
                          : build_list<G, false>(X, S.defects[colour], nd, nv, x, S.lists.l[colour][x], lane)) && fits;
        if (lane == 0 && !fits) S.lists.usable[colour] = 0;
      }
    }
    __syncthreads();
  }
  if constexpr (SharedT<G, L>::kLists) {
    for (int r = 0; r < rpw; ++r) {
      const int i = (group * rpw + r) * kWarps + warp;
      if (i >= restarts) break;
      __syncwarp();  // the warp's previous reference is written out
      greedy_restart<G, L>(X, C, K, shot, i, mode, init, cbits, S, warp, lane);
    }
  } else {  // one restart per warp (rpw is 1 without lists)
    const int i = group * kWarps + warp;
    if (i < restarts) greedy_restart<G, L>(X, C, K, shot, i, mode, init, cbits, S, warp, lane);
  }
}

}  // namespace greedy
}  // namespace xzzx
