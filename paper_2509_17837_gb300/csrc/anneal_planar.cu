// Annealing on the planar layout (the paper's own lattice; Alg. 2 with the
// Metropolis step of Alg. 3), in the same four forms as xzzx_anneal_variant:
// sweep order colour (stabilizer-index order) or random site, minimum per
// colour phase / sweep or per attempt.
//
// State.  One chain per thread.  Row r of the (2d-1)^2 grid holds its qubits
// (columns c = 2k + (r&1)) as two bits per slot k (bit 2k = Z, 2k+1 = X), one
// 64-bit word per row, in shared memory laid out [row][thread] so that a
// warp's 32 words of one row are contiguous whichever rows the lanes touch.
//
// Face (i, j): left and right corners are slots kl and kl+1 of row i
// (kl = (j - 1 - (i&1)) >> 1), up and down the slot kl + (i&1) of rows i-1 and
// i+1.  Signature left | right<<2 | up<<4 | down<<6 for a bulk face, the three
// present corners in that order for a boundary face, indexes the planar part
// of the per-sweep (dE, A) table.
//
// Draws.  Colour order: the face's draw is lane ia&3 of Philox(seed;
// (colour<<16) | (ib<<8) | (ia>>2), sweep, chain_lo, 3 | chain_hi<<8) with
// ia = i>>1, ib = j>>2, computed only when a move can be accepted (A > 0); the
// index order (colour, ib, ia) makes the faces of one block consecutive, so a
// one-block cache serves them.  Random site: as xzzx_anneal_variant.
#include "anneal_core.cuh"

namespace xzzx {
namespace {

constexpr int kPThreads = 128;
constexpr int kPLut = kSigPlanar;

struct PlanarArgs {
  PhiloxKeys keys;
  uint64_t chain0;
  int64_t n_chains;
  int d, g, m, W;  // distance, grid side 2d-1, generators, words per plane
  int order, emin;
  int colour_start[5];
  int n_sweeps, n_classes;
  int32_t Wt[4];
  const int16_t* face_a;
  const int16_t* face_b;
  const uint32_t* T;
  const int2* sig;  // the schedule's full table; planar entries from kSigRot
  const uint32_t* init;
  int32_t* best_E;
  uint32_t* best_cfg;
  int32_t* final_E;
  uint32_t* final_cfg;
};

// Face descriptor: i (bits 0-5), kl+1 (6-11), shape (12-14), colour (15-16),
// ia (17-21), ib (22-25).
__device__ __forceinline__ uint32_t planar_desc(int i, int j, int d) {
  const int g = 2 * d - 1;
  const int kl = (j - 1 - (i & 1)) >> 1;
  int shape = kPBulk;
  if (i == 0) shape = kPNoUp;
  else if (i == g - 1) shape = kPNoDown;
  else if (j == 0) shape = kPNoLeft;
  else if (j == g - 1) shape = kPNoRight;
  const uint32_t colour = (uint32_t)((i & 1) | ((((i + j - 1) >> 1) & 1) << 1));
  return (uint32_t)i | ((uint32_t)(kl + 1) << 6) | ((uint32_t)shape << 12) | (colour << 15) |
         ((uint32_t)(i >> 1) << 17) | ((uint32_t)(j >> 2) << 22);
}

struct PMove {
  uint32_t idx;  // into the planar table (0-based)
  int i, ku;
  uint64_t m_mid, m_ud;
  bool up, down;
};

__device__ __forceinline__ PMove planar_move(uint32_t fd, const uint64_t* rows) {
  PMove mv;
  mv.i = (int)(fd & 63u);
  const int kl = (int)((fd >> 6) & 63u) - 1;
  const int shape = (int)((fd >> 12) & 7u);
  mv.ku = kl + (mv.i & 1);
  const uint32_t su = 2u * (uint32_t)mv.ku;
  mv.up = shape != kPNoUp;
  mv.down = shape != kPNoDown;
  const uint64_t mid = rows[(size_t)mv.i * kPThreads];
  const uint32_t up = mv.up ? (uint32_t)(rows[(size_t)(mv.i - 1) * kPThreads] >> su) & 3u : 0u;
  const uint32_t dn = mv.down ? (uint32_t)(rows[(size_t)(mv.i + 1) * kPThreads] >> su) & 3u : 0u;
  mv.m_ud = 1ull << su;  // Z on the up and down corners
  switch (shape) {
    case kPNoLeft: {  // right | up<<2 | down<<4, right in slot 0
      mv.idx = (uint32_t)(planar_sig_base(kPNoLeft) - kSigRot) + (((uint32_t)mid & 3u) | (up << 2) | (dn << 4));
      mv.m_mid = 2ull;
      break;
    }
    case kPNoRight: {  // left | up<<2 | down<<4
      const uint32_t sl = 2u * (uint32_t)kl;
      mv.idx = (uint32_t)(planar_sig_base(kPNoRight) - kSigRot) + (((uint32_t)(mid >> sl) & 3u) | (up << 2) | (dn << 4));
      mv.m_mid = 2ull << sl;
      break;
    }
    default: {  // bulk, no-up, no-down: left | right<<2 then the present Z corners
      const uint32_t sl = 2u * (uint32_t)kl;
      const uint32_t lr = (uint32_t)(mid >> sl) & 0xFu;
      if (shape == kPNoUp) mv.idx = (uint32_t)(planar_sig_base(kPNoUp) - kSigRot) + (lr | (dn << 4));
      else if (shape == kPNoDown) mv.idx = (uint32_t)(planar_sig_base(kPNoDown) - kSigRot) + (lr | (up << 4));
      else mv.idx = lr | (up << 4) | (dn << 6);
      mv.m_mid = 0xAull << sl;  // X on left and right
      break;
    }
  }
  return mv;
}

__device__ __forceinline__ void planar_apply(const PMove& mv, uint64_t* rows) {
  rows[(size_t)mv.i * kPThreads] ^= mv.m_mid;
  if (mv.up) rows[(size_t)(mv.i - 1) * kPThreads] ^= mv.m_ud;
  if (mv.down) rows[(size_t)(mv.i + 1) * kPThreads] ^= mv.m_ud;
}

__device__ __forceinline__ int row_start(int d, int r) { return (r >> 1) * (2 * d - 1) + ((r & 1) ? d : 0); }
__device__ __forceinline__ int row_len(int d, int r) { return (r & 1) ? d - 1 : d; }

// Rows (stride kPThreads) -> planar words (x plane then z plane).
__device__ void store_planar(const uint64_t* rows, int d, int g, int W, uint32_t* __restrict__ cfg) {
  const int nq = d * d + (d - 1) * (d - 1);
  int r = 0;
  for (int j = 0; j < W; ++j) {
    uint32_t wx = 0u, wz = 0u;
    const int lo = 32 * j, hi = min(lo + 32, nq);
    while (r + 1 < g && row_start(d, r + 1) <= lo) ++r;
    for (int rr = r; rr < g && row_start(d, rr) < hi; ++rr) {
      const uint64_t v = rows[(size_t)rr * kPThreads];
      const uint32_t fz = core::gather2(v), fx = core::gather2(v >> 1);
      const int start = row_start(d, rr) - lo;
      if (start >= 0) {
        wz |= fz << start;
        wx |= fx << start;
      } else {
        wz |= fz >> (-start);
        wx |= fx >> (-start);
      }
    }
    cfg[j] = wx;
    cfg[W + j] = wz;
  }
}

__device__ __forceinline__ void copy_rows(const uint64_t* src, uint64_t* dst, int g) {
  for (int r = 0; r < g; ++r) dst[(size_t)r * kPThreads] = src[(size_t)r * kPThreads];
}

__device__ __forceinline__ void build_lut(uint2* __restrict__ dst, const int2* __restrict__ sig_static,
                                          const uint32_t* __restrict__ Trow, int lane) {
  for (int idx = lane; idx < kPLut; idx += 32) {
    const int2 s = sig_static[idx];
    dst[idx] = make_uint2((uint32_t)s.x, s.y >= 0 ? __ldg(&Trow[s.y]) : 0u);
  }
}

size_t planar_smem_bytes(int d, int m) {
  const int g = 2 * d - 1;
  size_t b = kPLut * sizeof(int2) + (kPThreads / 32) * kPLut * sizeof(uint2) + (size_t)m * sizeof(uint32_t);
  b = (b + 15) & ~(size_t)15;
  return b + 2 * (size_t)g * kPThreads * sizeof(uint64_t);
}

__global__ void __launch_bounds__(kPThreads) anneal_planar_kernel(const __grid_constant__ PlanarArgs A) {
  extern __shared__ __align__(16) uint8_t smem[];
  int2* sig_static = reinterpret_cast<int2*>(smem);
  uint2* lut_all = reinterpret_cast<uint2*>(smem + kPLut * sizeof(int2));
  uint32_t* faces = reinterpret_cast<uint32_t*>(smem + kPLut * sizeof(int2) + (kPThreads / 32) * kPLut * sizeof(uint2));
  size_t off = kPLut * sizeof(int2) + (kPThreads / 32) * kPLut * sizeof(uint2) + (size_t)A.m * sizeof(uint32_t);
  off = (off + 15) & ~(size_t)15;
  const int tid = threadIdx.x, lane = tid & 31;
  uint64_t* rows = reinterpret_cast<uint64_t*>(smem + off) + tid;
  uint64_t* best = rows + (size_t)A.g * kPThreads;
  uint2* L = lut_all + (tid >> 5) * kPLut;

  const int64_t c_raw = (int64_t)blockIdx.x * kPThreads + tid;
  const bool active = c_raw < A.n_chains;
  const int64_t c = active ? c_raw : A.n_chains - 1;  // inactive threads shadow a real chain
  const uint64_t chain = A.chain0 + (uint64_t)c;
  const uint32_t c2 = (uint32_t)chain;
  const uint32_t c3_sa = kTagSA | ((uint32_t)(chain >> 32) << 8);
  const uint32_t c3_site = kTagSite | ((uint32_t)(chain >> 32) << 8);
  const int d = A.d, g = A.g, m = A.m, P = (int)(c & 3);

  for (int k = tid; k < kPLut; k += kPThreads) sig_static[k] = __ldg(&A.sig[kSigRot + k]);
  for (int f = tid; f < m; f += kPThreads) faces[f] = planar_desc(A.face_a[f], A.face_b[f], d);
  __syncthreads();
  if (A.n_sweeps > 0) build_lut(L, sig_static, A.T, lane);

  // R_i L_P: L_X = X on column 0 (slot 0 of the even rows), L_Z = Z on row 0.
  const uint32_t* init = A.init + (size_t)(c >> 2) * 2 * A.W;
  int32_t nx = 0, ny = 0, nz = 0;
  for (int r = 0; r < g; ++r) {
    const int s0 = row_start(d, r), len = row_len(d, r);
    const uint32_t x = core::plane_field(init, A.W, s0, len);
    const uint32_t z = core::plane_field(init + A.W, A.W, s0, len);
    uint64_t v = core::spread2(z) | (core::spread2(x) << 1);
    if ((P == 1 || P == 2) && (r & 1) == 0) v ^= 2ull;
    if ((P == 2 || P == 3) && r == 0) v ^= 0x5555555555555555ull & ((1ull << (2 * d)) - 1ull);
    rows[(size_t)r * kPThreads] = v;
    best[(size_t)r * kPThreads] = v;
    const uint64_t zz = v & 0x5555555555555555ull, xx = (v >> 1) & 0x5555555555555555ull;
    ny += __popcll(xx & zz);
    nx += __popcll(xx & ~zz);
    nz += __popcll(zz & ~xx);
  }
  int32_t E = nx * A.Wt[2] + ny * A.Wt[3] + nz * A.Wt[1];
  int32_t E_best = E;
  const bool per_attempt = A.emin == 1;

  for (int t = 0; t < A.n_sweeps; ++t) {
    const uint32_t tt = (uint32_t)t;
    if (A.order == 1) {
      uint4 r = make_uint4(0u, 0u, 0u, 0u);
      for (int k = 0; k < m; ++k) {
        if ((k & 1) == 0) r = philox4x32_10((uint32_t)(k >> 1), tt, c2, c3_site, A.keys);
        const uint32_t u_site = (k & 1) ? r.z : r.x, u_acc = (k & 1) ? r.w : r.y;
        const int f = (int)__umulhi(u_site, (uint32_t)m);
        const PMove mv = planar_move(faces[f], rows);
        const uint2 e = L[mv.idx];
        const int32_t dE = (int32_t)e.x;
        if ((dE <= 0) | (u_acc < e.y)) {
          planar_apply(mv, rows);
          E += dE;
        }
        if (per_attempt && E < E_best) {
          E_best = E;
          copy_rows(rows, best, g);
        }
      }
      if (E < E_best) {
        E_best = E;
        copy_rows(rows, best, g);
      }
    } else {
      uint32_t cached = 0xFFFFFFFFu;
      uint4 rc = make_uint4(0u, 0u, 0u, 0u);
      for (int colour = 0; colour < 4; ++colour) {
        for (int f = A.colour_start[colour]; f < A.colour_start[colour + 1]; ++f) {
          const uint32_t fd = faces[f];
          const PMove mv = planar_move(fd, rows);
          const uint2 e = L[mv.idx];
          const int32_t dE = (int32_t)e.x;
          bool acc = dE <= 0;
          if (!acc && e.y != 0u) {
            const uint32_t ia = (fd >> 17) & 31u, ib = (fd >> 22) & 15u;
            const uint32_t c0 = ((uint32_t)colour << 16) | (ib << 8) | (ia >> 2);
            if (c0 != cached) {
              rc = philox4x32_10(c0, tt, c2, c3_sa, A.keys);
              cached = c0;
            }
            acc = lane_of(rc, (int)(ia & 3u)) < e.y;
          }
          if (acc) {
            planar_apply(mv, rows);
            E += dE;
          }
          if (per_attempt && E < E_best) {
            E_best = E;
            copy_rows(rows, best, g);
          }
        }
        if (E < E_best) {
          E_best = E;
          copy_rows(rows, best, g);
        }
      }
    }
    if (t + 1 < A.n_sweeps) {  // next sweep's thresholds, once every lane is done with these
      __syncwarp();
      build_lut(L, sig_static, A.T + (size_t)(t + 1) * A.n_classes, lane);
      __syncwarp();
    }
  }

  if (!active) return;
  A.best_E[c] = E_best;
  if (A.final_E) A.final_E[c] = E;
  if (A.final_cfg) store_planar(rows, d, g, A.W, A.final_cfg + (size_t)c * 2 * A.W);
  if (A.best_cfg) store_planar(best, d, g, A.W, A.best_cfg + (size_t)c * 2 * A.W);
}

}  // namespace

xzzx_status launch_anneal_planar_reg(const xzzx_code* code, const xzzx_schedule* sched, uint64_t seed, uint64_t shot0,
                                     int n_shots, int restarts, const uint32_t* init, int32_t* best_E,
                                     uint32_t* best_cfg, int32_t* final_E, uint32_t* final_cfg, cudaStream_t stream);

// Launch for a planar code (arguments checked by the caller): the colour sweep
// with per-phase minima runs register-resident up to d = 15, everything else
// in the table-driven kernel below.
xzzx_status launch_anneal_planar(const xzzx_code* code, const xzzx_schedule* sched, uint64_t seed, uint64_t shot0,
                                 int n_shots, int restarts, int order, int emin, const uint32_t* init, int32_t* best_E,
                                 uint32_t* best_cfg, int32_t* final_E, uint32_t* final_cfg, cudaStream_t stream) {
  if (order == 0 && emin == 0 && code->d <= 15)
    return launch_anneal_planar_reg(code, sched, seed, shot0, n_shots, restarts, init, best_E, best_cfg, final_E,
                                    final_cfg, stream);
  PlanarArgs A;
  A.keys = philox_keys(seed);
  A.chain0 = shot0 * (uint64_t)restarts * 4u;
  A.n_chains = (int64_t)n_shots * restarts * 4;
  A.d = code->d;
  A.g = 2 * code->d - 1;
  A.m = code->ns;
  A.W = code->w;
  A.order = order;
  A.emin = emin;
  for (int k = 0; k < 5; ++k) A.colour_start[k] = code->colour_start[k];
  A.n_sweeps = sched->n_sweeps;
  A.n_classes = sched->n_classes;
  for (int k = 0; k < 4; ++k) A.Wt[k] = sched->noise.W[k];
  A.face_a = code->dev.face_a;
  A.face_b = code->dev.face_b;
  A.T = sched->d_T;
  A.sig = sched->d_sig;
  A.init = init;
  A.best_E = best_E;
  A.best_cfg = best_cfg;
  A.final_E = final_E;
  A.final_cfg = final_cfg;
  const size_t smem = planar_smem_bytes(A.d, A.m);
  static DeviceOnce once;
  xzzx_status st = once.run([&]() -> xzzx_status {
    const int most = (int)planar_smem_bytes(kMaxD, 2 * kMaxD * (kMaxD - 1));
    XZZX_CUDA_TRY(cudaFuncSetAttribute(anneal_planar_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, most));
    return XZZX_OK;
  });
  if (st) return st;
  const int64_t grid = (A.n_chains + kPThreads - 1) / kPThreads;
  if (grid > 0x7FFFFFFF) return fail(XZZX_EINVAL, "too many chains for one launch");
  anneal_planar_kernel<<<(unsigned)grid, kPThreads, smem, stream>>>(A);
  XZZX_CUDA_TRY(cudaGetLastError());
  return XZZX_OK;
}

}  // namespace xzzx
