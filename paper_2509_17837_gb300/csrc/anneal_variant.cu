// Annealing in the literal forms of Alg. 2 and Alg. 3, next to the colour
// sweep of the main kernels:
//   order 0 (colour):      each sweep visits the generators in stabilizer-index
//                          order (colour by colour), draws as in the main
//                          kernels -- with emin 0 the results equal xzzx_anneal;
//   order 1 (random site): each sweep makes N_stab attempts on generators
//                          drawn uniformly at random (Alg. 3);
//   emin 0: the minimum is taken at the start and after every colour phase
//           (order 0) or every sweep (order 1);
//   emin 1: the minimum is taken after every attempt (Alg. 2).
// One chain per thread.  A random site needs rows by run-time index, so the
// rows live in shared memory, laid out [row][thread]: the 64-bit words of one
// row of a warp's 32 chains are contiguous, whichever rows the lanes touch.
#include "anneal_core.cuh"

namespace xzzx {
namespace {

using core::kLutN;

constexpr int kVarThreads = 128;

struct VariantArgs {
  PhiloxKeys keys;
  uint64_t chain0;
  int64_t n_chains;
  int d, m, W;  // distance, generators, planar words per plane
  int order, emin;
  int colour_start[5];
  int n_sweeps, n_classes;
  int32_t Wt[4];
  const int16_t* face_a;
  const int16_t* face_b;
  const uint32_t* T;
  const int2* sig;
  const uint32_t* init;
  int32_t* best_E;
  uint32_t* best_cfg;
  int32_t* final_E;
  uint32_t* final_cfg;
};

// Face descriptor: a+1 (bits 0-7), b+1 (8-15), shape (16-23), colour (24-31).
__device__ __forceinline__ uint32_t face_desc(int a, int b, int d) {
  int type = kBulk;
  if (a == -1) type = kTop;
  else if (a == d - 1) type = kBottom;
  else if (b == -1) type = kLeft;
  else if (b == d - 1) type = kRight;
  const uint32_t colour = (uint32_t)((a & 1) | ((b & 1) << 1));
  return (uint32_t)(a + 1) | ((uint32_t)(b + 1) << 8) | ((uint32_t)type << 16) | (colour << 24);
}

// Signature-table index of a face and the XOR masks of G_f on rows r0, r0+1.
struct Move {
  uint32_t idx;
  int r0;
  uint64_t m0, m1;
};

__device__ __forceinline__ Move face_move(uint32_t fd, const uint64_t* rows, int d) {
  const int a = (int)(fd & 0xFFu) - 1, b = (int)((fd >> 8) & 0xFFu) - 1, type = (int)((fd >> 16) & 0xFFu);
  Move mv;
  mv.m1 = 0;
  switch (type) {
    case kTop: {  // BL | BR << 2 on row 0
      const uint32_t s = 2u * (uint32_t)b;
      mv.r0 = 0;
      mv.idx = sig_base(kTop) + ((uint32_t)(rows[0] >> s) & 0xFu);
      mv.m0 = 0x9ull << s;
      break;
    }
    case kBottom: {  // TL | TR << 2 on row d-1
      const uint32_t s = 2u * (uint32_t)b;
      mv.r0 = d - 1;
      mv.idx = sig_base(kBottom) + ((uint32_t)(rows[(size_t)(d - 1) * kVarThreads] >> s) & 0xFu);
      mv.m0 = 0x6ull << s;
      break;
    }
    case kLeft: {  // TR | BR << 2, column 0
      mv.r0 = a;
      const uint64_t v0 = rows[(size_t)a * kVarThreads], v1 = rows[(size_t)(a + 1) * kVarThreads];
      mv.idx = sig_base(kLeft) + (((uint32_t)v0 & 3u) | (((uint32_t)v1 & 3u) << 2));
      mv.m0 = 1ull;
      mv.m1 = 2ull;
      break;
    }
    case kRight: {  // TL | BL << 2, column d-1
      const uint32_t s = 2u * (uint32_t)(d - 1);
      mv.r0 = a;
      const uint64_t v0 = rows[(size_t)a * kVarThreads], v1 = rows[(size_t)(a + 1) * kVarThreads];
      mv.idx = sig_base(kRight) + (((uint32_t)(v0 >> s) & 3u) | (((uint32_t)(v1 >> s) & 3u) << 2));
      mv.m0 = 2ull << s;
      mv.m1 = 1ull << s;
      break;
    }
    default: {  // TL | TR << 2 | BL << 4 | BR << 6
      const uint32_t s = 2u * (uint32_t)b;
      mv.r0 = a;
      const uint64_t v0 = rows[(size_t)a * kVarThreads], v1 = rows[(size_t)(a + 1) * kVarThreads];
      mv.idx = ((uint32_t)(v0 >> s) & 0xFu) | (((uint32_t)(v1 >> s) & 0xFu) << 4);
      mv.m0 = 0x6ull << s;
      mv.m1 = 0x9ull << s;
      break;
    }
  }
  return mv;
}

__device__ __forceinline__ void apply_move(const Move& mv, uint64_t* rows) {
  rows[(size_t)mv.r0 * kVarThreads] ^= mv.m0;
  if (mv.m1) rows[(size_t)(mv.r0 + 1) * kVarThreads] ^= mv.m1;
}

// Rows (stride kVarThreads) -> planar words (x plane then z plane).
__device__ void store_rows_rt(const uint64_t* rows, int d, int W, uint32_t* __restrict__ cfg) {
  const int nq = d * d;
  for (int j = 0; j < W; ++j) {
    uint32_t wx = 0u, wz = 0u;
    const int lo = 32 * j, hi = min(lo + 32, nq);
    for (int r = lo / d; r * d < hi; ++r) {
      const uint64_t v = rows[(size_t)r * kVarThreads];
      const uint32_t fz = core::gather2(v), fx = core::gather2(v >> 1);
      const int start = r * d - lo;
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

__device__ __forceinline__ void copy_rows(const uint64_t* src, uint64_t* dst, int d) {
  for (int r = 0; r < d; ++r) dst[(size_t)r * kVarThreads] = src[(size_t)r * kVarThreads];
}

// Shared memory: static (dE, class) table, per-warp sweep tables, face
// descriptors, then current and minimum-energy rows of every chain.
size_t variant_smem_bytes(int d, int m) {
  size_t b = kLutN * sizeof(int2) + (kVarThreads / 32) * kLutN * sizeof(uint2) + (size_t)m * sizeof(uint32_t);
  b = (b + 15) & ~(size_t)15;
  return b + 2 * (size_t)d * kVarThreads * sizeof(uint64_t);
}

__global__ void __launch_bounds__(kVarThreads) anneal_variant_kernel(const __grid_constant__ VariantArgs A) {
  extern __shared__ __align__(16) uint8_t smem[];
  int2* sig_static = reinterpret_cast<int2*>(smem);
  uint2* lut_all = reinterpret_cast<uint2*>(smem + kLutN * sizeof(int2));
  uint32_t* faces = reinterpret_cast<uint32_t*>(smem + kLutN * sizeof(int2) + (kVarThreads / 32) * kLutN * sizeof(uint2));
  size_t off = kLutN * sizeof(int2) + (kVarThreads / 32) * kLutN * sizeof(uint2) + (size_t)A.m * sizeof(uint32_t);
  off = (off + 15) & ~(size_t)15;
  const int tid = threadIdx.x, lane = tid & 31;
  uint64_t* rows = reinterpret_cast<uint64_t*>(smem + off) + tid;
  uint64_t* best = rows + (size_t)A.d * kVarThreads;
  uint2* L = lut_all + (tid >> 5) * kLutN;

  const int64_t c_raw = (int64_t)blockIdx.x * kVarThreads + tid;
  const bool active = c_raw < A.n_chains;
  const int64_t c = active ? c_raw : A.n_chains - 1;  // inactive threads shadow a real chain
  const uint64_t chain = A.chain0 + (uint64_t)c;
  const uint32_t c2 = (uint32_t)chain;
  const uint32_t c3_sa = kTagSA | ((uint32_t)(chain >> 32) << 8);
  const uint32_t c3_site = kTagSite | ((uint32_t)(chain >> 32) << 8);
  const int d = A.d, m = A.m, P = (int)(c & 3);

  for (int i = tid; i < kLutN; i += kVarThreads) sig_static[i] = __ldg(&A.sig[i]);
  for (int f = tid; f < m; f += kVarThreads) faces[f] = face_desc(A.face_a[f], A.face_b[f], d);
  __syncthreads();
  if (A.n_sweeps > 0) core::build_lut_warp(L, sig_static, A.T, lane);

  // R_i L_P (L_X: column 0, X on even rows and Z on odd rows; L_Z: row 0, Z on
  // even columns and X on odd columns).
  const uint32_t* init = A.init + (size_t)(c >> 2) * 2 * A.W;
  int32_t nx = 0, ny = 0, nz = 0;
  for (int r = 0; r < d; ++r) {
    const uint32_t x = core::plane_field(init, A.W, r * d, d);
    const uint32_t z = core::plane_field(init + A.W, A.W, r * d, d);
    uint64_t v = core::spread2(z) | (core::spread2(x) << 1);
    if (P == 1 || P == 2) v ^= (r & 1) ? 1ull : 2ull;
    if ((P == 2 || P == 3) && r == 0) v ^= 0x9999999999999999ull & ((1ull << (2 * d)) - 1ull);
    rows[(size_t)r * kVarThreads] = v;
    best[(size_t)r * kVarThreads] = v;
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
        const Move mv = face_move(faces[f], rows, d);
        const uint2 e = L[mv.idx];
        const int32_t dE = (int32_t)e.x;
        if ((dE <= 0) | (u_acc < e.y)) {
          apply_move(mv, rows);
          E += dE;
        }
        if (per_attempt && E < E_best) {
          E_best = E;
          copy_rows(rows, best, d);
        }
      }
      if (E < E_best) {
        E_best = E;
        copy_rows(rows, best, d);
      }
    } else {
      for (int colour = 0; colour < 4; ++colour) {
        for (int f = A.colour_start[colour]; f < A.colour_start[colour + 1]; ++f) {
          const uint32_t fd = faces[f];
          const Move mv = face_move(fd, rows, d);
          const uint2 e = L[mv.idx];
          const int32_t dE = (int32_t)e.x;
          bool acc = dE <= 0;
          if (!acc) {
            const uint32_t ia = (fd & 0xFFu) >> 1, ib = ((fd >> 8) & 0xFFu) >> 1;  // (a+1)>>1, (b+1)>>1
            const uint4 r = philox4x32_10(((uint32_t)colour << 16) | (ib << 8) | (ia >> 2), tt, c2, c3_sa, A.keys);
            acc = lane_of(r, (int)(ia & 3u)) < e.y;
          }
          if (acc) {
            apply_move(mv, rows);
            E += dE;
          }
          if (per_attempt && E < E_best) {
            E_best = E;
            copy_rows(rows, best, d);
          }
        }
        if (E < E_best) {
          E_best = E;
          copy_rows(rows, best, d);
        }
      }
    }
    if (t + 1 < A.n_sweeps) {  // next sweep's thresholds, once every lane is done with these
      __syncwarp();
      core::build_lut_warp(L, sig_static, A.T + (size_t)(t + 1) * A.n_classes, lane);
      __syncwarp();
    }
  }

  if (!active) return;
  A.best_E[c] = E_best;
  if (A.final_E) A.final_E[c] = E;
  if (A.final_cfg) store_rows_rt(rows, d, A.W, A.final_cfg + (size_t)c * 2 * A.W);
  if (A.best_cfg) store_rows_rt(best, d, A.W, A.best_cfg + (size_t)c * 2 * A.W);
}

}  // namespace

xzzx_status check_anneal_args(const xzzx_code* code, const xzzx_schedule* sched, int n_shots, int restarts);
xzzx_status launch_anneal_planar(const xzzx_code* code, const xzzx_schedule* sched, uint64_t seed, uint64_t shot0,
                                 int n_shots, int restarts, int order, int emin, const uint32_t* init, int32_t* best_E,
                                 uint32_t* best_cfg, int32_t* final_E, uint32_t* final_cfg, cudaStream_t stream);

}  // namespace xzzx

using namespace xzzx;

extern "C" xzzx_status xzzx_anneal_variant(const xzzx_code* code, const xzzx_schedule* sched, uint64_t seed,
                                           uint64_t shot0, int n_shots, int restarts, int order, int emin,
                                           const uint32_t* init, int32_t* best_E, uint32_t* best_cfg,
                                           int32_t* final_E, uint32_t* final_cfg, void* stream) {
  xzzx_status st = check_anneal_args(code, sched, n_shots, restarts);
  if (st) return st;
  if (order != 0 && order != 1) return fail(XZZX_EINVAL, "order must be 0 (colour sweep) or 1 (random site)");
  if (emin != 0 && emin != 1) return fail(XZZX_EINVAL, "emin must be 0 (per phase) or 1 (per attempt)");
  if (n_shots == 0) return XZZX_OK;
  if ((st = check_ptr(init, "init")) || (st = check_ptr(best_E, "best_E"))) return st;
  if (code->layout == kLayoutPlanar)
    return launch_anneal_planar(code, sched, seed, shot0, n_shots, restarts, order, emin, init, best_E, best_cfg,
                                final_E, final_cfg, (cudaStream_t)stream);
  VariantArgs A;
  A.keys = philox_keys(seed);
  A.chain0 = shot0 * (uint64_t)restarts * 4u;
  A.n_chains = (int64_t)n_shots * restarts * 4;
  A.d = code->d;
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
  const size_t smem = variant_smem_bytes(A.d, A.m);
  static DeviceOnce once;
  if ((st = once.run([&]() -> xzzx_status {
         XZZX_CUDA_TRY(cudaFuncSetAttribute(anneal_variant_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)variant_smem_bytes(kMaxD, kMaxD * kMaxD - 1)));
         return XZZX_OK;
       })))
    return st;
  const int64_t grid = (A.n_chains + kVarThreads - 1) / kVarThreads;
  if (grid > 0x7FFFFFFF) return fail(XZZX_EINVAL, "too many chains for one launch");
  anneal_variant_kernel<<<(unsigned)grid, kVarThreads, smem, (cudaStream_t)stream>>>(A);
  XZZX_CUDA_TRY(cudaGetLastError());
  return XZZX_OK;
}
