// Register-resident annealing on the planar layout (colour sweep, minimum per
// colour phase): the planar counterpart of anneal_cta, for d <= 15.
//
// State.  One chain per thread, one 32-bit word per grid row in registers
// (row r holds its 2d-1 or d-1 qubits as two bits per slot k, column
// c = 2k + (r&1)), so a face's corners are fields of rows i-1, i and i+1 at
// shifts fixed by the column step.
//
// Sweep.  Colour C holds the faces (i, j) with i & 1 = C & 1 and
// ((i+j-1)/2) & 1 = C >> 1.  With m = i >> 1 (the row inside the class) and
// t = j >> 2 (the column step), the faces of one step t sit in every row of
// the class at slot kl = 2t + kl0(m), kl0 alternating with m; their draw block
// (C, t, m>>2) serves four consecutive rows, exactly as four faces of one
// column share a block on the rotated lattice.  The step loop runs at run
// time with the rows unrolled; the edge steps of the odd-row class (left
// boundary at t = 0, right boundary at the last step) are peeled.
//
// Results equal anneal_planar_kernel in order 0 / emin 0 (same draws, same
// acceptance, same per-phase minimum), which the parity tests check.
#include "anneal_core.cuh"

namespace xzzx {
namespace {

constexpr int kRThreads = 128;
constexpr int kRLut = kSigPlanar;
constexpr uint32_t kPOffNoUp = (uint32_t)(planar_sig_base(kPNoUp) - kSigRot);
constexpr uint32_t kPOffNoDown = (uint32_t)(planar_sig_base(kPNoDown) - kSigRot);
constexpr uint32_t kPOffNoLeft = (uint32_t)(planar_sig_base(kPNoLeft) - kSigRot);
constexpr uint32_t kPOffNoRight = (uint32_t)(planar_sig_base(kPNoRight) - kSigRot);

template <int D>
struct PShape {
  static constexpr int G = 2 * D - 1;
  static constexpr int NQ = D * D + (D - 1) * (D - 1);
  static constexpr int kW = (NQ + 31) / 32;
};

__host__ __device__ constexpr int prow_start(int d, int r) { return (r >> 1) * (2 * d - 1) + ((r & 1) ? d : 0); }
__host__ __device__ constexpr int prow_len(int d, int r) { return (r & 1) ? d - 1 : d; }

struct RegArgs {
  PhiloxKeys keys;
  uint64_t chain0;
  int64_t n_chains;
  int n_sweeps, n_classes;
  int32_t W[4];
  const uint32_t* T;
  const int2* sig;
  const uint32_t* init;
  int32_t* best_E;
  uint32_t* best_cfg;
  int32_t* final_E;
  uint32_t* final_cfg;
};

template <int D>
__device__ __forceinline__ void pload(const uint32_t* __restrict__ cfg, uint32_t (&R)[PShape<D>::G]) {
  constexpr int W = PShape<D>::kW;
#pragma unroll
  for (int r = 0; r < PShape<D>::G; ++r) {
    const uint32_t x = core::plane_field(cfg, W, prow_start(D, r), prow_len(D, r));
    const uint32_t z = core::plane_field(cfg + W, W, prow_start(D, r), prow_len(D, r));
    R[r] = (uint32_t)(core::spread2(z) | (core::spread2(x) << 1));
  }
}

template <int D>
__device__ __forceinline__ void pstore(const uint32_t (&R)[PShape<D>::G], uint32_t* __restrict__ cfg) {
  constexpr int W = PShape<D>::kW;
  uint32_t px[W], pz[W];
#pragma unroll
  for (int j = 0; j < W; ++j) px[j] = pz[j] = 0u;
#pragma unroll
  for (int r = 0; r < PShape<D>::G; ++r) {
    const uint32_t fz = core::gather2(R[r]), fx = core::gather2((uint64_t)R[r] >> 1);
    const int start = prow_start(D, r), len = prow_len(D, r), wi = start >> 5, off = start & 31;
    pz[wi] |= fz << off;
    px[wi] |= fx << off;
    if (wi + 1 < W && off + len > 32) {
      pz[wi + 1] |= fz >> (32 - off);
      px[wi + 1] |= fx >> (32 - off);
    }
  }
#pragma unroll
  for (int j = 0; j < W; ++j) {
    cfg[j] = px[j];
    cfg[W + j] = pz[j];
  }
}

// Face kinds of one row at one step.
enum { kKBulk = 0, kKNoUp = 1, kKNoDown = 2, kKNoLeft = 3, kKNoRight = 4, kKNone = 5 };

// kl0 of row m of colour C: the slot of its face at step 0.
template <int C>
__host__ __device__ constexpr int kl0_of(int m) {
  return (C & 1) ? -(((C >> 1) - m - 1) & 1) : (((C >> 1) - m) & 1);
}

// Kind of the face of row m at a step of the given position (0 interior,
// 1 first step of the odd-row class, 2 its last step).
template <int D, int C, int POS>
__host__ __device__ constexpr int kind_of(int m) {
  return (C & 1) == 0 ? (m == 0 ? kKNoUp : (m == D - 1 ? kKNoDown : kKBulk))
                      : (POS == 0 ? kKBulk
                                  : POS == 1 ? (kl0_of<C>(m) == -1 ? kKNoLeft : kKBulk)
                                             : (kl0_of<C>(m) == -1 ? kKNoRight : kKNone));
}

// All faces of colour C at column step `step` (POS as kind_of) of sweep `sweep`.
template <int D, int C, int POS>
__device__ __forceinline__ void pstep(uint32_t (&R)[PShape<D>::G], int32_t& E, const uint2* __restrict__ L,
                                      uint32_t step, uint32_t sweep, uint32_t c2, uint32_t c3, const PhiloxKeys& K) {
  constexpr int CL = C & 1;
  constexpr int M = CL ? D - 1 : D;
  constexpr int NG = (M + 3) / 4;
  constexpr int G = PShape<D>::G;
  uint2 e[M];
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const int i = 2 * m + CL;
    const int kind = kind_of<D, C, POS>(m);
    // slot kl = 2 step + kl0: left corner at bit 2kl of row i, up/down at 2(kl + CL) of rows i -+ 1
    const int sm = 4 * (int)step + 2 * kl0_of<C>(m);
    const uint32_t smid = (uint32_t)(sm < 0 ? 0 : sm), sud = (uint32_t)(sm + 2 * CL);
    e[m] = make_uint2(0u, 0u);
    if (kind == kKNone) continue;
    const uint32_t up = (kind != kKNoUp) ? (R[i > 0 ? i - 1 : 0] >> sud) & 3u : 0u;
    const uint32_t dn = (kind != kKNoDown) ? (R[i + 1 < G ? i + 1 : i] >> sud) & 3u : 0u;
    uint32_t idx;
    if (kind == kKNoLeft) {
      idx = kPOffNoLeft + ((R[i] & 3u) | (up << 2) | (dn << 4));
    } else if (kind == kKNoRight) {
      idx = kPOffNoRight + (((R[i] >> smid) & 3u) | (up << 2) | (dn << 4));
    } else {
      const uint32_t lr = (R[i] >> smid) & 0xFu;
      if (kind == kKNoUp) idx = kPOffNoUp + (lr | (dn << 4));
      else if (kind == kKNoDown) idx = kPOffNoDown + (lr | (up << 4));
      else idx = lr | (up << 4) | (dn << 6);
    }
    e[m] = L[idx];
  }
  uint4 r[NG];
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    uint32_t need = 0;
#pragma unroll
    for (int m = 0; m < M; ++m)
      if ((m >> 2) == g) need |= e[m].y;
    r[g] = make_uint4(0u, 0u, 0u, 0u);
    if (__any_sync(0xFFFFFFFFu, need != 0u))
      r[g] = philox4x32_10(((uint32_t)C << 16) | (step << 8) | (uint32_t)g, sweep, c2, c3, K);
  }
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const int kind = kind_of<D, C, POS>(m);
    if (kind == kKNone) continue;
    const int i = 2 * m + CL;
    const int sm = 4 * (int)step + 2 * kl0_of<C>(m);
    const uint32_t smid = (uint32_t)(sm < 0 ? 0 : sm), sud = (uint32_t)(sm + 2 * CL);
    const uint32_t u = lane_of(r[m >> 2], m & 3);
    const int32_t dE = (int32_t)e[m].x;
    if ((dE <= 0) | (u < e[m].y)) {
      E += dE;
      if (kind == kKNoLeft) R[i] ^= 2u;
      else if (kind == kKNoRight) R[i] ^= 2u << smid;
      else R[i] ^= 0xAu << smid;
      const uint32_t mud = 1u << sud;
      if (kind != kKNoUp) R[i > 0 ? i - 1 : 0] ^= mud;
      if (kind != kKNoDown) R[i + 1 < G ? i + 1 : i] ^= mud;
    }
  }
}

// One colour phase: the column steps of colour C.
template <int D, int C>
__device__ __forceinline__ void pphase(uint32_t (&R)[PShape<D>::G], int32_t& E, const uint2* __restrict__ L,
                                       uint32_t sweep, uint32_t c2, uint32_t c3, const PhiloxKeys& K) {
  constexpr int NS = (D - 1) / 2;  // column steps of the even-row class; the odd-row class has NS + 1
  if ((C & 1) == 0) {
#pragma unroll 1
    for (int s = 0; s < NS; ++s) pstep<D, C, 0>(R, E, L, (uint32_t)s, sweep, c2, c3, K);
  } else {
    pstep<D, C, 1>(R, E, L, 0u, sweep, c2, c3, K);
#pragma unroll 1
    for (int s = 1; s < NS; ++s) pstep<D, C, 0>(R, E, L, (uint32_t)s, sweep, c2, c3, K);
    pstep<D, C, 2>(R, E, L, (uint32_t)NS, sweep, c2, c3, K);
  }
}

__device__ __forceinline__ void build_lut_planar(uint2* __restrict__ dst, const int2* __restrict__ sig_static,
                                                 const uint32_t* __restrict__ Trow, int lane) {
  for (int idx = lane; idx < kRLut; idx += 32) {
    const int2 s = sig_static[idx];
    dst[idx] = make_uint2((uint32_t)s.x, s.y >= 0 ? __ldg(&Trow[s.y]) : 0u);
  }
}

template <int D>
constexpr size_t reg_smem_bytes() {
  return kRLut * sizeof(int2) + (kRThreads / 32) * kRLut * sizeof(uint2) +
         (size_t)PShape<D>::G * kRThreads * sizeof(uint32_t);
}

template <int D>
__global__ void __launch_bounds__(kRThreads) anneal_planar_reg_kernel(const __grid_constant__ RegArgs A) {
  constexpr int G = PShape<D>::G;
  constexpr int W = PShape<D>::kW;
  extern __shared__ __align__(16) uint8_t smem[];
  int2* sig_static = reinterpret_cast<int2*>(smem);
  uint2* lut_all = reinterpret_cast<uint2*>(smem + kRLut * sizeof(int2));
  uint32_t* best_rows = reinterpret_cast<uint32_t*>(smem + kRLut * sizeof(int2) + (kRThreads / 32) * kRLut * sizeof(uint2));
  const int tid = threadIdx.x, lane = tid & 31;
  uint2* L = lut_all + (tid >> 5) * kRLut;
  const int64_t c_raw = (int64_t)blockIdx.x * kRThreads + tid;
  const bool active = c_raw < A.n_chains;
  const int64_t c = active ? c_raw : A.n_chains - 1;  // inactive threads shadow a real chain
  const uint64_t chain = A.chain0 + (uint64_t)c;
  const uint32_t c2 = (uint32_t)chain;
  const uint32_t c3 = kTagSA | ((uint32_t)(chain >> 32) << 8);
  const int P = (int)(c & 3);

  for (int k = tid; k < kRLut; k += kRThreads) sig_static[k] = __ldg(&A.sig[kSigRot + k]);
  __syncthreads();
  if (A.n_sweeps > 0) build_lut_planar(L, sig_static, A.T, lane);

  uint32_t R[G];
  pload<D>(A.init + (size_t)(c >> 2) * 2 * W, R);
  // L_X: X on column 0 (slot 0 of the even rows); L_Z: Z on every qubit of row 0.
  if (P == 1 || P == 2) {
#pragma unroll
    for (int r = 0; r < G; r += 2) R[r] ^= 2u;
  }
  if (P == 2 || P == 3) R[0] ^= (uint32_t)(0x55555555u & ((1u << (2 * D)) - 1u));
  int32_t nx = 0, ny = 0, nz = 0;
#pragma unroll
  for (int r = 0; r < G; ++r) {
    const uint32_t z = R[r] & 0x55555555u, x = (R[r] >> 1) & 0x55555555u;
    ny += __popc(x & z);
    nx += __popc(x & ~z);
    nz += __popc(z & ~x);
  }
  int32_t E = nx * A.W[2] + ny * A.W[3] + nz * A.W[1];
  int32_t E_best = E;
#pragma unroll
  for (int r = 0; r < G; ++r) best_rows[r * kRThreads + tid] = R[r];

  for (int t = 0; t < A.n_sweeps; ++t) {
    const uint32_t tt = (uint32_t)t;
#define XZZX_PPHASE(CC)                                                              \
  pphase<D, CC>(R, E, L, tt, c2, c3, A.keys);                                        \
  if (E < E_best) {                                                                  \
    E_best = E;                                                                      \
    _Pragma("unroll") for (int r = 0; r < G; ++r) best_rows[r * kRThreads + tid] = R[r]; \
  }
    XZZX_PPHASE(0)
    XZZX_PPHASE(1)
    XZZX_PPHASE(2)
    XZZX_PPHASE(3)
#undef XZZX_PPHASE
    if (t + 1 < A.n_sweeps) {
      __syncwarp();
      build_lut_planar(L, sig_static, A.T + (size_t)(t + 1) * A.n_classes, lane);
      __syncwarp();
    }
  }

  if (!active) return;
  A.best_E[c] = E_best;
  if (A.final_E) A.final_E[c] = E;
  if (A.final_cfg) pstore<D>(R, A.final_cfg + (size_t)c * 2 * W);
  if (A.best_cfg) {
#pragma unroll
    for (int r = 0; r < G; ++r) R[r] = best_rows[r * kRThreads + tid];
    pstore<D>(R, A.best_cfg + (size_t)c * 2 * W);
  }
}

template <int D>
xzzx_status launch_d(const RegArgs& A, cudaStream_t stream) {
  const size_t smem = reg_smem_bytes<D>();
  static DeviceOnce once;
  xzzx_status st = once.run([&]() -> xzzx_status {
    XZZX_CUDA_TRY(cudaFuncSetAttribute(anneal_planar_reg_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    return XZZX_OK;
  });
  if (st) return st;
  const int64_t grid = (A.n_chains + kRThreads - 1) / kRThreads;
  if (grid > 0x7FFFFFFF) return fail(XZZX_EINVAL, "too many chains for one launch");
  anneal_planar_reg_kernel<D><<<(unsigned)grid, kRThreads, smem, stream>>>(A);
  XZZX_CUDA_TRY(cudaGetLastError());
  return XZZX_OK;
}

}  // namespace

// Colour sweep with per-phase minima on a planar code, d <= 15 (arguments
// checked by the caller).
xzzx_status launch_anneal_planar_reg(const xzzx_code* code, const xzzx_schedule* sched, uint64_t seed, uint64_t shot0,
                                     int n_shots, int restarts, const uint32_t* init, int32_t* best_E,
                                     uint32_t* best_cfg, int32_t* final_E, uint32_t* final_cfg, cudaStream_t stream) {
  RegArgs A;
  A.keys = philox_keys(seed);
  A.chain0 = shot0 * (uint64_t)restarts * 4u;
  A.n_chains = (int64_t)n_shots * restarts * 4;
  A.n_sweeps = sched->n_sweeps;
  A.n_classes = sched->n_classes;
  for (int k = 0; k < 4; ++k) A.W[k] = sched->noise.W[k];
  A.T = sched->d_T;
  A.sig = sched->d_sig;
  A.init = init;
  A.best_E = best_E;
  A.best_cfg = best_cfg;
  A.final_E = final_E;
  A.final_cfg = final_cfg;
  switch (code->d) {
    case 3: return launch_d<3>(A, stream);
    case 5: return launch_d<5>(A, stream);
    case 7: return launch_d<7>(A, stream);
    case 9: return launch_d<9>(A, stream);
    case 11: return launch_d<11>(A, stream);
    case 13: return launch_d<13>(A, stream);
    case 15: return launch_d<15>(A, stream);
    default: return fail(XZZX_EUNSUPPORTED, "no register-resident planar kernel for this distance");
  }
}

}  // namespace xzzx
