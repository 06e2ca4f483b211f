// Code-capacity noise sampling and syndrome extraction (Sec. "Simulation
// setting"; Eqs. noise_map, G_f_comm_anticomm).  One warp per shot: the lanes
// draw the qubits four at a time from Philox, assemble the two bit planes in
// shared memory, then evaluate every generator's parity and ballot the
// syndrome words.
#include <cmath>

#include "internal.h"
#include "philox.cuh"

namespace xzzx {
namespace {

constexpr int kWarps = 4;
constexpr int kMaxWords = 64;  // words per bit plane: 59 for the planar d = 31 code

struct SampleArgs {
  DevCode code;
  PhiloxKeys keys;
  uint64_t shot0;
  int n_shots;
  uint64_t Tx, Txy, Txyz;  // cumulative thresholds floor(p 2^32)
  uint32_t* errors;        // n_shots x 2w or null
  uint32_t* syndromes;     // n_shots x sw
};

__global__ void __launch_bounds__(kWarps * 32) sample_kernel(const __grid_constant__ SampleArgs A) {
  __shared__ uint32_t planes[kWarps][2 * kMaxWords];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t k = (int64_t)blockIdx.x * kWarps + warp;
  if (k >= A.n_shots) return;
  const DevCode& C = A.code;
  const int w = C.w, d = C.d;
  uint32_t* P = planes[warp];
  for (int i = lane; i < 2 * w; i += 32) P[i] = 0u;
  __syncwarp();
  const uint64_t shot = A.shot0 + (uint64_t)k;
  const int n_blocks = (C.nq + 3) >> 2;
  for (int blk = lane; blk < n_blocks; blk += 32) {
    const uint4 r = philox4x32_10((uint32_t)blk, (uint32_t)shot, (uint32_t)(shot >> 32), kTagNoise, A.keys);
    for (int j = 0; j < 4; ++j) {
      const int q = 4 * blk + j;
      if (q >= C.nq) break;
      const uint64_t u = lane_of(r, j);
      const bool x = u < A.Txy;                       // X or Y
      const bool z = u >= A.Tx && u < A.Txyz;         // Y or Z
      if (x) atomicOr(&P[q >> 5], 1u << (q & 31));
      if (z) atomicOr(&P[w + (q >> 5)], 1u << (q & 31));
    }
  }
  __syncwarp();
  if (A.errors) {
    uint32_t* out = A.errors + (size_t)k * 2 * w;
    for (int i = lane; i < 2 * w; i += 32) out[i] = P[i];
  }
  // s_f: X corners (rotated TL, BR; planar left, right) see the Z bit, Z
  // corners (rotated TR, BL; planar up, down) see the X bit.
  const bool planar = C.layout == kLayoutPlanar;
  const int g = planar ? 2 * d - 1 : d;
  for (int base = 0; base < C.ns; base += 32) {
    const int f = base + lane;
    int bit = 0;
    if (f < C.ns) {
      const int a = C.face_a[f], b = C.face_b[f];
      int rr[4], cc[4];
      if (planar) {  // left, up, down, right
        rr[0] = a; cc[0] = b - 1;
        rr[1] = a - 1; cc[1] = b;
        rr[2] = a + 1; cc[2] = b;
        rr[3] = a; cc[3] = b + 1;
      } else {  // TL, TR, BL, BR
        rr[0] = a; cc[0] = b;
        rr[1] = a; cc[1] = b + 1;
        rr[2] = a + 1; cc[2] = b;
        rr[3] = a + 1; cc[3] = b + 1;
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (rr[c] < 0 || rr[c] >= g || cc[c] < 0 || cc[c] >= g) continue;
        const int q = planar ? planar_qubit(d, rr[c], cc[c]) : rr[c] * d + cc[c];
        const int plane = (c == 0 || c == 3) ? w : 0;
        bit ^= (P[plane + (q >> 5)] >> (q & 31)) & 1;
      }
    }
    const uint32_t word = __ballot_sync(0xFFFFFFFFu, bit);
    if (lane == 0) A.syndromes[(size_t)k * C.sw + (base >> 5)] = word;
  }
}

}  // namespace
}  // namespace xzzx

using namespace xzzx;

extern "C" xzzx_status xzzx_sample_errors(const xzzx_code* code, const xzzx_noise* noise, uint64_t seed,
                                          uint64_t shot0, int n_shots, uint32_t* errors, uint32_t* syndromes,
                                          void* stream) {
  xzzx_status st = check_code(code);
  if (st) return st;
  if (!noise) return fail(XZZX_EINVAL, "noise is NULL");
  if (n_shots < 0) return fail(XZZX_EINVAL, "n_shots < 0");
  if (n_shots == 0) return XZZX_OK;
  if ((st = check_ptr(syndromes, "syndromes"))) return st;
  if (!(noise->px >= 0 && noise->py >= 0 && noise->pz >= 0 && noise->px + noise->py + noise->pz <= 1.0))
    return fail(XZZX_EINVAL, "probabilities out of range");
  SampleArgs A;
  A.code = code->dev;
  A.keys = philox_keys(seed);
  A.shot0 = shot0;
  A.n_shots = n_shots;
  const uint64_t Tx = (uint64_t)std::floor(std::ldexp(noise->px, 32));
  const uint64_t Ty = (uint64_t)std::floor(std::ldexp(noise->py, 32));
  const uint64_t Tz = (uint64_t)std::floor(std::ldexp(noise->pz, 32));
  A.Tx = Tx;
  A.Txy = Tx + Ty;
  A.Txyz = Tx + Ty + Tz;
  A.errors = errors;
  A.syndromes = syndromes;
  const unsigned grid = (unsigned)((n_shots + kWarps - 1) / kWarps);
  sample_kernel<<<grid, kWarps * 32, 0, (cudaStream_t)stream>>>(A);
  XZZX_CUDA_TRY(cudaGetLastError());
  return XZZX_OK;
}
