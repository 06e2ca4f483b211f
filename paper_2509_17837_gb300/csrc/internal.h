// Private declarations of libxzzx (GB300 path).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/xzzx.h"

namespace xzzx {

// ---------------------------------------------------------------------------
// Error reporting: thread-local message behind xzzx_last_error().
// ---------------------------------------------------------------------------
xzzx_status fail(xzzx_status st, const std::string& msg);
xzzx_status ok();
xzzx_status cuda_fail(cudaError_t e, const char* what);

// One-time setup per device (a kernel's dynamic shared memory limit belongs to
// the device context it is set on).  Two threads may both run the setup; it
// is idempotent.
class DeviceOnce {
 public:
  // Runs fn() unless it already ran for the current device.
  template <typename F>
  xzzx_status run(F fn) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    const uint64_t bit = dev < 64 ? (1ull << dev) : 0ull;
    if (bit && (done_.load(std::memory_order_acquire) & bit)) return XZZX_OK;
    xzzx_status st = fn();
    if (st == XZZX_OK && bit) done_.fetch_or(bit, std::memory_order_acq_rel);
    return st;
  }

 private:
  std::atomic<uint64_t> done_{0};
};

// NVTX range around the host-side enqueue of one step of the path, so a
// timeline tool shows greedy (K1), annealing (K2) and decision (K3) launches by
// name.  Costs a few nanoseconds when no tool is attached.
class NvtxRange {
 public:
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

#define XZZX_CUDA_TRY(expr)                                    \
  do {                                                         \
    cudaError_t e_ = (expr);                                   \
    if (e_ != cudaSuccess) return ::xzzx::cuda_fail(e_, #expr); \
  } while (0)

// Largest distance the kernels are built for (one 64-bit interleaved word per
// lattice row: 2 bits per qubit).
constexpr int kMaxD = 31;

// Philox purposes (top byte layout of the last counter word).  kTagSite keys
// the site and acceptance draws of the random-site Metropolis variant.
constexpr uint32_t kTagNoise = 1, kTagGreedy = 2, kTagSA = 3, kTagSite = 4;

// Sentinel index of the virtual boundary vertex in greedy pair keys.
constexpr uint32_t kBoundary = 0xFFFFu;

// Code layouts: the rotated d x d lattice and the paper's planar lattice
// (qubits on the sites (r, c), r + c even, of a (2d-1) x (2d-1) grid).
constexpr int kLayoutRotated = 0, kLayoutPlanar = 1;

// Rotated generator shapes: the bulk weight-4 face and the four weight-2
// boundary faces, by which corners exist.  Signature bits: TL 0-1, TR 2-3,
// BL 4-5, BR 6-7.
enum FaceType { kBulk = 0, kTop = 1, kBottom = 2, kLeft = 3, kRight = 4, kNumTypes = 5 };
constexpr int kCornerMask[kNumTypes] = {0xF, 0xC, 0x3, 0xA, 0x5};  // bit k = corner k present
// Compact signature table of the rotated shapes: the 256 bulk signatures, then
// 16 entries per weight-2 shape indexed by its two present corners (the first
// present corner in bits 0-1, the second in bits 2-3).
constexpr int kSigRot = 256 + 4 * 16;
__host__ __device__ constexpr int sig_base(int type) { return type == kBulk ? 0 : 256 + 16 * (type - 1); }

// Planar generator shapes.  Corner order left, right, up, down (Paulis X, X,
// Z, Z); the bulk signature is left | right<<2 | up<<4 | down<<6, a
// three-body shape's signature its three present corners in that order.
enum PlanarShape { kPBulk = 0, kPNoUp = 1, kPNoDown = 2, kPNoLeft = 3, kPNoRight = 4, kNumPShapes = 5 };
constexpr int kPlanarCornerMask[kNumPShapes] = {0xF, 0xB, 0x7, 0xE, 0xD};
constexpr int kSigPlanar = 256 + 4 * 64;
__host__ __device__ constexpr int planar_sig_base(int shape) {
  return kSigRot + (shape == kPBulk ? 0 : 256 + 64 * (shape - 1));
}
// The schedule's (dE, class) table holds both: rotated entries [0, kSigRot),
// planar entries [kSigRot, kSigTable).
constexpr int kSigTable = kSigRot + kSigPlanar;

// Round keys of Philox4x32-10 for one seed, in kernel-parameter space.
struct PhiloxKeys {
  uint32_t k0[10], k1[10];
};
PhiloxKeys philox_keys(uint64_t seed);

// Device view of a code (pointers into the tables owned by xzzx_code).
struct DevCode {
  int d, nq, ns, w, sw;
  int layout;                // kLayoutRotated or kLayoutPlanar
  int colour_start[5];
  const int16_t* face_a;     // ns (planar: row i of the face site)
  const int16_t* face_b;     // ns (planar: column j)
  const uint8_t* face_c2;    // ns, decoding-graph colour
  const int16_t* face_at;    // rotated (d+1)^2 at (a+1)*(d+1)+(b+1); planar (2d-1)^2 at i*(2d-1)+j; -1 = none
  const uint32_t* logical;   // 2 x 2w words: L_X then L_Z, bit planes
  uint32_t* err;             // kErrWords: device-side error flags of work done with this code
};

// Device-side error area of a code (kErrWords words): [0] the OR of the
// XZZX_DEVERR_* flags raised, [1] how many times one was raised, [2] flags
// the host asks the kernels to raise as if the failure had happened (a test
// hook that faults nothing), [3] unused.
constexpr int kErrWords = 4;

#ifdef __CUDACC__
__device__ __forceinline__ void raise_device_error(uint32_t* err, uint32_t flag) {
  atomicOr(&err[0], flag);
  atomicAdd(&err[1], 1u);
}
__device__ __forceinline__ bool injected(const uint32_t* err, uint32_t flag) {
  return (*(volatile const uint32_t*)&err[2] & flag) != 0u;
}
#endif

// Bounds checks of the XZZX_CHECKS build: a failed check raises
// XZZX_DEVERR_BOUNDS and the caller skips the access.  The plain build
// compiles them out.
#ifdef XZZX_CHECKS
#define XZZX_CHECK(err, cond) ((cond) ? true : (::xzzx::raise_device_error((err), XZZX_DEVERR_BOUNDS), false))
#else
#define XZZX_CHECK(err, cond) true
#endif

// Planar qubit index of site (r, c), r + c even, inside the (2d-1)^2 grid:
// row-major over the qubit sites.
__host__ __device__ inline int planar_qubit(int d, int r, int c) {
  return (r >> 1) * (2 * d - 1) + ((r & 1) ? d : 0) + (c >> 1);
}

}  // namespace xzzx

struct xzzx_code {
  int d = 0, nq = 0, ns = 0, w = 0, sw = 0;
  int layout = 0;
  int colour_start[5] = {0, 0, 0, 0, 0};
  int device = -1;
  std::vector<int16_t> a, b;
  std::vector<uint8_t> c2, c4;
  std::vector<int32_t> corners;   // 4 per face
  std::vector<int16_t> face_at;
  std::vector<uint32_t> logical;  // L_X (2w) then L_Z (2w)
  void* dev_block = nullptr;      // one allocation holding the device tables
  xzzx::DevCode dev{};
};

struct xzzx_schedule {
  int kind = 0, n_sweeps = 0;
  double beta0 = 0, beta1 = 0;
  xzzx_noise noise{};
  int device = -1;
  int n_classes = 0;
  std::vector<int32_t> dE_class;        // positive dE values, ascending
  std::vector<uint32_t> T;              // n_sweeps x n_classes
  std::vector<int32_t> sig_dE;          // kSigTable entries
  std::vector<int32_t> sig_class;       // kSigTable entries, class index or -1 (dE <= 0)
  uint32_t* d_T = nullptr;              // device copy of T (at least one row)
  int2* d_sig = nullptr;                // device (dE, class) per compact signature
};

namespace xzzx {
// Validation helpers shared by the entry points.
xzzx_status check_code(const xzzx_code* code);
xzzx_status check_device(int device);
xzzx_status check_ptr(const void* p, const char* name);
}  // namespace xzzx
