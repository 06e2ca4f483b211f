// xzzx_decode_batch_static: the whole decoder without any device allocation.
//
// Some callers cannot allocate device memory once they are running.  A
// decoder embedded in a control loop may have its GPU memory plan fixed at
// start-up and must not risk an allocation that stalls or fails mid-run.  A
// plain C host may only receive device buffers from another component and
// has no allocator of its own to call.  This entry point serves them: the
// intermediates live in a scratch array compiled into the library, so the
// call itself allocates nothing.  The caller still passes inputs and outputs.
//
// Limits and sharing:
//  * the scratch is kStaticScratchBytes (16 MiB) per GPU; every GPU that loads
//    the library holds it until the process exits;
//  * a batch whose intermediates do not fit is rejected with XZZX_EINVAL
//    (split it into smaller batches);
//  * every call shares the one array; calls whose work overlaps on the GPU
//    (different streams, or different host threads) race on it and must be
//    serialised by the caller;
//  * nothing in the scratch needs to start at zero: each call writes every
//    scratch byte before reading it, so leftovers from the last call do not
//    matter;
//  * the first call on a device looks up the array's device address with
//    cudaGetSymbolAddress (device current, once per device); make that first
//    call before any stream capture.  With lazy module loading (the CUDA
//    default) that lookup is also what loads this file's module on the
//    device, so the 16 MiB are committed by the first call, not when the
//    library is loaded.  A caller that must not allocate later makes one
//    warm-up call with n_shots = 0 at start-up: it does the lookup and
//    decodes nothing;
//  * the address is cached per device index for the life of the process; a
//    cudaDeviceReset of a device destroys the array it points to, so the
//    entry point must not be used on that device after such a reset.
#include <mutex>

#include "internal.h"

namespace xzzx {
namespace {

constexpr size_t kStaticScratchBytes = XZZX_STATIC_SCRATCH_BYTES;
static_assert(kStaticScratchBytes == ((size_t)16 << 20), "the header states 16 MiB");
constexpr int kMaxDevices = 64;

// The array's name is only a host-side stand-in for it; host code must pass
// the address obtained from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

xzzx_status scratch_address(void** out) {
  int dev = -1;
  XZZX_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(XZZX_EINVAL, "device index beyond the static scratch table");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return XZZX_OK;
}

}  // namespace
}  // namespace xzzx

using namespace xzzx;

extern "C" xzzx_status xzzx_decode_batch_static(const xzzx_code* code, const xzzx_noise* noise,
                                                const xzzx_schedule* sched, uint64_t seed, uint64_t shot0,
                                                int n_shots, int restarts, int randomised, const uint32_t* syndromes,
                                                const uint32_t* true_errors, uint8_t* cls, int32_t* E4,
                                                uint32_t* recovery, uint32_t* best_cfg_out, uint8_t* fail_out,
                                                void* stream) {
  if (!code) return fail(XZZX_EINVAL, "code is NULL");
  size_t need = 0;
  xzzx_status st = xzzx_decode_workspace_size(code, n_shots, restarts, best_cfg_out != nullptr, &need);
  if (st) return st;
  if (need > kStaticScratchBytes)
    return fail(XZZX_EINVAL, "batch needs " + std::to_string(need) + " bytes of scratch but the built-in scratch holds " +
                                 std::to_string(kStaticScratchBytes) + "; split the batch");
  void* scratch = nullptr;
  if ((st = scratch_address(&scratch))) return st;
  return xzzx_decode_batch(code, noise, sched, seed, shot0, n_shots, restarts, randomised, syndromes, true_errors,
                           cls, E4, recovery, best_cfg_out, fail_out, scratch, kStaticScratchBytes, stream);
}
