// Private declarations shared by the batch translation units.
#pragma once

#include "internal.h"

namespace xzzx {
namespace batch {

constexpr int kNT = 128;  // chains per CTA in every batched anneal launch

// One homogeneous segment of a batch, as the kernels see it.
struct SegDev {
  DevCode code;
  uint64_t shot0;
  int n_shots, restarts, randomised, greedy_groups;
  int32_t Wt_x, Wt_z;
  const uint32_t* syndromes;
  const uint32_t* true_errors;
  uint8_t* cls;
  int32_t* E4;
  uint32_t* recovery;
  uint8_t* fail;
  uint32_t* init;     // workspace: n_shots x restarts x 2w words
  uint8_t* cbits;     // workspace: n_shots x restarts
  int32_t* chain_E;   // workspace: n_shots x restarts x 4
};

// kNT consecutive chains of one segment (one CTA's work).
struct ChunkDev {
  int seg, d, first_chain, n_chains;
  const uint32_t* T;
  const int2* sig;
  int n_sweeps, n_classes;
  int32_t W[4];
};

struct AnnealLaunch {
  PhiloxKeys keys;
  const SegDev* segs;
  const ChunkDev* chunks;
  int chunk0, n_chunks;
  int* head;  // persistent queue head (reset to 0 before the launch)
};

// Per-distance chunk kernel (one CTA per chunk) and persistent kernels
// serving every odd distance up to DMAX.
xzzx_status launch_chunks(int d, const AnnealLaunch& L, cudaStream_t stream);
xzzx_status launch_persistent(int dmax, const AnnealLaunch& L, int grid, cudaStream_t stream);
xzzx_status persistent_occupancy(int dmax, int* ctas_per_sm);
xzzx_status configure_kernels(int dmax);

}  // namespace batch
}  // namespace xzzx
