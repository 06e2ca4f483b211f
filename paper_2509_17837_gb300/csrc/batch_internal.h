// Private declarations shared by the batch translation units.
#pragma once

#include <vector>

#include "internal.h"

namespace xzzx {
namespace batch {

constexpr int kNT = 128;  // default chains per CTA of the batched anneal launches (128 or 256)

// One homogeneous segment of a batch, as the kernels see it.
struct SegDev {
  DevCode code;
  uint64_t shot0;
  int n_shots, restarts, randomised, greedy_groups, greedy_rpw;
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
  // schedule (also carried by every chunk of the segment)
  const uint32_t* T;
  const int2* sig;
  int n_sweeps, n_classes;
  int32_t W[4];
};

// Up to NT (the plan's chains per CTA) consecutive chains of one segment (one
// CTA's work).
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

struct DistanceRange {
  int d;
  int seg_begin, seg_end;        // segments [begin, end) (ordered by distance)
  int chunk_begin, chunk_end;    // chunks_byd range
  int warp_smem = 0;             // mode 2: shared memory per CTA of the warp kernel (0: its own need)
};

// Distance classes of the persistent kernels: d <= 15, 17..21, 23..31.
constexpr int kNumClasses = 3;
constexpr int kClassDmax[kNumClasses] = {15, 21, 31};
inline int class_of(int d) { return d <= 15 ? 0 : (d <= 21 ? 1 : 2); }

struct ClassRange {
  int cls;                       // index into kClassDmax
  int chunk_begin, chunk_end;    // chunks_bycls range (longest first within the class)
};

// Host images of a plan: segment and chunk descriptors, prefix sums and the
// per-distance ranges.  Segment workspace pointers are assigned from a device
// base address given to build_plan.
struct Plan {
  int nt = kNT;     // chains per CTA (chunk size): 128 or 256
  int unroll = 1;   // sweep-loop unroll of the annealing kernels: 1 or 2
  std::vector<SegDev> segs;
  std::vector<ChunkDev> lpt, byd, bycls;  // longest first; by distance; by class, longest first
  std::vector<ClassRange> classes;
  std::vector<int64_t> cta_prefix, shot_prefix, chain_prefix;
  std::vector<DistanceRange> ranges;
  int dmax = 0;
  double attempts = 0;
  int64_t total_shots = 0, total_ctas = 0;
  int64_t list_cta_end = 0;  // greedy CTAs [0, list_cta_end) are of segments with d <= 17
  size_t workspace_bytes = 0;
};

// Device addresses of a plan's descriptors (one blob) and queue head.
struct PlanDev {
  SegDev* segs;
  ChunkDev* lpt;
  ChunkDev* byd;
  ChunkDev* bycls;
  int64_t* cta_prefix;
  int64_t* shot_prefix;
  int64_t* chain_prefix;
  int* head;  // 1 + kNumClasses queue heads: mode 0's, then one per class (mode 4)
};

// Validate segments and build host images; workspace pointers start at
// ws_base (may be null to size only).  order: 0 = longest chunks first.  nt:
// chains per CTA (128 or 256), unroll: sweep-loop unroll (1 or 2).
xzzx_status build_plan(const xzzx_segment* segs, int n_segs, int device, int order, char* ws_base, Plan& out,
                       int nt = kNT, int unroll = 1);
// Bytes of the descriptor blob and the layout of PlanDev inside it.
size_t descriptor_bytes(const Plan& p);
PlanDev descriptor_layout(const Plan& p, char* dev_base);
void pack_descriptors(const Plan& p, char* host_blob);
// Enqueue the decode of a plan (mode 0: batched, 1: one launch per distance,
// 2: one launch per distance with one warp per chain).  Modes 3 and 4 need
// side streams and are issued by the batch handle.
xzzx_status launch_plan(const Plan& p, const PlanDev& d, const PhiloxKeys& K, int grid, int mode,
                        cudaStream_t stream);
// Configure the chunk kernels of (nt, unroll) and the persistent kernel of
// dmax's distance class; its resident CTAs per SM go to *ctas_per_sm.
xzzx_status configure_plan_kernels(int dmax, int nt, int unroll, int* ctas_per_sm);
// The persistent kernel of a distance class: configure it (resident CTAs per
// SM to *ctas_per_sm) and launch it.
xzzx_status configure_persistent(int dmax, int nt, int unroll, int* ctas_per_sm);
xzzx_status launch_persistent(int dmax, int nt, int unroll, const AnnealLaunch& L, int grid, cudaStream_t stream);
AnnealLaunch anneal_launch(const PlanDev& d, const PhiloxKeys& K, const ChunkDev* chunks, int chunk0, int n,
                           int* head);

// Per-distance chunk kernel (one CTA per chunk).
xzzx_status launch_chunks(int d, int nt, int unroll, const AnnealLaunch& L, cudaStream_t stream);
// Resident CTAs per SM of the distance-d chunk kernel (configured first).
xzzx_status occupancy_chunks(int d, int nt, int unroll, int* ctas_per_sm);

// The variants, instantiated in batch_chunks_nt*_u*.cu and batch_persist*.cu.
template <int NT, int U>
xzzx_status launch_chunks_v(int d, const AnnealLaunch& L, cudaStream_t stream);
template <int NT, int U>
xzzx_status configure_chunks_v();
template <int NT, int U>
xzzx_status occupancy_chunks_v(int d, int* ctas_per_sm);
template <int DMAX, int NT, int U>
xzzx_status launch_persistent_v(const AnnealLaunch& L, int grid, cudaStream_t stream);
template <int DMAX, int NT, int U>
xzzx_status configure_persistent_v(int* ctas_per_sm);

// Per-distance warp-per-chain kernel over the chains [chain0, chain0 + n).
struct WarpLaunch {
  PhiloxKeys keys;
  const SegDev* segs;
  const int64_t* chain_prefix;
  int n_segs;
  int64_t chain0, n_chains;
  int smem;  // dynamic shared memory per CTA; below the kernel's need means its need
};
xzzx_status launch_warp_chains(int d, const WarpLaunch& L, cudaStream_t stream);
// Configure the distance-d warp kernel for at most cap resident CTAs per SM
// (0: no cap) by padding its shared memory: bytes per CTA to *smem, the
// resulting resident CTAs per SM to *ctas_per_sm.
xzzx_status configure_warp_chains(int d, int cap, int* smem, int* ctas_per_sm);

}  // namespace batch
}  // namespace xzzx
