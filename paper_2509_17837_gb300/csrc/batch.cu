// Batches of many homogeneous segments decoded together (uneven distances,
// noise classes, schedules and restarts in one run).
//
// A batch is built once (xzzx_batch_create): segments are ordered by distance,
// their intermediates get one workspace allocation owned by the batch, and
// their chains are cut into chunks of kNT chains (one CTA each).  A run then
// issues, on the caller's stream:
//   mode 0 (batched): one greedy launch over every (segment, shot, restart
//          group), one persistent annealing launch whose CTAs pull chunks,
//          longest first, from an atomic counter, and one decision launch;
//   mode 1 (plain):   the same three kernels once per distance.
// Every chain uses the chain id it would get from xzzx_decode_batch on its
// segment alone, so both modes, and per-segment calls, agree bit for bit.
// xzzx_batch_run_graph captures mode 0 into a CUDA graph on its first call
// and replays that graph afterwards.
#include <algorithm>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "batch_internal.h"
#include "greedy_core.cuh"
#include "reduce_core.cuh"

namespace xzzx {
namespace batch {

xzzx_status launch_persistent_15(const AnnealLaunch&, int, cudaStream_t);
xzzx_status launch_persistent_21(const AnnealLaunch&, int, cudaStream_t);
xzzx_status launch_persistent_31(const AnnealLaunch&, int, cudaStream_t);
xzzx_status configure_persistent_15();
xzzx_status configure_persistent_21();
xzzx_status configure_persistent_31();
xzzx_status occupancy_persistent_15(int*);
xzzx_status occupancy_persistent_21(int*);
xzzx_status occupancy_persistent_31(int*);
xzzx_status configure_chunk_kernels();

namespace {

constexpr int kGreedyWarps = greedy::kWarps;
constexpr int kReduceWarps = 4;

// Index of the segment whose [prefix[s], prefix[s+1]) range holds x.
__device__ __forceinline__ int find_segment(const int64_t* __restrict__ prefix, int n_segs, int64_t x) {
  int lo = 0, hi = n_segs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

struct GreedyLaunch {
  PhiloxKeys keys;
  const SegDev* segs;
  const int64_t* cta_prefix;  // n_segs + 1
  int n_segs;
  int64_t cta0;
};

__global__ void __launch_bounds__(kGreedyWarps * 32) greedy_batch_kernel(const __grid_constant__ GreedyLaunch G) {
  __shared__ greedy::Shared S;
  const int64_t b = G.cta0 + blockIdx.x;
  const int s = find_segment(G.cta_prefix, G.n_segs, b);
  const SegDev& sg = G.segs[s];
  const int64_t local = b - G.cta_prefix[s];
  const int64_t k = local / sg.greedy_groups;
  const int group = (int)(local % sg.greedy_groups);
  greedy::greedy_cta(sg.code, G.keys, sg.shot0 + (uint64_t)k, group, sg.restarts, sg.randomised, sg.Wt_x, sg.Wt_z,
                     sg.syndromes + (size_t)k * sg.code.sw, sg.init + (size_t)k * sg.restarts * 2 * sg.code.w,
                     sg.cbits + (size_t)k * sg.restarts, S);
}

struct ReduceLaunch {
  const SegDev* segs;
  const int64_t* shot_prefix;  // n_segs + 1
  int n_segs;
  int64_t shot0, n_shots;      // global shot range of this launch
};

__global__ void __launch_bounds__(kReduceWarps * 32) reduce_batch_kernel(const __grid_constant__ ReduceLaunch L) {
  const int64_t g = (int64_t)blockIdx.x * kReduceWarps + (threadIdx.x >> 5);
  if (g >= L.n_shots) return;
  const int64_t x = L.shot0 + g;
  const int s = find_segment(L.shot_prefix, L.n_segs, x);
  const SegDev& sg = L.segs[s];
  const int64_t k = x - L.shot_prefix[s];
  const int R = sg.restarts, w = sg.code.w;
  reduce::reduce_warp(sg.code, R, sg.init + (size_t)k * R * 2 * w, sg.cbits + (size_t)k * R,
                      sg.chain_E + (size_t)k * 4 * R, nullptr,
                      sg.true_errors ? sg.true_errors + (size_t)k * 2 * w : nullptr, sg.cls + k, sg.E4 + 4 * k,
                      sg.recovery + (size_t)k * 2 * w, nullptr, sg.fail ? sg.fail + k : nullptr);
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

struct DistanceRange {
  int d;
  int seg_begin, seg_end;        // segments [begin, end) (ordered by distance)
  int chunk_begin, chunk_end;    // chunks_byd range
};

}  // namespace batch
}  // namespace xzzx

struct xzzx_batch {
  int device = -1;
  uint64_t seed = 0;
  xzzx::PhiloxKeys keys{};
  int n_segs = 0, n_chunks = 0, dmax = 0;
  int grid = 0;
  int64_t total_greedy_ctas = 0, total_shots = 0;
  double attempts = 0;
  std::vector<xzzx::batch::DistanceRange> ranges;
  void* dev_block = nullptr;  // descriptors + workspace
  xzzx::batch::SegDev* d_segs = nullptr;
  xzzx::batch::ChunkDev* d_chunks_lpt = nullptr;
  xzzx::batch::ChunkDev* d_chunks_byd = nullptr;
  int64_t* d_cta_prefix = nullptr;
  int64_t* d_shot_prefix = nullptr;
  int* d_head = nullptr;
  std::vector<int64_t> cta_prefix, shot_prefix;
  size_t workspace_bytes = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
};

namespace xzzx {
namespace batch {
namespace {

xzzx_status run_greedy(const xzzx_batch* b, int64_t cta0, int64_t n_ctas, cudaStream_t stream) {
  if (n_ctas <= 0) return XZZX_OK;
  GreedyLaunch G;
  G.keys = b->keys;
  G.segs = b->d_segs;
  G.cta_prefix = b->d_cta_prefix;
  G.n_segs = b->n_segs;
  G.cta0 = cta0;
  if (n_ctas > 0x7FFFFFFF) return fail(XZZX_EINVAL, "too many greedy CTAs in one launch");
  greedy_batch_kernel<<<(unsigned)n_ctas, kGreedyWarps * 32, 0, stream>>>(G);
  XZZX_CUDA_TRY(cudaGetLastError());
  return XZZX_OK;
}

xzzx_status run_reduce(const xzzx_batch* b, int64_t shot0, int64_t n_shots, cudaStream_t stream) {
  if (n_shots <= 0) return XZZX_OK;
  ReduceLaunch L;
  L.segs = b->d_segs;
  L.shot_prefix = b->d_shot_prefix;
  L.n_segs = b->n_segs;
  L.shot0 = shot0;
  L.n_shots = n_shots;
  const int64_t grid = (n_shots + kReduceWarps - 1) / kReduceWarps;
  reduce_batch_kernel<<<(unsigned)grid, kReduceWarps * 32, 0, stream>>>(L);
  XZZX_CUDA_TRY(cudaGetLastError());
  return XZZX_OK;
}

AnnealLaunch anneal_launch(const xzzx_batch* b, const ChunkDev* chunks, int chunk0, int n_chunks) {
  AnnealLaunch L;
  L.keys = b->keys;
  L.segs = b->d_segs;
  L.chunks = chunks;
  L.chunk0 = chunk0;
  L.n_chunks = n_chunks;
  L.head = b->d_head;
  return L;
}

xzzx_status run_batch(xzzx_batch* b, int mode, cudaStream_t stream) {
  xzzx_status st;
  if (mode == 0) {
    if ((st = run_greedy(b, 0, b->total_greedy_ctas, stream))) return st;
    if (b->n_chunks > 0) {
      XZZX_CUDA_TRY(cudaMemsetAsync(b->d_head, 0, sizeof(int), stream));
      const AnnealLaunch L = anneal_launch(b, b->d_chunks_lpt, 0, b->n_chunks);
      const int grid = std::min(b->grid, b->n_chunks);
      if (b->dmax <= 15) st = launch_persistent_15(L, grid, stream);
      else if (b->dmax <= 21) st = launch_persistent_21(L, grid, stream);
      else st = launch_persistent_31(L, grid, stream);
      if (st) return st;
    }
    return run_reduce(b, 0, b->total_shots, stream);
  }
  for (const DistanceRange& r : b->ranges) {
    if ((st = run_greedy(b, b->cta_prefix[r.seg_begin], b->cta_prefix[r.seg_end] - b->cta_prefix[r.seg_begin],
                         stream)))
      return st;
    if ((st = launch_chunks(r.d, anneal_launch(b, b->d_chunks_byd, r.chunk_begin, r.chunk_end - r.chunk_begin),
                            stream)))
      return st;
    if ((st = run_reduce(b, b->shot_prefix[r.seg_begin], b->shot_prefix[r.seg_end] - b->shot_prefix[r.seg_begin],
                         stream)))
      return st;
  }
  return XZZX_OK;
}

void free_batch(xzzx_batch* b) {
  if (!b) return;
  if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->dev_block) cudaFree(b->dev_block);
  delete b;
}

}  // namespace
}  // namespace batch
}  // namespace xzzx

using namespace xzzx;
using namespace xzzx::batch;

extern "C" {

xzzx_status xzzx_batch_create(const xzzx_segment* segs, int n_segs, uint64_t seed, const xzzx_batch_cfg* cfg,
                              xzzx_batch** out) {
  if (!out) return fail(XZZX_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_segs < 1 || !segs) return fail(XZZX_EINVAL, "need at least one segment");
  int device = -1;
  XZZX_CUDA_TRY(cudaGetDevice(&device));
  // Validate and order segments by distance (stable).
  std::vector<int> order(n_segs);
  std::iota(order.begin(), order.end(), 0);
  for (int i = 0; i < n_segs; ++i) {
    const xzzx_segment& s = segs[i];
    xzzx_status st = check_code(s.code);
    if (st) return st;
    if (!s.noise || !s.sched) return fail(XZZX_EINVAL, "segment " + std::to_string(i) + ": noise or schedule is NULL");
    if (!s.sched->d_sig) return fail(XZZX_EINVAL, "segment schedule has no device tables");
    if (s.code->device != device || s.sched->device != device)
      return fail(XZZX_EINVAL, "segment " + std::to_string(i) + ": handles belong to another device");
    if (s.n_shots < 0 || s.restarts < 1 || s.restarts > 65535)
      return fail(XZZX_EINVAL, "segment " + std::to_string(i) + ": bad n_shots or restarts");
    if (s.noise->Wt_x <= 0 || s.noise->Wt_z <= 0) return fail(XZZX_EINVAL, "matching weights must be positive");
    int32_t wmax = 0;
    for (int k = 0; k < 4; ++k) wmax = std::max(wmax, s.sched->noise.W[k]);
    if ((int64_t)wmax * s.code->nq * 2 > 0x7FFFFFFFll) return fail(XZZX_EINVAL, "energies would overflow int32");
    if (s.n_shots > 0 && (!s.syndromes || !s.cls || !s.E4 || !s.recovery))
      return fail(XZZX_EINVAL, "segment " + std::to_string(i) + ": NULL syndromes or outputs");
    if (s.fail && !s.true_errors) return fail(XZZX_EINVAL, "fail needs true_errors");
  }
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return segs[x].code->d < segs[y].code->d; });

  xzzx_batch* b = new (std::nothrow) xzzx_batch();
  if (!b) return fail(XZZX_ENOMEM, "host allocation");
  b->device = device;
  b->seed = seed;
  b->keys = philox_keys(seed);
  b->n_segs = n_segs;

  // Workspace layout and descriptors.
  std::vector<SegDev> hs(n_segs);
  std::vector<size_t> o_init(n_segs), o_cb(n_segs), o_E(n_segs);
  size_t ws = 0;
  b->cta_prefix.assign(n_segs + 1, 0);
  b->shot_prefix.assign(n_segs + 1, 0);
  for (int j = 0; j < n_segs; ++j) {
    const xzzx_segment& s = segs[order[j]];
    const size_t n = (size_t)s.n_shots, R = (size_t)s.restarts, w = (size_t)s.code->w;
    o_init[j] = ws;
    ws = align256(ws + sizeof(uint32_t) * n * R * 2 * w);
    o_cb[j] = ws;
    ws = align256(ws + n * R);
    o_E[j] = ws;
    ws = align256(ws + sizeof(int32_t) * n * R * 4);
    const int groups = (s.restarts + kGreedyWarps - 1) / kGreedyWarps;
    b->cta_prefix[j + 1] = b->cta_prefix[j] + (int64_t)s.n_shots * groups;
    b->shot_prefix[j + 1] = b->shot_prefix[j] + s.n_shots;
    b->dmax = std::max(b->dmax, s.code->d);
  }
  b->total_greedy_ctas = b->cta_prefix[n_segs];
  b->total_shots = b->shot_prefix[n_segs];
  b->workspace_bytes = ws;

  std::vector<ChunkDev> chunks;
  for (int j = 0; j < n_segs; ++j) {
    const xzzx_segment& s = segs[order[j]];
    const int64_t nch = (int64_t)s.n_shots * s.restarts * 4;
    for (int64_t c = 0; c < nch; c += kNT) {
      if (c > 0x7FFFFFFF) {
        free_batch(b);
        return fail(XZZX_EINVAL, "segment too large");
      }
      ChunkDev ch;
      ch.seg = j;
      ch.d = s.code->d;
      ch.first_chain = (int)c;
      ch.n_chains = (int)std::min<int64_t>(kNT, nch - c);
      ch.T = s.sched->d_T;
      ch.sig = s.sched->d_sig;
      ch.n_sweeps = s.sched->n_sweeps;
      ch.n_classes = s.sched->n_classes;
      for (int k = 0; k < 4; ++k) ch.W[k] = s.sched->noise.W[k];
      chunks.push_back(ch);
    }
    b->attempts += (double)nch * s.sched->n_sweeps * s.code->ns;
  }
  if (chunks.size() > 0x7FFFFFFF) {
    free_batch(b);
    return fail(XZZX_EINVAL, "too many chunks");
  }
  b->n_chunks = (int)chunks.size();
  std::vector<ChunkDev> byd = chunks;  // already grouped by distance (segments are)
  std::vector<ChunkDev> lpt = chunks;
  const int order_policy = cfg ? cfg->order : 0;
  if (order_policy == 0)
    std::stable_sort(lpt.begin(), lpt.end(), [](const ChunkDev& x, const ChunkDev& y) {
      return (int64_t)x.n_sweeps * (x.d * x.d - 1) > (int64_t)y.n_sweeps * (y.d * y.d - 1);
    });
  for (int j = 0; j < n_segs;) {
    DistanceRange r;
    r.d = segs[order[j]].code->d;
    r.seg_begin = j;
    while (j < n_segs && segs[order[j]].code->d == r.d) ++j;
    r.seg_end = j;
    r.chunk_begin = (int)(std::lower_bound(byd.begin(), byd.end(), r.seg_begin,
                                           [](const ChunkDev& c, int sidx) { return c.seg < sidx; }) -
                          byd.begin());
    r.chunk_end = (int)(std::lower_bound(byd.begin(), byd.end(), r.seg_end,
                                         [](const ChunkDev& c, int sidx) { return c.seg < sidx; }) -
                        byd.begin());
    b->ranges.push_back(r);
  }

  // One device allocation: descriptors then workspace.
  const size_t o_segs = 0;
  const size_t o_lpt = align256(o_segs + sizeof(SegDev) * n_segs);
  const size_t o_byd = align256(o_lpt + sizeof(ChunkDev) * std::max<size_t>(chunks.size(), 1));
  const size_t o_cta = align256(o_byd + sizeof(ChunkDev) * std::max<size_t>(chunks.size(), 1));
  const size_t o_shot = align256(o_cta + sizeof(int64_t) * (n_segs + 1));
  const size_t o_head = align256(o_shot + sizeof(int64_t) * (n_segs + 1));
  const size_t o_ws = align256(o_head + sizeof(int));
  const size_t total = o_ws + ws;
  cudaError_t e = cudaMalloc(&b->dev_block, total);
  if (e != cudaSuccess) {
    free_batch(b);
    return cuda_fail(e, "xzzx_batch_create allocation");
  }
  char* base = (char*)b->dev_block;
  for (int j = 0; j < n_segs; ++j) {
    const xzzx_segment& s = segs[order[j]];
    SegDev& d = hs[j];
    d.code = s.code->dev;
    d.shot0 = s.shot0;
    d.n_shots = s.n_shots;
    d.restarts = s.restarts;
    d.randomised = s.randomised ? 1 : 0;
    d.greedy_groups = (s.restarts + kGreedyWarps - 1) / kGreedyWarps;
    d.Wt_x = s.noise->Wt_x;
    d.Wt_z = s.noise->Wt_z;
    d.syndromes = s.syndromes;
    d.true_errors = s.true_errors;
    d.cls = s.cls;
    d.E4 = s.E4;
    d.recovery = s.recovery;
    d.fail = s.fail;
    d.init = (uint32_t*)(base + o_ws + o_init[j]);
    d.cbits = (uint8_t*)(base + o_ws + o_cb[j]);
    d.chain_E = (int32_t*)(base + o_ws + o_E[j]);
  }
  b->d_segs = (SegDev*)(base + o_segs);
  b->d_chunks_lpt = (ChunkDev*)(base + o_lpt);
  b->d_chunks_byd = (ChunkDev*)(base + o_byd);
  b->d_cta_prefix = (int64_t*)(base + o_cta);
  b->d_shot_prefix = (int64_t*)(base + o_shot);
  b->d_head = (int*)(base + o_head);
  std::vector<char> blob(o_ws, 0);
  std::memcpy(blob.data() + o_segs, hs.data(), sizeof(SegDev) * n_segs);
  if (!chunks.empty()) {
    std::memcpy(blob.data() + o_lpt, lpt.data(), sizeof(ChunkDev) * chunks.size());
    std::memcpy(blob.data() + o_byd, byd.data(), sizeof(ChunkDev) * chunks.size());
  }
  std::memcpy(blob.data() + o_cta, b->cta_prefix.data(), sizeof(int64_t) * (n_segs + 1));
  std::memcpy(blob.data() + o_shot, b->shot_prefix.data(), sizeof(int64_t) * (n_segs + 1));
  e = cudaMemcpy(b->dev_block, blob.data(), o_ws, cudaMemcpyHostToDevice);
  xzzx_status st = XZZX_OK;
  if (e != cudaSuccess) st = cuda_fail(e, "xzzx_batch_create upload");
  // Kernel attributes are set here so that runs (and graph captures) only launch.
  if (!st) st = configure_chunk_kernels();
  if (!st) st = b->dmax <= 15 ? configure_persistent_15() : b->dmax <= 21 ? configure_persistent_21()
                                                                          : configure_persistent_31();
  int per_sm = 0;
  if (!st) st = b->dmax <= 15 ? occupancy_persistent_15(&per_sm) : b->dmax <= 21 ? occupancy_persistent_21(&per_sm)
                                                                                  : occupancy_persistent_31(&per_sm);
  int n_sm = 0;
  if (!st) {
    e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) st = cuda_fail(e, "cudaDeviceGetAttribute");
  }
  if (st) {
    free_batch(b);
    return st;
  }
  if (per_sm < 1) per_sm = 1;
  if (cfg && cfg->ctas_per_sm > 0) per_sm = std::min(per_sm, cfg->ctas_per_sm);
  b->grid = n_sm * per_sm;
  *out = b;
  return XZZX_OK;
}

xzzx_status xzzx_batch_run(xzzx_batch* b, int mode, void* stream) {
  if (!b) return fail(XZZX_EINVAL, "batch is NULL");
  if (mode != 0 && mode != 1) return fail(XZZX_EINVAL, "mode must be 0 (batched) or 1 (one launch per distance)");
  xzzx_status st = check_device(b->device);
  if (st) return st;
  return run_batch(b, mode, (cudaStream_t)stream);
}

xzzx_status xzzx_batch_run_graph(xzzx_batch* b, void* stream) {
  if (!b) return fail(XZZX_EINVAL, "batch is NULL");
  if (!stream) return fail(XZZX_EINVAL, "graph capture needs a non-default stream");
  xzzx_status st = check_device(b->device);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if (!b->graph_exec) {
    XZZX_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    st = run_batch(b, 0, s);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s, &g);
    if (st) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    const cudaError_t e2 = cudaGraphInstantiate(&exec, g, 0);
    if (e2 != cudaSuccess) {
      cudaGraphDestroy(g);
      return cuda_fail(e2, "cudaGraphInstantiate");
    }
    b->graph = g;
    b->graph_exec = exec;
  }
  XZZX_CUDA_TRY(cudaGraphLaunch(b->graph_exec, s));
  return XZZX_OK;
}

xzzx_status xzzx_batch_get_info(const xzzx_batch* b, xzzx_batch_info* out) {
  if (!b || !out) return fail(XZZX_EINVAL, "NULL argument");
  out->n_segments = b->n_segs;
  out->n_chunks = b->n_chunks;
  out->n_distances = (int)b->ranges.size();
  out->persistent_grid = std::min(b->grid, std::max(b->n_chunks, 1));
  out->launches_batched = 3;
  out->launches_plain = 3 * (int)b->ranges.size();
  out->workspace_bytes = b->workspace_bytes;
  out->move_attempts = b->attempts;
  out->total_shots = b->total_shots;
  return XZZX_OK;
}

void xzzx_batch_destroy(xzzx_batch* b) { free_batch(b); }

}  // extern "C"
