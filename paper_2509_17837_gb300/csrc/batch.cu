// Batches of many homogeneous segments decoded together (uneven distances,
// noise classes, schedules and restarts in one run).
//
// A plan (build_plan) orders segments by distance, lays their intermediates
// out in a workspace, and cuts their chains into chunks of NT chains (one CTA
// each; NT = 128 or 256, a tuning knob like the sweep unroll of the kernels).  launch_plan then issues, on one stream:
//   mode 0 (batched): one greedy launch over every (segment, shot, restart
//          group), one persistent annealing launch whose CTAs pull chunks,
//          longest first, from an atomic counter, and one decision launch;
//   mode 1 (plain):   the same three kernels once per distance;
//   mode 2 (latency): as mode 1 with one warp per chain (colour-parallel lanes).
// Every chain uses the chain id it would get from xzzx_decode_batch on its
// segment alone, so both modes, and per-segment calls, agree bit for bit.
//
// xzzx_batch_* owns one allocation holding a plan's descriptors and
// workspace; xzzx_batch_run_graph captures mode 0 into a CUDA graph on its
// first call and replays it afterwards.  The decode server (serve.cu) builds
// plans into memory it allocated up front.
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

// Runtime choice of a (chains per CTA, sweep unroll) variant.
#define XZZX_VARIANTS(CALL)                                                        \
  if (nt == 128 && unroll == 1) return CALL(128, 1);                                \
  if (nt == 128 && unroll == 2) return CALL(128, 2);                                \
  if (nt == 256 && unroll == 1) return CALL(256, 1);                                \
  if (nt == 256 && unroll == 2) return CALL(256, 2);                                \
  return fail(XZZX_EINVAL, "chains per CTA must be 128 or 256 and sweep unroll 1 or 2");

xzzx_status launch_chunks(int d, int nt, int unroll, const AnnealLaunch& L, cudaStream_t stream) {
#define XZZX_CALL(NT, U) launch_chunks_v<NT, U>(d, L, stream)
  XZZX_VARIANTS(XZZX_CALL)
#undef XZZX_CALL
}

xzzx_status occupancy_chunks(int d, int nt, int unroll, int* ctas_per_sm) {
#define XZZX_CALL(NT, U) occupancy_chunks_v<NT, U>(d, ctas_per_sm)
  XZZX_VARIANTS(XZZX_CALL)
#undef XZZX_CALL
}

static xzzx_status configure_chunk_kernels(int nt, int unroll) {
#define XZZX_CALL(NT, U) configure_chunks_v<NT, U>()
  XZZX_VARIANTS(XZZX_CALL)
#undef XZZX_CALL
}

xzzx_status launch_persistent(int dmax, int nt, int unroll, const AnnealLaunch& L, int grid, cudaStream_t stream) {
  if (dmax <= 15) {
#define XZZX_CALL(NT, U) launch_persistent_v<15, NT, U>(L, grid, stream)
    XZZX_VARIANTS(XZZX_CALL)
#undef XZZX_CALL
  }
  if (dmax <= 21) {
#define XZZX_CALL(NT, U) launch_persistent_v<21, NT, U>(L, grid, stream)
    XZZX_VARIANTS(XZZX_CALL)
#undef XZZX_CALL
  }
#define XZZX_CALL(NT, U) launch_persistent_v<31, NT, U>(L, grid, stream)
  XZZX_VARIANTS(XZZX_CALL)
#undef XZZX_CALL
}

xzzx_status configure_persistent(int dmax, int nt, int unroll, int* ctas_per_sm) {
  if (dmax <= 15) {
#define XZZX_CALL(NT, U) configure_persistent_v<15, NT, U>(ctas_per_sm)
    XZZX_VARIANTS(XZZX_CALL)
#undef XZZX_CALL
  }
  if (dmax <= 21) {
#define XZZX_CALL(NT, U) configure_persistent_v<21, NT, U>(ctas_per_sm)
    XZZX_VARIANTS(XZZX_CALL)
#undef XZZX_CALL
  }
#define XZZX_CALL(NT, U) configure_persistent_v<31, NT, U>(ctas_per_sm)
  XZZX_VARIANTS(XZZX_CALL)
#undef XZZX_CALL
}
#undef XZZX_VARIANTS

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

template <bool L>
__global__ void __launch_bounds__(kGreedyWarps * 32, L ? greedy::RotGeo::kMinCtasLists : 1)
    greedy_batch_kernel(const __grid_constant__ GreedyLaunch G) {
  __shared__ greedy::SharedT<greedy::RotGeo, L> S;
  const int64_t b = G.cta0 + blockIdx.x;
  const int s = find_segment(G.cta_prefix, G.n_segs, b);
  const SegDev& sg = G.segs[s];
  const int64_t local = b - G.cta_prefix[s];
  const int64_t k = local / sg.greedy_groups;
  const int group = (int)(local % sg.greedy_groups);
  greedy::greedy_cta<greedy::RotGeo, L>(sg.code, G.keys, sg.shot0 + (uint64_t)k, group, sg.restarts, sg.greedy_rpw,
                                        sg.randomised, sg.Wt_x, sg.Wt_z, sg.syndromes + (size_t)k * sg.code.sw,
                                        sg.init + (size_t)k * sg.restarts * 2 * sg.code.w,
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

xzzx_status run_greedy(const Plan& p, const PlanDev& d, const PhiloxKeys& K, int64_t cta0, int64_t n_ctas,
                       cudaStream_t stream) {
  if (n_ctas <= 0) return XZZX_OK;
  if (n_ctas > 0x7FFFFFFF) return fail(XZZX_EINVAL, "too many greedy CTAs in one launch");
  GreedyLaunch G;
  G.keys = K;
  G.segs = d.segs;
  G.cta_prefix = d.cta_prefix;
  G.n_segs = (int)p.segs.size();
  // Segments are ordered by distance: CTAs before list_cta_end (d <= 17) run
  // the kernel with candidate lists, the rest the one without.
  const int64_t end = cta0 + n_ctas, split = std::min(std::max(p.list_cta_end, cta0), end);
  if (split > cta0) {
    G.cta0 = cta0;
    greedy_batch_kernel<true><<<(unsigned)(split - cta0), kGreedyWarps * 32, 0, stream>>>(G);
  }
  if (end > split) {
    G.cta0 = split;
    greedy_batch_kernel<false><<<(unsigned)(end - split), kGreedyWarps * 32, 0, stream>>>(G);
  }
  XZZX_CUDA_TRY(cudaGetLastError());
  return XZZX_OK;
}

xzzx_status run_reduce(const Plan& p, const PlanDev& d, int64_t shot0, int64_t n_shots, cudaStream_t stream) {
  if (n_shots <= 0) return XZZX_OK;
  ReduceLaunch L;
  L.segs = d.segs;
  L.shot_prefix = d.shot_prefix;
  L.n_segs = (int)p.segs.size();
  L.shot0 = shot0;
  L.n_shots = n_shots;
  const int64_t grid = (n_shots + kReduceWarps - 1) / kReduceWarps;
  reduce_batch_kernel<<<(unsigned)grid, kReduceWarps * 32, 0, stream>>>(L);
  XZZX_CUDA_TRY(cudaGetLastError());
  return XZZX_OK;
}

}  // namespace

AnnealLaunch anneal_launch(const PlanDev& d, const PhiloxKeys& K, const ChunkDev* chunks, int chunk0, int n,
                           int* head) {
  AnnealLaunch L;
  L.keys = K;
  L.segs = d.segs;
  L.chunks = chunks;
  L.chunk0 = chunk0;
  L.n_chunks = n;
  L.head = head ? head : d.head;
  return L;
}

xzzx_status build_plan(const xzzx_segment* segs, int n_segs, int device, int order_policy, char* ws_base, Plan& P,
                       int nt, int unroll) {
  if (n_segs < 1 || !segs) return fail(XZZX_EINVAL, "need at least one segment");
  if ((nt != 128 && nt != 256) || (unroll != 1 && unroll != 2))
    return fail(XZZX_EINVAL, "chains per CTA must be 128 or 256 and sweep unroll 1 or 2");
  std::vector<int> order(n_segs);
  std::iota(order.begin(), order.end(), 0);
  for (int i = 0; i < n_segs; ++i) {
    const xzzx_segment& s = segs[i];
    xzzx_status st = check_code(s.code);
    if (st) return st;
    if (s.code->layout != kLayoutRotated)
      return fail(XZZX_EUNSUPPORTED, "segment " + std::to_string(i) + ": batches take rotated codes only");
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
    if (s.randomised < 0 || s.randomised > 2) return fail(XZZX_EINVAL, "init mode must be 0, 1 or 2");
  }
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return segs[x].code->d < segs[y].code->d; });

  P = Plan();
  P.nt = nt;
  P.unroll = unroll;
  P.segs.resize(n_segs);
  P.cta_prefix.assign(n_segs + 1, 0);
  P.shot_prefix.assign(n_segs + 1, 0);
  P.chain_prefix.assign(n_segs + 1, 0);
  size_t ws = 0;
  std::vector<ChunkDev> chunks;
  // Restarts per greedy warp: the largest count that leaves the whole greedy
  // launch enough CTAs.
  int rpw = 1;
  for (int r = greedy::kMaxRestartsPerWarp; r > 1 && rpw == 1; r >>= 1) {
    int64_t ctas = 0;
    for (int j = 0; j < n_segs; ++j)
      ctas += (int64_t)segs[j].n_shots *
              greedy::greedy_groups(segs[j].restarts, segs[j].code->d <= greedy::kListMaxD ? r : 1);
    if (ctas >= greedy::kMinGreedyCtas) rpw = r;
  }
  for (int j = 0; j < n_segs; ++j) {
    const xzzx_segment& s = segs[order[j]];
    const size_t n = (size_t)s.n_shots, R = (size_t)s.restarts, w = (size_t)s.code->w;
    SegDev& d = P.segs[j];
    d.code = s.code->dev;
    d.shot0 = s.shot0;
    d.n_shots = s.n_shots;
    d.restarts = s.restarts;
    d.randomised = s.randomised;
    d.greedy_rpw = s.code->d <= greedy::kListMaxD ? rpw : 1;  // several per warp only with candidate lists
    d.greedy_groups = greedy::greedy_groups(s.restarts, d.greedy_rpw);
    d.Wt_x = s.noise->Wt_x;
    d.Wt_z = s.noise->Wt_z;
    d.syndromes = s.syndromes;
    d.true_errors = s.true_errors;
    d.cls = s.cls;
    d.E4 = s.E4;
    d.recovery = s.recovery;
    d.fail = s.fail;
    d.init = (uint32_t*)(ws_base ? ws_base + ws : nullptr);
    ws = align256(ws + sizeof(uint32_t) * n * R * 2 * w);
    d.cbits = (uint8_t*)(ws_base ? ws_base + ws : nullptr);
    ws = align256(ws + n * R);
    d.chain_E = (int32_t*)(ws_base ? ws_base + ws : nullptr);
    ws = align256(ws + sizeof(int32_t) * n * R * 4);
    d.T = s.sched->d_T;
    d.sig = s.sched->d_sig;
    d.n_sweeps = s.sched->n_sweeps;
    d.n_classes = s.sched->n_classes;
    for (int k = 0; k < 4; ++k) d.W[k] = s.sched->noise.W[k];
    P.cta_prefix[j + 1] = P.cta_prefix[j] + (int64_t)s.n_shots * d.greedy_groups;
    if (s.code->d <= greedy::kListMaxD) P.list_cta_end = P.cta_prefix[j + 1];
    P.shot_prefix[j + 1] = P.shot_prefix[j] + s.n_shots;
    P.chain_prefix[j + 1] = P.chain_prefix[j] + (int64_t)s.n_shots * s.restarts * 4;
    P.dmax = std::max(P.dmax, s.code->d);
    const int64_t nch = (int64_t)s.n_shots * s.restarts * 4;
    if (nch > 0x7FFFFFFFll) return fail(XZZX_EINVAL, "segment too large");
    for (int64_t c = 0; c < nch; c += nt) {
      ChunkDev ch;
      ch.seg = j;
      ch.d = s.code->d;
      ch.first_chain = (int)c;
      ch.n_chains = (int)std::min<int64_t>(nt, nch - c);
      ch.T = s.sched->d_T;
      ch.sig = s.sched->d_sig;
      ch.n_sweeps = s.sched->n_sweeps;
      ch.n_classes = s.sched->n_classes;
      for (int k = 0; k < 4; ++k) ch.W[k] = s.sched->noise.W[k];
      chunks.push_back(ch);
    }
    P.attempts += (double)nch * s.sched->n_sweeps * s.code->ns;
  }
  if (chunks.size() > 0x7FFFFFFF) return fail(XZZX_EINVAL, "too many chunks");
  P.total_ctas = P.cta_prefix[n_segs];
  P.total_shots = P.shot_prefix[n_segs];
  P.workspace_bytes = ws;
  P.byd = chunks;  // grouped by distance already (segments are)
  P.lpt = chunks;
  auto work = [](const ChunkDev& c) { return (int64_t)c.n_sweeps * (c.d * c.d - 1); };
  if (order_policy == 0)
    std::stable_sort(P.lpt.begin(), P.lpt.end(),
                     [&](const ChunkDev& x, const ChunkDev& y) { return work(x) > work(y); });
  P.bycls = chunks;
  std::stable_sort(P.bycls.begin(), P.bycls.end(), [&](const ChunkDev& x, const ChunkDev& y) {
    const int cx = class_of(x.d), cy = class_of(y.d);
    if (cx != cy) return cx < cy;
    return order_policy == 0 && work(x) > work(y);
  });
  for (int c = 0, k = 0; c < kNumClasses; ++c) {
    ClassRange r;
    r.cls = c;
    r.chunk_begin = k;
    while (k < (int)P.bycls.size() && class_of(P.bycls[k].d) == c) ++k;
    r.chunk_end = k;
    if (r.chunk_end > r.chunk_begin) P.classes.push_back(r);
  }
  for (int j = 0; j < n_segs;) {
    DistanceRange r;
    r.d = segs[order[j]].code->d;
    r.seg_begin = j;
    while (j < n_segs && segs[order[j]].code->d == r.d) ++j;
    r.seg_end = j;
    auto by_seg = [](const ChunkDev& c, int sidx) { return c.seg < sidx; };
    r.chunk_begin = (int)(std::lower_bound(P.byd.begin(), P.byd.end(), r.seg_begin, by_seg) - P.byd.begin());
    r.chunk_end = (int)(std::lower_bound(P.byd.begin(), P.byd.end(), r.seg_end, by_seg) - P.byd.begin());
    P.ranges.push_back(r);
  }
  return XZZX_OK;
}

namespace {
struct BlobLayout {
  size_t segs, lpt, byd, bycls, cta, shot, chain, head, total;
};
BlobLayout blob_layout(const Plan& p) {
  BlobLayout L;
  const size_t nc = std::max<size_t>(p.lpt.size(), 1);
  L.segs = 0;
  L.lpt = align256(L.segs + sizeof(SegDev) * p.segs.size());
  L.byd = align256(L.lpt + sizeof(ChunkDev) * nc);
  L.bycls = align256(L.byd + sizeof(ChunkDev) * nc);
  L.cta = align256(L.bycls + sizeof(ChunkDev) * nc);
  L.shot = align256(L.cta + sizeof(int64_t) * p.cta_prefix.size());
  L.chain = align256(L.shot + sizeof(int64_t) * p.shot_prefix.size());
  L.head = align256(L.chain + sizeof(int64_t) * p.chain_prefix.size());
  L.total = align256(L.head + sizeof(int) * (1 + kNumClasses));
  return L;
}
}  // namespace

size_t descriptor_bytes(const Plan& p) { return blob_layout(p).total; }

PlanDev descriptor_layout(const Plan& p, char* base) {
  const BlobLayout L = blob_layout(p);
  PlanDev d;
  d.segs = (SegDev*)(base + L.segs);
  d.lpt = (ChunkDev*)(base + L.lpt);
  d.byd = (ChunkDev*)(base + L.byd);
  d.bycls = (ChunkDev*)(base + L.bycls);
  d.cta_prefix = (int64_t*)(base + L.cta);
  d.shot_prefix = (int64_t*)(base + L.shot);
  d.chain_prefix = (int64_t*)(base + L.chain);
  d.head = (int*)(base + L.head);
  return d;
}

void pack_descriptors(const Plan& p, char* blob) {
  const BlobLayout L = blob_layout(p);
  std::memset(blob, 0, L.total);
  std::memcpy(blob + L.segs, p.segs.data(), sizeof(SegDev) * p.segs.size());
  if (!p.lpt.empty()) {
    std::memcpy(blob + L.lpt, p.lpt.data(), sizeof(ChunkDev) * p.lpt.size());
    std::memcpy(blob + L.byd, p.byd.data(), sizeof(ChunkDev) * p.byd.size());
    std::memcpy(blob + L.bycls, p.bycls.data(), sizeof(ChunkDev) * p.bycls.size());
  }
  std::memcpy(blob + L.cta, p.cta_prefix.data(), sizeof(int64_t) * p.cta_prefix.size());
  std::memcpy(blob + L.shot, p.shot_prefix.data(), sizeof(int64_t) * p.shot_prefix.size());
  std::memcpy(blob + L.chain, p.chain_prefix.data(), sizeof(int64_t) * p.chain_prefix.size());
}

xzzx_status configure_plan_kernels(int dmax, int nt, int unroll, int* ctas_per_sm) {
  xzzx_status st = configure_chunk_kernels(nt, unroll);
  if (st) return st;
  return configure_persistent(dmax, nt, unroll, ctas_per_sm);
}

xzzx_status launch_plan(const Plan& p, const PlanDev& d, const PhiloxKeys& K, int grid, int mode,
                        cudaStream_t stream) {
  NvtxRange nvtx_range(mode == 0 ? "xzzx batch (persistent)" : "xzzx batch (per distance)");
  xzzx_status st;
  const int n_chunks = (int)p.lpt.size();
  if (mode == 0) {
    if ((st = run_greedy(p, d, K, 0, p.total_ctas, stream))) return st;
    if (n_chunks > 0) {
      XZZX_CUDA_TRY(cudaMemsetAsync(d.head, 0, sizeof(int), stream));
      const AnnealLaunch L = anneal_launch(d, K, d.lpt, 0, n_chunks, nullptr);
      const int g = std::max(1, std::min(grid, n_chunks));
      if ((st = launch_persistent(p.dmax, p.nt, p.unroll, L, g, stream))) return st;
    }
    return run_reduce(p, d, 0, p.total_shots, stream);
  }
  for (const DistanceRange& r : p.ranges) {
    if ((st = run_greedy(p, d, K, p.cta_prefix[r.seg_begin], p.cta_prefix[r.seg_end] - p.cta_prefix[r.seg_begin],
                         stream)))
      return st;
    if (mode == 2) {
      WarpLaunch W;
      W.keys = K;
      W.segs = d.segs;
      W.chain_prefix = d.chain_prefix;
      W.n_segs = (int)p.segs.size();
      W.chain0 = p.chain_prefix[r.seg_begin];
      W.n_chains = p.chain_prefix[r.seg_end] - p.chain_prefix[r.seg_begin];
      W.smem = r.warp_smem;
      if ((st = launch_warp_chains(r.d, W, stream))) return st;
    } else if ((st = launch_chunks(r.d, p.nt, p.unroll,
                                   anneal_launch(d, K, d.byd, r.chunk_begin, r.chunk_end - r.chunk_begin, nullptr), stream))) {
      return st;
    }
    if ((st = run_reduce(p, d, p.shot_prefix[r.seg_begin], p.shot_prefix[r.seg_end] - p.shot_prefix[r.seg_begin],
                         stream)))
      return st;
  }
  return XZZX_OK;
}

}  // namespace batch
}  // namespace xzzx

struct xzzx_batch {
  int device = -1;
  xzzx::PhiloxKeys keys{};
  int grid = 0;
  xzzx::batch::Plan plan;
  xzzx::batch::PlanDev dev{};
  void* dev_block = nullptr;  // descriptors + workspace
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  int graph_mode = 0;
  int class_grid[xzzx::batch::kNumClasses] = {0, 0, 0};  // mode 4: persistent grid of each class
  int warp_per_sm = 0;  // mode 2: resident warp-kernel CTAs per SM (fewest over the distances)
  // modes 3 and 4: one side stream and one completion event per distance (or
  // class), and the fork event, created on first use
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> done;
  cudaEvent_t fork = nullptr;
};

namespace {
void free_batch(xzzx_batch* b) {
  if (!b) return;
  if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (cudaStream_t s : b->side) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->done) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->dev_block) cudaFree(b->dev_block);
  delete b;
}
xzzx_status ensure_side_streams(xzzx_batch* b, size_t n) {
  while (b->side.size() < n) {
    cudaStream_t s = nullptr;
    XZZX_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    b->side.push_back(s);
    cudaEvent_t e = nullptr;
    XZZX_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    b->done.push_back(e);
  }
  if (!b->fork) XZZX_CUDA_TRY(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
  return XZZX_OK;
}

// Mode 3: greedy for all segments on `stream`, each distance's chunk kernel on
// its own side stream (largest distance first), decisions after the join.
xzzx_status launch_concurrent(xzzx_batch* b, cudaStream_t stream) {
  using namespace xzzx::batch;
  const Plan& p = b->plan;
  const PlanDev& d = b->dev;
  const size_t n = p.ranges.size();
  xzzx_status st = ensure_side_streams(b, n);
  if (st) return st;
  st = run_greedy(p, d, b->keys, 0, p.total_ctas, stream);
  if (st) return st;
  XZZX_CUDA_TRY(cudaEventRecord(b->fork, stream));
  for (size_t k = 0; k < n; ++k) {
    const DistanceRange& r = p.ranges[n - 1 - k];  // ranges ascend in d
    XZZX_CUDA_TRY(cudaStreamWaitEvent(b->side[k], b->fork, 0));
    if ((st = launch_chunks(r.d, p.nt, p.unroll,
                            anneal_launch(d, b->keys, d.byd, r.chunk_begin, r.chunk_end - r.chunk_begin, nullptr), b->side[k])))
      return st;
    XZZX_CUDA_TRY(cudaEventRecord(b->done[k], b->side[k]));
    XZZX_CUDA_TRY(cudaStreamWaitEvent(stream, b->done[k], 0));
  }
  return run_reduce(p, d, 0, p.total_shots, stream);
}

// Mode 4: greedy for all segments on `stream`, then one persistent launch per
// distance class (d <= 15, 17..21, 23..31), each on its own side stream with
// its own chunk queue (longest first) and the register allocation of its
// class, largest class first; decisions after the join.  Small-distance chunks
// so keep their own occupancy while the large ones fill the GPU's tails.
xzzx_status launch_class_persistent(xzzx_batch* b, cudaStream_t stream) {
  using namespace xzzx::batch;
  const Plan& p = b->plan;
  const PlanDev& d = b->dev;
  const size_t n = p.classes.size();
  xzzx_status st = ensure_side_streams(b, n);
  if (st) return st;
  if ((st = run_greedy(p, d, b->keys, 0, p.total_ctas, stream))) return st;
  XZZX_CUDA_TRY(cudaEventRecord(b->fork, stream));
  for (size_t k = 0; k < n; ++k) {
    const ClassRange& r = p.classes[n - 1 - k];
    int* head = d.head + 1 + r.cls;
    const int n_chunks = r.chunk_end - r.chunk_begin;
    XZZX_CUDA_TRY(cudaStreamWaitEvent(b->side[k], b->fork, 0));
    XZZX_CUDA_TRY(cudaMemsetAsync(head, 0, sizeof(int), b->side[k]));
    const int g = std::max(1, std::min(b->class_grid[r.cls], n_chunks));
    if ((st = launch_persistent(kClassDmax[r.cls], p.nt, p.unroll,
                                anneal_launch(d, b->keys, d.bycls, r.chunk_begin, n_chunks, head), g, b->side[k])))
      return st;
    XZZX_CUDA_TRY(cudaEventRecord(b->done[k], b->side[k]));
    XZZX_CUDA_TRY(cudaStreamWaitEvent(stream, b->done[k], 0));
  }
  return run_reduce(p, d, 0, p.total_shots, stream);
}

xzzx_status run_mode(xzzx_batch* b, int mode, cudaStream_t stream) {
  if (mode == 3) return launch_concurrent(b, stream);
  if (mode == 4) return launch_class_persistent(b, stream);
  return xzzx::batch::launch_plan(b->plan, b->dev, b->keys, b->grid, mode, stream);
}

}  // namespace

using namespace xzzx;
using namespace xzzx::batch;

extern "C" {

xzzx_status xzzx_batch_create(const xzzx_segment* segs, int n_segs, uint64_t seed, const xzzx_batch_cfg* cfg,
                              xzzx_batch** out) {
  if (!out) return fail(XZZX_EINVAL, "out is NULL");
  *out = nullptr;
  int device = -1;
  XZZX_CUDA_TRY(cudaGetDevice(&device));
  const int nt = (cfg && cfg->chains_per_cta) ? cfg->chains_per_cta : kNT;
  const int unroll = (cfg && cfg->sweep_unroll) ? cfg->sweep_unroll : 1;
  Plan sizing;
  xzzx_status st = build_plan(segs, n_segs, device, cfg ? cfg->order : 0, nullptr, sizing, nt, unroll);
  if (st) return st;
  xzzx_batch* b = new (std::nothrow) xzzx_batch();
  if (!b) return fail(XZZX_ENOMEM, "host allocation");
  b->device = device;
  b->keys = philox_keys(seed);
  const size_t desc = descriptor_bytes(sizing);
  cudaError_t e = cudaMalloc(&b->dev_block, desc + sizing.workspace_bytes);
  if (e != cudaSuccess) {
    free_batch(b);
    return cuda_fail(e, "xzzx_batch_create allocation");
  }
  char* base = (char*)b->dev_block;
  if ((st = build_plan(segs, n_segs, device, cfg ? cfg->order : 0, base + desc, b->plan, nt, unroll))) {
    free_batch(b);
    return st;
  }
  b->dev = descriptor_layout(b->plan, base);
  std::vector<char> blob(desc);
  pack_descriptors(b->plan, blob.data());
  e = cudaMemcpy(base, blob.data(), desc, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    free_batch(b);
    return cuda_fail(e, "xzzx_batch_create upload");
  }
  int per_sm = 0, n_sm = 0;
  if ((st = configure_plan_kernels(b->plan.dmax, nt, unroll, &per_sm))) {
    free_batch(b);
    return st;
  }
  e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) {
    free_batch(b);
    return cuda_fail(e, "cudaDeviceGetAttribute");
  }
  if (per_sm < 1) per_sm = 1;
  if (cfg && cfg->ctas_per_sm > 0) per_sm = std::min(per_sm, cfg->ctas_per_sm);
  b->grid = n_sm * per_sm;
  for (const ClassRange& r : b->plan.classes) {
    int cls_per_sm = 0;
    if ((st = configure_persistent(kClassDmax[r.cls], nt, unroll, &cls_per_sm))) {
      free_batch(b);
      return st;
    }
    if (cls_per_sm < 1) cls_per_sm = 1;
    if (cfg && cfg->ctas_per_sm > 0) cls_per_sm = std::min(cls_per_sm, cfg->ctas_per_sm);
    b->class_grid[r.cls] = n_sm * cls_per_sm;
  }
  b->warp_per_sm = 0;
  for (DistanceRange& r : b->plan.ranges) {
    int w_per_sm = 0;
    if ((st = configure_warp_chains(r.d, cfg ? cfg->ctas_per_sm : 0, &r.warp_smem, &w_per_sm))) {
      free_batch(b);
      return st;
    }
    b->warp_per_sm = b->warp_per_sm ? std::min(b->warp_per_sm, w_per_sm) : w_per_sm;
  }
  b->graph_mode = cfg ? cfg->graph_mode : 0;
  if (b->graph_mode != 0 && b->graph_mode != 3 && b->graph_mode != 4) {
    free_batch(b);
    return fail(XZZX_EINVAL, "graph_mode must be 0, 3 or 4");
  }
  *out = b;
  return XZZX_OK;
}

xzzx_status xzzx_batch_run(xzzx_batch* b, int mode, void* stream) {
  if (!b) return fail(XZZX_EINVAL, "batch is NULL");
  if (mode < 0 || mode > 4)
    return fail(XZZX_EINVAL,
                "mode must be 0 (batched), 1 (one launch per distance), 2 (one warp per chain), 3 (concurrent "
                "per-distance launches) or 4 (concurrent per-class persistent launches)");
  xzzx_status st = check_device(b->device);
  if (st) return st;
  return run_mode(b, mode, (cudaStream_t)stream);
}

xzzx_status xzzx_batch_run_graph(xzzx_batch* b, void* stream) {
  if (!b) return fail(XZZX_EINVAL, "batch is NULL");
  if (!stream) return fail(XZZX_EINVAL, "graph capture needs a non-default stream");
  xzzx_status st = check_device(b->device);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if (!b->graph_exec) {
    XZZX_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    st = run_mode(b, b->graph_mode, s);
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
  out->n_segments = (int)b->plan.segs.size();
  out->n_chunks = (int)b->plan.lpt.size();
  out->n_distances = (int)b->plan.ranges.size();
  out->persistent_grid = std::min(b->grid, std::max((int)b->plan.lpt.size(), 1));
  // Mode 0: greedy (one launch per side of d = 15 present), the persistent anneal, the decision.
  out->launches_batched = 2 + (b->plan.list_cta_end > 0 ? 1 : 0) + (b->plan.list_cta_end < b->plan.total_ctas ? 1 : 0);
  out->n_classes = (int)b->plan.classes.size();
  out->launches_plain = 3 * (int)b->plan.ranges.size();
  out->workspace_bytes = b->plan.workspace_bytes;
  out->move_attempts = b->plan.attempts;
  out->total_shots = b->plan.total_shots;
  out->chains_per_cta = b->plan.nt;
  out->sweep_unroll = b->plan.unroll;
  out->warp_ctas_per_sm = b->warp_per_sm;
  return XZZX_OK;
}

void xzzx_batch_destroy(xzzx_batch* b) { free_batch(b); }

}  // extern "C"
