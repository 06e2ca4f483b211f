// Decode server with continuous batching.
//
// Requests are single syndromes of registered (distance, noise) classes.  The
// code tables and schedules of every class stay on the device; so does a pool
// of in-flight slots, allocated once at start (the HBM budget split evenly),
// each with its own stream, descriptor area, workspace and staging buffers.
//
// A dispatcher thread forms a batch whenever a slot is free: it takes pending
// requests in arrival order (of one distance, so the batch's work finishes
// together) while they fit the slot's memory and the register budget: a
// number of GPU-fulls of the kernels' resident CTAs (two by default, so that
// under load the next batch's CTAs already wait in hardware when a batch
// ends).  The batch is decoded by the batched plan (one greedy launch, one
// annealing launch of the batch distance's own kernel, one decision launch;
// small batches on a lightly loaded GPU anneal with one warp per chain
// instead, for latency) between a
// host-to-device
// copy of the syndromes and a device-to-host copy of the results; batches in
// different slots overlap on the GPU.  A host callback on the slot's stream
// stamps the completion time.  Requests that arrive while others run are
// admitted as soon as a slot and budget free up.
//
// Determinism: each request is its own one-shot segment with shot index =
// request id, so its chains draw exactly what xzzx_decode_batch(..., shot0 =
// req_id, n_shots = 1, ...) draws, whatever else shares its batch.
//
// Every host wait is bounded (condition-variable timeouts); nothing on the
// device waits on the host.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "batch_internal.h"

namespace xzzx {
namespace serve {

using Clock = std::chrono::steady_clock;

struct Class {
  xzzx_code* code = nullptr;
  xzzx_schedule* sched = nullptr;
  xzzx_noise noise{};
  int d = 0, group = 0;
  size_t bytes = 0;      // conservative device bytes per request
  int64_t regs = 0;      // registers per request while resident
};

struct Req {
  uint64_t id;
  int cls;
  Clock::time_point t_submit;
  uint32_t syn[32];
};

struct Slot {
  cudaStream_t stream = nullptr;
  char* dev = nullptr;       // slot_bytes of device memory
  char* host_in = nullptr;   // pinned: descriptors + syndromes
  char* host_out = nullptr;  // pinned: results
  bool busy = false;
  bool warp_mode = false;  // anneal this batch with one warp per chain
  int64_t warps = 0;       // warps it occupies while it does
  int64_t regs = 0;
  std::vector<Req> reqs;
  size_t off_out = 0, out_stride = 0;
  Clock::time_point t_done;
  xzzx_server* server = nullptr;
  int index = 0;
};

constexpr size_t kOutStride = 512;  // bytes per request result in the output area

}  // namespace serve
}  // namespace xzzx

struct xzzx_server {
  xzzx_serve_cfg cfg{};
  int device = -1, n_sm = 0;
  xzzx::PhiloxKeys keys{};
  std::vector<xzzx::serve::Class> classes;
  std::vector<xzzx::serve::Slot> slots;
  size_t slot_bytes = 0, staging_bytes = 0;
  int64_t regs_total = 0, regs_in_use = 0;
  int64_t warp_inflight = 0;  // warps of batches annealing one warp per chain
  bool started = false, stop = false;
  bool blocked = false;  // pending requests wait for budget freed by a completion
  std::deque<xzzx::serve::Req> pending;
  std::vector<xzzx_result> done;
  std::vector<double> lat_us;
  std::vector<int> completed_slots;
  int64_t submitted = 0, rejected = 0, dispatched = 0, completed = 0, batches = 0;
  xzzx_status sticky = XZZX_OK;
  std::string sticky_msg;
  uint32_t* d_err = nullptr;     // device error area shared by the classes' codes
  uint32_t device_errors = 0;    // OR of the XZZX_DEVERR_* flags seen after batches
  std::mutex mu;
  std::condition_variable cv, cv_done;
  std::thread dispatcher;
  std::vector<std::thread> replayers;
};

namespace xzzx {
namespace serve {
namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

void CUDART_CB on_complete(void* p) {
  Slot* s = (Slot*)p;
  xzzx_server* sv = s->server;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    s->t_done = Clock::now();
    sv->completed_slots.push_back(s->index);
  }
  sv->cv.notify_all();
}

// Issue one batch on a slot (called without the server lock; the slot is busy
// and owned by the dispatcher).
xzzx_status issue(xzzx_server* sv, Slot& slot) {
  using namespace xzzx::batch;
  const int n = (int)slot.reqs.size();
  std::vector<xzzx_segment> segs(n);
  // Layout of the slot: [descriptors | syndromes | outputs | workspace]; the
  // pinned staging buffer mirrors the first two parts.
  size_t syn_bytes = 0;
  for (const Req& r : slot.reqs) syn_bytes += align256(sizeof(uint32_t) * sv->classes[r.cls].code->sw);
  const size_t out_bytes = (size_t)n * kOutStride;
  // First pass sizes the plan; pointers are filled in the second pass.
  Plan plan;
  for (int i = 0; i < n; ++i) {
    const Class& c = sv->classes[slot.reqs[i].cls];
    xzzx_segment& s = segs[i];
    std::memset(&s, 0, sizeof(s));
    s.code = c.code;
    s.noise = &c.noise;
    s.sched = c.sched;
    s.shot0 = slot.reqs[i].id;
    s.n_shots = 1;
    s.restarts = sv->cfg.restarts;
    s.randomised = 1;
    s.syndromes = (const uint32_t*)(uintptr_t)256;  // placeholders for sizing
    s.cls = (uint8_t*)(uintptr_t)256;
    s.E4 = (int32_t*)(uintptr_t)256;
    s.recovery = (uint32_t*)(uintptr_t)256;
  }
  xzzx_status st = build_plan(segs.data(), n, sv->device, 0, nullptr, plan);
  if (st) return st;
  const size_t desc = descriptor_bytes(plan);
  const size_t o_syn = align256(desc);
  const size_t o_out = align256(o_syn + syn_bytes);
  const size_t o_ws = align256(o_out + out_bytes);
  if (o_ws + plan.workspace_bytes > sv->slot_bytes) return fail(XZZX_ENOMEM, "batch exceeds the slot's device memory");
  if (o_out > sv->staging_bytes) return fail(XZZX_ENOMEM, "batch exceeds the slot's staging buffer");
  size_t so = 0;
  for (int i = 0; i < n; ++i) {
    const Class& c = sv->classes[slot.reqs[i].cls];
    xzzx_segment& s = segs[i];
    s.syndromes = (const uint32_t*)(slot.dev + o_syn + so);
    std::memcpy(slot.host_in + o_syn + so, slot.reqs[i].syn, sizeof(uint32_t) * c.code->sw);
    so += align256(sizeof(uint32_t) * c.code->sw);
    char* o = slot.dev + o_out + (size_t)i * kOutStride;
    s.cls = (uint8_t*)o;
    s.E4 = (int32_t*)(o + 16);
    s.recovery = (uint32_t*)(o + 32);
  }
  if ((st = build_plan(segs.data(), n, sv->device, 0, slot.dev + o_ws, plan))) return st;
  pack_descriptors(plan, slot.host_in);
  const PlanDev pd = descriptor_layout(plan, slot.dev);
  slot.off_out = o_out;
  XZZX_CUDA_TRY(cudaMemcpyAsync(slot.dev, slot.host_in, desc, cudaMemcpyHostToDevice, slot.stream));
  XZZX_CUDA_TRY(cudaMemcpyAsync(slot.dev + o_syn, slot.host_in + o_syn, syn_bytes, cudaMemcpyHostToDevice,
                                slot.stream));
  // One distance per batch: its own chunk kernel (mode 1) runs with that
  // distance's register allocation; the persistent form's queue over distances
  // has nothing to balance here.
  if ((st = launch_plan(plan, pd, sv->keys, (int)plan.lpt.size(), slot.warp_mode ? 2 : 1, slot.stream))) return st;
  XZZX_CUDA_TRY(cudaMemcpyAsync(slot.host_out, slot.dev + o_out, out_bytes, cudaMemcpyDeviceToHost, slot.stream));
  // the device error flags after this batch, read beside its results
  XZZX_CUDA_TRY(cudaMemcpyAsync(slot.host_out + (size_t)sv->cfg.max_batch * kOutStride, sv->d_err,
                                2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, slot.stream));
  XZZX_CUDA_TRY(cudaLaunchHostFunc(slot.stream, on_complete, &slot));
  return XZZX_OK;
}

// Move finished slots' results out (server lock held).
void harvest(xzzx_server* sv) {
  for (int si : sv->completed_slots) {
    Slot& s = sv->slots[si];
    for (size_t i = 0; i < s.reqs.size(); ++i) {
      const Req& r = s.reqs[i];
      const Class& c = sv->classes[r.cls];
      const char* o = s.host_out + i * kOutStride;
      xzzx_result res;
      std::memset(&res, 0, sizeof(res));
      res.req_id = r.id;
      res.d = c.d;
      res.class_id = r.cls;
      res.cls = *(const uint8_t*)o;
      std::memcpy(res.E4, o + 16, sizeof(res.E4));
      std::memcpy(res.recovery, o + 32, sizeof(uint32_t) * 2 * c.code->w);
      res.latency_us = std::chrono::duration<double, std::micro>(s.t_done - r.t_submit).count();
      sv->lat_us.push_back(res.latency_us);
      sv->done.push_back(res);
      ++sv->completed;
    }
    sv->device_errors |= *(const uint32_t*)(s.host_out + (size_t)sv->cfg.max_batch * kOutStride);
    sv->regs_in_use -= s.regs;
    sv->warp_inflight -= s.warps;
    s.reqs.clear();
    s.regs = 0;
    s.warps = 0;
    s.busy = false;
  }
  if (!sv->completed_slots.empty()) sv->cv_done.notify_all();
  sv->completed_slots.clear();
}

// Pick the next batch for a free slot (server lock held): requests of the
// oldest pending request's distance, in arrival order, while they fit.  One
// distance per batch keeps a batch's CTAs finishing together, so the budget
// they hold is released without idle tails.
bool form_batch(xzzx_server* sv, Slot& slot) {
  if (sv->pending.empty()) return false;
  const int group = sv->classes[sv->pending.front().cls].d;
  size_t bytes = 4096;
  int64_t regs = 0;
  std::vector<size_t> take;
  for (size_t i = 0; i < sv->pending.size() && (int)take.size() < sv->cfg.max_batch; ++i) {
    const Class& c = sv->classes[sv->pending[i].cls];
    if (c.d != group) continue;
    if (bytes + c.bytes > sv->slot_bytes) break;
    if (sv->regs_in_use + regs + c.regs > sv->regs_total && !(take.empty() && sv->regs_in_use == 0)) break;
    bytes += c.bytes;
    regs += c.regs;
    take.push_back(i);
  }
  if (take.empty()) return false;
  std::vector<Req> reqs;
  reqs.reserve(take.size());
  std::deque<Req> rest;
  size_t t = 0;
  for (size_t i = 0; i < sv->pending.size(); ++i) {
    if (t < take.size() && take[t] == i) {
      reqs.push_back(sv->pending[i]);
      ++t;
    } else {
      rest.push_back(sv->pending[i]);
    }
  }
  sv->pending.swap(rest);
  slot.reqs.swap(reqs);
  slot.regs = regs;
  // A small batch anneals one warp per chain while the warps of all batches
  // doing so stay within 16 per SM: a lightly loaded GPU has the room, and
  // each chain's sequential work is shorter.  Past that the batch runs one
  // thread per chain, which has the higher throughput.
  const int warp_max = sv->cfg.warp_max_requests == 0 ? 16 : sv->cfg.warp_max_requests;
  const int64_t warps = (int64_t)slot.reqs.size() * 4 * sv->cfg.restarts;
  slot.warp_mode = (int)slot.reqs.size() <= warp_max && sv->warp_inflight + warps <= (int64_t)sv->n_sm * 16;
  slot.warps = slot.warp_mode ? warps : 0;
  sv->warp_inflight += slot.warps;
  slot.busy = true;
  sv->regs_in_use += regs;
  sv->dispatched += (int64_t)slot.reqs.size();
  ++sv->batches;
  return true;
}

void dispatcher_main(xzzx_server* sv) {
  cudaSetDevice(sv->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  for (;;) {
    sv->cv.wait_for(lk, std::chrono::milliseconds(2), [&] {
      if (!sv->completed_slots.empty()) return true;
      if (sv->stop) return true;
      if (sv->pending.empty() || sv->blocked) return false;
      for (const Slot& s : sv->slots)
        if (!s.busy) return true;
      return false;
    });
    if (!sv->completed_slots.empty()) sv->blocked = false;
    harvest(sv);
    bool any_busy = false;
    for (const Slot& s : sv->slots) any_busy |= s.busy;
    if (sv->stop && sv->pending.empty() && !any_busy) break;
    if (sv->sticky) {
      if (!any_busy) break;
      continue;
    }
    if (sv->stop && !any_busy && !sv->pending.empty()) {
      // Stopping with nothing in flight: whatever cannot be dispatched now
      // never will be (no completion is coming to free budget), so it is
      // dropped and counted as rejected rather than waited on.
      bool formed = false;
      for (Slot& s : sv->slots)
        if (!s.busy && form_batch(sv, s)) {
          formed = true;
          lk.unlock();
          const xzzx_status st = issue(sv, s);
          lk.lock();
          if (st) {
            sv->sticky = st;
            sv->sticky_msg = std::string("dispatch failed: ") + xzzx_last_error();
            sv->regs_in_use -= s.regs;
            sv->warp_inflight -= s.warps;
            s.reqs.clear();
            s.regs = s.warps = 0;
            s.busy = false;
          }
          break;
        }
      if (!formed) {
        sv->rejected += (int64_t)sv->pending.size();
        sv->pending.clear();
      }
      continue;
    }
    for (Slot& s : sv->slots) {
      if (s.busy) continue;
      if (!form_batch(sv, s)) {
        sv->blocked = !sv->pending.empty();
        break;
      }
      lk.unlock();
      const xzzx_status st = issue(sv, s);
      lk.lock();
      if (st) {
        sv->sticky = st;
        sv->sticky_msg = std::string("dispatch failed: ") + xzzx_last_error();
        sv->regs_in_use -= s.regs;
        sv->warp_inflight -= s.warps;
        s.reqs.clear();
        s.regs = 0;
        s.warps = 0;
        s.busy = false;
        break;
      }
    }
  }
  sv->cv_done.notify_all();
}

}  // namespace
}  // namespace serve
}  // namespace xzzx

using namespace xzzx;
using namespace xzzx::serve;

extern "C" {

xzzx_status xzzx_serve_create(const xzzx_serve_cfg* cfg, xzzx_server** out) {
  if (!cfg || !out) return fail(XZZX_EINVAL, "NULL argument");
  *out = nullptr;
  if (cfg->restarts < 1 || cfg->restarts > 65535) return fail(XZZX_EINVAL, "restarts must be in [1, 65535]");
  if (cfg->n_sweeps < 0) return fail(XZZX_EINVAL, "n_sweeps < 0");
  if (cfg->max_batch < 1 || cfg->max_batch > 4096 || cfg->n_slots < 1 || cfg->n_slots > 64)
    return fail(XZZX_EINVAL, "max_batch must be in [1, 4096] and n_slots in [1, 64]");
  if (cfg->queue_capacity < 1) return fail(XZZX_EINVAL, "queue_capacity must be positive");
  if (cfg->resident_waves < 0 || cfg->resident_waves > 64) return fail(XZZX_EINVAL, "resident_waves must be in [0, 64]");
  xzzx_server* sv = new (std::nothrow) xzzx_server();
  if (!sv) return fail(XZZX_ENOMEM, "host allocation");
  sv->cfg = *cfg;
  sv->keys = philox_keys(cfg->seed);
  cudaError_t e = cudaGetDevice(&sv->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sv->n_sm, cudaDevAttrMultiProcessorCount, sv->device);
  if (e != cudaSuccess) {
    delete sv;
    return cuda_fail(e, "xzzx_serve_create");
  }
  *out = sv;
  return XZZX_OK;
}

xzzx_status xzzx_serve_add_class(xzzx_server* sv, int d, const xzzx_noise* noise, int* class_id) {
  if (!sv || !noise || !class_id) return fail(XZZX_EINVAL, "NULL argument");
  if (sv->started) return fail(XZZX_EINVAL, "classes must be added before xzzx_serve_start");
  Class c;
  c.d = d;
  c.noise = *noise;
  c.group = d <= 15 ? 0 : 1;
  xzzx_status st = xzzx_make_code(d, 0, &c.code);
  if (st) return st;
  st = xzzx_make_schedule(noise, sv->cfg.sched_kind, sv->cfg.n_sweeps, sv->cfg.beta0, sv->cfg.beta1, &c.sched);
  if (st) {
    xzzx_free_code(c.code);
    return st;
  }
  const size_t R = (size_t)sv->cfg.restarts, w = (size_t)c.code->w;
  // descriptors (segment + chunks + prefixes), workspace, syndrome, output row
  const size_t chunks = (4 * R + batch::kNT - 1) / batch::kNT;
  c.bytes = sizeof(batch::SegDev) + chunks * 2 * sizeof(batch::ChunkDev) + 2 * sizeof(int64_t) +
            align256(sizeof(uint32_t) * R * 2 * w) + align256(R) + align256(sizeof(int32_t) * 4 * R) +
            align256(sizeof(uint32_t) * c.code->sw) + kOutStride;
  c.regs = 0;  // filled at start, from the kernel's register use
  *class_id = (int)sv->classes.size();
  sv->classes.push_back(c);
  return XZZX_OK;
}

xzzx_status xzzx_serve_start(xzzx_server* sv) {
  if (!sv) return fail(XZZX_EINVAL, "server is NULL");
  if (sv->started) return fail(XZZX_EINVAL, "already started");
  if (sv->classes.empty()) return fail(XZZX_EINVAL, "no classes registered");
  xzzx_status st = check_device(sv->device);
  if (st) return st;
  // On-chip budget: a request's CTAs take the share of an SM that its
  // distance's chunk kernel occupies.
  int regs_per_sm = 0;
  XZZX_CUDA_TRY(cudaDeviceGetAttribute(&regs_per_sm, cudaDevAttrMaxRegistersPerMultiprocessor, sv->device));
  sv->regs_total = (int64_t)regs_per_sm * sv->n_sm * (sv->cfg.resident_waves > 0 ? sv->cfg.resident_waves : 2);
  for (Class& c : sv->classes) {
    int per_sm = 0;
    if ((st = batch::configure_plan_kernels(c.d, batch::kNT, 1, &per_sm))) return st;
    if ((st = batch::occupancy_chunks(c.d, batch::kNT, 1, &per_sm))) return st;
    if (per_sm < 1) per_sm = 1;
    const int64_t ctas = (4 * (int64_t)sv->cfg.restarts + batch::kNT - 1) / batch::kNT;
    c.regs = ctas * (regs_per_sm / per_sm);
  }
  const size_t budget = sv->cfg.hbm_budget_bytes ? sv->cfg.hbm_budget_bytes : ((size_t)256 << 20);
  sv->slot_bytes = budget / sv->cfg.n_slots & ~(size_t)255;
  sv->staging_bytes = ((size_t)64 << 10) + (size_t)sv->cfg.max_batch * 1024;
  // Every class must fit one request into an empty slot (memory and staging),
  // or requests of that class could never be dispatched.
  for (const Class& c : sv->classes)
    if (4096 + c.bytes > sv->slot_bytes || 4096 + c.bytes > sv->staging_bytes)
      return fail(XZZX_ENOMEM, "one request of distance " + std::to_string(c.d) + " needs " +
                                   std::to_string(4096 + c.bytes) + " bytes but a slot holds " +
                                   std::to_string(sv->slot_bytes) + " (raise hbm_budget_bytes or lower n_slots)");
  // One device error area for every class's code, so that each batch's flags
  // can be read back with its results.
  XZZX_CUDA_TRY(cudaMalloc((void**)&sv->d_err, 256));
  XZZX_CUDA_TRY(cudaMemset(sv->d_err, 0, 256));
  for (Class& c : sv->classes) c.code->dev.err = sv->d_err;
  sv->slots.resize(sv->cfg.n_slots);
  for (int i = 0; i < sv->cfg.n_slots; ++i) {
    Slot& s = sv->slots[i];
    s.server = sv;
    s.index = i;
    cudaError_t e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc((void**)&s.dev, sv->slot_bytes);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&s.host_in, sv->staging_bytes);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&s.host_out, (size_t)sv->cfg.max_batch * kOutStride + 256);
    if (e != cudaSuccess) return cuda_fail(e, "xzzx_serve_start slot allocation");
  }
  sv->started = true;
  sv->dispatcher = std::thread(dispatcher_main, sv);
  return XZZX_OK;
}

static xzzx_status submit_locked(xzzx_server* sv, uint64_t req_id, int class_id, const uint32_t* syn) {
  if (sv->sticky) return fail(sv->sticky, sv->sticky_msg);
  if ((int)sv->pending.size() >= sv->cfg.queue_capacity) {
    ++sv->rejected;
    return fail(XZZX_EBUSY, "request queue full");
  }
  Req r;
  r.id = req_id;
  r.cls = class_id;
  r.t_submit = Clock::now();
  std::memset(r.syn, 0, sizeof(r.syn));
  std::memcpy(r.syn, syn, sizeof(uint32_t) * sv->classes[class_id].code->sw);
  sv->pending.push_back(r);
  ++sv->submitted;
  return XZZX_OK;
}

xzzx_status xzzx_serve_submit(xzzx_server* sv, uint64_t req_id, int class_id, const uint32_t* syndrome_host) {
  if (!sv || !syndrome_host) return fail(XZZX_EINVAL, "NULL argument");
  if (!sv->started) return fail(XZZX_EINVAL, "server not started");
  if (class_id < 0 || class_id >= (int)sv->classes.size()) return fail(XZZX_EINVAL, "unknown class");
  xzzx_status st;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    st = submit_locked(sv, req_id, class_id, syndrome_host);
  }
  if (!st) sv->cv.notify_all();
  return st;
}

xzzx_status xzzx_serve_replay(xzzx_server* sv, int n, const uint64_t* req_ids, const int32_t* class_ids,
                              const uint32_t* syndromes, const double* arrival_us) {
  if (!sv || n < 0 || (n > 0 && (!req_ids || !class_ids || !syndromes || !arrival_us)))
    return fail(XZZX_EINVAL, "bad arguments");
  if (!sv->started) return fail(XZZX_EINVAL, "server not started");
  for (int i = 0; i < n; ++i)
    if (class_ids[i] < 0 || class_ids[i] >= (int)sv->classes.size()) return fail(XZZX_EINVAL, "unknown class");
  std::vector<uint64_t> ids(req_ids, req_ids + n);
  std::vector<int32_t> cls(class_ids, class_ids + n);
  std::vector<uint32_t> syn(syndromes, syndromes + (size_t)n * 32);
  std::vector<double> at(arrival_us, arrival_us + n);
  sv->replayers.emplace_back([sv, ids, cls, syn, at]() {
    const Clock::time_point t0 = Clock::now();
    for (size_t i = 0; i < ids.size(); ++i) {
      const Clock::time_point due = t0 + std::chrono::nanoseconds((int64_t)(at[i] * 1e3));
      for (;;) {
        const Clock::time_point now = Clock::now();
        if (now >= due) break;
        if (due - now > std::chrono::microseconds(200)) std::this_thread::sleep_for(due - now - std::chrono::microseconds(100));
      }
      {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->stop) return;
        submit_locked(sv, ids[i], cls[i], &syn[i * 32]);
      }
      sv->cv.notify_all();
    }
  });
  return XZZX_OK;
}

xzzx_status xzzx_serve_poll(xzzx_server* sv, xzzx_result* out, int cap, int* n_out, int timeout_ms) {
  if (!sv || !n_out || (cap > 0 && !out)) return fail(XZZX_EINVAL, "NULL argument");
  std::unique_lock<std::mutex> lk(sv->mu);
  if (sv->done.empty() && timeout_ms > 0)
    sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return !sv->done.empty() || sv->sticky; });
  const int n = std::min<int>(cap, (int)sv->done.size());
  for (int i = 0; i < n; ++i) out[i] = sv->done[i];
  sv->done.erase(sv->done.begin(), sv->done.begin() + n);
  *n_out = n;
  if (sv->sticky) return fail(sv->sticky, sv->sticky_msg);
  if (n == 0 && timeout_ms > 0) return fail(XZZX_ETIMEOUT, "no result within the timeout");
  return XZZX_OK;
}

xzzx_status xzzx_serve_get_stats(xzzx_server* sv, xzzx_serve_stats* out, int reset) {
  if (!sv || !out) return fail(XZZX_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  std::memset(out, 0, sizeof(*out));
  out->submitted = sv->submitted;
  out->rejected = sv->rejected;
  out->dispatched = sv->dispatched;
  out->completed = sv->completed;
  out->batches = sv->batches;
  out->pending = (int64_t)sv->pending.size();
  for (const Slot& s : sv->slots) out->in_flight += (int64_t)s.reqs.size();
  out->mean_batch = sv->batches ? (double)sv->dispatched / sv->batches : 0.0;
  out->device_errors = sv->device_errors;
  if (!sv->lat_us.empty()) {
    std::vector<double> v = sv->lat_us;
    std::sort(v.begin(), v.end());
    auto pct = [&](double q) { return v[std::min(v.size() - 1, (size_t)(q * (v.size() - 1) + 0.5))]; };
    out->p50_us = pct(0.50);
    out->p99_us = pct(0.99);
    out->max_us = v.back();
    double sum = 0;
    for (double x : v) sum += x;
    out->mean_us = sum / v.size();
  }
  if (reset) {
    sv->lat_us.clear();
    sv->submitted = sv->rejected = sv->dispatched = sv->completed = sv->batches = 0;
  }
  return XZZX_OK;
}

void xzzx_serve_destroy(xzzx_server* sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv.notify_all();
  for (std::thread& t : sv->replayers)
    if (t.joinable()) t.join();
  if (sv->dispatcher.joinable()) sv->dispatcher.join();
  for (Slot& s : sv->slots) {
    if (s.stream) {
      cudaStreamSynchronize(s.stream);
      cudaStreamDestroy(s.stream);
    }
    if (s.dev) cudaFree(s.dev);
    if (s.host_in) cudaFreeHost(s.host_in);
    if (s.host_out) cudaFreeHost(s.host_out);
  }
  if (sv->d_err) cudaFree(sv->d_err);
  for (Class& c : sv->classes) {
    xzzx_free_schedule(c.sched);
    xzzx_free_code(c.code);
  }
  delete sv;
}

}  // extern "C"
