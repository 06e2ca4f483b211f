// Host side of libxzzx: error reporting, code tables, noise weights and the
// FP64 acceptance-threshold table.  All of it runs once per handle; the
// kernels only read the uploaded tables.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <set>

#include "internal.h"

namespace xzzx {

static thread_local std::string g_last_error;

xzzx_status fail(xzzx_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

xzzx_status ok() { return XZZX_OK; }

xzzx_status cuda_fail(cudaError_t e, const char* what) {
  return fail(XZZX_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

PhiloxKeys philox_keys(uint64_t seed) {
  PhiloxKeys K;
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    K.k0[r] = k0;
    K.k1[r] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return K;
}

xzzx_status check_code(const xzzx_code* code) {
  if (!code || code->d < 3) return fail(XZZX_EINVAL, "invalid code handle");
  if (!code->dev_block) return fail(XZZX_EINVAL, "code handle has no device tables (created without a GPU)");
  return check_device(code->device);
}

xzzx_status check_device(int device) {
  int cur = -1;
  XZZX_CUDA_TRY(cudaGetDevice(&cur));
  if (cur != device)
    return fail(XZZX_EINVAL, "handle was created on device " + std::to_string(device) + " but device " +
                                 std::to_string(cur) + " is current");
  return XZZX_OK;
}

xzzx_status check_ptr(const void* p, const char* name) {
  if (!p) return fail(XZZX_EINVAL, std::string(name) + " is NULL");
  return XZZX_OK;
}

namespace {

// Face (a, b) of the rotated layout: the bulk squares plus the weight-2 faces
// that alternate along each side (top: odd b, bottom: even b, left: even a,
// right: odd a), so that every boundary qubit component is detected.
bool rotated_face(int d, int a, int b) {
  const bool a_in = 0 <= a && a <= d - 2;
  const bool b_in = 0 <= b && b <= d - 2;
  if (a_in && b_in) return true;
  if (b_in && a == -1) return (b & 1) == 1;
  if (b_in && a == d - 1) return (b & 1) == 0;
  if (a_in && b == -1) return (a & 1) == 0;
  if (a_in && b == d - 1) return (a & 1) == 1;
  return false;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// True when a CUDA device is usable; handles built without one keep only their
// host tables.
bool has_device() {
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return n > 0;
}

// Schedule value at sweep t (see xzzx_make_schedule).
double beta_of(int kind, int n, double beta0, double beta1, int t) {
  if (kind == XZZX_SCHED_LINEAR) {
    if (n <= 1) return beta0;
    return beta0 + (beta1 - beta0) * (double)t / (double)(n - 1);
  }
  const double gamma = n >= 2 ? (beta1 / beta0 - 1.0) / std::log((double)n) : 0.0;
  return beta0 * (1.0 + gamma * std::log((double)(t + 1)));
}

// floor(2^32 exp(-beta dE / scale)), saturated at 2^32 - 1.
uint32_t threshold_of(double beta, int32_t dE, int32_t scale) {
  const double x = beta * (double)dE / (double)scale;
  const double v = std::ldexp(std::exp(-x), 32);
  if (v >= 4294967295.0) return 0xFFFFFFFFu;
  return (uint32_t)v;
}

}  // namespace
}  // namespace xzzx

using namespace xzzx;

extern "C" {

const char* xzzx_last_error(void) { return g_last_error.c_str(); }

const char* xzzx_version(void) { return "xzzx-gb300 0.1 (sm_103a)"; }

size_t xzzx_abi_struct_size(int which) {
  switch (which) {
    case 0: return sizeof(xzzx_noise);
    case 1: return sizeof(xzzx_code_info);
    case 2: return sizeof(xzzx_segment);
    case 3: return sizeof(xzzx_batch_cfg);
    case 4: return sizeof(xzzx_batch_info);
    case 5: return sizeof(xzzx_serve_cfg);
    case 6: return sizeof(xzzx_result);
    case 7: return sizeof(xzzx_serve_stats);
    default: return 0;
  }
}

namespace xzzx {
namespace {

// The planar layout: faces (i, j), i + j odd, of the (2d-1)^2 grid, indexed in
// the order (colour, j>>2, i>>1) with colour = (i&1) | (((i+j-1)/2 & 1) << 1);
// corners left, up, down, right; L_Z = Z on row 0, L_X = X on column 0.
void build_planar(xzzx_code* c) {
  const int d = c->d, g = 2 * d - 1;
  c->nq = d * d + (d - 1) * (d - 1);
  c->w = (c->nq + 31) / 32;
  c->face_at.assign((size_t)g * g, -1);
  struct F {
    int colour, ib, ia, i, j;
  };
  std::vector<F> fs;
  for (int i = 0; i < g; ++i)
    for (int j = 0; j < g; ++j)
      if ((i + j) & 1) fs.push_back({(i & 1) | ((((i + j - 1) >> 1) & 1) << 1), j >> 2, i >> 1, i, j});
  std::sort(fs.begin(), fs.end(), [](const F& x, const F& y) {
    if (x.colour != y.colour) return x.colour < y.colour;
    if (x.ib != y.ib) return x.ib < y.ib;
    return x.ia < y.ia;
  });
  for (int k = 0; k < 5; ++k) c->colour_start[k] = 0;
  auto site = [&](int r, int col) {
    return (r >= 0 && r < g && col >= 0 && col < g) ? planar_qubit(d, r, col) : -1;
  };
  for (const F& f : fs) {
    c->face_at[(size_t)f.i * g + f.j] = (int16_t)c->a.size();
    c->a.push_back((int16_t)f.i);
    c->b.push_back((int16_t)f.j);
    c->c2.push_back((uint8_t)(f.i & 1));
    c->c4.push_back((uint8_t)f.colour);
    c->colour_start[f.colour + 1]++;
    c->corners.push_back(site(f.i, f.j - 1));
    c->corners.push_back(site(f.i - 1, f.j));
    c->corners.push_back(site(f.i + 1, f.j));
    c->corners.push_back(site(f.i, f.j + 1));
  }
  for (int k = 0; k < 4; ++k) c->colour_start[k + 1] += c->colour_start[k];
  c->ns = (int)c->a.size();
  c->sw = (c->ns + 31) / 32;
  const int w = c->w;
  c->logical.assign(4 * w, 0u);
  uint32_t* LX = c->logical.data();
  uint32_t* LZ = c->logical.data() + 2 * w;
  for (int col = 0; col < g; col += 2) {
    const int q = planar_qubit(d, 0, col);
    LZ[w + (q >> 5)] |= 1u << (q & 31);  // Z
  }
  for (int r = 0; r < g; r += 2) {
    const int q = planar_qubit(d, r, 0);
    LX[q >> 5] |= 1u << (q & 31);  // X
  }
}

}  // namespace
}  // namespace xzzx

xzzx_status xzzx_make_code(int d, int layout, xzzx_code** out) {
  if (!out) return fail(XZZX_EINVAL, "out is NULL");
  *out = nullptr;
  if (layout != kLayoutRotated && layout != kLayoutPlanar)
    return fail(XZZX_EUNSUPPORTED, "layout must be 0 (rotated) or 1 (planar)");
  if (d < 3 || d > kMaxD || (d & 1) == 0) return fail(XZZX_EINVAL, "d must be odd and in [3, 31]");
  xzzx_code* c = new (std::nothrow) xzzx_code();
  if (!c) return fail(XZZX_ENOMEM, "host allocation");
  c->d = d;
  c->layout = layout;
  if (layout == kLayoutPlanar) build_planar(c);
  c->nq = layout == kLayoutPlanar ? c->nq : d * d;
  c->w = (c->nq + 31) / 32;
  if (layout == kLayoutRotated) c->face_at.assign((d + 1) * (d + 1), -1);
  for (int colour = 0; colour < 4 && layout == kLayoutRotated; ++colour) {
    c->colour_start[colour] = (int)c->a.size();
    const int pa = colour & 1, pb = colour >> 1;
    for (int a = -1; a <= d - 1; ++a) {
      if ((a & 1) != pa) continue;
      for (int b = -1; b <= d - 1; ++b) {
        if ((b & 1) != pb || !rotated_face(d, a, b)) continue;
        c->face_at[(a + 1) * (d + 1) + (b + 1)] = (int16_t)c->a.size();
        c->a.push_back((int16_t)a);
        c->b.push_back((int16_t)b);
        c->c2.push_back((uint8_t)((a + b) & 1));
        c->c4.push_back((uint8_t)colour);
        const int rr[4] = {a, a, a + 1, a + 1}, cc[4] = {b, b + 1, b, b + 1};
        for (int k = 0; k < 4; ++k) {
          const bool in = rr[k] >= 0 && rr[k] < d && cc[k] >= 0 && cc[k] < d;
          c->corners.push_back(in ? rr[k] * d + cc[k] : -1);
        }
      }
    }
  }
  if (layout == kLayoutRotated) {
    c->colour_start[4] = (int)c->a.size();
    c->ns = (int)c->a.size();
    c->sw = (c->ns + 31) / 32;
    // L_X: column 0 alternating X, Z; L_Z: row 0 alternating Z, X.
    const int w = c->w;
    c->logical.assign(4 * w, 0u);
    uint32_t* LX = c->logical.data();
    uint32_t* LZ = c->logical.data() + 2 * w;
    for (int r = 0; r < d; ++r) {
      const int q = r * d;
      (r % 2 == 0 ? LX : LX + w)[q >> 5] |= 1u << (q & 31);
    }
    for (int col = 0; col < d; ++col) {
      const int q = col;
      (col % 2 == 0 ? LZ + w : LZ)[q >> 5] |= 1u << (q & 31);
    }
  }
  // Upload the device tables in one block.
  const size_t o_a = 0;
  const size_t o_b = align256(o_a + sizeof(int16_t) * c->ns);
  const size_t o_c2 = align256(o_b + sizeof(int16_t) * c->ns);
  const size_t o_at = align256(o_c2 + c->ns);
  const size_t o_log = align256(o_at + sizeof(int16_t) * c->face_at.size());
  const size_t o_err = align256(o_log + sizeof(uint32_t) * c->logical.size());
  const size_t total = align256(o_err + sizeof(uint32_t) * kErrWords);
  if (!has_device()) {  // host tables only; launches on this handle are refused
    *out = c;
    return XZZX_OK;
  }
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaMalloc(&c->dev_block, total);
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e, "xzzx_make_code device tables");
  }
  std::vector<char> blob(total, 0);
  std::memcpy(blob.data() + o_a, c->a.data(), sizeof(int16_t) * c->ns);
  std::memcpy(blob.data() + o_b, c->b.data(), sizeof(int16_t) * c->ns);
  std::memcpy(blob.data() + o_c2, c->c2.data(), c->ns);
  std::memcpy(blob.data() + o_at, c->face_at.data(), sizeof(int16_t) * c->face_at.size());
  std::memcpy(blob.data() + o_log, c->logical.data(), sizeof(uint32_t) * c->logical.size());
  e = cudaMemcpy(c->dev_block, blob.data(), total, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(c->dev_block);
    delete c;
    return cuda_fail(e, "xzzx_make_code upload");
  }
  char* base = (char*)c->dev_block;
  DevCode& dv = c->dev;
  dv.d = d;
  dv.layout = layout;
  dv.nq = c->nq;
  dv.ns = c->ns;
  dv.w = c->w;
  dv.sw = c->sw;
  for (int k = 0; k < 5; ++k) dv.colour_start[k] = c->colour_start[k];
  dv.face_a = (const int16_t*)(base + o_a);
  dv.face_b = (const int16_t*)(base + o_b);
  dv.face_c2 = (const uint8_t*)(base + o_c2);
  dv.face_at = (const int16_t*)(base + o_at);
  dv.logical = (const uint32_t*)(base + o_log);
  dv.err = (uint32_t*)(base + o_err);  // zeroed with the blob
  *out = c;
  return XZZX_OK;
}

xzzx_status xzzx_get_code_info(const xzzx_code* code, xzzx_code_info* out) {
  if (!code || !out) return fail(XZZX_EINVAL, "NULL argument");
  out->d = code->d;
  out->n_qubits = code->nq;
  out->n_stab = code->ns;
  out->words = code->w;
  out->syn_words = code->sw;
  for (int k = 0; k < 5; ++k) out->colour_start[k] = code->colour_start[k];
  return XZZX_OK;
}

xzzx_status xzzx_code_faces(const xzzx_code* code, int32_t* a, int32_t* b, int32_t* corners) {
  if (!code) return fail(XZZX_EINVAL, "NULL code");
  for (int f = 0; f < code->ns; ++f) {
    if (a) a[f] = code->a[f];
    if (b) b[f] = code->b[f];
    if (corners)
      for (int k = 0; k < 4; ++k) corners[4 * f + k] = code->corners[4 * f + k];
  }
  return XZZX_OK;
}

void xzzx_free_code(xzzx_code* code) {
  if (!code) return;
  if (code->dev_block) cudaFree(code->dev_block);
  delete code;
}

xzzx_status xzzx_device_errors(const xzzx_code* code, uint32_t* flags, uint32_t* count, int clear, void* stream) {
  xzzx_status st = check_code(code);
  if (st) return st;
  const cudaStream_t s = (cudaStream_t)stream;
  uint32_t words[2] = {0u, 0u};
  XZZX_CUDA_TRY(cudaMemcpyAsync(words, code->dev.err, sizeof(words), cudaMemcpyDeviceToHost, s));
  if (clear) XZZX_CUDA_TRY(cudaMemsetAsync(code->dev.err, 0, sizeof(words), s));
  XZZX_CUDA_TRY(cudaStreamSynchronize(s));
  if (flags) *flags = words[0];
  if (count) *count = words[1];
  return XZZX_OK;
}

xzzx_status xzzx_debug_inject(const xzzx_code* code, uint32_t flags, void* stream) {
  xzzx_status st = check_code(code);
  if (st) return st;
  if (flags & ~(uint32_t)(XZZX_DEVERR_GREEDY_WALK | XZZX_DEVERR_BOUNDS)) return fail(XZZX_EINVAL, "unknown flag");
  // The value lives in a stream-ordered upload from a host word that must
  // outlive the copy: a static per flag combination.
  static const uint32_t kValues[4] = {0u, 1u, 2u, 3u};
  XZZX_CUDA_TRY(cudaMemcpyAsync(code->dev.err + 2, &kValues[flags], sizeof(uint32_t), cudaMemcpyHostToDevice,
                                (cudaStream_t)stream));
  return XZZX_OK;
}

xzzx_status xzzx_make_noise(double px, double py, double pz, int32_t scale, xzzx_noise* out) {
  if (!out) return fail(XZZX_EINVAL, "out is NULL");
  if (!(px > 0.0) || !(py > 0.0) || !(pz > 0.0))
    return fail(XZZX_EINVAL, "px, py and pz must be positive");
  if (scale <= 0 || scale > (1 << 20)) return fail(XZZX_EINVAL, "scale must be in [1, 2^20]");
  const double p = px + py + pz;
  if (!(p < 0.5)) return fail(XZZX_EINVAL, "p = px+py+pz must be below 1/2");
  const double s = (double)scale, q = 1.0 - p;
  out->px = px;
  out->py = py;
  out->pz = pz;
  out->scale = scale;
  out->W[0] = 0;
  out->W[1] = (int32_t)std::llround(s * -std::log(pz / q));  // Z
  out->W[2] = (int32_t)std::llround(s * -std::log(px / q));  // X
  out->W[3] = (int32_t)std::llround(s * -std::log(py / q));  // Y
  out->Wt_x = (int32_t)std::llround(s * -std::log((px + py) / q));
  out->Wt_z = (int32_t)std::llround(s * -std::log((pz + py) / q));
  return XZZX_OK;
}

xzzx_status xzzx_noise_from_eta(double p, double eta, int convention, int32_t scale, xzzx_noise* out) {
  if (!(p > 0.0) || !(eta > 0.0) || !std::isfinite(eta)) return fail(XZZX_EINVAL, "p and eta must be positive");
  double px, py;
  if (convention == 0) {
    py = p * eta / (eta + 1.0);
    px = p / (2.0 * (eta + 1.0));
  } else if (convention == 1) {
    py = p * eta / (eta + 2.0);
    px = p / (eta + 2.0);
  } else {
    return fail(XZZX_EINVAL, "convention must be 0 or 1");
  }
  return xzzx_make_noise(px, py, px, scale, out);
}

xzzx_status xzzx_make_schedule(const xzzx_noise* noise, int kind, int n_sweeps, double beta0, double beta1,
                               xzzx_schedule** out) {
  if (!out || !noise) return fail(XZZX_EINVAL, "NULL argument");
  *out = nullptr;
  if (kind != XZZX_SCHED_LINEAR && kind != XZZX_SCHED_PAPER_LOG) return fail(XZZX_EINVAL, "unknown schedule kind");
  if (n_sweeps < 0 || n_sweeps > (1 << 24)) return fail(XZZX_EINVAL, "n_sweeps must be in [0, 2^24]");
  if (!(beta0 >= 0.0) || !(beta1 >= 0.0) || !std::isfinite(beta0) || !std::isfinite(beta1))
    return fail(XZZX_EINVAL, "beta0 and beta1 must be finite and non-negative");
  if (kind == XZZX_SCHED_PAPER_LOG && !(beta0 > 0.0)) return fail(XZZX_EINVAL, "PAPER_LOG needs beta0 > 0");
  if (noise->scale <= 0) return fail(XZZX_EINVAL, "noise not initialised");
  xzzx_schedule* s = new (std::nothrow) xzzx_schedule();
  if (!s) return fail(XZZX_ENOMEM, "host allocation");
  s->kind = kind;
  s->n_sweeps = n_sweeps;
  s->beta0 = beta0;
  s->beta1 = beta1;
  s->noise = *noise;
  // Energy change of each generator shape for each corner signature.  Rotated
  // (compact table: bulk by its 8-bit signature TL|TR<<2|BL<<4|BR<<6, weight-2
  // shapes by their two present corners): X flips the x bit of TL and BR, Z
  // flips the z bit of TR and BL.  Planar (bulk left|right<<2|up<<4|down<<6,
  // three-body shapes by their present corners): X on left and right, Z on up
  // and down.
  s->sig_dE.assign(kSigTable, 0);
  s->sig_class.assign(kSigTable, -1);
  std::set<int32_t> positive;
  auto fill = [&](int base, int mask, const int* flip) {
    int present[4], np = 0;
    for (int k = 0; k < 4; ++k)
      if ((mask >> k) & 1) present[np++] = k;
    for (int code = 0; code < (1 << (2 * np)); ++code) {
      int64_t dE = 0;
      for (int j = 0; j < np; ++j) {
        const int lab = (code >> (2 * j)) & 3;
        dE += (int64_t)noise->W[lab ^ flip[present[j]]] - (int64_t)noise->W[lab];
      }
      s->sig_dE[base + code] = (int32_t)dE;
      if (dE > 0) positive.insert((int32_t)dE);
    }
  };
  const int flip_rot[4] = {2, 1, 1, 2}, flip_planar[4] = {2, 2, 1, 1};
  for (int y = 0; y < kNumTypes; ++y) fill(sig_base(y), kCornerMask[y], flip_rot);
  for (int y = 0; y < kNumPShapes; ++y) fill(planar_sig_base(y), kPlanarCornerMask[y], flip_planar);
  s->dE_class.assign(positive.begin(), positive.end());
  s->n_classes = (int)s->dE_class.size();
  for (int i = 0; i < kSigTable; ++i) {
    const int32_t dE = s->sig_dE[i];
    if (dE > 0)
      s->sig_class[i] = (int32_t)(std::lower_bound(s->dE_class.begin(), s->dE_class.end(), dE) - s->dE_class.begin());
  }
  s->T.assign((size_t)n_sweeps * s->n_classes, 0u);
  for (int t = 0; t < n_sweeps; ++t) {
    const double beta = beta_of(kind, n_sweeps, beta0, beta1, t);
    for (int k = 0; k < s->n_classes; ++k)
      s->T[(size_t)t * s->n_classes + k] = threshold_of(beta, s->dE_class[k], noise->scale);
  }
  std::vector<int2> sig(kSigTable);
  for (int i = 0; i < kSigTable; ++i) sig[i] = make_int2(s->sig_dE[i], s->sig_class[i]);
  if (!has_device()) {  // host tables only; launches with this handle are refused
    *out = s;
    return XZZX_OK;
  }
  const size_t tbytes = sizeof(uint32_t) * std::max<size_t>(s->T.size(), 1);
  cudaError_t e = cudaGetDevice(&s->device);
  if (e == cudaSuccess) e = cudaMalloc((void**)&s->d_T, tbytes);
  if (e == cudaSuccess) e = cudaMalloc((void**)&s->d_sig, sizeof(int2) * sig.size());
  if (e == cudaSuccess && !s->T.empty())
    e = cudaMemcpy(s->d_T, s->T.data(), sizeof(uint32_t) * s->T.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->d_sig, sig.data(), sizeof(int2) * sig.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    xzzx_free_schedule(s);
    return cuda_fail(e, "xzzx_make_schedule upload");
  }
  *out = s;
  return XZZX_OK;
}

void xzzx_free_schedule(xzzx_schedule* s) {
  if (!s) return;
  if (s->d_T) cudaFree(s->d_T);
  if (s->d_sig) cudaFree(s->d_sig);
  delete s;
}

xzzx_status xzzx_schedule_table(const xzzx_schedule* s, int* n_classes, int32_t* dE, int cap_classes, uint32_t* T) {
  if (!s || !n_classes) return fail(XZZX_EINVAL, "NULL argument");
  *n_classes = s->n_classes;
  if (dE) {
    if (cap_classes < s->n_classes) return fail(XZZX_EINVAL, "dE capacity too small");
    for (int k = 0; k < s->n_classes; ++k) dE[k] = s->dE_class[k];
  }
  if (T && !s->T.empty()) std::memcpy(T, s->T.data(), sizeof(uint32_t) * s->T.size());
  return XZZX_OK;
}

}  // extern "C"
