/*
 * xzzx.h -- C ABI of the GB300 simulated-annealing decoder for the XZZX code
 * (T. Sakashita, "Simulated-annealing decoder for the XZZX code with
 * greedy-matching initialization", arXiv:2509.17837).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every function returns an xzzx_status; XZZX_OK is 0.  On failure
 *   xzzx_last_error() returns a message for the calling thread.  No C++
 *   exception crosses this boundary.
 * - The library owns only opaque handles (xzzx_code, xzzx_schedule,
 *   xzzx_server) and the device tables they hold; xzzx_free_* releases them.
 *   The caller owns every data buffer.  Buffers marked "device" must be device
 *   memory of the GPU that was current when the handle was created; buffers
 *   marked "host" are ordinary host memory.
 * - Device calls take a cudaStream_t passed as void* (NULL = legacy default
 *   stream), validate every size on the host before launching anything, and
 *   run asynchronously on that stream.  A kernel fault surfaces as
 *   XZZX_ECUDA from the launch or from a later synchronising call.
 * - Rotated layout (layout 0): data qubit (r, c), 0 <= r, c < d, has index
 *   q = r*d + c; the d*d - 1 generators are indexed colour by colour (colour =
 *   (a&1) | ((b&1)<<1) of the face (a, b)), then by a, then by b.
 * - Planar layout (layout 1, the paper's lattice): the sites (r, c) of a
 *   (2d-1) x (2d-1) grid; data qubits on the sites with r + c even
 *   (n = d*d + (d-1)*(d-1)), indexed row-major over those sites
 *   (q = (r>>1)(2d-1) + (r odd ? d : 0) + (c>>1)); faces on the sites with
 *   r + c odd (2d(d-1) generators X_left Z_up Z_down X_right, three-body on
 *   the boundary), indexed by colour = (i&1) | (((i+j-1)/2 & 1) << 1) of face
 *   (i, j), then by j>>2, then by i>>1.  L_Z is Z on row 0, L_X is X on
 *   column 0.
 * - Configuration layout ("2w words"): w = ceil(n/32) for n data qubits;
 *   words [0, w) hold the X bits, words [w, 2w) the Z bits; qubit q is bit
 *   (q & 31) of word q >> 5.  Pauli I, X, Y, Z is (x, z) = (0,0), (1,0),
 *   (1,1), (0,1).
 * - Syndrome layout ("sw words"): sw = ceil(n_stab/32); generator f is bit
 *   (f & 31) of word f >> 5.
 * - Logical classes are indexed I=0, X=1, Y=2, Z=3.
 * - Randomness: Philox4x32-10 keyed by the 64-bit seed.  A draw depends only on
 *   (seed, purpose, shot, restart/chain, sweep, face), so results do not
 *   depend on how shots are split across calls or launches.
 */
#ifndef XZZX_H
#define XZZX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  XZZX_OK = 0,
  XZZX_EINVAL = 1,      /* bad argument, size or handle */
  XZZX_ENOMEM = 2,      /* host or device allocation failed */
  XZZX_ECUDA = 3,       /* a CUDA runtime call or kernel launch failed */
  XZZX_ETIMEOUT = 4,    /* a bounded device or host wait ran out */
  XZZX_EBUSY = 5,       /* no capacity left (server admission) */
  XZZX_EUNSUPPORTED = 6 /* valid request this build does not implement */
} xzzx_status;

/* Message describing the last failure on the calling thread ("" if none). */
const char* xzzx_last_error(void);

/* Device-side error flags.  Kernels never trap: a failure they detect is
 * recorded in the error area of the code handle the work used and the work
 * goes on.  XZZX_DEVERR_GREEDY_WALK: a greedy path walk or matching round
 * could not complete (never expected on a valid code; that reference then
 * does not reproduce its syndrome, and bit 7 of its cbits byte is set).
 * XZZX_DEVERR_BOUNDS: a bounds check of the checked build (compiled with
 * -DXZZX_CHECKS) found an index outside its buffer and skipped the access. */
#define XZZX_DEVERR_GREEDY_WALK 0x1u
#define XZZX_DEVERR_BOUNDS 0x2u

/* Library version string. */
const char* xzzx_version(void);

/* Size in bytes of public struct number which, as compiled into the library:
 * 0 xzzx_noise, 1 xzzx_code_info, 2 xzzx_segment, 3 xzzx_batch_cfg,
 * 4 xzzx_batch_info, 5 xzzx_serve_cfg, 6 xzzx_result, 7 xzzx_serve_stats;
 * 0 for any other number.  Host only (no device needed), for bindings to
 * check their own copies of the layouts.  The paper has no counterpart. */
size_t xzzx_abi_struct_size(int which);

/* ------------------------------------------------------------------------ */
/* Code tables (Sec. "The XZZX code", Eq. stabilizer_generator).           */
/* ------------------------------------------------------------------------ */

typedef struct xzzx_code xzzx_code;

typedef struct {
  int32_t d;
  int32_t n_qubits;        /* rotated d*d; planar d*d + (d-1)*(d-1) */
  int32_t n_stab;          /* n_qubits - 1 */
  int32_t words;           /* w: words per bit plane; a configuration is 2w words */
  int32_t syn_words;       /* sw: words per syndrome */
  int32_t colour_start[5]; /* generators of colour c are [start[c], start[c+1]) */
} xzzx_code_info;

/* Build the distance-d XZZX code (Eq. stabilizer_generator).  layout 0: the
 * rotated lattice, G_f = X_TL Z_TR Z_BL X_BR on the corners of face f inside
 * the lattice, L_Z along row 0 and L_X along column 0.  layout 1: the paper's
 * planar lattice (Sec. "The XZZX code"), G_f = X_left Z_up Z_down X_right.
 * d must be odd, 3 <= d <= 31; another layout returns XZZX_EUNSUPPORTED.
 * Planar codes run through sampling, greedy initialisation, xzzx_anneal,
 * xzzx_anneal_variant, the decision and xzzx_decode_batch; the warp-per-chain
 * kernel, batches and the server take rotated codes only (XZZX_EUNSUPPORTED).
 * Uploads the tables to the current device.  *out is owned by the caller and
 * released with xzzx_free_code. */
xzzx_status xzzx_make_code(int d, int layout, xzzx_code** out);
xzzx_status xzzx_get_code_info(const xzzx_code* code, xzzx_code_info* out);
void xzzx_free_code(xzzx_code* code);

/* Read the device-side error flags raised by work done with this code (OR
 * of XZZX_DEVERR_*) into *flags and how many times one was raised into
 * *count (either may be NULL), after the work already queued on stream;
 * with clear != 0 they are reset to zero after the read.  Synchronises
 * stream.  Work on other streams is included once it has finished. */
xzzx_status xzzx_device_errors(const xzzx_code* code, uint32_t* flags, uint32_t* count, int clear, void* stream);

/* Test hook: ask the kernels that use this code to raise the given
 * XZZX_DEVERR_* flags as if the failure had happened, without faulting
 * anything (flags = 0 turns it off).  GREEDY_WALK marks restart 0 of every
 * shot in xzzx_greedy_init (bit 7 of its cbits byte; the reference itself is
 * unchanged); in the checked build, BOUNDS makes the bounds check of the
 * annealing kernels' table lookup fail, which skips the lookup (the move is
 * then taken with dE = 0, so energies are no longer meaningful) and raises
 * the flag.  The plain build ignores BOUNDS.  Ordered on stream. */
xzzx_status xzzx_debug_inject(const xzzx_code* code, uint32_t flags, void* stream);

/* Generator f as four corner qubits (-1 outside) in the order of its X, Z, Z,
 * X factors (rotated TL, TR, BL, BR; planar left, up, down, right) and its
 * face coordinates (rotated (a, b); planar (i, j)); host arrays of n_stab
 * entries (corners: 4*n_stab).  Any pointer may be NULL. */
xzzx_status xzzx_code_faces(const xzzx_code* code, int32_t* a, int32_t* b, int32_t* corners);

/* ------------------------------------------------------------------------ */
/* Noise and energies (Eqs. noise_map, coeff_in_energy, energy,            */
/* coeff_in_distance).                                                      */
/* ------------------------------------------------------------------------ */

typedef struct {
  double px, py, pz; /* per-qubit X, Y, Z probabilities, p = px+py+pz < 1/2 */
  int32_t scale;     /* fixed-point scale of the energies */
  int32_t W[4];      /* integer energy of one qubit by (x<<1)|z: I, Z, X, Y;
                        W_P = llround(scale * -ln(p_P / (1-p))) */
  int32_t Wt_x, Wt_z;/* matching weights llround(scale * -ln((px+py)/(1-p)))
                        and llround(scale * -ln((pz+py)/(1-p))) */
} xzzx_noise;

/* Fill *out from (px, py, pz).  Each p_P must be > 0 and p < 1/2; scale > 0
 * and small enough that d*d*max(W) fits in int32 for the codes used. */
xzzx_status xzzx_make_noise(double px, double py, double pz, int32_t scale, xzzx_noise* out);

/* Bias helpers.  convention 0: py = p*eta/(eta+1), px = pz = p/(2(eta+1));
 * convention 1 (the paper's px:py:pz = 1:eta:1, Sec. "Simulation setting"):
 * py = p*eta/(eta+2), px = pz = p/(eta+2). */
xzzx_status xzzx_noise_from_eta(double p, double eta, int convention, int32_t scale, xzzx_noise* out);

/* ------------------------------------------------------------------------ */
/* Annealing schedule and acceptance thresholds (Eqs. beta_i, beta_ratio,   */
/* Alg. 3).                                                                 */
/* ------------------------------------------------------------------------ */

typedef struct xzzx_schedule xzzx_schedule;

enum { XZZX_SCHED_LINEAR = 0, XZZX_SCHED_PAPER_LOG = 1 };

/* Build the threshold table of an n_sweeps schedule for the energies of
 * *noise.  Inverse temperatures are in units of the Nishimori value:
 * LINEAR: beta_t = beta0 + (beta1-beta0) t/(n_sweeps-1) (beta0 if n_sweeps=1);
 * PAPER_LOG: beta_t = beta0 (1 + gamma ln(t+1)), gamma = (beta1/beta0-1)/ln N.
 * For every sweep t and every positive energy change dE a generator move can
 * produce, T[t][dE] = min(2^32-1, floor(2^32 exp(-beta_t dE/scale))) in FP64;
 * a move is accepted when dE <= 0 or its uint32 draw u < T.  0 <= n_sweeps,
 * beta0, beta1 >= 0 and finite.  The table is copied to the current device.
 * *out is released with xzzx_free_schedule. */
xzzx_status xzzx_make_schedule(const xzzx_noise* noise, int kind, int n_sweeps, double beta0,
                               double beta1, xzzx_schedule** out);
void xzzx_free_schedule(xzzx_schedule* sched);

/* Copy the host threshold table: *n_classes distinct positive dE values into
 * dE (host, capacity cap_classes) and n_sweeps x n_classes thresholds into T
 * (host, row-major).  Pass NULL arrays to query *n_classes only. */
xzzx_status xzzx_schedule_table(const xzzx_schedule* sched, int* n_classes, int32_t* dE, int cap_classes,
                                uint32_t* T);

/* ------------------------------------------------------------------------ */
/* Hot path.                                                                */
/* ------------------------------------------------------------------------ */

/* Sample code-capacity errors and their syndromes (Sec. "Simulation
 * setting"): qubit q of shot s is X, Y, Z or I as its draw u falls below
 * floor(px 2^32), +floor(py 2^32), +floor(pz 2^32).  errors: device,
 * n_shots x 2w words (may be NULL); syndromes: device, n_shots x sw words.
 * Row k belongs to shot shot0 + k. */
xzzx_status xzzx_sample_errors(const xzzx_code* code, const xzzx_noise* noise, uint64_t seed, uint64_t shot0,
                               int n_shots, uint32_t* errors, uint32_t* syndromes, void* stream);

/* Initial references for every (shot, restart).  randomised is the init mode:
 * 1 = greedy matching with random tie-breaking (Alg. 6), 0 = greedy matching
 * with lexicographic ties (Alg. 5; every restart then gets the same R, as in
 * Alg. 1), 2 = "boundary": every defect joined to the nearer boundary of its
 * decoding graph (Sec. "Effect of initial error configuration").  Greedy
 * matching pairs the defects of each decoding-graph colour in the order
 * (w(u,v), key, u, v), w = min(w_int, w(u,b) + w(v,b)) (Eq.
 * distance_u_v_def_new), key = a Philox draw per pair in mode 1 and 0
 * otherwise, a pair kept when both ends are free; a virtual boundary vertex
 * joins an odd defect set; each kept pair is joined by a canonical shortest
 * path, added modulo two.  syndromes: device, n_shots x sw words.  init:
 * device, n_shots x restarts x 2w words (R_i of restart i).  cbits: device,
 * n_shots x restarts bytes, bit 0 = R_i anticommutes with L_Z, bit 1 = with
 * L_X.  1 <= restarts <= 65535. */
xzzx_status xzzx_greedy_init(const xzzx_code* code, const xzzx_noise* noise, uint64_t seed, uint64_t shot0,
                             int n_shots, int restarts, int randomised, const uint32_t* syndromes, uint32_t* init,
                             uint8_t* cbits, void* stream);

/* Simulated annealing of every chain (Alg. 2 with the Metropolis step of
 * Alg. 3).  Chain (k, i, P), k < n_shots, i < restarts, P in I,X,Y,Z, has
 * index c = (k*restarts + i)*4 + P, starts from init[k][i] * L_P and draws
 * with chain id (shot0+k)*restarts*4 + i*4 + P.  A sweep visits the
 * generators colour by colour; the lowest energy and its configuration are
 * recorded at the start and after every colour phase.  init: device,
 * n_shots x restarts x 2w words.  best_E: device, n_chains int32.  best_cfg:
 * device, n_chains x 2w words, or NULL.  final_E / final_cfg: device, the
 * state after the last sweep, or NULL. */
xzzx_status xzzx_anneal(const xzzx_code* code, const xzzx_schedule* sched, uint64_t seed, uint64_t shot0,
                        int n_shots, int restarts, const uint32_t* init, int32_t* best_E, uint32_t* best_cfg,
                        int32_t* final_E, uint32_t* final_cfg, void* stream);

/* xzzx_anneal with one warp per chain instead of one thread: the lanes take a
 * colour's faces in parallel (rows in shared memory, accepted moves applied
 * with shared atomics), cutting each chain's sequential work up to 32-fold
 * for latency-bound use.  Same arguments, draws and results as xzzx_anneal. */
xzzx_status xzzx_anneal_warp(const xzzx_code* code, const xzzx_schedule* sched, uint64_t seed, uint64_t shot0,
                             int n_shots, int restarts, const uint32_t* init, int32_t* best_E, uint32_t* best_cfg,
                             int32_t* final_E, uint32_t* final_cfg, void* stream);

/* Annealing in the literal forms of Alg. 2 and Alg. 3, for comparison with
 * the colour sweep of xzzx_anneal.  order 0: each sweep visits the
 * generators in stabilizer-index order with the draws of xzzx_anneal;
 * order 1: each sweep makes N_stab attempts on generators drawn uniformly at
 * random (Alg. 3), attempt k of sweep t taking its site draw u and
 * acceptance draw from lanes 2(k&1) and 2(k&1)+1 of Philox(seed; k>>1, t,
 * chain_lo, 4 | chain_hi<<8), the site being floor(u * N_stab / 2^32).
 * emin 0: the minimum is taken at the start and after every colour phase
 * (order 0) or every sweep (order 1); emin 1: after every attempt as well
 * (Alg. 2).  With order 0 and emin 0 the results equal xzzx_anneal.  One
 * chain per thread, rows in shared memory (slower than xzzx_anneal).  Other
 * arguments as xzzx_anneal; XZZX_EINVAL for an order or emin outside {0, 1}. */
xzzx_status xzzx_anneal_variant(const xzzx_code* code, const xzzx_schedule* sched, uint64_t seed, uint64_t shot0,
                                int n_shots, int restarts, int order, int emin, const uint32_t* init,
                                int32_t* best_E, uint32_t* best_cfg, int32_t* final_E, uint32_t* final_cfg,
                                void* stream);

/* Coset relabelling and decision (Alg. 7, Eqs. coset_correspondence,
 * determine_P_from_E): chain (i, P) belongs to coset Q_i P with
 * [L_Q] = [R_i R_1]; E4[P] is the minimum over coset P; cls = argmin with
 * ties in the order I, X, Y, Z; recovery = R_1 L_cls.  best_cfg_out is the
 * configuration of the lowest-index chain reaching E4[cls] inside coset cls
 * (needs chain_cfg).  fail = [C_true recovery] != [I] (needs true_errors).
 * Inputs are the outputs of xzzx_greedy_init and xzzx_anneal (device).
 * Outputs (device): cls n_shots bytes, E4 4 x n_shots int32, recovery
 * n_shots x 2w words; best_cfg_out, fail and the matching inputs may be NULL. */
xzzx_status xzzx_decode_reduce(const xzzx_code* code, int n_shots, int restarts, const uint32_t* init,
                               const uint8_t* cbits, const int32_t* chain_E, const uint32_t* chain_cfg,
                               const uint32_t* true_errors, uint8_t* cls, int32_t* E4, uint32_t* recovery,
                               uint32_t* best_cfg_out, uint8_t* fail, void* stream);

/* Bytes of device workspace xzzx_decode_batch needs for this batch. */
xzzx_status xzzx_decode_workspace_size(const xzzx_code* code, int n_shots, int restarts, int want_best_cfg,
                                       size_t* bytes);

/* The whole decoder (Alg. 7) for n_shots syndromes: greedy_init, anneal and
 * decode_reduce on one stream with intermediates in the caller's workspace
 * (device, at least xzzx_decode_workspace_size bytes, 256-byte aligned).
 * Same layouts and optional outputs as the three calls above. */
xzzx_status xzzx_decode_batch(const xzzx_code* code, const xzzx_noise* noise, const xzzx_schedule* sched,
                              uint64_t seed, uint64_t shot0, int n_shots, int restarts, int randomised,
                              const uint32_t* syndromes, const uint32_t* true_errors, uint8_t* cls, int32_t* E4,
                              uint32_t* recovery, uint32_t* best_cfg_out, uint8_t* fail, void* workspace,
                              size_t workspace_bytes, void* stream);

/* ------------------------------------------------------------------------ */
/* Batches of uneven segments (many distances, noise classes, schedules).   */
/* ------------------------------------------------------------------------ */

/* One homogeneous segment: n_shots syndromes of one code, noise, schedule and
 * restart count.  Its shots are decoded exactly as xzzx_decode_batch(code,
 * noise, sched, seed, shot0, n_shots, restarts, randomised, ...) would decode
 * them alone.  Buffers are device memory owned by the caller and must stay
 * valid for the life of the batch; their contents may change between runs. */
typedef struct {
  const xzzx_code* code;
  const xzzx_noise* noise;
  const xzzx_schedule* sched;
  uint64_t shot0;
  int32_t n_shots, restarts, randomised;
  const uint32_t* syndromes;   /* n_shots x sw words */
  const uint32_t* true_errors; /* n_shots x 2w words, or NULL */
  uint8_t* cls;                /* n_shots */
  int32_t* E4;                 /* 4 x n_shots */
  uint32_t* recovery;          /* n_shots x 2w words */
  uint8_t* fail;               /* n_shots, or NULL (needs true_errors) */
} xzzx_segment;

typedef struct {
  int32_t ctas_per_sm;    /* persistent grid = SMs x this; 0 = the occupancy maximum.  Mode 2: resident
                             CTAs (4 chains each) per SM capped at this by padding each CTA's shared memory */
  int32_t order;          /* chunk queue: 0 = longest chunks first, 1 = segment order */
  int32_t graph_mode;     /* the mode xzzx_batch_run_graph captures: 0, 3 or 4 */
  int32_t chains_per_cta; /* chains per CTA of the annealing launches (chunk size): 128 or 256; 0 = 128 */
  int32_t sweep_unroll;   /* unroll of the annealing kernels' sweep loop: 1 or 2; 0 = 1 */
} xzzx_batch_cfg;

typedef struct {
  int32_t n_segments, n_chunks, n_distances, persistent_grid;
  int32_t launches_batched, launches_plain; /* kernel launches of modes 0 and 1 */
  size_t workspace_bytes;
  double move_attempts;  /* per run */
  int64_t total_shots;
  int32_t chains_per_cta, sweep_unroll;
  int32_t n_classes;     /* distance classes present (d <= 15, 17..21, 23..31): mode 4's launches */
  int32_t warp_ctas_per_sm; /* mode 2: resident CTAs (4 chains each) per SM, fewest over the distances */
} xzzx_batch_info;

typedef struct xzzx_batch xzzx_batch;

/* Plan a batch (Alg. 7 applied to every segment).  Chains are cut into chunks
 * of cfg->chains_per_cta (128 or 256) chains of one segment, one CTA each;
 * the chunk size and the sweep unroll are tuning knobs that never change a
 * result (XZZX_EINVAL for other values).  The batch owns its descriptors and the
 * intermediates of every segment (one device allocation).  seed keys every
 * draw; cfg may be NULL. */
xzzx_status xzzx_batch_create(const xzzx_segment* segs, int n_segs, uint64_t seed, const xzzx_batch_cfg* cfg,
                              xzzx_batch** out);
/* Decode every segment on the stream.  mode 0: one greedy launch (two when
 * the batch has distances both up to 17 and above), one persistent annealing
 * launch whose CTAs pull chunks (longest first) from an atomic counter, one
 * decision launch.  mode 1: the three kernels once per
 * distance (the plain form).  mode 2: as mode 1 with one warp per chain
 * (xzzx_anneal_warp).  mode 3: one greedy launch, then each distance's own
 * annealing kernel on its own stream forked from this one (largest distance
 * first, so the hardware fills one distance's tail with the next one's CTAs),
 * joined back before one decision launch; the batch owns those streams.
 * mode 4: as mode 0, with one persistent launch per distance class (d <= 15,
 * 17..21, 23..31), each with its own chunk queue and the register allocation
 * of its class, concurrently on forked streams.  All modes give identical
 * outputs. */
xzzx_status xzzx_batch_run(xzzx_batch* b, int mode, void* stream);
/* cfg->graph_mode (0, 3 or 4) captured into a CUDA graph on the first call (stream must not be the
 * legacy default stream), replayed on every call. */
xzzx_status xzzx_batch_run_graph(xzzx_batch* b, void* stream);
xzzx_status xzzx_batch_get_info(const xzzx_batch* b, xzzx_batch_info* out);
void xzzx_batch_destroy(xzzx_batch* b);

/* ------------------------------------------------------------------------ */
/* Decode server with continuous batching.                                   */
/* ------------------------------------------------------------------------ */

typedef struct {
  uint64_t seed;            /* keys every draw; request r uses shot index r */
  int32_t restarts;         /* greedy restarts per request (4x chains) */
  int32_t n_sweeps;         /* annealing sweeps */
  int32_t sched_kind;       /* XZZX_SCHED_LINEAR or XZZX_SCHED_PAPER_LOG */
  double beta0, beta1;      /* schedule endpoints (units of the Nishimori beta) */
  int32_t max_batch;        /* requests per dispatched batch (<= 4096) */
  int32_t n_slots;          /* batches in flight at once, one stream each (1..64) */
  int32_t queue_capacity;   /* pending requests before submit returns XZZX_EBUSY */
  size_t hbm_budget_bytes;  /* device memory for all slots, split evenly (0 = 256 MiB) */
  int32_t warp_max_requests;/* a batch of at most this many requests anneals with one warp per
                               chain (lower latency) while the warps of all batches doing so
                               stay within 16 per SM; otherwise one thread per chain, which
                               has the higher throughput (0 = 16, -1 = never) */
  int32_t resident_waves;   /* register budget of all batches in flight, in GPU-fulls of the
                               annealing kernels' resident CTAs (0 = 2).  1: every admitted
                               request is resident at once; 2 or more lets CTAs queue in hardware
                               behind running ones, which keeps the GPU busy between batches
                               under heavy load (light loads form small batches either way) */
} xzzx_serve_cfg;

typedef struct {
  uint64_t req_id;
  int32_t class_id, d, cls;  /* cls: decoded logical class (I=0, X=1, Y=2, Z=3) */
  int32_t E4[4];             /* coset minimum energies */
  uint32_t recovery[62];     /* R_1 L_cls, 2w words (w = ceil(d*d/32)) */
  double latency_us;         /* submit to completion */
} xzzx_result;

typedef struct {
  int64_t submitted, rejected, dispatched, completed, batches, pending, in_flight;
  double mean_batch, p50_us, p99_us, max_us, mean_us;
  uint32_t device_errors;  /* OR of the XZZX_DEVERR_* flags raised by any batch since start */
} xzzx_serve_stats;

typedef struct xzzx_server xzzx_server;

/* Server for single-syndrome requests (the decoder of Alg. 7 per request).
 * Code tables, schedules and a pool of in-flight slots stay on the current
 * device.  A dispatcher thread forms a batch whenever a slot is free, taking
 * pending requests in arrival order (one distance per batch) while they
 * fit the slot's memory and the register budget (resident_waves), decodes it
 * with the batched launches (the batch distance's own annealing kernel), and
 * overlaps batches of different slots on the GPU.
 * Requests that arrive while others run are admitted as slots and budget free
 * up.  A request's result depends only on (seed, request id, class,
 * syndrome), never on the batch it shared.  All host waits are bounded. */
xzzx_status xzzx_serve_create(const xzzx_serve_cfg* cfg, xzzx_server** out);
/* Register a (distance, noise) class before start; its tables stay resident. */
xzzx_status xzzx_serve_add_class(xzzx_server* s, int d, const xzzx_noise* noise, int* class_id);
/* Allocate the slot pool (device + pinned host) and start the dispatcher. */
xzzx_status xzzx_serve_start(xzzx_server* s);
/* Enqueue one request; syndrome_host: sw words of the class's code (host).
 * XZZX_EBUSY when the queue is full (counted as rejected). */
xzzx_status xzzx_serve_submit(xzzx_server* s, uint64_t req_id, int class_id, const uint32_t* syndrome_host);
/* Submit n requests from a server thread at the given arrival offsets (us,
 * ascending, relative to this call); syndromes: n x 32 words (host, copied). */
xzzx_status xzzx_serve_replay(xzzx_server* s, int n, const uint64_t* req_ids, const int32_t* class_ids,
                              const uint32_t* syndromes, const double* arrival_us);
/* Move up to cap finished results to out (host); waits up to timeout_ms for
 * the first one (XZZX_ETIMEOUT if none). */
xzzx_status xzzx_serve_poll(xzzx_server* s, xzzx_result* out, int cap, int* n_out, int timeout_ms);
/* Counters and latency percentiles since start or the last reset. */
xzzx_status xzzx_serve_get_stats(xzzx_server* s, xzzx_serve_stats* out, int reset);
/* Drain pending and in-flight requests, stop, and free everything. */
void xzzx_serve_destroy(xzzx_server* s);

/* Size of the scratch array built into the library for
 * xzzx_decode_batch_static (per GPU, held until the process exits). */
#define XZZX_STATIC_SCRATCH_BYTES ((size_t)16 << 20)

/* The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory while they run, for example a decoder
 * inside a control loop whose GPU memory is fixed at start-up, or a C host
 * that only receives device buffers from another component.  It does what
 * xzzx_decode_batch does, with the same arguments minus the workspace: the
 * intermediates live in a scratch array compiled into the library, so the
 * call performs no allocation (no cudaMalloc, no allocating library call).
 * Returns XZZX_EINVAL when the batch's intermediates
 * (xzzx_decode_workspace_size) exceed XZZX_STATIC_SCRATCH_BYTES; split such
 * batches.  All calls share the one array: calls whose work overlaps on the
 * GPU race on it, so the caller must serialise them.  No scratch byte needs
 * to start at zero (each call writes what it reads).  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress, once
 * per device, that device current); make that first call before any stream
 * capture.  Under lazy module loading (the CUDA default) that first call is
 * also when the array's 16 MiB are committed on the device, so a caller that
 * must not allocate later makes a warm-up call with n_shots = 0 at start-up
 * (it only does this set-up).  The cached address does not survive a
 * cudaDeviceReset of the device; do not call this entry point on a device
 * after resetting it. */
xzzx_status xzzx_decode_batch_static(const xzzx_code* code, const xzzx_noise* noise, const xzzx_schedule* sched,
                                     uint64_t seed, uint64_t shot0, int n_shots, int restarts, int randomised,
                                     const uint32_t* syndromes, const uint32_t* true_errors, uint8_t* cls,
                                     int32_t* E4, uint32_t* recovery, uint32_t* best_cfg_out, uint8_t* fail,
                                     void* stream);

#ifdef __cplusplus
}
#endif

#endif /* XZZX_H */
