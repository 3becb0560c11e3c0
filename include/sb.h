/*
 * sb.h -- C ABI of the GB300 simulated-bifurcation (SB) tracking library.
 *
 * The library solves the triplet QUBO of track reconstruction (Okawa, Zeng,
 * Tao, Yung, arXiv:2402.14718) with ballistic / discrete / adiabatic
 * simulated bifurcation on one GPU, and carries the host-side pieces that
 * feed and score it: a synthetic barrel event generator, the triplet-QUBO
 * builder and track assembly with efficiency / purity.
 *
 * Conventions (every entry point):
 *  - a status code is returned; SB_OK = 0. On failure sb_last_error() gives a
 *    thread-local message. No C++ exception crosses this boundary.
 *  - inputs are copied; the caller keeps ownership of every buffer it passes.
 *  - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *    global memory of the current device (e.g. a torch tensor's data_ptr()).
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *    stream. Calls documented "asynchronous" only enqueue work on `stream`.
 *  - CSR matrices hold both triangles of a symmetric matrix, columns strictly
 *    ascending within a row, no diagonal entry, int32 indices.
 *  - SB state is replica-minor: element (i, r) of an N x R array lives at
 *    [i * R + r].
 *  - A context belongs to the device that was current when it was created;
 *    call it with that device current. A context is not thread-safe: calls on
 *    one context must not overlap; different contexts are independent.
 */
#ifndef SB_H
#define SB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SB_OK = 0,
  SB_ERR_ARG = 1,      /* invalid argument (null pointer, size out of range) */
  SB_ERR_CSR = 2,      /* malformed CSR: unsorted, out of range, diagonal, asymmetric */
  SB_ERR_CUDA = 3,     /* a CUDA runtime call failed; see sb_last_error() */
  SB_ERR_OOM = 4,      /* device or host allocation failed (no C++ exception crosses this API) */
  SB_ERR_TIMEOUT = 5,  /* a bounded device-side wait gave up */
  SB_ERR_STATE = 6,    /* call out of order (e.g. readout before any run) */
  SB_ERR_BOUNDS = 7    /* bounds-checked build: a kernel met an index outside its array */
} sb_status;

typedef enum { SB_ASB = 0, SB_BSB = 1, SB_DSB = 2 } sb_variant;
typedef enum { SB_J_FP32 = 0, SB_J_BF16 = 1 } sb_jprec;

/* Thread-local text of the last error raised on this thread ("" if none). */
const char* sb_last_error(void);

/* Library version string. */
const char* sb_version(void);

/* ======================================================================
 * Host side: synthetic events, triplet QUBO, tracks. No GPU involved.
 * ====================================================================== */

/*
 * Synthetic barrel event; stands in for the TrackML events of section
 * "Dataset" (tt-bar + pile-up, barrel only, 10 layers, 2 T).
 * Tracks: q = +-1, 1/pT ~ U[inv_pt_min, inv_pt_max] GeV^-1, eta ~ U(-eta_max,
 * eta_max), phi0 ~ U[0, 2pi), z0 ~ N(0, z0_sigma); helix in B = bz tesla
 * (Rc[mm] = 1000 pT / (0.3 bz)); one hit per cylinder radius, r*phi and z
 * smeared by N(0, smear_rphi) and N(0, smear_z); floor(noise_frac * n_true +
 * 0.5) uniform noise hits. Random numbers: Philox4x32-10 keyed by the seed.
 * Hits are sorted by (layer, phi in [-pi, pi), generation index).
 */
typedef struct {
  int32_t n_tracks;
  int32_t n_layers;        /* <= 16; radii[0..n_layers-1] ascending, mm */
  double radii[16];
  double noise_frac;
  double bz;               /* tesla */
  double inv_pt_min, inv_pt_max;
  double eta_max;
  double z0_sigma;         /* mm */
  double smear_rphi;       /* mm */
  double smear_z;          /* mm */
} sb_event_params;

/* Fill `p` with the defaults: 100 tracks, 10 layers at 32..1000 mm, 10 % noise,
 * 2 T, 1/pT in [0.1, 1], |eta| < 1, sigma_z0 = 5 mm, 0.1 mm smear. */
void sb_event_params_default(sb_event_params* p);

typedef struct sb_event sb_event;  /* opaque; owns its hit arrays */

/* Generate one event. *out must be released with sb_event_destroy. */
sb_status sb_event_generate(uint64_t seed, const sb_event_params* p, sb_event** out);
int32_t sb_event_num_hits(const sb_event* ev);
int32_t sb_event_num_true(const sb_event* ev);
/* Copy hit arrays (each of sb_event_num_hits entries; any pointer may be NULL).
 * particle = generating track index, -1 for a noise hit. */
sb_status sb_event_hits(const sb_event* ev, int32_t* layer, double* r, double* phi,
                        double* z, double* x, double* y, int32_t* particle);
void sb_event_destroy(sb_event* ev);

/*
 * Triplet QUBO builder: sections "QUBO Formulation" (Eq. 13) and "QUBO
 * Generation and Track Finding" (Eq. 16, 17, pruning).
 *  doublets: consecutive layers, |wrap(dphi)| <= dphi_slope (r_out - r_in) +
 *            dphi_margin / r_in, |z_in - r_in (z_out - z_in)/(r_out - r_in)| <= z0_max;
 *  triplets: doublets sharing the middle hit, |kappa| <= kappa_max (signed
 *            curvature of the circle through the 3 transverse points, mm^-1)
 *            and |theta_bc - theta_ab| <= dtheta_max (Eq. 16);
 *  quadruplets: (a,b,c),(b,c,d) with |kappa_t - kappa_u| <= dkappa_max (Eq. 17);
 *  pruning: with five_hit_rule a quadruplet must have a consistent neighbour
 *            on either side; triplets in no kept quadruplet are dropped;
 *  weights: b = -1 consistent pair, +w_c conflict (shared hit, same or
 *            adjacent start layer, not consistent), else 0;
 *            a_i = w_q * (|kappa_i|/kappa_max + dtheta_i/dtheta_max) / 2.
 *  coupling_mode = 1 (paper Eq. 14, 17): consistent pairs carry b = -S_ij,
 *            S_ij = 1 - (|kappa_i - kappa_j| + max(dtheta_i, dtheta_j)) / 2 (no
 *            holes), and a quadruplet also needs S_ij > s_min.
 *  bias_mode = 1 (paper Eq. 15, decaying-exponential reading): quality_i =
 *            alpha (1 - exp(-|d0|/gamma)) + beta (1 - exp(-|z0|/lambda)), d0 the
 *            closest approach of the triplet's circle to the beam line, z0 the
 *            r = 0 intercept of its a-c line in r-z (mm).
 * Triplets are indexed in lexicographic (hit a, hit b, hit c) order.
 */
typedef struct {
  double dphi_slope, dphi_margin, z0_max;
  double kappa_max, dtheta_max, dkappa_max;
  double w_q, w_c;
  int32_t five_hit_rule;
  int32_t coupling_mode;   /* 0: -1 for consistent pairs; 1: -S_ij (Eq. 14) */
  int32_t bias_mode;       /* 0: curvature/angle quality; 1: Eq. 15 */
  double s_min;            /* Eq. 17 cut on S_ij (0.2) */
  double alpha, beta, gamma, lambda;  /* Eq. 15 (0.5, 0.2, 1.0, 0.5) */
} sb_build_params;

void sb_build_params_default(sb_build_params* p);

typedef struct sb_qubo sb_qubo;  /* opaque; owns its arrays */

sb_status sb_qubo_build(const sb_event* ev, const sb_build_params* p, sb_qubo** out);
sb_status sb_qubo_sizes(const sb_qubo* q, int32_t* n, int64_t* nnz);
/* Copy out (host buffers; any may be NULL): rowptr[n+1], col[nnz], val[nnz]
 * (b_ij), lin[n] (a_i), cls[nnz] (0 consistent, 1 conflict), quality[n],
 * trip[3n] (hit ids a,b,c), kappa[n], dtheta[n]. */
sb_status sb_qubo_arrays(const sb_qubo* q, int32_t* rowptr, int32_t* col, double* val,
                         double* lin, int8_t* cls, double* quality, int32_t* trip,
                         double* kappa, double* dtheta);
void sb_qubo_destroy(sb_qubo* q);

/*
 * sb_qubo_factor -- the shared-hit structure of the builder's conflict
 * couplings (Eq. 13, "any conflict" read as two triplets that share a hit and
 * start on the same or adjacent layers), for sb_set_factor. A triplet holding
 * hit h at position p (0, 1, 2 for a, b, c) starts on layer(h) - p, so two
 * triplets that share h at positions p, p' start |p - p'| layers apart and
 * conflict exactly when |p - p'| <= 1 (unless they are a consistent pair).
 * Outputs (host, caller-allocated): member[3 n] = the triplets' hit ids
 * (row-major, position p at 3 i + p), couple[9] = W[p][p'] = 1 iff
 * |p - p'| <= 1, *w = the conflict weight w_c the QUBO was built with,
 * *n_ids = the event's hit count (ids lie in [0, n_ids)). SB_ERR_ARG on a
 * NULL argument.
 */
sb_status sb_qubo_factor(const sb_qubo* q, int32_t* member, uint8_t* couple, double* w,
                         int32_t* n_ids);

/*
 * sb_qubo_build_device -- the builder above run on the current GPU (hits
 * uploaded from the host event; count / scan / write passes over doublets,
 * triplets, hit incidences and triplet pairs). The result is the same sb_qubo
 * as sb_qubo_build: identical structure (triplets, rows, columns, classes) and
 * identical values except where they pass through atan2 (segment angles) or exp
 * (Eq. 15 bias), whose device results may differ from the host's in the last
 * place. out_device_ms (may be NULL): device time of the build, CUDA events on
 * `stream`. Synchronous.
 */
sb_status sb_qubo_build_device(const sb_event* ev, const sb_build_params* p, sb_qubo** out,
                               double* out_device_ms, void* stream);

/*
 * Track finding and scoring (last paragraph of "QUBO Generation and Track
 * Finding"; Eq. 18-19). T[n] (host, 0/1) selects triplets; their doublets are
 * merged, hits with more than one selected outgoing or incoming doublet lose
 * them all, the rest is chained, candidates with < min_hits hits are dropped.
 * Outputs (host, any may be NULL): n_tracks; track_ptr[n_tracks+1] and
 * track_hits[] (capacity num_hits + 1 and num_hits suffice), tracks ordered by
 * first hit; counts[3] = TP, FP, FN on doublets; eff_pur[2] = efficiency,
 * purity (0 when a denominator is 0).
 */
sb_status sb_tracks(const sb_event* ev, const sb_qubo* q, const uint8_t* T, int32_t min_hits,
                    int32_t* n_tracks, int32_t* track_ptr, int32_t* track_hits,
                    int64_t* counts, double* eff_pur);

/* ======================================================================
 * Device side: the SB solver on one GPU.
 * ====================================================================== */

typedef struct sb_ctx sb_ctx;  /* opaque; owns every device buffer it allocates */

/*
 * sb_create -- QUBO (Eq. 13) -> Ising problem on the device.
 * Host inputs: CSR (rowptr[n+1], col[nnz], qval[nnz] = b_ij) and qlin[n] = a_i.
 * The CSR is validated on the host (SB_ERR_CSR). The arrays are copied to the
 * device, where the conversion runs in FP64 (T = (1+s)/2):
 *   J_ij = -b_ij / 4,  h_i = -(a_i/2 + sum_j b_ij / 4),
 *   offset = sum_i a_i / 2 + sum_{i<j} b_ij / 4,
 *   sigma_J = sqrt(sum_{i!=j} J_ij^2 / (n (n-1))),  c0_auto = 0.5 / (sqrt(n) sigma_J).
 * J is stored as `prec` (FP32 or BF16) for the SB step and b, a stay in FP64
 * for the energies. Synchronous. 1 <= n < 2^31 - 1, 0 <= nnz < 2^31.
 */
sb_status sb_create(int32_t n, int64_t nnz, const int32_t* rowptr, const int32_t* col,
                    const double* qval, const double* qlin, sb_jprec prec, sb_ctx** out);

/*
 * sb_create_batch -- many independent QUBOs (events) in one context, solved
 * together by every later call. Host inputs: n_events, n_per_event[E],
 * nnz_per_event[E] and the per-event CSRs concatenated (each rowptr of length
 * n_e + 1 starting at 0, local column indices), qval and qlin concatenated.
 * Each event keeps its own h, offset, sigma_J and c0. Synchronous.
 */
sb_status sb_create_batch(int32_t n_events, const int32_t* n_per_event,
                          const int64_t* nnz_per_event, const int32_t* rowptr,
                          const int32_t* col, const double* qval, const double* qlin,
                          sb_jprec prec, sb_ctx** out);

/* Release every device buffer of the context (waits for the device first).
 * NULL is accepted. */
void sb_destroy(sb_ctx* ctx);

/* Sizes and FP64 scalars of event `e` (0 for a single QUBO). Any pointer may be NULL. */
sb_status sb_info(const sb_ctx* ctx, int32_t e, int32_t* n, int64_t* nnz, double* offset,
                  double* sigma_j, double* c0_auto);
int32_t sb_num_events(const sb_ctx* ctx);
int32_t sb_total_rows(const sb_ctx* ctx);

/* Row-group tables of the step kernel (SB_OPT_ROWS_PER_WARP), built on the
 * first run that uses them: rows per warp (0: not built) and the number of
 * union entries, each of which reads one neighbour row per step (the step's
 * on-chip gather is union_entries x R x 4 bytes). Either pointer may be NULL. */
sb_status sb_step_info(const sb_ctx* ctx, int32_t* rows_per_warp, int64_t* union_entries);

/*
 * sb_set_factor -- factored form of the coupling product of Eq. 2 / 6 / 10 for
 * QUBOs in which one weight w is shared by whole groups of rows (Eq. 13: every
 * conflict pair carries w_c). Rows (triplets) belong to group blocks (hits)
 * through K slots (positions); with T_{g,s} = sum of x_i over the rows i whose
 * slot s names block g, and the K x K 0/1 slot-coupling pattern W, the
 * product becomes
 *   sum_j J_ij x_j = jf sum_s U_{member[i][s], s} + sum_j Rs_ij x_j,
 *   U_{g,s} = sum_{s'} W[s][s'] T_{g,s'},   jf = -w / 4 (J = -b / 4),
 * where the residual Rs = J - jf M^T W M (M: the row-to-(block, slot)
 * incidence; diagonal included) is formed here, exactly, from the context's
 * J values (so a factored row uses the same couplings as its CSR row, J
 * rounded to the context's precision included). Each step then forms the U rows (one pass over the
 * members of the blocks in use) and, per row, reads its K U rows and its
 * residual row instead of its whole CSR row. A row stays in plain CSR form
 * when its residual is not exactly representable in the context's J
 * precision or when it would read more (its K U rows, its K memberships and
 * its residual against its CSR length). The factor changes only the rounding
 * order of the FP32 coupling sums (for dSB with weights that are multiples of
 * 1/4 every partial sum is exact and the states equal the plain kernels' bit
 * for bit). Used by aSB / bSB when R / 4 is a power of two <= 32 or a
 * multiple of 32, and by dSB with sign bytes when R / 8 is a power of two
 * <= 32 or a multiple of 32 (U rows in BF16 while no U element sums more
 * than 256 members, else in FP32; both exact); other
 * runs use the plain kernels. SB_OPT_FACTOR switches it off.
 * Inputs (host, copied): n_ids (ids lie in [0, n_ids)); k slots, 1 <= k <= 4;
 * member[n k] (block id of row i's slot s at k i + s, -1 for none); couple[k
 * k] (symmetric 0/1); w (finite, non-zero, -w / 4 exact in FP32). In a batched
 * context every block's members must lie in one event (offset the ids per
 * event). n_ids = 0 with member and couple NULL removes the factor.
 * Errors: SB_ERR_ARG on invalid arguments (nothing changes). sb_set_weights
 * removes the factor (its weight and residual belong to the old couplings).
 * Synchronous.
 */
sb_status sb_set_factor(sb_ctx* ctx, int32_t n_ids, int32_t k, const int32_t* member,
                        const uint8_t* couple, double w);

/* Sizes of the factored form: out[7] = {set (0/1), rows in factored form,
 * residual nonzeros, U rows, group blocks in use, their member entries, most
 * members behind one U element}. */
sb_status sb_factor_info(const sb_ctx* ctx, int64_t* out);

/*
 * sb_gather_probe -- a diagnostic of the on-chip bound of the coupling product
 * (no SB arithmetic): the rate at which the GPU reads whole rows of an array
 * at random row indices, as the step reads neighbour rows. array_bytes: size
 * of the array (e.g. the state x, N x R x 4); row_bytes: one row (R x 4 for
 * FP32 positions), a positive multiple of 512; about 64 reads per row (at most
 * 2^23), indices from splitmix64(seed). Each warp reads two rows at a time with
 * 16-byte loads per lane, all SMs fully occupied; the best of `repeats` timed
 * launches (CUDA events on `stream`, after one untimed one) is returned in
 * *out_bytes_per_s (host). Allocates and frees its own device memory;
 * synchronises the stream. SB_ERR_ARG for bad sizes, SB_ERR_OOM / SB_ERR_CUDA.
 */
sb_status sb_gather_probe(int64_t array_bytes, int32_t row_bytes, int32_t repeats, uint64_t seed,
                          double* out_bytes_per_s, void* stream);

/*
 * sb_run -- SB time evolution, section "Simulated Bifurcation":
 *   aSB (Eq. 1-2), bSB (Eq. 5-8, wall at |x| > 1), dSB (Eq. 9-12, sgn(x_j) in
 *   the coupling), symplectic Euler: y += dt (-(a0 - a_k) x [- x^3 for aSB]
 *   + c0 (sum_j J_ij g(x_j) + h_i)); x += dt a0 y; wall (bSB, dSB):
 *   |x| > 1 -> x = sgn(x), y = 0.
 * Initial state: x, y ~ U(-0.01, 0.01) from Philox4x32-10, counter
 * (row within event, replica, 3, event), key = seed.
 * c0 > 0 is used for every event; c0 = 0 selects each event's c0_auto; c0 < 0
 * selects -c0 times each event's c0_auto (a scale relative to the automatic
 * value, per event). a_sched: device FP32 array of `steps`
 * values a_k, or NULL for the linear ramp a_k = a0 k / (steps - 1).
 * Allocates the N x R state on first use (kept for later calls with the same
 * R). 1 <= replicas <= 65535, 0 <= steps. Asynchronous on `stream`.
 */
sb_status sb_run(sb_ctx* ctx, sb_variant variant, double a0, double c0, double dt,
                 int32_t steps, int32_t replicas, uint64_t seed, const float* a_sched,
                 void* stream);

/*
 * sb_advance -- continue the current state for `steps` more steps; a_sched
 * (device, `steps` values) is required. Used for checkpoint / resume.
 * Asynchronous on `stream`.
 */
sb_status sb_advance(sb_ctx* ctx, sb_variant variant, double a0, double c0, double dt,
                     int32_t steps, const float* a_sched, void* stream);

/*
 * sb_set_state / sb_get_state -- copy the N x R FP32 state (x, y) in or out
 * (replica-minor). on_device = 0: host buffers; 1: device buffers. set_state
 * fixes R = replicas (allocating if needed). Synchronous.
 */
sb_status sb_set_state(sb_ctx* ctx, const float* x, const float* y, int32_t replicas,
                       int32_t on_device);
sb_status sb_get_state(const sb_ctx* ctx, float* x, float* y, int32_t on_device);

/*
 * sb_energy -- QUBO energies O(T) of Eq. 13 in FP64 for R spin vectors.
 * spins: host int8 [N x R] (replica-minor, +1 selects the triplet, anything
 * else does not), or NULL to read sgn(x) of the current state (x > 0 -> T = 1).
 * out_E: host double [E x R] (event-major). Synchronous.
 */
sb_status sb_energy(sb_ctx* ctx, const int8_t* spins, int32_t replicas, double* out_E);

/*
 * sb_best -- readout of the current state: FP64 QUBO energy of every replica
 * of every event, arg-min over replicas (ties -> lowest replica index), and the
 * best replica's 0/1 selection. Host outputs, any may be NULL:
 * out_T[N] (all events' rows), out_E[E], out_replica[E]. Synchronous.
 */
sb_status sb_best(sb_ctx* ctx, uint8_t* out_T, double* out_E, int32_t* out_replica);

/*
 * sb_readout_device -- sb_best with device outputs, asynchronous on `stream`:
 * d_E_all[E x R] (may be NULL), d_best_E[E], d_best_r[E], d_T[N] (may be NULL).
 */
sb_status sb_readout_device(sb_ctx* ctx, double* d_E_all, double* d_best_E, int32_t* d_best_r,
                            uint8_t* d_T, void* stream);

/*
 * sb_set_weights -- set the QUBO weights from class tags (section "QUBO
 * Formulation", Eq. 13): b_ij = -1 where cls = 0 (consistent pair) and
 * b_ij = w_c where cls = 1 (conflict); a_i = w_q * quality_i. Host inputs:
 * cls[nnz] (aligned with the CSR given to sb_create, symmetric), quality[n].
 * The Ising conversion is redone on the device and the tags are kept, which
 * lets sb_backward return gradients with respect to w_q and w_c.
 * Single-event contexts only. Synchronous.
 */
sb_status sb_set_weights(sb_ctx* ctx, const int8_t* cls, const double* quality, double w_q,
                         double w_c);

/*
 * sb_backward -- gradient of the mean relaxed Ising energy of a bSB run
 * (section "Simulated Bifurcation", Eq. 5-8, with the field term of sb_run):
 *   L = (1/R) sum_r [ -(1/2) x_S,r^T J x_S,r - h^T x_S,r ],
 * x_S the positions after `steps` bSB steps from the Philox start of `seed`.
 * The run is repeated on the device with (x, y) kept at the start of every
 * `ckpt_every`-step segment; the last segment records, as it runs, the
 * pre-wall momentum, the wall mask and J x, each earlier one is recomputed
 * with that recording, and every segment is then reversed. With
 * ckpt_every >= steps the whole run is recorded once and nothing is
 * recomputed (fastest; memory grows with steps). The wall is treated as the piecewise map it is:
 * where it fires the new position is a constant and no adjoint flows through.
 * c0 (> 0) is an input of the gradient path (no automatic c0 here).
 * Outputs (host, may be NULL): out_loss; out_grads[4] = dL/d dt, dL/d c0,
 * dL/d w_q, dL/d w_c (the last two are NaN unless sb_set_weights was called);
 * d_grad_sched: device FP64 [steps] = dL/d a_k (may be NULL).
 * a_sched: device FP32 [steps] or NULL for the linear ramp. Single-event
 * contexts only. Work memory: 2 (ceil(steps / ckpt_every) - 1) + 3 K + 5
 * state-sized FP32 arrays plus K byte masks, K = min(ckpt_every, steps); it
 * stays with the context for the next call of the same (steps, replicas, K)
 * and is freed by a call of another shape or by sb_destroy.
 * Synchronous; discards the current state.
 */
sb_status sb_backward(sb_ctx* ctx, double a0, double c0, double dt, int32_t steps,
                      int32_t replicas, uint64_t seed, const float* a_sched, int32_t ckpt_every,
                      double* out_loss, double* out_grads, double* d_grad_sched, void* stream);

/*
 * sb_energy_noalloc -- the FP64 readout of sb_energy / sb_readout_device
 * (QUBO energies of R replicas, arg-min over replicas with ties to the lowest
 * index) for callers that cannot allocate device memory. The paper has no
 * counterpart: it is an interface for embedding the solver in host frameworks
 * that own every device allocation themselves (an online trigger or
 * reconstruction framework running under a fixed memory budget, or a
 * latency-bound loop where the implicit device synchronisation of cudaMalloc /
 * cudaFree is not acceptable). It calls no cudaMalloc, cudaFree or allocating
 * library routine, and needs no sb_ctx.
 *
 * Inputs (device pointers, one QUBO): the same CSR and linear terms as
 * sb_create takes (rowptr[n+1], col[nnz], qval[nnz], qlin[n]; not validated
 * here, all four required), and exactly one of x (FP32 [n x R], T_i = 1 iff
 * x > 0) or spins (int8 [n x R], T_i = 1 iff spin > 0), both replica-minor.
 * Outputs (device): E[R] (QUBO energies, FP64); best_E[1] and best_r[1] (both
 * or neither). Asynchronous on `stream`. A NULL required pointer, or sizes
 * beyond the scratch, return SB_ERR_ARG before anything is launched.
 *
 * Scratch: a static device array of 8 MiB inside the library. A call needs
 * 8 * ceil(n / B) * R bytes of it plus a small row table (B = 64 rows when
 * R >= 16, 128 or 256 for fewer replicas): e.g. n <= 261,000 rows at R = 256.
 * Larger problems are rejected with SB_ERR_ARG and a message (use sb_energy or
 * sb_readout_device, which allocate).
 * First call on a device: the array sits in its own code module, which CUDA
 * loads lazily, so the first call in a context loads that module and commits
 * the 8 MiB there (a driver allocation, which can synchronise the device or
 * fail when device memory is exhausted). Make that first call while memory is
 * still available and no stream is being captured. The array's device address
 * is then cached per device and context and looked up again when the calling
 * thread's current context changes (e.g. after cudaDeviceReset); the array
 * stays committed until that context is destroyed.
 * Sharing: every call in a context uses the one array and it keeps the last
 * call's contents (each call writes every scratch entry it reads, so nothing
 * needs clearing); calls that overlap on the GPU (other streams, other
 * threads) race on it and must be serialised by the caller.
 */
sb_status sb_energy_noalloc(int32_t n, const int32_t* rowptr, const int32_t* col,
                            const double* qval, const double* qlin, const float* x,
                            const int8_t* spins, int32_t replicas, double* E, double* best_E,
                            int32_t* best_r, void* stream);

/*
 * sb_set_option -- per-context switches.
 *   SB_OPT_GRAPH (0): 1 (default) replays runs of >= 8 steps from a captured
 *   CUDA graph; 0 launches one kernel per step directly on the stream.
 *   SB_OPT_TILED (1): 1 uses the row-block tiled step kernel (shared-memory
 *   staging of each row block's neighbour union) when R is a multiple of 32;
 *   0 (default) the untiled kernel. Both give bit-identical states (same FMA
 *   order).
 *   SB_OPT_STEP_RT (2): replica-tile width of the untiled kernel (4 x a power
 *   of two, <= 128, dividing R; 0 = automatic).
 *   SB_OPT_STEP_RPC (3): rows per CTA of the untiled kernel (0 = one row per
 *   thread group, -1 = one wave of CTAs over the SMs); a CTA walks a contiguous
 *   row chunk so rows in flight share neighbour rows in L1.
 *   SB_OPT_STEP_UNROLL (4): neighbour rows gathered at once per thread (4).
 *   SB_OPT_DSB_SIGNS (5): 1 (default) lets dSB gather one byte per sign of x
 *   (written by the step that writes x) instead of FP32 positions; taken only
 *   while every |J_ij| < 2^118 (bounded through sigma_J), else positions.
 *   SB_OPT_REPLICA_GROUPS (6): run the replicas as this many groups one after
 *   another, each for all steps (R / groups replicas per group, a multiple of 4
 *   with R / (4 groups) a power of two <= 32), so a group's state stays in L2.
 *   None of these changes results.
 */
#define SB_OPT_GRAPH 0
#define SB_OPT_TILED 1
#define SB_OPT_STEP_RT 2
#define SB_OPT_STEP_RPC 3
#define SB_OPT_STEP_UNROLL 4
#define SB_OPT_DSB_SIGNS 5
#define SB_OPT_REPLICA_GROUPS 6
/* SB_OPT_L2_PERSIST (7): 1 marks each step's source positions as L2-persisting
 * (stream access-policy window; the persisting L2 set-aside of this process's
 * context is raised to the device maximum). 0 (or sb_destroy) returns every
 * persisting line to normal and puts the set-aside back. Does not change
 * results. */
#define SB_OPT_L2_PERSIST 7
/* SB_OPT_STREAM (8): 1 uses the streamed step kernel when R is a multiple of
 * 64: one CTA per SM walks a contiguous chunk of rows in blocks of 32; a
 * producer warp copies each block's union of neighbour x rows (one replica
 * tile of 256, 128 or 64 replicas) into a shared-memory ring with bulk
 * asynchronous copies and eight consumer warps (four rows each) accumulate
 * from it. Same FMA order as the untiled kernel, so the states are identical.
 * Its waits are bounded (SB_OPT_WAIT_NS, 2 s by default): if one gives up,
 * the kernel returns early and the next of sb_best, sb_energy (current state)
 * or sb_get_state returns SB_ERR_TIMEOUT once (the state of that run is not
 * valid; the context stays usable).
 * Applies to every variant (dSB gathers FP32 positions on this path). */
#define SB_OPT_STREAM 8
/* SB_OPT_ROWS_PER_WARP (9): 2 or 4 uses the row-group step kernel when R is a
 * multiple of 128: one warp owns a group of that many rows (grouped on the
 * host, on first use, so that they share neighbours) and walks the sorted
 * union of their columns, loading each neighbour row of x once for all of
 * them. 0 turns it off. -1 (default) chooses: groups of 2 for aSB and bSB
 * unless SB_OPT_TILED or SB_OPT_STEP_RT is set, off for dSB. Same
 * FMA order as the untiled kernel, so the states are identical. With it,
 * SB_OPT_STEP_RPC sets rows per CTA (divided by the group size) and
 * SB_OPT_STEP_RT = 128 makes a warp cover 128 replicas instead of 256. */
#define SB_OPT_ROWS_PER_WARP 9
/* SB_OPT_HEAVY_FIRST (10): 1 dispatches the row-group kernel's CTAs (chunks
 * of consecutive row groups) in order of decreasing cost, so that the CTAs
 * that start last in a step are the light ones; 0 dispatches them in row
 * order, which keeps the neighbour rows of the CTAs in flight together in L2;
 * -1 (default) takes 1 when the gathered array (x, or the dSB sign bytes)
 * fits in half of the L2, else 0. Each group is computed the same way either
 * way: same states. */
#define SB_OPT_HEAVY_FIRST 10
/* SB_OPT_R1_LANES (11): with one replica (R = 1), 8, 16 or 32 lanes share a
 * row: they load its couplings and gather its neighbours' positions in
 * parallel, then form the coupling sum in CSR order as the one-thread kernel
 * does (same states). 0: one thread per row. -1 (default): the widest group
 * for which rows x lanes fit in the SMs' resident threads, else 0. */
#define SB_OPT_R1_LANES 11
/* SB_OPT_WAIT_NS (12): limit, in nanoseconds of the GPU's global timer, of
 * every wait of the streamed step kernel (SB_OPT_STREAM) on its shared-memory
 * pipeline; 2e9 (2 s) by default, accepted in [1e3, 6e10]. */
#define SB_OPT_WAIT_NS 12
/* SB_OPT_TEST_SKIP_STAGE (13): test hook of the time-out path of the streamed
 * step kernel. A stage index s >= 0 makes the producer warp of CTA 0 leave
 * its s-th ring stage unissued (no barrier arrival, no copy started), so the
 * consumer warps' wait for that stage runs out after SB_OPT_WAIT_NS, they
 * record the time-out and return, and the producer drains its copies in
 * flight with a bound and returns. -1 (default) turns it off. Nothing
 * faults or hangs either way: every wait is bounded. */
#define SB_OPT_TEST_SKIP_STAGE 13
/* SB_OPT_FACTOR (14): -1 (default) or 1 runs the factored coupling product
 * whenever sb_set_factor has set one and the run is supported; 0 runs the
 * plain kernels. sb_autotune times both and sets this option. */
#define SB_OPT_FACTOR 14
/* SB_OPT_TEST_BAD_COL (15): test hook of the bounds-checked build only
 * (sb_checked_build() == 1; SB_ERR_ARG in the release build). Value p in
 * [0, nnz) overwrites the context's device copy of CSR column p with n + 7,
 * an index outside the state, so that the next step or energy kernel that
 * reads it records it (sb_check_bounds) and reads row 0 instead. The host
 * copies and the context's other tables are not changed. */
#define SB_OPT_TEST_BAD_COL 15
sb_status sb_set_option(sb_ctx* ctx, int32_t key, int64_t value);

/*
 * sb_autotune -- pick the step-kernel configuration (tiled, untiled or
 * row-group kernel, replica-tile width, rows per CTA) for this context, variant and replica
 * count by timing each candidate for `trial_steps` steps with CUDA events on
 * `stream`, and set it on the context. Results do not depend on the choice.
 * Outputs (host, may be NULL): out_cfg[8] = {tiled, tile width, rows per CTA, unroll,
 * replica groups, L2 persist, rows per warp, factored product (sb_set_factor)},
 * out_us_per_step = the best time. Synchronous; discards the current state.
 */
sb_status sb_autotune(sb_ctx* ctx, sb_variant variant, int32_t replicas, int32_t trial_steps,
                      int32_t* out_cfg, float* out_us_per_step, void* stream);

/*
 * Bounds-checked build -- the device-side stand-in for a memory checker
 * (no counterpart in the paper). The library built with SB_CHECKED=1
 * (libsbtrack_checked.so) tests, in the step kernels (plain, sign-byte,
 * one-replica, row-group, factored: CSR columns, row-pointer pairs, U rows,
 * group members) and the energy kernel, every index it reads before using
 * it. An index outside its array is recorded -- the first one per kernel
 * module -- and replaced by 0, so the access stays inside the array and
 * nothing traps; a row-pointer pair outside [0, nnz] reads as an empty row.
 * Results are then wrong but the device stays usable. Not covered: the
 * tiled and streamed step options, the adjoint kernels and the device QUBO
 * builder. The release build compiles the tests away.
 *
 * sb_checked_build: 1 in the bounds-checked build, 0 in the release build.
 *
 * sb_check_bounds: synchronises the current device, then reads and clears
 * the recorded index of every kernel module. Returns SB_OK with *first = 0
 * when none was recorded (always so in the release build); otherwise
 * SB_ERR_BOUNDS, *first = module << 48 | site << 32 | index (module 1: plain,
 * sign-byte, one-replica and energy kernels; 2: factored kernels; 3:
 * row-group kernel; site 1: CSR column, 2: row-pointer pair (its end), 3: U
 * row, 4: group member, 5: row-group union column; index: the offending
 * value, as 32 bits) for the first module that recorded one, and
 * sb_last_error() names it. SB_ERR_ARG when first is NULL, SB_ERR_CUDA when a
 * copy fails.
 */
int32_t sb_checked_build(void);
sb_status sb_check_bounds(uint64_t* first);

#ifdef __cplusplus
}
#endif
#endif /* SB_H */
