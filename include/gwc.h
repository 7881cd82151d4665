/*
 * gwc.h -- C ABI of the GB300 dark-siren hierarchical likelihood library (libgwc.so).
 *
 * The library evaluates, for a batch of K hyperparameter points Lambda, the
 * hierarchical log-likelihood of a gravitational-wave event catalogue with a galaxy
 * catalogue prior (Papadopoulos et al., "Scalable Dark Siren Cosmology with gwcosmo"):
 *
 *   ln L(Lambda) = sum_i ln L_i(Lambda) - N_det ln xi(Lambda)            (Eqs. 2-4)
 *   ln L_i       = ln( (1/N_i) sum_k w_ik )                              (Eqs. 5-6, kernel width -> 0)
 *   w_ik         = p_LOS(z_ik | pixel_ik) psi(z)/(1+z) / N_z
 *                  * p(m1_s) p(m2_s | m1_s) / [(1+z)^2 d d_L/dz] / pi_PE  (Eq. hier_pixels, Eq. 6)
 *   ln xi        = ln( (1/N_draw) sum_m w~_m )   with the pixel-averaged LOS prior and
 *                  the injections' draw density in place of pi_PE       (Eq. 4, Eq. hier_pixels)
 *   N_eff,i      = (sum_k w_ik)^2 / sum_k w_ik^2                          (Eq. 7, applied per event)
 *
 * z solves d_L = (c/H0)(1+z) int_0^z dz'/E(z'), E = sqrt(Om (1+z)^3 + 1 - Om) (Eq. 1, flat).
 * The mass model is a power law plus a Gaussian peak with a low-mass smoothing window
 * (GWC_MASS_PLP), or the multi-peak model of the paper's simulated catalogue (App. A,
 * Table 2; GWC_MASS_MULTIPEAK): a power law plus two Gaussian peaks, mixed as
 * (1 - lambda_g) P + lambda_g [lambda_low G_low + (1 - lambda_low) G_high], every
 * component normalised on [m_min, m_max], with the same smoothing.  psi is the
 * Madau-Dickinson rate shape with psi(0) = 1.
 *
 * Lambda layout: P doubles per point, in this order, where P = GWC_NUM_PARAMS (13) for
 * GWC_MASS_PLP and GWC_NUM_PARAMS_MULTIPEAK (16) for GWC_MASS_MULTIPEAK (the context's
 * options.mass_model; gwc_get_info reports P):
 *   [H0 (km/s/Mpc), Om, alpha, beta, m_min, m_max, delta_m, mu_g, sigma_g, lambda_peak,
 *    gamma, kappa, z_p]
 * and for the multi-peak model, where (mu_g, sigma_g, lambda_peak) are the low peak's
 * (mu_low, sigma_low) and lambda_g, three more: [..., mu_high, sigma_high, lambda_low].
 * Every [K][P] array below (Lambda points, gradients, HMC states) has this width.
 * Domain: H0 > 0, 0 <= Om <= 1, m_min > 0, m_max > m_min, delta_m >= 0,
 * m_min + delta_m < m_max, sigma_g > 0, 0 <= lambda_peak <= 1, z_p > -1, all finite; the
 * multi-peak model adds sigma_high > 0 and 0 <= lambda_low <= 1.  Its gradient is the
 * interior derivative: at lambda_g or lambda_low equal to 0 or 1 the two components
 * d/d lambda_g and d/d lambda_low are NaN (the other components stay exact).
 * A point outside the domain is not an error: its flags bit 0 is set and its
 * log-likelihood outputs are -inf.
 *
 * Memory: gwc_create copies every host input into device memory owned by the context;
 * the caller may free its inputs on return.  The per-call Lambda and output buffers are
 * caller-owned device memory, read and written asynchronously on the given stream
 * (a cudaStream_t passed as void*, NULL for the legacy default stream).  A context
 * serves one stream at a time.  The per-call path allocates nothing, synchronises
 * nothing and touches no host memory, except gwc_loglik_grad_host, which stages
 * through the context's pinned buffers and synchronises its stream.
 *
 * Errors: every entry point returns a gwc_status; no exception crosses the ABI.
 * gwc_last_error returns the message of the last failure (per context, or
 * thread-local when the context is NULL).
 */
#ifndef GWC_H
#define GWC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GWC_NUM_PARAMS 13              /* Lambda entries, power law + peak */
#define GWC_NUM_PARAMS_MULTIPEAK 16    /* Lambda entries, multi-peak */
#define GWC_MASS_PLP 0
#define GWC_MASS_MULTIPEAK 1

typedef enum {
  GWC_OK = 0,
  GWC_E_INVALID = -1,     /* malformed inputs, sizes or options */
  GWC_E_CUDA = -2,        /* a CUDA call failed; gwc_last_error has its message */
  GWC_E_NOMEM = -3,       /* a device or pinned allocation failed (nothing leaked) */
  GWC_E_TIMEOUT = -4,     /* reserved: the kernels contain no waits */
  GWC_E_UNSUPPORTED = -5  /* no usable CUDA device, or an option this build lacks */
} gwc_status;

/* flags[k] bits */
#define GWC_FLAG_DOMAIN 1       /* Lambda outside its domain */
#define GWC_FLAG_NEFF_EVENT 2   /* some event has N_eff below options.neff_min_event */
#define GWC_FLAG_NEFF_SEL 4     /* N_eff,sel below options.neff_min_sel (when > 0) */
#define GWC_FLAG_XI_ZERO 8      /* every injection weight is zero */
/* any flag makes lnL_total -inf and grad_total zero */

#define GWC_LOS_F32 0
#define GWC_LOS_BF16 1

typedef struct gwc_ctx gwc_ctx;

/* Posterior samples, CSR by event (host memory, structure of arrays).
 * offsets[n_events + 1]: offsets[0] = 0, strictly increasing (every event has at least
 * one sample); sample k of event i is k in [offsets[i], offsets[i+1]).  Detector-frame
 * masses m1_det >= m2_det are expected (pairs with m2_det > m1_det get zero weight),
 * dl_mpc is the luminosity distance in Mpc (d_L <= 0 gets zero weight), ln_pe_prior the
 * natural log of the parameter-estimation prior density in (m1_det, m2_det, d_L), and
 * pix the sample's sky pixel, 0 <= pix < n_pix.  All values finite. */
typedef struct {
  int32_t n_events;
  const int64_t* offsets;
  const float* m1_det;
  const float* m2_det;
  const float* dl_mpc;
  const float* ln_pe_prior;
  const int32_t* pix;
} gwc_events;

/* Line-of-sight redshift priors: row-major [n_pix][n_z] (host memory), row j tabulated at
 * z_j = j z_max / (n_z - 1) and linearly interpolated in between (zero outside
 * [0, z_max]).  dtype GWC_LOS_F32 (float) or GWC_LOS_BF16 (uint16 bfloat16 bits).
 * n_pix >= 1, n_z >= 2, z_max > 0; values finite and >= 0. */
typedef struct {
  int32_t n_pix;
  int32_t n_z;
  double z_max;
  int32_t dtype;
  const void* p_z;
} gwc_los;

/* Detected injections (host memory): n_found >= 1 rows, drawn from a known density
 * whose natural log in (m1_det, m2_det, d_L) is ln_p_draw; n_draw >= n_found is the
 * number of draws made. */
typedef struct {
  int64_t n_found;
  double n_draw;
  const float* m1_det;
  const float* m2_det;
  const float* dl_mpc;
  const float* ln_p_draw;
} gwc_injections;

typedef struct {
  double neff_min_event; /* per-event N_eff threshold (default 2) */
  double neff_min_sel;   /* selection N_eff threshold; 0 = report only (default) */
  int32_t accum;         /* 0: plain FP32 per-lane sums; 1: compensated (Kahan) sums */
  int32_t los_dtype;     /* device storage of the LOS table: GWC_LOS_F32 or GWC_LOS_BF16 */
  int32_t n_x_table;     /* nodes of the per-Lambda z(d_L) inversion table, a multiple of 4
                            in [16, 4096] (default 512) */
  int32_t max_K;         /* largest Lambda batch a call may pass (default 256) */
  int32_t chunk;         /* samples per work item, 64..4096 (default 2048) */
  int32_t lambda_tile;   /* Lambda points per CTA tile, 0..256 (0 = default 256); a tile
                            holds at most 512 / lambda_group points */
  int32_t lambda_group;  /* warps of a CTA sharing one Lambda point: 1, 2, 4, 8 (0 = automatic:
                            1 for a batch of 8 or more points, else the largest power of two
                            <= 8 / K, so that a small batch keeps every warp of a CTA busy) */
  int32_t cap_per_pixel; /* > 0: keep at most this many samples of each (event, pixel), chosen
                            at random as the paper's memory option does (it quotes 2500);
                            0 = keep all (default).  The kept samples of a group are those
                            with the smallest key, the (k+1)-th output of the SplitMix64
                            generator (Steele, Lea and Flood 2014) started at cap_seed for
                            input sample k, so a caller can reproduce the choice; N_i
                            counts the kept samples, and every later output (per-sample
                            terms included) refers to the kept samples only. */
  uint64_t cap_seed;     /* seed of that choice (default 0) */
  int32_t mass_model;    /* GWC_MASS_PLP (default) or GWC_MASS_MULTIPEAK; sets the Lambda width */
} gwc_options;

/* Fill *o with the defaults listed above. */
void gwc_default_options(gwc_options* o);

/* Validate the inputs, copy them to the current CUDA device and build the context.
 * opts may be NULL (defaults).  On success *out owns all device memory. */
gwc_status gwc_create(const gwc_events* events, const gwc_los* los,
                      const gwc_injections* inj, const gwc_options* opts, gwc_ctx** out);

/* Log-likelihood for K Lambda points (1 <= K <= max_K).  Device pointers:
 *   d_lambda[K][P] (in), d_lnL_event[K][n_events], d_neff_event[K][n_events],
 *   d_ln_xi[K], d_neff_sel[K], d_lnL_total[K], d_flags[K] (out).
 * d_lnL_event and d_neff_event may be NULL when n_events == 0. */
gwc_status gwc_loglik(gwc_ctx* ctx, int32_t K, const double* d_lambda, double* d_lnL_event,
                      double* d_neff_event, double* d_ln_xi, double* d_neff_sel,
                      double* d_lnL_total, int32_t* d_flags, void* stream);

/* As gwc_loglik, plus d_grad_total[K][P] = d lnL_total / d Lambda (zero where a flag
 * is set).  Each sample's derivative is recomputed in the same pass as its weight. */
gwc_status gwc_loglik_grad(gwc_ctx* ctx, int32_t K, const double* d_lambda, double* d_lnL_event,
                           double* d_neff_event, double* d_ln_xi, double* d_neff_sel,
                           double* d_lnL_total, int32_t* d_flags, double* d_grad_total,
                           void* stream);

/* The paper's KDE form of the event term (Eqs. 5-7; value only).  For each event and
 * each sky pixel j holding its samples: a Gaussian kernel density estimate in z of the
 * pixel's samples, weighted by w' = p_pop(z, m1, m2 | Lambda) / pi_PE (Eq. 6: the
 * Monte-Carlo weight without its LOS factor), evaluated on n_grid points uniform on
 * [0, z_max], multiplied by the pixel's LOS prior there and integrated by the trapezoid
 * rule; L_i = (1/N_i) sum over the pixels whose N_eff = (sum w')^2 / sum w'^2 (Eq. 7)
 * reaches neff_min_pixel.  The bandwidth of each pixel comes from its samples' z
 * (unweighted), by the appendix's rules: Scott 1.06 sigma n^-1/5 (sample sigma with an
 * n-1 divisor), Silverman 0.9 min(sigma, IQR/1.34) n^-1/5 (quartiles linear between
 * order statistics), biweight 1.06 s_bi n^-1/5 (s_bi^2 the printed biweight
 * midvariance about the median, u = (z - Q)/(9 MAD)); a pixel with fewer than two
 * samples in [0, z_max] or a zero bandwidth is dropped.  Kernels are summed over the
 * grid points within 6 h of each sample, rounded out to aligned blocks of 4 points (the
 * kernel's mass beyond 6 h is 2e-9).  The
 * selection term is the Monte-Carlo sum of gwc_loglik.  Outputs as gwc_loglik, except
 * that d_neff_event[K][n_events] receives the effective number of kept pixels,
 * (sum_j L_ij)^2 / sum_j L_ij^2, and flag bit 1 is never set (no per-event cut); an
 * event with no kept pixel makes the total -inf.  kopt may be NULL (defaults).  The
 * first call (and a call with another n_grid) allocates the form's device buffers:
 * about max_K x (groups + work items) x 92 bytes plus n_pix x n_grid floats (rows rounded
 * up to a multiple of 4).  Needs the
 * LOS table stored as FP32 (GWC_E_UNSUPPORTED otherwise). */
enum { GWC_BW_SCOTT = 0, GWC_BW_SILVERMAN = 1, GWC_BW_BIWEIGHT = 2 };
typedef struct {
  int32_t bw_rule;        /* GWC_BW_* (default Scott) */
  int32_t n_grid;         /* KDE grid points on [0, z_max] (default 256) */
  double neff_min_pixel;  /* per-pixel N_eff threshold (default 2) */
} gwc_kde_options;
void gwc_default_kde_options(gwc_kde_options* o);
gwc_status gwc_loglik_kde(gwc_ctx* ctx, int32_t K, const double* d_lambda,
                          const gwc_kde_options* kopt, double* d_lnL_event, double* d_neff_event,
                          double* d_ln_xi, double* d_neff_sel, double* d_lnL_total,
                          int32_t* d_flags, void* stream);

/* The parts of the likelihood that shards of a catalogue combine (event sharding or
 * batching: one exchange of K (5 + 2P) numbers).  A context built from a subset of the
 * events and a subset of the found injections, with n_draw of the whole injection set,
 * gives for its share: d_lnL_event, d_neff_event, d_ln_xi (ln of its injections' sum
 * over the whole n_draw), d_neff_sel and d_flags as gwc_loglik; d_sum_events[K] = the sum
 * of its events' ln L_i (-inf if one has no weight); and, when both are non-NULL,
 * d_grad_events[K][P] (gradient of that sum) and d_grad_ln_xi[K][P] (gradient of its
 * ln xi).  Shards combine exactly: xi = sum over shards of xi_r, so
 *   ln L = sum_r sum_events_r - N_det ln(sum_r xi_r)
 *   grad = sum_r grad_events_r - N_det sum_r (xi_r / xi) grad_ln_xi_r
 * with N_det the number of events over all shards, and N_eff,sel = (sum xi_r)^2 /
 * sum (xi_r^2 / N_eff,sel,r).  No total is formed here. */
gwc_status gwc_loglik_parts(gwc_ctx* ctx, int32_t K, const double* d_lambda, double* d_lnL_event,
                            double* d_neff_event, double* d_ln_xi, double* d_neff_sel,
                            double* d_sum_events, int32_t* d_flags, double* d_grad_events,
                            double* d_grad_ln_xi, void* stream);

/* Combination of event shards (Eq. 3 with the selection function of Eq. 4 as a
 * Monte-Carlo sum over injections, which splits into the shards' sums): the exchange step
 * of event sharding.  parts[R][K][5 + 2P] (FP64, row-major) holds, for shard r and point
 * k, the outputs of that shard's gwc_loglik_parts: d_sum_events, d_ln_xi, d_neff_sel,
 * d_flags (as a double), the shard's number of events, then (P = 13 or 16) its
 * d_grad_events and d_grad_ln_xi rows; P = 0 leaves the gradients out.  Receives
 * lnL_total[K], ln_xi[K] (of the whole injection set), neff_sel[K], flags[K] and, when
 * P > 0 and grad_total is not NULL, grad_total[K][P], with the formulas of
 * gwc_loglik_parts; flag bits 0 and 1 carry over, bit 3 follows the merged ln xi, bit 2
 * (a shard's own selection cut) is dropped (apply a threshold to the merged neff_sel).
 * on_device = 1: every pointer is device memory and one kernel runs on `stream`
 * (asynchronous, no allocation); on_device = 0: every pointer is host memory and the
 * same FP64 arithmetic runs on the calling thread (no CUDA call; stream is ignored).
 * Shards are combined in index order, so the result does not depend on the device.
 * GWC_E_INVALID for R < 1, K < 1, P not in {0, 13, 16} or a NULL output. */
gwc_status gwc_merge_parts(int32_t R, int32_t K, int32_t P, const double* parts, int32_t on_device,
                           double* lnL_total, double* ln_xi, double* neff_sel, int32_t* flags,
                           double* grad_total, void* stream);

/* The plain single-Lambda path, kept as the speed-up baseline: the same per-sample
 * arithmetic, one Lambda per launch sequence, every sample re-read from memory for each
 * Lambda, per-sample weights (and, for the gradient, per-sample weighted derivatives)
 * written to device memory and reduced in separate passes.  Same outputs as
 * gwc_loglik_grad (d_grad_total may be NULL for the value only).  Power law + peak
 * contexts only (GWC_E_UNSUPPORTED for the multi-peak model). */
gwc_status gwc_loglik_plain(gwc_ctx* ctx, int32_t K, const double* d_lambda,
                            double* d_lnL_event, double* d_neff_event, double* d_ln_xi,
                            double* d_neff_sel, double* d_lnL_total, int32_t* d_flags,
                            double* d_grad_total, void* stream);

/* Host-memory convenience form of gwc_loglik_grad: h_lambda[K][P] in; h_lnL_total[K],
 * h_flags[K] and h_grad_total[K][P] out (h_grad_total may be NULL for the value only).
 * Copies through the context's pinned staging buffers and synchronises the stream. */
gwc_status gwc_loglik_grad_host(gwc_ctx* ctx, int32_t K, const double* h_lambda,
                                double* h_lnL_total, int32_t* h_flags, double* h_grad_total,
                                void* stream);

/* A recorded call.  gwc_graph_create records one gwc_loglik (want_grad = 0) or
 * gwc_loglik_grad (want_grad = 1) call on the given device pointers as a CUDA graph --
 * the prologue, the persistent fused kernel and the merge, three kernel nodes -- and
 * gwc_graph_launch replays it on a stream.  A replay reads the current contents of
 * d_lambda, so a sampler writes its next K points there and replays; the outputs are the
 * same as a direct call's.  The paper has no counterpart: it serves callers that issue
 * many calls of one shape (a sampler's steps), where the launch sequence is recorded
 * once.  The graph uses the context's per-call scratch: replays of graphs of one context
 * must not overlap (one stream at a time), and every graph must be destroyed before its
 * context (a replay after gwc_destroy fails with GWC_E_INVALID).  Profiling events are
 * not recorded inside graphs.  want_grad = 0 ignores d_grad_total. */
typedef struct gwc_graph gwc_graph;
gwc_status gwc_graph_create(gwc_ctx* ctx, int32_t K, const double* d_lambda, int32_t want_grad,
                            double* d_lnL_event, double* d_neff_event, double* d_ln_xi,
                            double* d_neff_sel, double* d_lnL_total, int32_t* d_flags,
                            double* d_grad_total, gwc_graph** out);
gwc_status gwc_graph_launch(gwc_graph* graph, void* stream);
void gwc_graph_destroy(gwc_graph* graph);   /* NULL is a no-op */

/* One Hamiltonian Monte Carlo trajectory for K independent chains, recorded once as a
 * CUDA graph and replayed by gwc_hmc_launch.  The paper samples with nested sampling
 * and has no counterpart; this uses the gradient of gwc_loglik_grad for the leapfrog
 * integrator of HMC (Duane et al. 1987; Neal 2011, "MCMC using Hamiltonian dynamics").
 * With M^-1 = diag(d_inv_mass[P]) and step eps_k = d_eps[k], a replay evaluates lnL and
 * its gradient at q, takes n_leapfrog leapfrog steps
 *     p += eps/2 grad lnL(q);  q += eps M^-1 p;  p += eps/2 grad lnL(q)
 * (n_leapfrog + 1 evaluations, the half kicks between steps merged into full ones), and
 * accepts the end point when log_u_k < H(start) - H(end), H = -lnL + p.M^-1.p / 2.
 * Device arrays, all caller-owned: d_q[K][P] (in: start; out: the accepted end point or
 * the start again), d_p[K][P] (in: initial momenta, drawn by the caller from N(0, M);
 * out: final momenta of the proposal), d_log_u[K] (in: log of uniform(0,1) numbers drawn
 * by the caller), d_lnL[K] and d_grad[K][P] (out: at the returned point), d_accept[K]
 * (out: 1 or 0), d_H[K][2] (out: H at the start and the end).  A chain whose path meets
 * a flagged point (outside the domain, or an N_eff cut) stops moving and is rejected.
 * The graph holds its own evaluation buffers (allocated here) and uses the context's
 * per-call scratch: replays must not overlap other calls on the context, and the object
 * must be destroyed before the context. */
typedef struct gwc_hmc gwc_hmc;
gwc_status gwc_hmc_create(gwc_ctx* ctx, int32_t K, int32_t n_leapfrog, const double* d_eps,
                          const double* d_inv_mass, double* d_q, double* d_p,
                          const double* d_log_u, double* d_lnL, double* d_grad,
                          int32_t* d_accept, double* d_H, gwc_hmc** out);
gwc_status gwc_hmc_launch(gwc_hmc* hmc, void* stream);
void gwc_hmc_destroy(gwc_hmc* hmc);   /* NULL is a no-op */

/* Launch-shape autotuner.  Times whole calls (gwc_loglik_grad when want_grad != 0,
 * gwc_loglik otherwise) on the caller's K points d_lambda[K][P] (device) at every
 * shape of chunk in {1024, 1536, 2048} x Lambda tile in {16, 32, 64, 128, 256} (clamped to K)
 * x warp group in {1, 2, 4, 8} with tile x group <= 512: one untimed call, then two
 * timed with CUDA events on the
 * stream.  The fastest shape becomes the context's chunk, lambda_tile and lambda_group
 * for later calls (a new chunk re-splits the work items; results then differ from the
 * old shape's only by FP32 rounding order).  Synchronises the device, allocates scratch
 * for the trial outputs, and must not overlap other calls on the context.  Fails with
 * GWC_E_INVALID while a graph or HMC object of the context exists (their recorded
 * launches hold the work-item layout).  The paper has no counterpart.  *out (may be NULL) receives the chosen shape, its time per call
 * and the number of shapes timed. */
typedef struct {
  int32_t chunk;
  int32_t lambda_tile;
  int32_t lambda_group;
  int32_t n_tried;
  double ms;
} gwc_tune_result;
gwc_status gwc_autotune(gwc_ctx* ctx, int32_t K, const double* d_lambda, int32_t want_grad,
                        void* stream, gwc_tune_result* out);

/* Release every resource of the context (NULL is a no-op). */
void gwc_destroy(gwc_ctx* ctx);

/* Message of the last failure on ctx, or of the calling thread when ctx is NULL. */
const char* gwc_last_error(const gwc_ctx* ctx);

/* Sizes of a context (for callers and tests). */
typedef struct {
  int32_t n_events;
  int64_t n_samples;
  int64_t n_injections;
  int32_t n_pix;
  int32_t n_z;
  int32_t n_items;       /* work items (sample chunks) the kernels iterate over */
  int32_t chunk;
  int32_t n_x_table;
  int32_t max_K;
  int64_t device_bytes;  /* device memory held by the context */
  int32_t n_params;      /* P: Lambda entries of the context's mass model (13 or 16) */
  int32_t mass_model;
} gwc_info;

gwc_status gwc_get_info(const gwc_ctx* ctx, gwc_info* out);

/* Per-sample terms for one Lambda point (diagnostics and element-wise tests).  For every
 * event sample, in the context's order (events in input order; within an event, samples
 * stably sorted by pixel id, then by dl_mpc), followed by every injection in the
 * context's order (stably sorted by dl_mpc, then each consecutive block of 256 stably
 * sorted by m1_det):
 *   d_lnw[n_samples + n_found]          ln w minus the per-Lambda constant c (-inf where w = 0)
 *   d_dlnw[P][n_samples + n_found]      (optional, may be NULL) d(ln w - c)/d Lambda
 *   d_c[1 + P]                          c and dc/d Lambda, so ln w = d_lnw + c
 *   d_cell[n_samples + n_found]         (optional, may be NULL) the LOS grid cell j whose
 *                                       nodes z_j, z_j+1 the sample's prior is interpolated
 *                                       between (Sec. 2.1's pixelised LOS prior), from the same
 *                                       arithmetic as the likelihood kernels: the floor of the
 *                                       sample's grid position z (n_z - 1) / z_max, clamped to
 *                                       [0, n_z - 2]; -1 where d_L maps outside [0, z_max]
 * d_lambda points to P doubles on the device.  Uses the context's per-call scratch. */
gwc_status gwc_sample_terms(gwc_ctx* ctx, const double* d_lambda, float* d_lnw, float* d_dlnw,
                            double* d_c, int32_t* d_cell, void* stream);

/* Per-sample terms without allocating: the outputs d_lnw, d_dlnw and d_c of
 * gwc_sample_terms, computed from caller-owned device arrays instead of a context.  The paper has no counterpart;
 * this entry point serves callers that cannot allocate device memory when they need an
 * evaluation -- code running while a CUDA graph is being captured (cudaMalloc is not
 * allowed then), code inside a framework whose caching allocator owns the device's
 * memory, or callbacks that must leave the memory state untouched -- and so cannot hold
 * a gwc_ctx.  It calls no cudaMalloc, cudaFree or other allocating routine: its scratch
 * (one Lambda point's constants and tables, the pixel-mean LOS row and its partial sums
 * over 8 slabs of pixels, about 340 KB) is a
 * fixed device array inside the library, held by every GPU that loads the library until
 * the process exits.  It evaluates the power law + peak model (13-entry Lambda).
 *   d_lambda[13]                      Lambda (device, doubles)
 *   d_samples[n_samples][4]           {m1_det, m2_det, d_L, ln pi_PE} (device, 16-byte aligned)
 *   d_pix[n_samples]                  pixel of each sample, in [0, n_pix); the library does
 *                                     not read these on the host, so it cannot reject a bad
 *                                     one up front: a sample whose pixel lies outside the
 *                                     range reads no LOS row and gets w = 0 (d_lnw = -inf,
 *                                     d_dlnw = 0)
 *   d_injections[n_inj][4]            {m1_det, m2_det, d_L, ln p_draw} (device, 16-byte aligned)
 *   d_los[n_pix][n_z]                 LOS priors on z_j = j z_max / (n_z - 1) (device, float)
 *   n_x_table                         inversion-table nodes, a multiple of 4 in [16, 1024]
 *   d_lnw[n_samples + n_inj], d_dlnw[13][n_samples + n_inj] (may be NULL), d_c[14]:
 *                                     as for gwc_sample_terms, samples in the caller's order
 * Sizes beyond the scratch (n_z > 4096, n_x_table > 1024) are rejected with
 * GWC_E_INVALID and a message from gwc_last_error(NULL).  The first call on a device
 * looks up the scratch array's device address and uploads the quadrature constants, so
 * make that first call before any stream capture begins.  Every call shares the one
 * scratch array and overwrites what it reads, so nothing carries over between calls, but
 * calls whose kernels overlap on the GPU (several streams or host threads at once) race on
 * it: serialise them. */
gwc_status gwc_sample_terms_noalloc(const double* d_lambda, int64_t n_samples,
                                    const float* d_samples, const int32_t* d_pix, int64_t n_inj,
                                    const float* d_injections, int32_t n_pix, int32_t n_z,
                                    double z_max, const float* d_los, int32_t n_x_table,
                                    float* d_lnw, float* d_dlnw, double* d_c, void* stream);

/* Per-kernel timing.  While enabled, every call records CUDA events on its stream around
 * its three stages (the prologue kernel, the sample kernel or the plain path's sample
 * passes, and the merge kernel; for gwc_loglik_kde the first stage also holds the
 * injections' Monte-Carlo sum and the second is the KDE kernel alone).  gwc_profile_read
 * waits for the recorded events,
 * returns ms[0..2] = summed stage times in milliseconds and *n_calls = calls recorded
 * since the last read, then resets the sums.  Enabling creates the events (no per-call
 * allocation); disabling destroys them.  Not for use inside stream capture. */
gwc_status gwc_profile_enable(gwc_ctx* ctx, int32_t enable);
gwc_status gwc_profile_read(gwc_ctx* ctx, double* ms, int64_t* n_calls);

/* The library's LOS grid cell index, for tests of bit-exact indexing: for each z (device
 * array of n floats) d_cell receives floor(z * ((n_z - 1) / z_max)) evaluated in double
 * precision and clamped to [0, n_z - 2] (the index the linear interpolation uses, with
 * the -1 marker for z < 0 or z > z_max).  The fused kernels reach the same cells through
 * their split-precision position tables. */
gwc_status gwc_los_cell_index(const float* d_z, int64_t n, int32_t n_z, double z_max,
                              int32_t* d_cell, void* stream);

/* Path census of the likelihood kernels' per-(sample, Lambda) arithmetic (measurement
 * only; the paper has no counterpart).  For the K points d_lambda[K][P] (device) and
 * every event sample and injection of the context, the value arithmetic of the fused
 * kernel is run once and d_counts[GWC_CENSUS_N] (device, uint64, overwritten) receives
 * how many (sample, Lambda) evaluations reached each stage, so that a roofline can
 * charge each evaluation only the work it did:
 *   [0] evaluations at a live (in-domain) Lambda       [1] d_L maps into [0, z_max]
 *   [2] of those, m2_det <= m1_det                     [3] of those, inside the mass support
 *   [4] the whole value computed (LOS prior > 0)       [5] of [4], m1 inside the smoothing window
 *   [6] of [4], m2 inside the smoothing window         [7] weight > 0 (the gradient's share)
 *   [8] of [7], m1 inside the window                   [9] of [7], m2 inside the window
 * Uses the context's per-call scratch and must not overlap other calls on it. */
#define GWC_CENSUS_N 10
gwc_status gwc_path_census(gwc_ctx* ctx, int32_t K, const double* d_lambda, uint64_t* d_counts,
                           void* stream);

/* Path census of the KDE form's kernel (measurement only; the paper has no counterpart):
 * for the K points d_lambda[K][P] (device) and the options kopt (NULL: defaults), runs the
 * KDE kernel of gwc_loglik_kde once and d_counts[GWC_KDE_CENSUS_N] (device, uint64,
 * overwritten) receives
 *   [0] (sample, Lambda) evaluations of the first pass (weights, moments, bandwidth)
 *   [1] (event, pixel group, Lambda) pairs kept (N_eff and bandwidth tests passed)
 *   [2] (sample, Lambda) evaluations of the second pass with a weight
 *   [3] kernel terms summed on the grid (the grid points within 6 h of each of [2])
 * so that a roofline can charge the kernel its work.  Errors as gwc_loglik_kde; uses the
 * context's per-call scratch and must not overlap other calls on it. */
#define GWC_KDE_CENSUS_N 4
gwc_status gwc_kde_census(gwc_ctx* ctx, int32_t K, const double* d_lambda, const gwc_kde_options* kopt,
                          uint64_t* d_counts, void* stream);

/* Throughput probes of the arithmetic units (measurement only; the paper has no
 * counterpart): one kernel of `blocks` CTAs x 256 threads on the stream, each thread
 * running `iters` iterations of 8 independent dependency chains of one operation:
 *   GWC_UNIT_FFMA   FP32 fused multiply-add           GWC_UNIT_FFMA2  packed f32x2 FMA
 *   GWC_UNIT_EX2, GWC_UNIT_LG2, GWC_UNIT_RCP, GWC_UNIT_RSQRT   special-function unit
 *                   approximations (each chain also adds a constant in FP32)
 *   GWC_UNIT_DFMA   FP64 fused multiply-add
 *   GWC_UNIT_DFMA_LANE1  the same with only lane 0 of each warp active
 * *ops (host, may be NULL) receives the operations the launch performs (a packed FMA
 * counts as two; DFMA_LANE1 counts only the active lanes' operations); the caller times
 * the launch, e.g. with CUDA events on the stream. */
enum { GWC_UNIT_FFMA = 0, GWC_UNIT_FFMA2 = 1, GWC_UNIT_EX2 = 2, GWC_UNIT_LG2 = 3,
       GWC_UNIT_RCP = 4, GWC_UNIT_RSQRT = 5, GWC_UNIT_DFMA = 6, GWC_UNIT_DFMA_LANE1 = 7 };
gwc_status gwc_alu_probe(int32_t unit, int32_t blocks, int32_t iters, double* ops, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GWC_H */
