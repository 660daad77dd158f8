/*
 * pcv.h -- C ABI of the GB300 (sm_103a) parallel cross-validation library.
 *
 * The library evaluates the parallel cross-validation loss of Gerber & Nychka,
 * "Parallel cross-validation: a scalable fitting method for Gaussian process
 * models" (arXiv 1912.13132), for batches of covariance-parameter
 * configurations, and kriging predictions at new locations.
 *
 * Model (Sec. 2.1, Eq. 1; exponential covariance of Sec. 3):
 *     y ~ N(0, sigma2 * Sigma(rho) + tau2 * I),   Sigma_ab = exp(-||s_a - s_b|| / rho).
 * The paper names the nugget variance "tau"; this ABI calls it tau2.  Kriging
 * depends only on lambda = tau2 / sigma2 and rho (Eq. 3 and the remark after it).
 *
 * Subsets (Sec. 2.3, Eq. 5-6; Fig. 1): the domain D is cut into disjoint
 * rectangles D_1..D_N ("cores").  Subset i predicts the VALID points of D_i from
 * the TRAIN points of D_i and of its shell of width delta.  The loss of one
 * configuration is Eq. 6:   CV~ = sum_i CV(y~_T^i, y_V^i, zeta),
 * CV(.) being the sum of squared prediction errors (SSPE, Eq. 4).  Algorithm 1
 * (parallel evaluation) maps to one persistent GPU launch over all
 * (subset, configuration) tasks followed by a fixed-order device sum.
 *
 * Readings of points the paper leaves open (fixed by this ABI):
 *   - cores are half-open [x0, x1) x [y0, y1), closed on D's upper edges;
 *   - the shell is the closed L-infinity band: the training window of subset i
 *     is [x0 - delta, x1 + delta] x [y0 - delta, y1 + delta];
 *   - only TRAIN points enter training sets; VALID points are predicted only by
 *     the subset whose core holds them; IGNORE points are never used;
 *   - regular layouts cut [X0, X1] at X0 + ((X1 - X0) * c) / nx, evaluated in
 *     FP64 in that order (c = 1..nx-1), subset index i = cy * nx + cx;
 *   - subsets without validation data are skipped (Sec. 4.3.1): their local SSPE
 *     is 0 and they are not factorised;
 *   - membership lists are in ascending input-index order.
 *
 * Conventions:
 *   - every function returns a pcv_status; no exceptions cross the ABI;
 *     pcv_last_error() gives a message for the calling thread's last failure;
 *   - host buffers belong to the caller; the library copies what it needs and
 *     keeps no caller pointer after a call returns;
 *   - device buffers passed to *_device functions belong to the caller and must
 *     stay valid until the work queued on `stream` has finished;
 *   - `stream` is a cudaStream_t (NULL = legacy default stream);
 *   - one pcv_ctx must not be used by two threads at the same time.
 */
#ifndef PCV_H
#define PCV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pcv_ctx pcv_ctx;
typedef struct pcv_plan pcv_plan;

typedef enum {
    PCV_OK = 0,
    PCV_ERR_ARG = 1,          /* invalid argument (message in pcv_last_error) */
    PCV_ERR_OOM = 2,          /* host or device allocation failed */
    PCV_ERR_CUDA = 3,         /* a CUDA call failed */
    PCV_ERR_TIMEOUT = 4,      /* a bounded device wait ran out */
    PCV_ERR_BUSY = 5,         /* the context is in use */
    PCV_NOT_SPD = 6,          /* a subset matrix was not numerically positive definite */
    PCV_REFINE_FALLBACK = 7,  /* mixed precision: refinement needed the FP64 fallback (warning) */
    PCV_ERR_UNSUPPORTED = 8   /* feature not available in this build / on this device */
} pcv_status;

enum { PCV_ROLE_TRAIN = 0, PCV_ROLE_VALID = 1, PCV_ROLE_IGNORE = 2 };

/* Arithmetic of the hot path.
 *   PCV_PREC_FP64:  every step in FP64 (reference GPU path).
 *   PCV_PREC_MIXED: matrix factorised in a lower precision, solution refined
 *                   against double-float residuals; same results to the stated
 *                   tolerance (1e-6 relative on losses, 1e-5 on predictions), with
 *                   the context's factorisation engine (pcv_options.factor_engine;
 *                   for the CV loss, size buckets with autotuned engines).
 *   The other modes are the mixed path with one operand scheme for the tensor-core
 *   factorisation, for every subset of the call (trailing updates and panels on
 *   tcgen05 with FP32 accumulation):
 *   PCV_PREC_MIXED_TF32:   values rounded to TF32 (11 significant bits), one product;
 *                          refinement converges only for well-conditioned matrices,
 *                          other tasks are recomputed in FP64 (status
 *                          PCV_REFINE_FALLBACK) -- results meet the tolerance either way;
 *   PCV_PREC_MIXED_TF32X3: two TF32 terms (22 bits), three products;
 *   PCV_PREC_MIXED_BF16X3: three BF16 terms (24 bits), six products;
 *   PCV_PREC_MIXED_F16X2:  two FP16 terms (22 bits), three products (the default
 *                          engine's scheme).
 *   pcv_neg2loglik and pcv_gls in mixed precision need the FP16 scheme (or, for
 *   pcv_neg2loglik, the SIMT engine). */
enum {
    PCV_PREC_FP64 = 0,
    PCV_PREC_MIXED = 1,
    PCV_PREC_MIXED_TF32 = 2,
    PCV_PREC_MIXED_TF32X3 = 3,
    PCV_PREC_MIXED_BF16X3 = 4,
    PCV_PREC_MIXED_F16X2 = 5
};

enum { PCV_LAYOUT_RECTS = 0, PCV_LAYOUT_GRID = 1, PCV_LAYOUT_RECURSIVE = 2 };

typedef struct { double x0, x1, y0, y1; } pcv_rect;

/* Subset layout (Sec. 2.3).
 *   kind = PCV_LAYOUT_GRID:  regular nx x ny cores over the domain.
 *   kind = PCV_LAYOUT_RECTS: n_cores explicit cores (caller's array, copied).
 *   kind = PCV_LAYOUT_RECURSIVE: 2^q cores by the recursive division of Sec. 2.4
 *       (0 <= q <= 20): a rectangle is cut in two so that both halves, each together
 *       with its shell, hold similar amounts of data; the cuts alternate, the first
 *       at depth 0 across x (a line parallel to the y-axis), then across y, and so on.
 *       "Amount of data" counts every point, whatever its role, in the child's closed
 *       window of width delta, the shell taken in all of D (with delta = 0 the paper's
 *       512 subsets of its Sec. 4.3.2 hold 9765 or 9766 residuals each: all data, not
 *       only training data, are balanced).  Candidate cuts are the midpoints of
 *       consecutive distinct coordinates of the points inside the parent; the one with
 *       the smallest |count(left) - count(right)| wins, ties going to the smaller
 *       coordinate; a parent with fewer than two distinct coordinates is cut at its
 *       middle.  Cores are numbered depth first, left (lower) child first.
 *   has_domain = 0: the domain is the bounding box of all n points.
 *   delta >= 0: shell width.
 *   shell_cap > 0 (any kind): a subset whose shell holds more than shell_cap TRAIN
 *       points keeps shell_cap of them, drawn at random without replacement
 *       (Sec. 4.3.2 caps shells at 2000); the core's points are always kept.  The
 *       draw is reproducible: every shell point j of subset i gets as key output
 *       number w + 1 of the SplitMix64 generator (Steele, Lea and Flood, 2014) seeded
 *       with cap_seed, w = (i << 40) | j, i.e. mix(cap_seed + (w + 1) * 0x9E3779B97F4A7C15)
 *       with the generator's published output mix, arithmetic modulo 2^64; the
 *       shell_cap smallest keys (ties: smaller j) are kept, in ascending index order. */
typedef struct {
    int32_t kind;
    int32_t nx, ny;
    const pcv_rect* cores;
    int32_t n_cores;
    int32_t has_domain;
    pcv_rect domain;
    double delta;
    int32_t q;           /* PCV_LAYOUT_RECURSIVE: levels, 2^q cores */
    int32_t shell_cap;   /* 0 = no cap */
    uint64_t cap_seed;
} pcv_layout;

/* Tuning knobs; pass NULL for defaults.  Zero fields take defaults. */
typedef struct {
    int32_t struct_size;       /* sizeof(pcv_options) */
    int32_t max_slots;         /* concurrent tasks on the device (default: SM count) */
    double workspace_fraction; /* share of free device memory for workspaces (default 0.5) */
    int32_t refine_max_iter;   /* mixed path: maximum refinement corrections (default 6) */
    double refine_tol;         /* mixed path: stop once the error left after correction i,
                                  estimated as ||d_i|| * ||d_i|| / ||d_i-1||, is at most
                                  tol * ||x|| (max norms; default 2e-8: the local
                                  loss amplifies prediction errors by about
                                  |yhat| / |yhat - y|, so the solution is refined well
                                  past the loss's 1e-6 target); tasks whose
                                  corrections stop shrinking are recomputed in FP64 */
    int32_t factor_engine;     /* mixed path factorisation: 0 = tensor cores with FP32 values
                                  split in two FP16 terms, three products (default; a task
                                  whose values leave FP16 range, which needs tau2 / sigma2
                                  above ~6e4, is recomputed in FP64); 1 = FP32 SIMT;
                                  2 = tensor cores with three BF16 terms, six products
                                  (FP32 range, half again the operand bytes, twice the MMAs);
                                  3 = tensor cores with TF32 values, one product; 4 = two
                                  TF32 terms, three products */
    int32_t tc_stages;         /* tensor engines: depth of the TMA operand ring, 2 to 4 (0 =
                                  each engine's default: 3 for engines 0 and 4, 2 for engine
                                  2, 4 for engine 3); rings above 96 KB leave one CTA per SM */
    double refine_loss_tol;    /* mixed path, loss-aware stopping rule (default 2e-8; < 0
                                  turns it off): a CV-loss or prediction task whose solution
                                  rule (refine_tol) is not met yet, but whose error bound is
                                  within refine_loss_guard times it, also stops once the error
                                  left in its predictions, estimated as g |K d_i| (K the
                                  cross-covariances to the prediction points, d_i the last
                                  correction, g = c / (1 - c) with c the observed
                                  contraction |d_i| / |d_i-1|), changes its local SSPE by at
                                  most this fraction (|dz| <= 2 |yhat - y| |dyhat|) and moves
                                  no prediction by more than ten times this fraction of their
                                  RMS.  The SSPE amplifies prediction errors by about
                                  |yhat| / |yhat - y|, which the rule weighs subset by
                                  subset instead of refining every solution for the worst
                                  case.  Used where a task's prediction points are no more
                                  than its training points (their cost stays below a
                                  residual pass); the local log-likelihood and GLS keep the
                                  solution rule. */
    int32_t bucketing;         /* mixed CV loss with the default engine: 0 (default) = size
                                  buckets, the active subsets grouped by training size, each
                                  group with slots of its own size and the factorisation
                                  engine (tensor cores or FP32 SIMT) that an autotuner found
                                  fastest for it, the groups' persistent launches running
                                  side by side; 1 = one launch over all subsets in slots
                                  sized for the largest, engine factor_engine (also the
                                  behaviour whenever factor_engine is set to a non-default
                                  engine).  The tuner times both engines on a sample of each
                                  size class at the first mixed CV call of a context (that
                                  call synchronises) and caches its choice per process,
                                  keyed by the histogram of training sizes, the lattice flag
                                  and the device's SM count; pcv_buckets describes it. */
    int32_t graph;             /* mixed CV loss: 0 (default) = the second call with a given
                                  batch size (and the same optional outputs and timing
                                  state) captures the call's device work -- the buckets'
                                  launches, the FP64 fallback and the combine -- in a CUDA
                                  graph, which later calls of that shape replay (parameters
                                  and results pass through context buffers by
                                  device-to-device copies on the caller's stream); 1 = every
                                  call launches its kernels directly */
    int32_t alpha_cache;       /* kriging weights kept per context (default 32 configurations,
                                  < 0 = none): pcv_cv_loss (host buffers) and pcv_predict
                                  store the refined weights alpha = (Sigma + lambda I)^-1 y_T
                                  of every subset they solve, keyed by (rho, lambda =
                                  tau2 / sigma2, precision), least recently used replaced
                                  first, in T_off[N] doubles of device memory per
                                  configuration; pcv_predict with a configuration whose
                                  weights are kept for every subset it needs computes the
                                  predictions (Eq. 3) from them without any factorisation */
    double refine_loss_guard;  /* the loss-aware rule applies once the solution rule's error
                                  bound is within this factor of refine_tol (default 1000;
                                  < 0: always) */
    /* Test hooks of the tensor engines' bounded waits (leave 0): test_wait_us > 0 sets
     * their limit (default 2 s); test_withhold_task = t + 1 makes the TMA producer skip
     * the first operand stage of the launch's task t, so that the waits of that CTA run
     * out: the CTA drains the copies and products it issued, stops using the tensor path
     * and hands its tasks to the FP64 fallback (status PCV_REFINE_FALLBACK). */
    int32_t test_wait_us;
    int32_t test_withhold_task;
} pcv_options;

/* ---------------------------------------------------------------- host-only */

/* Build the subset membership of `layout` on the host (no device needed).
 *   xy:   n x 2 row-major point coordinates (FP64), finite.
 *   role: n entries in {PCV_ROLE_TRAIN, PCV_ROLE_VALID, PCV_ROLE_IGNORE}.
 * On success *out owns CSR arrays (see pcv_plan_info).  Errors: PCV_ERR_ARG for
 * n < 0, NULL pointers with n > 0, a bad role, non-finite coordinates, an empty
 * or inverted domain, nx/ny < 1, delta < 0 or non-finite; PCV_ERR_OOM. */
pcv_status pcv_plan_create(const double* xy, const uint8_t* role, int64_t n,
                           const pcv_layout* layout, pcv_plan** out);

/* Read-only views of the membership, valid until pcv_plan_destroy:
 *   subset i trains on T_idx[T_off[i] .. T_off[i+1]) and validates
 *   V_idx[V_off[i] .. V_off[i+1]), indices into the input arrays, ascending.
 * pcv_plan_cores writes the N core rectangles (x0, x1, y0, y1) to the caller's
 * array `cores` of N = *n_subsets entries. */
pcv_status pcv_plan_info(const pcv_plan* plan, int32_t* n_subsets, const int64_t** T_off,
                         const int64_t** T_idx, const int64_t** V_off, const int64_t** V_idx);
pcv_status pcv_plan_cores(const pcv_plan* plan, pcv_rect* cores);
void pcv_plan_destroy(pcv_plan* plan);

/* ------------------------------------------------------------ device context */

/* Create a context on CUDA device `device`: builds the plan (as pcv_plan_create),
 * copies locations, values and membership to device memory, where they stay
 * resident for the context's lifetime.  Work buffers are allocated on first use.
 *   v: n observed values (FP64), finite.
 * Errors: as pcv_plan_create, plus PCV_ERR_CUDA / PCV_ERR_OOM. */
pcv_status pcv_create(const double* xy, const double* v, const uint8_t* role, int64_t n,
                      const pcv_layout* layout, int32_t device, const pcv_options* opts,
                      pcv_ctx** out);

/* Membership of a context (same views as pcv_plan_info). */
pcv_status pcv_subset_info(const pcv_ctx* ctx, int32_t* n_subsets, const int64_t** T_off,
                           const int64_t** T_idx, const int64_t** V_off, const int64_t** V_idx);

/* Parallel-CV loss (Eq. 6) for B parameter configurations; host buffers.
 *   params:          B x 3 row-major (sigma2, rho, tau2).
 *   precision:       PCV_PREC_FP64 or PCV_PREC_MIXED.
 *   sspe:            out, B sums of local SSPEs (Eq. 6), FP64.
 *   sspe_per_subset: out or NULL, B x N local SSPEs z_i (0 for skipped subsets).
 *   yhat_valid:      out or NULL, B x n_valid predictions of the validation points
 *                    in membership order (subset 0's V list, then subset 1's, ...).
 *   n_valid:         out or NULL, number of validation points in all cores.
 *   status:          out or NULL, B per-configuration statuses: PCV_OK,
 *                    PCV_ERR_ARG (sigma2 <= 0, rho <= 0, tau2 < 0 or non-finite;
 *                    sspe = NaN), PCV_NOT_SPD (sspe = NaN), PCV_REFINE_FALLBACK.
 * Synchronises `stream`.  Returns PCV_OK unless the call itself failed. */
pcv_status pcv_cv_loss(pcv_ctx* ctx, const double* params, int32_t B, int32_t precision,
                       double* sspe, double* sspe_per_subset, double* yhat_valid,
                       int64_t* n_valid, int32_t* status, void* stream);

/* Same on device buffers (params, outputs in device memory); asynchronous on
 * `stream`: nothing is copied between host and device.  Any output may be NULL
 * except d_sspe. */
pcv_status pcv_cv_loss_device(pcv_ctx* ctx, const double* d_params, int32_t B,
                              int32_t precision, double* d_sspe, double* d_sspe_per_subset,
                              double* d_yhat_valid, int32_t* d_status, void* stream);

/* Local log-likelihood (Eq. 2) of the training data of every subset the CV loss
 * evaluates (those with validation data; the others contribute 0), a by-product of
 * the same factorisations:
 *   -2 log L_i = k_i log(2 pi) + log det(sigma2 Sigma_i + tau2 I)
 *                + y_T^T (sigma2 Sigma_i + tau2 I)^-1 y_T,
 * total[b] = the fixed-order sum over subsets (host buffers, like pcv_cv_loss;
 * per_subset B x N, may be NULL; status as pcv_cv_loss).  FP64: the log-determinant
 * from the FP64 factor.  Mixed: the quadratic form from the refined solution, the
 * log-determinant from the FP32 factor, so its error is that of the factorisation,
 * not the refinement's, and grows with the conditioning (measured: 2e-6 relative of
 * -2 log L on well-conditioned subsets, 4e-5 at condition ~1e5); mixed precision
 * needs the default tensor engine or the SIMT engine.  Synchronises. */
pcv_status pcv_neg2loglik(pcv_ctx* ctx, const double* params, int32_t B, int32_t precision, double* total,
                          double* per_subset, int32_t* status, void* stream);

/* Kriging predictions (Eq. 3) at m new locations with one configuration.
 * Each location is predicted by the subset whose core contains it (locations
 * outside D are first clamped onto D), from that subset's training data (core
 * and shell).  xy_new: m x 2 host array; yhat: m host outputs.  Synchronises. */
pcv_status pcv_predict(pcv_ctx* ctx, const double* params3, const double* xy_new, int64_t m,
                       int32_t precision, double* yhat, void* stream);

/* Non-stationary prediction with locally best parameters (Sec. 4.4, where each of the
 * paper's subsets is scored by its local RMSPE and the hold-out data are predicted
 * with every subset's best configuration).  Subset i takes the row b of params
 * (B x 3) with the smallest local SSPE sspe_per_subset[b * N + i] (B x N, as
 * pcv_cv_loss returns it; NaN rows never chosen, lowest b on ties); a subset without
 * validation data takes the row with the smallest sum of finite local losses.  Every
 * location is then predicted as by pcv_predict with the row of the subset whose core
 * contains it.  best: N host outputs, the chosen row per subset, or NULL; m may be 0
 * to get the choice alone.  Synchronises. */
pcv_status pcv_predict_local(pcv_ctx* ctx, const double* params, int32_t B, const double* sspe_per_subset,
                             const double* xy_new, int64_t m, int32_t precision, double* yhat, int32_t* best,
                             void* stream);

/* Generalised least squares for a linear mean (Sec. 5): with covariates X the model
 * becomes y ~ N(X beta, sigma2 Sigma + tau2 I) and
 *     beta = (X^T M^-1 X)^-1 X^T M^-1 y,   M = Sigma + lambda I,  lambda = tau2 / sigma2,
 * over the TRAIN points.  Sec. 5 rewrites M^-1 v = (v - H v) / lambda, H v the kriging
 * prediction of v at the observed locations, so M^-1 X comes from prediction
 * operations on the columns of X; here H v at a training point is the prediction from
 * the training data of the subset whose core holds the point (the parallel
 * approximation of H; exact when one subset covers D).  One factorisation per subset
 * serves all p + 1 columns (the covariates and y), each refined and predicted in turn;
 * the p x p system (X^T (X - H X)) beta = X^T (y - H y) is summed in subset order and
 * solved on the host.  X: n x p row-major, host, a row per input point (only TRAIN
 * rows are used), 1 <= p <= 64; params3 = (sigma2, rho, tau2) with tau2 > 0; beta: p
 * host outputs.  Mixed precision needs the default tensor engine.  Synchronises. */
pcv_status pcv_gls(pcv_ctx* ctx, const double* X, int32_t p, const double* params3, int32_t precision,
                   double* beta, void* stream);

/* The size buckets of the context's mixed CV launch as text (one line per bucket:
 * training-size range, subsets, engine, slot size, slots) into buf (NUL-terminated,
 * truncated to cap bytes); empty before the first mixed CV call.  Returns the length of
 * the full description. */
int32_t pcv_buckets(const pcv_ctx* ctx, char* buf, int32_t cap);

/* Use of the kriging-weight cache (pcv_options.alpha_cache): pcv_predict calls served
 * from kept weights (hits) and calls that solved (misses), and the configurations held.
 * Any output may be NULL. */
pcv_status pcv_alpha_cache_stats(const pcv_ctx* ctx, int64_t* hits, int64_t* misses, int32_t* rows_held);

/* Kernel timing for benchmarks.  When enabled, pcv_cv_loss* records CUDA events
 * on the launching stream around the task kernel and around the combine kernel;
 * pcv_kernel_time waits for the most recent call's end events and returns the
 * two durations in milliseconds.  PCV_ERR_ARG if timing is off or nothing ran. */
pcv_status pcv_set_timing(pcv_ctx* ctx, int32_t enable);
pcv_status pcv_kernel_time(pcv_ctx* ctx, double* task_ms, double* combine_ms);

/* Per-phase SM cycles of the mixed task kernel, summed over its CTAs since timing
 * was enabled (or since the last reset), 16 entries: 0 gather + FP32 assembly,
 * 1 tensor-core trailing updates, 2 diagonal-block factorisations and inverses,
 * 3 panel solves (tensor cores, against the diagonal block's inverse), 4 loads and
 * stores of the diagonal blocks and their BF16 planes,
 * 5 SIMT factorisation (FP32 engine), 6 FP32 triangular solves,
 * 7 double-float residuals, 8 prediction + loss, 9 whole tasks; entries 10 and 11
 * count residual passes and finished tasks, 12..14 tasks handed to the FP64
 * fallback because the factorisation broke down, a correction was not finite, or
 * the corrections stopped shrinking (counts, not cycles); others unused.
 * Synchronises the device. */
pcv_status pcv_phase_cycles(pcv_ctx* ctx, uint64_t* out, int32_t reset);

/* Destroy a context and free its device memory (synchronises the device). */
void pcv_destroy(pcv_ctx* ctx);

/* ------------------------------------------------------------------ serving
 *
 * A request loop over several device-resident datasets (contexts) for outer
 * optimisers that submit CV-loss evaluations one configuration at a time (the
 * paper evaluates its grid of configurations sequentially, Sec. 4.4) and for
 * prediction requests.  Continuous batching: every dataset has `lanes` lanes (the
 * caller's context and clones over the same data, each with a worker thread and a
 * stream); an idle lane takes the CV requests queued for its dataset (up to
 * max_batch) as one pcv_cv_loss batch, or all queued predictions with one
 * configuration as one pcv_predict call.  A request arriving while a batch runs
 * starts on an idle lane at once: its persistent launch takes the SMs the running
 * launch leaves free or frees as its last tasks finish, so the two overlap on the
 * device.  Predictions use the kriging weights CV evaluations kept (the lanes share
 * that cache, pcv_options.alpha_cache), so a prediction at a recently evaluated
 * configuration factors nothing.  Admission by device memory: a batch starts only
 * when its lane's work memory fits hbm_budget_bytes; idle lanes' work memory is
 * released (least recently used first) to make room.  Streams get priorities by work
 * per configuration (sum of k^3 over subsets), the smallest dataset highest, so that
 * waiting launches of short jobs are scheduled first.  CV results do not depend on
 * batching or lane (every subset task is computed on its own, lanes are identical,
 * the sums have a fixed order); predictions agree within the precision's tolerance
 * whether they come from kept weights or a fresh solve.  Creation reserves every
 * lane's work memory for batches of max_batch CV requests, budget permitting (a
 * device allocation waits for the kernels already running, so a lane that allocated
 * at its first batch would wait for the other lanes' launches); the size buckets
 * are built then when the process already holds the autotuner's choice for the
 * dataset, else at the lane's first CV batch.
 *
 * The server takes the contexts over: while it exists, no other thread may use
 * them (their clones' device copies of the data are the server's and are freed with
 * it).  Contexts should be created with max_slots set so that their work memory is
 * predictable.  Thread-safe: any thread may submit and wait. */
typedef struct pcv_server pcv_server;

typedef struct {
    int32_t struct_size;      /* sizeof(pcv_server_options) */
    int32_t max_batch;        /* CV requests per batch (default 16) */
    int32_t precision;        /* PCV_PREC_MIXED (default) or PCV_PREC_FP64 */
    double hbm_budget_bytes;  /* work-memory budget over all lanes; 0 = unlimited */
    int32_t lanes;            /* lanes per dataset, 1 to 4 (default 2) */
    int32_t priorities;       /* 0 (default) = stream priorities by work per configuration,
                                 the smallest dataset highest; 1 = all equal */
} pcv_server_options;

pcv_status pcv_server_create(pcv_ctx* const* ctxs, int32_t n_ctx, const pcv_server_options* opts,
                             pcv_server** out);
/* Queue a CV-loss evaluation of one configuration (sigma2, rho, tau2) on dataset
 * `dataset` (index into ctxs); *request_id identifies it. */
pcv_status pcv_server_submit_cv(pcv_server* s, int32_t dataset, const double* params3, int64_t* request_id);
/* Queue a prediction at m locations (m x 2, copied). */
pcv_status pcv_server_submit_predict(pcv_server* s, int32_t dataset, const double* params3,
                                     const double* xy_new, int64_t m, int64_t* request_id);
/* Wait up to timeout_s (<= 0: no limit) for a request and take its results: the
 * CV loss and per-configuration status (CV), or m predictions into yhat (caller's
 * array, may be NULL), and the latency from submission to completion in ms.  The
 * request is forgotten afterwards.  PCV_ERR_TIMEOUT if not done in time. */
pcv_status pcv_server_wait(pcv_server* s, int64_t request_id, double timeout_s, double* sspe,
                           int32_t* status, double* yhat, double* latency_ms);
/* Latency percentiles over all completed requests, CV evaluations per second from
 * the first submission to the last completion, counts of completed requests, batches and evictions. */
pcv_status pcv_server_stats(pcv_server* s, double* p50_ms, double* p99_ms, double* cv_evals_per_s,
                            int64_t* completed, int64_t* batches, int64_t* evictions);
/* Stop the workers (requests still queued are dropped) and free the server; the
 * contexts remain the caller's. */
void pcv_server_destroy(pcv_server* s);

/* ------------------------------------------------- allocation-free variant
 *
 * The paper has no counterpart to this entry point; it exists for callers that
 * cannot call cudaMalloc -- for example a host application that owns all device
 * memory through its own pool and forbids allocations behind its back, or a
 * latency-critical loop in which cudaMalloc/cudaFree (which may synchronise the
 * device) are not acceptable.  It evaluates the same FP64 cross-validation loss
 * as pcv_cv_loss_device with precision PCV_PREC_FP64, without a pcv_ctx and
 * without allocating: all work memory is one static device array of
 * PCV_STATIC_SCRATCH_BYTES bytes inside this library, which every GPU that loads
 * the library holds until the process exits.
 *
 * Inputs (caller's memory; d_ = device, h_ = host):
 *   d_x, d_y, d_v:   the n point coordinates and observed values (FP64);
 *   N:               number of subsets;
 *   h_T_off, d_T_idx: training membership in CSR form (as pcv_plan_info gives it),
 *                    offsets on the host (N + 1 entries), indices on the device
 *                    as int32;
 *   h_V_off:         validation offsets (host, N + 1 entries);
 *   d_Vx, d_Vy, d_Vv: coordinates and values of the validation points in
 *                    membership order (V_off[N] entries each, device);
 *   d_params:        B x 3 (sigma2, rho, tau2), device.
 * Outputs (device): d_sspe (B), d_sspe_per_subset (B x N, or NULL), d_status (B,
 * or NULL), with the meanings of pcv_cv_loss.  Asynchronous on `stream`.
 *
 * Limits: the layout needs 256 + 2 * 8 (N + 1) + 4 N + 12 B N bytes (each region
 * rounded up to 256) plus one matrix slot of 8 * ld^2 + 8 * (4 ld + m_max + 32)
 * bytes, ld = largest training set rounded up to 128, to fit in the scratch array;
 * otherwise PCV_ERR_ARG and nothing runs.  With one slot the largest training
 * set is about 2800 points; smaller sets run more slots (up to one per SM) in
 * parallel.
 *
 * Sharing: every call on a device uses the same array and finds the previous
 * call's contents there; the call resets what must start at zero.  Calls whose
 * work overlaps on the GPU (different streams, or other host threads) race on the
 * array and give wrong results: serialise them.  The first call on each device
 * looks up the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  The host offset
 * arrays are read during the call; the device arrays must stay valid until the
 * queued work has finished. */
#define PCV_STATIC_SCRATCH_BYTES ((size_t)64 << 20)
pcv_status pcv_cv_loss_fp64_static(const double* d_x, const double* d_y, const double* d_v, int32_t N,
                                   const int64_t* h_T_off, const int32_t* d_T_idx, const int64_t* h_V_off,
                                   const double* d_Vx, const double* d_Vy, const double* d_Vv,
                                   const double* d_params, int32_t B, double* d_sspe,
                                   double* d_sspe_per_subset, int32_t* d_status, void* stream);

/* ----------------------------------------------------------------- self-tests
 * The mixed path computes residuals and predictions in double-float arithmetic
 * (pairs of floats).  These evaluate its primitives elementwise so that tests can
 * compare them with FP64 references:  op 0: exp(-a) (a >= 0), 1: sqrt(a),
 * 2: a * b, 3: a + b; each input is first rounded to double-float.
 * pcv_selftest_df runs on the host (host arrays), pcv_selftest_df_device on the
 * device (device arrays, asynchronous on `stream`).  b may be NULL for ops 0, 1. */
pcv_status pcv_selftest_df(int32_t op, const double* a, const double* b, int64_t n, double* out);
pcv_status pcv_selftest_df_device(int32_t op, const double* d_a, const double* d_b, int64_t n,
                                  double* d_out, void* stream);

/* The tensor-core building block of the mixed path's factorisation on its own:
 * C (M x 128, row-major) = A (M x K, row-major) * B (128 x K, row-major)^T with
 * A and B split into three BF16 terms each and six tcgen05 products accumulated
 * in FP32 (TMA-loaded tiles, TMEM accumulators).  K must be a positive multiple
 * of 32.  Host arrays; allocates and frees its own device buffers; synchronous.
 * PCV_ERR_TIMEOUT if one of the kernel's bounded waits ran out. */
pcv_status pcv_selftest_umma(const float* A, int32_t M, const float* B, int32_t K, float* C);

/* The same product with the operand scheme of each tensor engine: scheme 0 = three BF16
 * terms (six products), 1 = two FP16 terms (three products), 2 = TF32 (one product,
 * tcgen05.mma kind::tf32), 3 = two TF32 terms (three products).  Same arguments, limits
 * and errors as pcv_selftest_umma (PCV_ERR_ARG for an unknown scheme). */
pcv_status pcv_selftest_umma_scheme(int32_t scheme, const float* A, int32_t M, const float* B, int32_t K, float* C);

/* Throughput probes for roofline denominators (the paper has no counterpart; they
 * measure the device, not the method).  kind: 0 FP64 fused multiply-add, 1 FP32 fused
 * multiply-add (SIMT pipes, every SM), 2 tcgen05 kind::tf32, 3 kind::f16 with BF16
 * operands, 4 kind::f16 with FP16 operands (dense M = 128, N = 256 MMAs, FP32
 * accumulators in TMEM, one CTA per SM).  Runs on the current device for about
 * `seconds` (0 < seconds <= 60) after a short calibration and writes the achieved
 * rate in TFLOP/s (2 flops per multiply-add) and the timed run's duration (may be
 * NULL).  Allocates and frees a few bytes of device memory; synchronous.
 * PCV_ERR_TIMEOUT if a bounded wait of the tensor probe ran out. */
pcv_status pcv_measure_peak(int32_t kind, double seconds, double* tflops, double* elapsed_s);

/* ----------------------------------------------------------------- utilities */
const char* pcv_status_str(int32_t status);
const char* pcv_last_error(void);
int32_t pcv_version(void);

/* 1 if the context's data took the lattice path, with the spacings; 0 otherwise.
 * The data are a lattice when every point lies on x0 + i hx, y0 + j hy for integers
 * 0 <= i, j < 2^31 (pcv_lattice_detect), and the path is taken when, in addition, the
 * index extent of every subset (training and validation points) fits a table of 2^21
 * entries.  On that path the mixed CV loss takes each covariance from a per-task table
 * indexed by the lattice offsets (|di|, |dj|), computed once per task in FP64 (Eq. 1
 * evaluated at the lattice distances), instead of evaluating the exponential per matrix
 * entry. */
int32_t pcv_lattice(const pcv_ctx* ctx, double* hx, double* hy);

/* Host-only lattice test of n points (xy: n x 2 row-major FP64, read only), the rule
 * pcv_create applies: per axis, h is the smallest gap between distinct values refined
 * over the whole range (span / round(span / gap)), and every value v must satisfy
 * |(v - v_min) / h - round(...)| <= 16 eps (max|v| / h + span / h), a few FP64 ulps
 * of the largest coordinate, so snapping to the lattice moves no point more than the
 * rounding of its coordinates already did.  One distinct value on an axis counts as a
 * lattice of spacing 1.  Returns 1 and writes the origin and spacings (any output
 * pointer may be NULL) if both axes pass; 0 otherwise (also for n <= 0, NULL xy or a
 * non-finite coordinate).  No device work; thread-safe. */
int32_t pcv_lattice_detect(const double* xy, int64_t n, double* x0, double* hx, double* y0, double* hy);

/* Number of kernels of this library launched by the calling thread since the
 * last reset (for launch accounting in benchmarks); reset when reset != 0. */
int64_t pcv_launch_count(int32_t reset);

#ifdef __cplusplus
}
#endif
#endif /* PCV_H */
