/*
 * dlm.h -- C-ABI of the GB300 dual-sweep solver for ridge-regularized
 * matching LPs.
 *
 * The problem (Sec. 3.1, Eq. primal; Sec. 3.3, Eq. dest-capacity):
 *
 *     min_x  sum_ij c_ij x_ij + (gamma/2) sum_ij x_ij^2
 *     s.t.   sum_i a_ij x_ij <= b_j            for every item j,
 *            x_i in C_i                        for every user i,
 *
 * over the eligible edges (i, j) only.  C_i is the simplex
 * {x_i >= 0, sum_j x_ij <= z} (DLM_SIMPLEX_LE), the simplex with equality
 * (DLM_SIMPLEX_EQ), the box [0, z]^n (DLM_BOX), or the box cut by one budget,
 * {0 <= x_ij <= z, sum_j x_ij <= cut} (DLM_BOX_CUT: the paper lists a box-cut
 * projection among its primitives, Table 1, without defining it; this is the
 * reading implemented).  Only the capacities carry
 * dual variables lam >= 0 (Sec. 3.2, Eq. dual).  Each iteration evaluates the
 * dual at a point y (Eq. primal-recovery: x(y) = Proj_C(-(A^T y + c)/gamma);
 * Eq. dual-gradient: grad g(y) = A x(y) - b), then takes a projected
 * accelerated step on lam >= 0 (Sec. 4.4) under a gamma-continuation schedule
 * (Sec. 6; App. B.2).
 *
 * Conventions for every call:
 *  - Every call returns a dlm_status and never aborts; on failure
 *    dlm_last_error() gives a thread-local message.
 *  - "device" pointers are CUDA global-memory addresses of the current device;
 *    "host" pointers are ordinary (preferably pinned) host memory.  Calls
 *    taking a dlm_memspace argument accept either.
 *  - All GPU work of a handle is ordered on the CUDA stream given at creation.
 *    Calls that return host-visible results (dlm_solve, dlm_get_stats,
 *    dlm_calculate's scalar, host-memspace reads) synchronize that stream.
 *  - A handle is not thread-safe; distinct handles are independent.
 *  - Array layouts are plain C order; all sizes are element counts.
 */
#ifndef DLM_H
#define DLM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DLM_OK = 0,
  DLM_ERR_INVALID_ARG = 1, /* bad sizes, pointers, NaN/Inf data, gamma <= 0, ... */
  DLM_ERR_OOM = 2,         /* a device or host allocation failed */
  DLM_ERR_CUDA = 3,        /* a CUDA runtime call failed */
  DLM_ERR_NUMERIC = 4,     /* a NaN/Inf appeared in the iteration */
  DLM_ERR_TIMEOUT = 5,     /* an iteration limit was reached before the target, or a bounded
                              device-side wait ran out */
  DLM_ERR_UNSUPPORTED = 6  /* valid input outside what this build handles */
} dlm_status;

typedef enum { DLM_F32 = 0, DLM_BF16 = 1 } dlm_dtype;
typedef enum { DLM_SIMPLEX_LE = 0, DLM_SIMPLEX_EQ = 1, DLM_BOX = 2, DLM_BOX_CUT = 3 } dlm_simple_kind;
typedef enum { DLM_MEM_DEVICE = 0, DLM_MEM_HOST = 1 } dlm_memspace;

/* The instance, as user-major CSR (the paper stores the same data as CSC with
 * one column per source, Sec. 4.1; one column per user is one CSR row here).
 *   row_ptr  int64 [num_users + 1], row_ptr[0] = 0, non-decreasing,
 *            row_ptr[num_users] = nnz
 *   item_idx int32 [nnz], 0 <= item_idx < num_items: the eligible items of
 *            each user, distinct within a row (the eligible set E of
 *            Sec. 3.3 is a set of (user, item) pairs; a repeated item in one
 *            row is rejected)
 *   c        [nnz] float32 (val_dtype DLM_F32) or bfloat16 bit patterns
 *            (DLM_BF16, stored as uint16); all finite
 *   a        [nnz x num_families], edge-major (a[e * m + k] is edge e's
 *            coefficient in capacity family k), same type; all finite
 *   b        float64 [num_families x num_items], family-major, finite, >= 0
 * With m = num_families > 1 (Def. 1: several coupling families, each with one
 * diagonal block per user; at most 4) every dual vector of the handle is
 * [m x num_items] family-major (lam[k * num_items + j]); such handles sweep
 * with a general kernel, take the static slice orders (mapping 1 or 2), and
 * do not combine with the count constraint or the warm start; they batch only
 * with handles of the same m.
 * The arrays live in `memspace`.  dlm_create copies them into its own layout;
 * the caller may free or reuse them once dlm_create has returned. */
struct dlm_shard;

typedef struct {
  int64_t num_users, num_items, nnz;
  const int64_t* row_ptr;
  const int32_t* item_idx;
  const void* c;
  const void* a;
  const double* b;
  int32_t val_dtype;    /* dlm_dtype */
  int32_t kind;         /* dlm_simple_kind */
  double z;             /* simplex radius or box bound, > 0 */
  int32_t memspace;     /* dlm_memspace of the arrays above */
  int32_t num_families; /* capacity families m, 1..4 (0 means 1) */
  double cut;           /* DLM_BOX_CUT: per-user budget sum_j x_ij <= cut, finite and > 0 (ignored
                           otherwise); such handles take one family and no count constraint, batch
                           only with other box-cut handles, and sweep with their own kernel */
  const struct dlm_shard* shard; /* NULL, or: these rows are one shard of a user-sharded instance
                                    (see "User-sharded instances" below) */
} dlm_problem_desc;

/* Solver options (zero-initialised fields take the defaults).  The mapping
 * fields change only how the sweep is laid onto the GPU: every mapping gives
 * the same item sums (they are exact), and mappings with the same coop_max
 * and short_rows give bit-identical iterates. */
typedef struct {
  int32_t gap_every;     /* iterations between certified-gap checks in dlm_solve (default 50) */
  int32_t precondition;  /* 1: row normalization (App. B.2) as the per-item step gamma/sum_i a_ij^2 */
  int32_t mapping;       /* slice-to-CTA assignment: 0 default (1 for a handle, 3 for a batch),
                            1 interleaved (CTA k sweeps slices k, k + grid, ... of every instance),
                            2 contiguous (equal-work ranges of the instances' slices in order),
                            3 dynamic (CTAs take work units -- slice ranges of one instance,
                              shrinking toward the end -- from a device counter; certificate
                              sweeps then use order 1 for a handle, 2 for a batch) */
  int32_t graph_iters;   /* iterations per captured CUDA graph (default 10) */
  int32_t ctas_per_sm;   /* persistent sweep CTAs per SM, 0..4 (0: 1 at 1024 threads, 2 at 512) */
  int32_t coop_max;      /* 0..33: rows whose simplex active set has four or more edges (the
                            threshold iteration) are handled one after another by all 32 lanes
                            of the warp while fewer than coop_max of its 32 rows need it
                            (default 12; 1 never, 33 always) */
  int32_t block_threads; /* threads per sweep CTA: 0 (default 1024), 512 or 1024 */
  int32_t restart;       /* 1: adaptive momentum restart besides the stage restarts -- theta = 1
                            after a step whose direction opposes the momentum in the step metric,
                            sum_j (lam+_j - y_j)(lam+_j - lam_j) / step_j < 0 (O'Donoghue &
                            Candes 2015); 0 (default): the paper's schedule-only restarts */
  int32_t topk;          /* one-family sweeps: largest values of a row tracked in the first pass, with
                            the positions of all but the last: 0 or 4 (default), or 8 -- rows with up
                            to seven active edges then take their threshold without the iteration
                            over the row (more work per edge, fewer re-reads of the row) */
  int32_t short_rows;    /* 1: iteration sweeps of a single one-family handle without a count
                            constraint (not box-cut) take the short-row kernel: each row of at most
                            32 edges is held in registers and sorted to find its threshold in one
                            scan, wider rows are read again for every pass of the threshold
                            iteration -- for instances whose rows are short and have many active
                            edges near the optimum; 0 (default): the general sweep.  Certificate
                            sweeps are unchanged; other handles ignore it. */
  int32_t reserved[1];
} dlm_options;

/* Result of a certified-gap evaluation at the current iterate lam (one extra
 * sweep at lam; App. B.1-style objective tracking):
 *   dual_obj    g(lam)
 *   primal_obj  P(x~), x~_ij = s_j x_ij(lam), s_j = min(1, b_j / (A x(lam))_j)
 *               (feasible for simplex-<= and box sets when a, b >= 0)
 *   rel_gap     (primal_obj - dual_obj) / max(|dual_obj|, 1e-30) (>= 0)
 *   uncert_gap  -lam^T (A x(lam) - b) / max(|dual_obj|, 1e-30)
 *   max_viol    max_j (A x(lam) - b)_j^+
 * For DLM_SIMPLEX_EQ or negative a the scaled point is not certified and
 * rel_gap is NaN. */
typedef struct {
  int64_t iter;   /* iterations taken so far */
  double gamma;   /* ridge of the current stage */
  double dual_obj, primal_obj, rel_gap, uncert_gap, max_viol;
  double seconds; /* wall time of the last dlm_solve */
  int32_t status; /* dlm_status of the device-side checks */
  int32_t converged;
} dlm_stats;

/* Iteration state for checkpoint / resume (besides the lam and y vectors). */
typedef struct {
  int64_t iter;  /* global iteration counter t */
  double theta;  /* accelerated-momentum scalar */
  int32_t stage; /* continuation stage index */
  int32_t reserved;
} dlm_state;

typedef struct dlm_problem dlm_problem;
typedef struct dlm_batch dlm_batch;

/* Create a solver handle for one instance (Sec. 3.3 matching LP).  Validates
 * the input (returns DLM_ERR_INVALID_ARG with a message on non-monotone
 * row_ptr, out-of-range items, an item repeated within a row, non-finite
 * values, b < 0, z <= 0), buckets
 * users by degree and lays the edges out for the sweep kernels.  `stream` is
 * a cudaStream_t; with NULL the handle creates its own blocking stream,
 * which is ordered with the legacy default stream in both directions.  Initial state: lam = 0,
 * fixed gamma = 1e-2, no preconditioning.  Synchronous.
 * Item limit: every sweep CTA holds the dual and the gradient sums of all
 * items in shared memory (12 bytes per item, about 19,000 items on a GPU with
 * 227 KB per block; with m > 1, (12 m + 16) bytes per item); certificate
 * sweeps of larger instances take one launch per window of items.  Beyond
 * the limit: DLM_ERR_UNSUPPORTED. */
dlm_status dlm_create(const dlm_problem_desc* desc, void* stream, dlm_problem** out);

/* gamma schedule (Sec. 6, App. B.2 "regularization decay"): iteration t is in
 * stage s = t / iters_per_stage; gamma_0 = gamma0 and
 * gamma_{s+1} = max(gamma_end, gamma_s * factor).  When gamma changes at a
 * stage boundary the momentum restarts (theta = 1, y = lam), lam is kept as the
 * warm start, and the step 1/L, L = max_j sum_i a_ij^2 / gamma, follows gamma.
 * gamma0 == gamma_end gives a fixed ridge.  Requires gamma_end > 0,
 * gamma0 >= gamma_end, 0 < factor <= 1 (factor == 1 only with
 * gamma0 == gamma_end), iters_per_stage >= 1; DLM_ERR_INVALID_ARG otherwise.
 * The stages down to gamma_end are tabulated; a schedule that needs more than
 * 2^20 stages to reach gamma_end returns DLM_ERR_UNSUPPORTED.  Resets the
 * iteration counter and momentum (lam is kept). */
dlm_status dlm_set_schedule(dlm_problem* p, double gamma0, double gamma_end, double factor,
                            int64_t iters_per_stage);

/* Global count constraint sum_{(i,j)} x_ij <= M (Sec. 5 names it as the
 * example of a new coupling constraint: one more dual coordinate mu >= 0,
 * added to every edge's cost, one more gradient entry sum x - M).  M >= 0;
 * INFINITY removes it.  While it is set, every dual vector of this handle --
 * dlm_set_lambda, dlm_get_lambda, dlm_calculate's lambda and grad,
 * dlm_get_state / dlm_set_state, dlm_ws_features' lam_prev -- has
 * num_items + 1 entries, the last being mu.  The steps use Gershgorin bounds of
 * A A^T with the count row: item j's curvature n_j + |s_j| (s_j = sum_i a_ij),
 * the count row's nnz + sum_j |s_j|; with row normalization each coordinate
 * takes gamma over its bound, otherwise all take gamma over the largest (slow
 * with a count row: use row normalization).  The certificate multiplies the
 * item-scaled point by min(1, M / sum x).  Sets mu to 0; call it before
 * iterating and before dlm_batch_create.  Meaningful for DLM_SIMPLEX_LE and
 * DLM_BOX (with DLM_SIMPLEX_EQ, sum x = z per user whatever mu); handles with
 * several capacity families or DLM_BOX_CUT return DLM_ERR_UNSUPPORTED. */
dlm_status dlm_set_count_limit(dlm_problem* p, double M);

/* Replace the handle's options (see dlm_options; out-of-range values return
 * DLM_ERR_INVALID_ARG).  Synchronizes the handle's stream when the launch
 * shape changes. */
dlm_status dlm_set_options(dlm_problem* p, const dlm_options* opt);
dlm_status dlm_get_options(dlm_problem* p, dlm_options* opt);

/* Mapping tuner (the paper has no counterpart; its kernels have one fixed
 * mapping).  Times `iters` iterations (after one warm-up iteration) of every
 * candidate mapping -- block_threads {1024, 512}, mapping {1, 2, 3},
 * coop_max {1, 6, 12, 20, 33}, then topk {4, 8} with the best of those (one
 * family, not DLM_BOX_CUT) -- from the handle's current state, restores
 * that state (lam, y, theta, counter) after each trial, and keeps the mapping
 * whose sweeps took the least device time.  Writes it to *chosen and the mean
 * sweep time of the winner in milliseconds to *sweep_ms (either may be NULL).
 * Allocates two num_items float arrays while it runs.  Synchronous. */
dlm_status dlm_autotune(dlm_problem* p, int32_t iters, dlm_options* chosen, double* sweep_ms);

/* Warm start: lam <- max(lambda0, 0), y <- lam, theta <- 1, iteration counter
 * kept.  lambda0 has num_items float32 entries in `memspace`.  The handle
 * keeps its iterate lam, y in FP64 (the sweeps read FP32 copies of it). */
dlm_status dlm_set_lambda(dlm_problem* p, const float* lambda0, int32_t memspace);

/* One dual evaluation (the paper's ObjectiveFunction.calculate, Table 1):
 * at lambda (device, num_items float32, >= 0 expected) and ridge gamma,
 * writes g(lambda) to *g (host double), grad g(lambda) = A x - b to grad
 * (device, num_items float32; may be NULL) and x(lambda) in the caller's
 * CSR edge order to x (device, nnz float32; may be NULL).  Synchronous. */
dlm_status dlm_calculate(dlm_problem* p, const float* lambda, double gamma, double* g, float* grad, float* x);

/* Run n_iters iterations (asynchronous on the handle's stream; replays
 * captured CUDA graphs). */
dlm_status dlm_step(dlm_problem* p, int64_t n_iters);

/* Iterate until the certified relative gap at lam is <= target_rel_gap while
 * gamma is at its final value, checking every gap_every iterations, or until
 * max_iters iterations in total (then DLM_ERR_TIMEOUT).  Fills *out (may be
 * NULL), including the wall time.  Synchronous. */
dlm_status dlm_solve(dlm_problem* p, double target_rel_gap, int64_t max_iters, dlm_stats* out);

/* Certified-gap evaluation at the current lam (one sweep; see dlm_stats). */
dlm_status dlm_get_stats(dlm_problem* p, dlm_stats* out);

/* Current lam (num_items float32: the FP32 copy of the FP64 iterate) into
 * `memspace`. */
dlm_status dlm_get_lambda(dlm_problem* p, float* out, int32_t memspace);

/* x(lam) for the current lam and gamma, in the caller's CSR edge order
 * (nnz float32) into `memspace`. */
dlm_status dlm_get_x(dlm_problem* p, float* out, int32_t memspace);

/* Checkpoint / resume: the FP64 iterate lam and momentum point y (num_items
 * float64 each, `memspace`) and the scalar state.  dlm_set_state restores
 * exactly the trajectory that dlm_get_state saved (same schedule and options
 * assumed). */
dlm_status dlm_get_state(dlm_problem* p, double* lam, double* y, dlm_state* s, int32_t memspace);
dlm_status dlm_set_state(dlm_problem* p, const double* lam, const double* y, const dlm_state* s, int32_t memspace);

/* Dual objective along the iteration (App. B.1 tracks it per iteration; the
 * paper's ObjectiveFunction.calculate returns it with the gradient, Table 1):
 * every iteration t records g(y_t) = sum_i (c x_i + gamma/2 ||x_i||^2) +
 * y_t^T (A x - b) at the point its sweep evaluated (x = x(y_t), gamma of
 * iteration t), from the sweep's exact fixed-point objective sum and an FP64
 * dot product.  Copies g(y_t) for t = first_iter .. first_iter + n - 1 to the
 * host array g_out.  The handle keeps the last 4096 iterations since the last
 * dlm_set_schedule / dlm_set_state; other ranges return DLM_ERR_INVALID_ARG.
 * Synchronous. */
dlm_status dlm_get_trajectory(dlm_problem* p, int64_t first_iter, int64_t n, double* g_out);

/* Run n_iters iterations as individual kernel launches with a CUDA event
 * recorded on the handle's stream between consecutive kernels, and return the
 * summed device time of the sweep kernels (*sweep_ms), of the update kernels
 * (*update_ms) and of the whole sequence (*total_ms) (each may be NULL).
 * Same arithmetic as dlm_step; used to measure kernel durations.
 * Synchronous. */
dlm_status dlm_step_timed(dlm_problem* p, int64_t n_iters, double* sweep_ms, double* update_ms, double* total_ms);

/* Sizes of the handle's instance and the bytes per iteration the sweep must
 * read (the algorithmic traffic: item index + c + a per edge, plus the row
 * pointer per user). */
dlm_status dlm_get_info(dlm_problem* p, int64_t* num_users, int64_t* num_items, int64_t* nnz,
                        int64_t* bytes_per_iter);

/* Wall-clock seconds dlm_create spent, by phase: out[0] host inputs copied
 * to the device (0 for device inputs), out[1] validation (row pointers,
 * items, values, distinct items per row, capacities), out[2] degree sort of
 * the users and slice sizes, out[3] slice layout and per-item sums, out[4]
 * the handle's own arrays, tables and schedule, out[5] the whole call.  The
 * first min(n, 6) entries are written (host array). */
dlm_status dlm_get_setup_seconds(dlm_problem* p, double* out, int32_t n);

/* Free the handle and its device memory.  The instance's large arrays (the
 * sliced layout, set-up scratch) come from a stream-ordered memory pool per
 * device that keeps freed memory for later handles, so that re-creating an
 * instance of similar size (the paper's recurring daily solves, Sec. 1) maps
 * no new device memory; dlm_release_cached_memory returns that memory to
 * the device. */
void dlm_destroy(dlm_problem* p);

/* Return the memory the library's pools keep after dlm_destroy (every device
 * the library has used) to the device.  Call it with no handle being created
 * or destroyed on another thread. */
dlm_status dlm_release_cached_memory(void);

/* Batches (the paper's experiments solve many independent instances; this
 * sweeps them together).  A batch runs n existing handles as one: each
 * iteration is one sweep launch over the slices of all members and one update
 * launch with one CTA per member, replayed as CUDA graphs.  Every member keeps
 * its own data, schedule, options' precondition flag, lam, y and state, and
 * its iterates are those it would take alone (bit-identical for the same
 * coop_max).  Members must share val_dtype, device and the number of
 * capacity families (several-family members sweep with the general kernel in
 * a static order); DLM_BOX_CUT handles batch only with each other; a handle
 * appears at most once.  Set each member's schedule, precondition flag and warm start
 * before dlm_batch_create (the batch captures them; set_lambda and set_state
 * on a member remain valid afterwards).  Work of the batch is ordered on
 * `stream` (NULL: the batch creates its own blocking stream); calls on a
 * member's own handle and on the batch act on the same state, so the caller
 * must not let them overlap.  Destroy the batch before its members. */
dlm_status dlm_batch_create(dlm_problem* const* probs, int32_t n, void* stream, dlm_batch** out);
/* Mapping fields of `opt` for the batch (mapping 0 means dynamic here);
 * gap_every and graph_iters apply to dlm_batch_solve and dlm_batch_step. */
dlm_status dlm_batch_set_options(dlm_batch* bt, const dlm_options* opt);
/* dlm_autotune over the whole batch (interleaved candidates only up to 8 members). */
dlm_status dlm_batch_autotune(dlm_batch* bt, int32_t iters, dlm_options* chosen, double* sweep_ms);
dlm_status dlm_batch_step(dlm_batch* bt, int64_t n_iters);
/* As dlm_step_timed, for the batch's launches. */
dlm_status dlm_batch_step_timed(dlm_batch* bt, int64_t n_iters, double* sweep_ms, double* update_ms,
                                double* total_ms);
/* Certified-gap evaluation of every member: out[i] for member i (n entries). */
dlm_status dlm_batch_get_stats(dlm_batch* bt, dlm_stats* out);
/* Iterate until every member meets the target of dlm_solve (its own final
 * gamma and certified gap <= target_rel_gap), checking every gap_every
 * iterations, or until max_iters more iterations (then DLM_ERR_TIMEOUT);
 * out[i] (may be NULL) gets member i's stats with `converged` per member. */
dlm_status dlm_batch_solve(dlm_batch* bt, double target_rel_gap, int64_t max_iters, dlm_stats* out);
void dlm_batch_destroy(dlm_batch* bt);

/* Learned warm start (the paper motivates warm starts for recurring solves,
 * Sec. 1, but fixes no predictor; this one is the project's).  A three-layer
 * perceptron of width H maps DLM_WS_FEATURES per-item features to an initial
 * dual: xn = (x - mu) / sd, h1 = relu(xn W1 + b1), h2 = relu(h1 W2 + b2),
 * lam0 = softplus(h2 . w3 + b3 + softplus^-1(max(x_4, 1e-6))) -- a correction
 * to the previous day's dual x_4, so lam0 >= 0 and an untrained last layer
 * returns x_4.  Products run on the tensor cores with bf16 operands (xn, h1,
 * h2, the weights and, in the backward pass, the pre-activation gradients) and
 * FP32 accumulation; the master weights, Adam moments and biases are FP32.
 * Training minimises the mean squared error against solved duals with Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8).  All reductions add in a fixed order:
 * results are deterministic.  A predictor is not thread-safe; its work is
 * ordered on its stream. */
#define DLM_WS_FEATURES 7
typedef struct dlm_ws dlm_ws;

/* width: 8..1024, a multiple of 8.  seed: initial weights (He-uniform W1, W2;
 * zero w3 and biases).  stream: cudaStream_t or NULL (own blocking stream).
 * Normalizer mu = 0, sd = 1 until fitted or set. */
dlm_status dlm_ws_create(int32_t width, uint64_t seed, void* stream, dlm_ws** out);
/* Parameter count P and layout of the flat FP32 vector theta:
 * W1 (F x H, row-major), b1 (H), W2 (H x H, row-major: row = input unit),
 * b2 (H), w3 (H), b3 (1). */
dlm_status dlm_ws_num_params(dlm_ws* w, int64_t* n);
/* Host copies of theta (P floats) and the normalizer (F floats each); any
 * pointer may be NULL.  Synchronous. */
dlm_status dlm_ws_get_params(dlm_ws* w, float* theta, float* mu, float* sd);
/* Replace theta (resets the Adam state) and/or the normalizer (both or
 * neither; sd > 0).  Host arrays; NULL keeps the current values. */
dlm_status dlm_ws_set_params(dlm_ws* w, const float* theta, const float* mu, const float* sd);
/* Item features of an instance, one row of DLM_WS_FEATURES floats per item
 * (device X, num_items x F, row-major):
 *   0 log(1 + b_j)          1 log(1 + deg_j)      2 mean_i(-c_ij)
 *   3 max_i(-c_ij)          4 lam_prev_j          5 log(gamma)
 *   6 G_j / (1 + b_j), G = A x(lam_prev) - b at ridge gamma (one dual sweep)
 * (2, 3 are 0 for an item without edges).  lam_prev: device, num_items.
 * Allocates temporary device memory; synchronous. */
dlm_status dlm_ws_features(dlm_problem* p, const float* lam_prev, double gamma, float* X);
/* mu, sd of the columns of X (device, n x F; population sd, 1 where < 1e-6). */
dlm_status dlm_ws_fit_normalizer(dlm_ws* w, const float* X, int64_t n);
/* Loss at the current weights on (X, y) (device; n rows) into *loss (host)
 * and its gradient (host, P floats, theta layout) into grad (may be NULL);
 * no update.  Synchronous. */
dlm_status dlm_ws_loss_grad(dlm_ws* w, const float* X, const float* y, int64_t n, double* loss, float* grad);
/* `steps` full-batch Adam steps of learning rate lr on (X, y) (device; fits
 * the normalizer first if none was fitted or set); the loss before each step
 * into losses (host, steps floats; may be NULL).  n <= 2^26.  Synchronous. */
dlm_status dlm_ws_train(dlm_ws* w, const float* X, const float* y, int64_t n, int32_t steps, float lr,
                        float* losses);
/* lam0 for n feature rows X (device) into out (device, n floats).
 * Synchronous, so a solver on another stream may read out at once. */
dlm_status dlm_ws_predict(dlm_ws* w, const float* X, int64_t n, float* out);
void dlm_ws_destroy(dlm_ws* w);

/* One dual evaluation straight from the caller's device CSR arrays, with no
 * device memory allocated by this call or any earlier one: for callers that
 * cannot call cudaMalloc (a process whose device memory belongs to another
 * framework's allocator, a fixed memory budget, code that must not allocate
 * after start-up).  The paper has no counterpart; it computes what
 * dlm_calculate computes (g(lambda), grad g(lambda) = A x - b, x(lambda))
 * for FP32 c and a, without a handle.
 *   row_ptr, item_idx, c, a, b, lambda: device arrays as in dlm_problem_desc
 *     (valid CSR; an out-of-range item or row pointer makes the call write
 *     NaN to g and grad instead of reading out of bounds, and x is then
 *     undefined: a row with a bad row pointer is skipped, its x entries
 *     keep whatever the buffer held);
 *   kind, z: the simple sets; gamma > 0: the ridge;
 *   g: device double (1), grad: device float (num_items) or NULL,
 *   x: device float (nnz, caller's edge order) or NULL.
 * Asynchronous on `stream` (a cudaStream_t; NULL = legacy default stream).
 * Scratch: one file-scope device array of about 0.5 MB (fixed-point item
 * sums for up to 65,536 items, objective partials, bounds), held on every GPU
 * that loads the library until the process exits; num_items > 65,536 returns
 * DLM_ERR_UNSUPPORTED.  The first call on a device looks the array's device
 * address up (cudaGetSymbolAddress) and keeps it for the life of the
 * process, so make that first call before any stream capture, and do not
 * call this entry point again after cudaDeviceReset on that device.  Every call clears the scratch it needs at its start and
 * leaves it cleared at its end; calls that overlap on the GPU share the
 * array and race, so issue them one after another on one stream. */
dlm_status dlm_calculate_static(int64_t num_users, int64_t num_items, int64_t nnz, const int64_t* row_ptr,
                                const int32_t* item_idx, const float* c, const float* a, const double* b,
                                int32_t kind, double z, const float* lambda, double gamma, double* g, float* grad,
                                float* x, void* stream);

/* User-sharded instances (Sec. 4.4: the paper splits the sources across
 * GPUs, sums the gradient on one rank and broadcasts lambda; here every rank
 * sums and updates).  Users are independent given the dual, so each rank
 * holds a contiguous range of users (its rows, in dlm_problem_desc) and the
 * full capacity vector b; after every sweep the ranks add their partial
 * item sums -- exact 64-bit fixed-point integers, so the sum is the same in
 * any order and on every rank -- and each rank takes the same update.  The
 * iterates are bit-identical to those of one handle holding every row.  One
 * capacity family; no batches.
 *
 * Set-up, on every rank:
 *  1. dlm_shard_local: validates the rows and fills the rank's statistics
 *     (nnz, active_users, max_abs_a, max_abs_c, a_nonneg) and its item
 *     degrees (host int64 [num_items]);
 *  2. the ranks combine them: nnz, active_users and the item degrees by
 *     sums, max_abs_a and max_abs_c by maxima, a_nonneg by minimum;
 *     max_item_degree = the largest summed item degree;
 *  3. dlm_shard_item_sums with the combined statistics: the rank's
 *     fixed-point sums of a_ij^2 and a_ij per item; the ranks add them
 *     (int64 sums) into item_sq and item_sum;
 *  4. dlm_create with desc.shard pointing at the combined dlm_shard, whose
 *     exchange buffers the caller allocates (device memory, kept for the
 *     handle's life).
 * Each iteration: dlm_shard_sweep, then the ranks add `exchange` (int64
 * sum, in place), then dlm_shard_update.  The iterates equal those of one
 * handle holding every row when both take every row's threshold in its own
 * lane (dlm_options.coop_max = 1): the warp-cooperative path for rows with
 * many active edges sums in another order, and whether a row takes it
 * depends on the other rows of its slice.  A certified gap: dlm_shard_cert_sweep,
 * the ranks add `cert_exchange` (int64) and `cert_obj` (float64), then
 * dlm_shard_cert_finish.  All work is ordered on the handle's stream; the
 * sums must be complete on that stream before the call that follows them.
 * dlm_step, dlm_solve and dlm_get_stats are not valid on a shard handle
 * (DLM_ERR_UNSUPPORTED): each rank alone sees only part of the sums. */
typedef struct dlm_shard {
  int64_t nnz;             /* edges, all shards */
  int64_t active_users;    /* users with at least one edge, all shards */
  int64_t max_item_degree; /* the largest item degree, degrees summed over the shards */
  double max_abs_a;        /* largest |a| over the shards */
  double max_abs_c;        /* largest |c| over the shards */
  int32_t a_nonneg;        /* 1 when no shard has a negative a */
  int32_t reserved;
  const int64_t* item_sq;  /* host [num_items]: fixed-point sum_i a_ij^2 over the shards */
  const int64_t* item_sum; /* host [num_items]: fixed-point sum_i a_ij over the shards */
  int64_t* exchange;       /* device [num_items + 2]: the iteration's partial sums (item sums, count, objective) */
  int64_t* cert_exchange;  /* device [3 num_items + 1]: the certificate's partial sums */
  double* cert_obj;        /* device [1]: the certificate's objective partial */
} dlm_shard;

/* Step 1 of the set-up above: statistics of this rank's rows (a
 * dlm_problem_desc without `shard`); item_degree: host int64 [num_items].
 * Validates as dlm_create does.  Synchronous. */
dlm_status dlm_shard_local(const dlm_problem_desc* desc, void* stream, dlm_shard* local, int64_t* item_degree);
/* Step 3: this rank's fixed-point item sums at the exponents the combined
 * statistics `global` (max_item_degree, max_abs_a) fix; item_sq, item_sum:
 * host int64 [num_items].  Synchronous. */
dlm_status dlm_shard_item_sums(const dlm_problem_desc* desc, const dlm_shard* global, void* stream, int64_t* item_sq,
                               int64_t* item_sum);
/* The iteration sweep at y: this rank's partial sums into `exchange`. */
dlm_status dlm_shard_sweep(dlm_problem* p);
/* The accelerated step from the summed `exchange` (identical on every rank);
 * clears `exchange` for the next sweep. */
dlm_status dlm_shard_update(dlm_problem* p);
/* The certificate sweep at lam: partial sums into `cert_exchange` and
 * `cert_obj`. */
dlm_status dlm_shard_cert_sweep(dlm_problem* p);
/* The certified gap from the summed certificate buffers (see dlm_stats);
 * clears them.  Synchronous. */
dlm_status dlm_shard_cert_finish(dlm_problem* p, dlm_stats* out);

/* Thread-local message describing the last failure on this thread ("" if none). */
const char* dlm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DLM_H */
