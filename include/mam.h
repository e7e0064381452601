/*
 * mam.h - C ABI of libmam, a GB300 (sm_103a) implementation of the Method of
 * Averaged Marginals (MAM) for fixed-support balanced and unbalanced
 * Wasserstein barycenters (Mimouni, Malisani, Zhu, de Oliveira,
 * arXiv 2309.05315).
 *
 * Problem (eq. HugeLP, eq. UWB):  M discrete measures
 *   nu^(m) = sum_s q^(m)_s delta_{zeta^(m)_s},  s = 1..S_m,
 * a fixed barycenter support xi_1..xi_R, weights alpha_m and costs
 *   c^(m)_{rs} = alpha_m * ||xi_r - zeta^(m)_s||^2   (or alpha_m * C^(m)_{rs}).
 * The library runs Algorithm 1 (MAM): Step 1 averages the row marginals of
 * the plans theta^(m) with the weights a_m of eq. (pr) (Prop. 2), the factor
 * t^k of Algorithm 1 switches between the balanced (gamma = inf) and the
 * unbalanced prox of eq. (Unbalanced-prox), Step 2 projects every plan
 * column onto the scaled simplex Delta_R(q_s) (Prop. 3, Remark 1) and
 * updates theta, Step 3 recomputes the marginals.  Index sets follow
 * Remark 2 (random bundles) or are all measures (deterministic MAM).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every function returns mam_status; no C++ exception crosses the ABI.
 *   On failure a message is available from mam_last_error(handle) (or
 *   mam_last_error(NULL) for a failed create, thread-local).
 * - Ownership: inputs are copied during the call; caller buffers may be
 *   freed as soon as the call returns.  The library owns every device buffer
 *   it allocates (plans, costs, marginals, scratch) and frees them in
 *   mam_destroy.  Outputs go to caller-provided buffers.
 * - Streams: all device work of a handle is ordered on its stream
 *   (mam_desc.stream, or a stream the library creates when NULL).  Only
 *   mam_objective, mam_solve, the mam_get_* calls and mam_backward
 *   synchronise that stream.
 * - Layout: supports are given measure after measure, unpruned (zero
 *   weights allowed): measure m occupies entries off_m .. off_m + S_m - 1
 *   where off_m = S_0 + ... + S_{m-1}.  Point arrays are row-major
 *   [n][dim].  Plans are stored pruned and column-contiguous: column s of
 *   measure m is R consecutive floats.
 * - Errors: invalid arguments -> MAM_ERR_INVALID_ARG with nothing
 *   allocated; device allocation failure -> MAM_ERR_OOM with nothing
 *   leaked; a CUDA error -> MAM_ERR_CUDA and the handle enters the error
 *   state, in which every later call except mam_destroy/mam_last_error
 *   returns MAM_ERR_STATE.  A non-finite residual -> MAM_ERR_NONFINITE.  A
 *   device-side wait that exceeded its bound -> MAM_ERR_TIMEOUT.
 */
#ifndef MAM_H_
#define MAM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MAM_OK = 0,
  MAM_ERR_INVALID_ARG = 1,
  MAM_ERR_CUDA = 2,
  MAM_ERR_OOM = 3,
  MAM_ERR_NONFINITE = 4,
  MAM_ERR_TIMEOUT = 5,
  MAM_ERR_STATE = 6,
  MAM_ERR_UNSUPPORTED = 7,
  MAM_ERR_COMM = 8,      /* the exchange callback of a sharded problem failed */
  MAM_ERR_CAPACITY = 9   /* sparse plan layout: a column's active set exceeded
                            sparse_slots (the iterate is invalid)           */
} mam_status;

/* Storage type of the cost c (theta is always FP32; p, objective and
 * residuals are FP64).  Costs are computed in FP64, rounded to FP32 (nearest)
 * and then, for BF16/F16, rounded again to nearest-even. */
typedef enum { MAM_F32 = 0, MAM_BF16 = 1, MAM_F16 = 2 } mam_cost_dtype;

/* How the costs are stored (mam_desc.cost_layout). */
typedef enum {
  MAM_COST_PER_COLUMN = 0,
  MAM_COST_SHARED = 1,
  MAM_COST_GENERATED = 2
} mam_cost_layout;

/* How the plans theta are stored (mam_desc.plan_layout). */
typedef enum { MAM_PLAN_DENSE = 0, MAM_PLAN_SPARSE = 1 } mam_plan_layout;

/* When the fused diagnostics (W-hat, dist_L(pi-hat), lower bound, residuals)
 * are computed. */
typedef enum {
  MAM_DIAG_LAST = 0,   /* last iteration of every mam_step call (default) */
  MAM_DIAG_NEVER = 1,  /* never (fastest; mam_objective then reports iter=-1) */
  MAM_DIAG_EVERY = 2   /* every iteration */
} mam_diag_mode;

typedef struct mam_problem mam_problem; /* opaque, library-owned */

/* Problem description (eq. HugeLP / eq. UWB data plus MAM parameters). */
typedef struct {
  int32_t M;            /* number of measures, >= 1                          */
  int32_t R;            /* barycenter support size, 1..12288                 */
  int32_t dim;          /* point dimension, 1..3                             */
  const int32_t* S;     /* host [M]: support sizes BEFORE pruning, >= 1      */
  const double* zeta;   /* host [sum S][dim]: support points of the measures */
  const double* q;      /* host [sum S]: weights q^(m)_s >= 0, finite; columns
                           with q = 0 are pruned (Section 4.3); every measure
                           needs at least one positive weight               */
  const double* alpha;  /* host [M]: alpha_m >= 0, folded into the cost      */
  const double* xi;     /* host [R][dim]: barycenter support points          */
  const double* cost;   /* host [sum S][R] general cost C (row s of measure m
                           = column s of C^(m)), or NULL for squared
                           Euclidean.  Scaled by alpha_m either way.         */
  double rho;           /* prox parameter of eq. (DR), in [1e-30, 1e30] (the
                           kernels use rho and 1/rho in FP32): the projected
                           vector is theta + 2 t d - c / rho (Alg. 1)        */
  double gamma;         /* unbalanced penalty >= 0; INFINITY = balanced.
                           Balanced problems need equal total masses unless
                           capped is set.                                    */
  int32_t n_bundles;    /* 0 or 1: deterministic MAM (all measures each
                           iteration).  nb > 1: Remark 2, measures split into
                           nb contiguous bundles, bundle i drawn with
                           probability sum_{m in A_i} alpha_m.               */
  uint64_t seed;        /* seed of the bundle draws (counter-based
                           SplitMix64; draw k uses seed + k*0x9E3779B97F4A7C15) */
  int32_t cost_dtype;   /* mam_cost_dtype                                    */
  int32_t theta0_mode;  /* 0: theta^0_{rs} = q_s / R;  1: theta^0 = 0       */
  int32_t diag_mode;    /* mam_diag_mode                                     */
  void* stream;         /* cudaStream_t to order work on, or NULL            */
  double eta;           /* capped only: mass penalty eta >= 0, finite; the
                           cost becomes alpha_m (d - eta) (or alpha_m (C - eta)
                           with a general cost).  Must be 0 when capped = 0. */
  int32_t capped;       /* 0: Step 2 projects column s onto Delta_R(q_s), so
                           every column carries its mass (Alg. 1).  1: the
                           full unbalanced extension of the paper ("Algorithm's
                           Extension: the Full Unbalanced Setting"): column s
                           is projected onto Delta_<=(q_s) = {u >= 0 :
                           sum u <= q_s} (clip at 0, then the simplex
                           projection if the clipped mass exceeds q_s), so a
                           column may carry less mass; masses may differ for
                           any gamma.  All problems of a batch share it.
                           Reverse mode needs capped = 0.                    */
  int32_t cost_layout;  /* 0 (MAM_COST_PER_COLUMN): c^(m) stored column by
                           column for every kept column (T x R values).
                           1 (MAM_COST_SHARED): every measure has the same
                           support points (the same S_m and zeta, before
                           pruning, as images on one pixel grid have), so
                           one matrix C_rs = ||xi_r - zeta_s||^2 (- eta when
                           capped) over that support serves every measure,
                           and c^(m) = alpha_m C (eq. HugeLP): S x R values
                           instead of T x R, read from L2 when they fit, and
                           alpha_m applied in the kernels (to 1/rho).  Needs
                           the squared Euclidean cost (cost = NULL); in a
                           batch every problem must have the same support,
                           xi and eta.  The stored C is rounded to cost_dtype
                           before alpha_m is applied.
                           2 (MAM_COST_GENERATED): no cost is stored; the
                           column kernel computes ||xi_r - zeta_s||^2 (- eta)
                           in FP32 from FP32 copies of the points (16 B per
                           row and per column, read through L2) whenever it
                           needs c: 8 B of HBM traffic per plan entry (theta
                           read and write) and no T x R cost buffer, for
                           problems whose costs would not fit or whose
                           columns are long.  Uses the one-column-per-cluster
                           kernel (kind 2) for every R; needs the squared
                           Euclidean cost (cost = NULL); cost_dtype is
                           ignored.  Reverse mode is not offered.            */
  int32_t plan_layout;  /* 0 (MAM_PLAN_DENSE): theta stored as FP32 [T][ld].
                           1 (MAM_PLAN_SPARSE): every step sets theta' = pihat
                           - d (Alg. 1) with pihat zero off the column's active
                           set and d one vector per measure, so a visited
                           column is stored as the (row, value) pairs of its
                           pihat (at most sparse_slots) and each measure keeps
                           the d of its last visit; theta_rs = pihat_rs - d_r
                           (one FP32 subtraction, the value the dense layout
                           stores: the iterates are bit for bit the dense
                           layout's).  Plan memory is 8 B x sparse_slots per
                           column instead of 4 B x ld, and a column step reads
                           its cost and pairs and writes pairs: the cost's
                           HBM traffic plus 16 B per active entry.  Runs on
                           the one-CTA-per-column kernel (kind 0, 1 stage,
                           R <= 12288); not with the generated cost layout or
                           the support step.  A column whose active set
                           exceeds sparse_slots fails the step with
                           MAM_ERR_CAPACITY; the handle is then unusable.
                           mam_get_theta and mam_get_theta_range expand the
                           plans on the device.  The order of a column's
                           pairs in a state blob is not deterministic.       */
  int32_t sparse_slots; /* sparse layout: pairs per column (even, 2..ld; 0:
                           min(ld, 1024)).  Active sets are largest in the
                           first iterations from theta^0.                    */
} mam_desc;

/* Diagnostics of the most recent diagnostic iteration k (all FP64). */
typedef struct {
  double w_hat;        /* sum_m <c^(m), pi-hat^(m)>.  Randomized index sets:
                          each column contributes the value of its last
                          diagnostic update (with MAM_DIAG_EVERY: its last
                          update, stale columns included, as p^(m) are).   */
  double dist_pihat;   /* dist_L(pi-hat) = sqrt(sum_m ||p^ - p^^(m)||^2/S_m) */
  double lower_bound;  /* sum_m sum_s q_s min_r (c_rs - rho d^(m)_r): a valid
                          lower bound of eq. (HugeLP)/(UWB) (deterministic
                          runs; randomized runs recompute it on demand).
                          Capped columns take q_s min(0, min_r (...)).      */
  double f_unbal;      /* w_hat + gamma * dist_pihat (= w_hat if balanced) */
  double fp_resid;     /* ||theta^{k+1} - theta^k||_2 over updated columns  */
  double dp_norm;      /* ||p^{k+1} - p^k||_2                               */
  double t;            /* t^k of Algorithm 1 used by iteration k            */
  double dist_theta;   /* dist_L(theta) of the current plans (text after
                          Algorithm 1)                                      */
  double t_next;       /* t of the next iteration (from the current plans)  */
  int64_t iter;        /* k + 1 = iterations done when measured, -1: none   */
  int64_t newton_passes; /* threshold-search passes summed over columns     */
} mam_objective_t;

/* Create a problem: validates, prunes zero-weight columns, builds the cost
 * on the device, sets theta^0 and the Step 0 marginals.  With randomized
 * index sets (n_bundles > 1) it also primes the stored thresholds: every
 * index set is projected once from theta^0 and only the thresholds are kept
 * (the state is reset to theta^0), so that a column's first visit starts its
 * threshold search from a nearby value instead of the cold bracket; the
 * iterates are those of Algorithm 1 from theta^0 either way.  On failure
 * *out is NULL and nothing is leaked.  Cites: eq. (HugeLP), Section 4.3,
 * Alg. 1 Step 0, Remark 2. */
mam_status mam_create(const mam_desc* desc, mam_problem** out);

/* ---------------------------------------------------------------------
 * Measure-sharded problems (one problem over several GPUs).
 *
 * Step 2 of Algorithm 1 is independent across measures, and Step 1 needs of
 * them only p = sum_m a_m p^(m) (eq. pr, Prop. 2) and, for t^k, the
 * distance D^2 = sum_m ||p - p^(m)||^2 / S_m.  A sharded problem gives each
 * rank a contiguous range of the measures; every iteration the rank runs the
 * column step on its own columns, forms its partial sum of a_m p^(m) as
 * 64-bit fixed-point integers and has the caller's callback sum those R
 * integers over all ranks; the sum is exact, so p (and with it every shift
 * and every plan) is bit for bit that of the unsharded solver.  When t^k is
 * needed (gamma finite) or diagnostics are taken, a second exchange sums four
 * FP64 values (D^2 and diagnostic distances; diagnostic iterations also sum
 * the R FP64 values of sum_m a_m pi-hat marginals).  Nothing else crosses
 * ranks.
 */

/* Exchange callback: sum `count` values of type `dtype` in the device buffer
 * `buf` over every rank, in place, ordered on the CUDA stream `stream` (a
 * cudaStream_t): the result must be in `buf` for work enqueued on `stream`
 * after the call returns.  Return 0 on success.  Every rank calls it the same
 * number of times with the same counts, in the same order. */
typedef enum { MAM_SUM_I64 = 0, MAM_SUM_F64 = 1 } mam_sum_dtype;
typedef int32_t (*mam_allreduce_fn)(void* buf, int64_t count, int32_t dtype, void* stream,
                                    void* user);

typedef struct {
  int32_t m_begin;            /* this rank owns measures m_begin .. m_end - 1 */
  int32_t m_end;              /* of the description (1 <= m_end - m_begin)   */
  mam_allreduce_fn allreduce; /* required                                    */
  void* user;                 /* passed to allreduce unchanged               */
} mam_shard;

/* Create this rank's part of a measure-sharded problem.  `desc` describes
 * the WHOLE problem (every measure) and must be identical on every rank;
 * the handle keeps the plans, costs and marginals of measures m_begin ..
 * m_end - 1 only (the averaging weights a_m, the fixed-point scale and the
 * bundles of Remark 2 come from all of them).  Collective: every rank calls
 * it, and it already calls the callback (the Step 0 average).  Afterwards
 * mam_step, mam_solve and mam_objective are collective too and give the same
 * p, t and diagnostics on every rank; mam_get_barycenter returns the global
 * p, mam_get_marginals/mam_get_theta/mam_get_pruned_sizes the rank's own
 * measures.  Single problem only; no CUDA-graph replay (every iteration
 * calls the callback); reverse mode and the free-support step are not
 * offered (MAM_ERR_INVALID_ARG).  A failing callback returns MAM_ERR_COMM and
 * puts the handle in the error state.  Ranks are usually one per GPU: the
 * range rule that balances the plan entries is to cut the measures into
 * contiguous groups of about equal sum_m S_m. */
mam_status mam_create_sharded(const mam_desc* desc, const mam_shard* shard, mam_problem** out);

/* Batch of n independent problems solved together: every iteration is one
 * launch of the column kernel over all problems' columns plus one averaging
 * launch, replayed from a captured CUDA graph.  All problems must share R,
 * dim, cost_dtype and diag_mode and be deterministic (n_bundles <= 1).  The
 * stream of descs[0] is used. */
mam_status mam_batch_create(int32_t n, const mam_desc* descs, mam_problem** out);

/* Run n_iters iterations of Algorithm 1 (asynchronous on the stream). */
mam_status mam_step(mam_problem* h, int32_t n_iters);

/* Iterate until gap <= gap_tol (checked every check_every iterations, which
 * must be >= 1) or max_iters.  gap = max(|F - ref| / |ref|,
 * dist_L(pi-hat) / Q) where F = f_unbal, Q = total mass and ref = w_ref if
 * w_ref > 0, else the lower bound (a certified gap when F is an upper
 * bound).  *iters_done (may be NULL) receives the iterations run; *gap_out
 * (may be NULL) the last gap.  Batched handles use the largest gap. */
mam_status mam_solve(mam_problem* h, int32_t max_iters, double gap_tol,
                     double w_ref, int32_t check_every, int32_t* iters_done,
                     double* gap_out);

/* Diagnostics of problem `index` (0 for a single problem); synchronises. */
mam_status mam_objective(mam_problem* h, int32_t index, mam_objective_t* out);

/* Diagnostics of every problem of the handle at once, out[n_problems]
 * (host array); synchronises.  Same values as mam_objective. */
mam_status mam_objective_all(mam_problem* h, mam_objective_t* out);

/* Barycenter p = sum_m a_m p^(m) of the current theta (Alg. 1 "Return"),
 * [n_problems][R] FP64.  device_ptr != 0: p_out is a device pointer. */
mam_status mam_get_barycenter(mam_problem* h, double* p_out, int32_t device_ptr);

/* Row marginals p^(m) = sum_s theta^(m)_{.s} of the current plans (Alg. 1
 * Step 3), [total measures][R] FP64.  device_ptr != 0: device pointer. */
mam_status mam_get_marginals(mam_problem* h, double* pm_out, int32_t device_ptr);

/* Current plans, pruned and column-contiguous: [T][R] FP32 where T is the
 * number of kept columns (mam_get_sizes).  Host pointer. */
mam_status mam_get_theta(mam_problem* h, float* theta_out);

/* Columns col0 .. col0 + ncols - 1 of the current plans (pruned order, as
 * in mam_get_theta), [ncols][R] FP32, host pointer; synchronises.  For
 * reading a sample of the columns of a plan too large to copy whole.
 * MAM_ERR_INVALID_ARG if the range leaves 0..T. */
mam_status mam_get_theta_range(mam_problem* h, int64_t col0, int64_t ncols, float* theta_out);

/* Work done by the column steps of Step 2 since the handle was created:
 * plan columns projected and plan entries updated (columns x R), summed
 * over the index sets M^k actually drawn (Remark 2: a randomized run updates
 * one bundle per iteration).  Host counters, no synchronisation; either
 * pointer may be NULL. */
mam_status mam_get_work(const mam_problem* h, int64_t* columns, int64_t* entries);

/* Sizes: n_problems, total measures, R, kept columns T, padded column
 * stride (floats) of the device plan buffer.  Any pointer may be NULL. */
mam_status mam_get_sizes(const mam_problem* h, int32_t* n_problems,
                         int32_t* n_measures, int32_t* R, int64_t* T,
                         int32_t* ld);

/* Kept (pruned) column count of every measure, [total measures]. */
mam_status mam_get_pruned_sizes(const mam_problem* h, int32_t* S_out);

/* Checkpoint: the whole iteration state (theta, marginals, thresholds,
 * iteration counter, bundle position).  Call with buf = NULL to get *bytes.
 * Resuming with mam_set_state reproduces an uninterrupted run bit for bit.
 * Infrastructure for long runs and for the autotuner: the paper has no
 * counterpart (its state is the plan theta^k of Algorithm 1).  A sharded
 * handle saves and restores its own measures; every rank must restore the
 * same iteration.  With the sparse plan layout the blob holds each column's
 * pairs and count and each measure's last shift in place of theta, and
 * restores only into a handle of the same layout and sparse_slots
 * (MAM_ERR_INVALID_ARG otherwise). */
mam_status mam_get_state(mam_problem* h, void* buf, size_t* bytes);
mam_status mam_set_state(mam_problem* h, const void* buf, size_t bytes);

/* Differentiation through K unrolled iterations (balanced, deterministic,
 * single problem).  mam_forward_record restarts from theta^0 and runs K
 * iterations.  The reverse step of an iteration needs only its active sets
 * (one bit per plan entry).  ckpt_every > 0: the state is kept every
 * ckpt_every iterations and mam_backward recomputes each segment (memory:
 * K/ckpt_every states and ckpt_every masks).  ckpt_every = 0 (automatic):
 * the masks of all K steps are kept from the forward pass when they fit in a
 * quarter of the free device memory, and mam_backward recomputes nothing;
 * otherwise as with ckpt_every = sqrt(K).  The gradients are the same either
 * way.  mam_backward
 * takes dL/dp^K [R] and writes dL/dq [sum S] (unpruned order, zeros for
 * pruned columns), dL/dzeta [sum S][dim] and dL/dxi [R][dim]; any output may
 * be NULL.  All host pointers.  Only squared Euclidean costs with
 * theta0_mode 0 or 1. */
mam_status mam_forward_record(mam_problem* h, int32_t K, int32_t ckpt_every);
mam_status mam_backward(mam_problem* h, const double* grad_p, double* grad_q,
                        double* grad_zeta, double* grad_xi);

/* Free-support step of Algorithm 2 (Prop. 4).  From the current state, the
 * plans pi-hat that the next column step would compute (Step 1 and the
 * projection of Step 2, Algorithm 1; theta is not changed) give the new
 * support
 *   xi_r = sum_m alpha_m sum_s zeta_s pi-hat_rs / sum_m alpha_m sum_s pi-hat_rs,
 * the minimiser of sum_m alpha_m sum_{r,s} ||xi_r - zeta_s||^2 pi-hat_rs; rows
 * that carry no mass keep their point.  The costs are then rebuilt for the
 * new support (FP64, rounded to the storage type; with eta when capped) and
 * theta, the marginals and the thresholds are kept as the warm start of the
 * following iterations.  Algorithm 2 alternates mam_step (or mam_solve) with
 * this call.  The costs follow the support, not mam_get_state/mam_set_state.
 * xi_out: host [R][dim], may be NULL; receives the new support.  Needs a
 * single problem, support points with the squared Euclidean cost (no general
 * cost matrix) and the deterministic index set, else MAM_ERR_INVALID_ARG.
 * The per-row sums are 64-bit fixed point (order-independent).  Synchronises
 * the handle's stream. */
mam_status mam_update_support(mam_problem* h, double* xi_out);

/* Algorithm 2 (free-support barycenter): `outer` rounds of
 *   (a) Algorithm 1 on the current support: inner_iters iterations
 *       (gap_tol = 0), or mam_solve to gap_tol with at most inner_iters
 *       iterations and a check every check_every (gap_tol > 0);
 *   (b) mam_update_support (Prop. 4).
 * theta is kept across rounds.  xi_out (host [R][dim], may be NULL) receives
 * the last support; iters_done (may be NULL) the iterations run.  Same
 * requirements and errors as mam_update_support and mam_solve. */
mam_status mam_free_support(mam_problem* h, int32_t outer, int32_t inner_iters, double gap_tol,
                            int32_t check_every, double* xi_out, int32_t* iters_done);

/* Kernel configuration of the column step.
 * kind 0: one CTA per column.  threads (multiple of 32, up to 1024 for vec
 *   1, 768 for 2, 512 for 3..4, 192 for 5..6, 384 for 8) x vec float4
 *   groups cover the column; stages (1..4) is the depth of the bulk-copy
 *   pipeline.  Any R up to 12288.
 * kind 2: one column per thread-block cluster of vec (2, 4, 8, 16) CTAs of
 *   threads (64..256) threads; each CTA keeps a slice of the column in shared
 *   memory (columns up to 786432 rows; the default above 12288); stages 1.
 * kind 1: one warp per column.  vec (1,2,4,7,8,13,16) float4 groups
 *   per lane cover the column (R up to 2048; the default for R up to
 *   1024); stages (>= threads/32) is the number of shared-memory ring
 *   slots; threads/32 warps per CTA.
 * ctas_per_sm: 0 = occupancy maximum.  bisect_depth (0..30): bisection steps
 * on a cold start.  Invalid combinations return MAM_ERR_INVALID_ARG. */
typedef struct {
  int32_t threads;
  int32_t vec;
  int32_t stages;
  int32_t ctas_per_sm;
  int32_t bisect_depth;
  int32_t kind;
} mam_kernel_config;
mam_status mam_get_config(const mam_problem* h, mam_kernel_config* cfg);
mam_status mam_set_config(mam_problem* h, const mam_kernel_config* cfg);

/* Autotuner of the column step (the batching form's launch shapes).  Saves
 * the state, then (1) times every candidate launch shape for `iters`
 * iterations from that state: one-CTA-per-column shapes (threads x float4
 * groups covering a column, copy-pipeline depth, resident CTAs per SM, which
 * fixes the columns each CTA of the persistent grid takes) and
 * warp-per-column shapes (width, ring slots, warps per CTA, CTAs per SM);
 * (2) on the fastest shape, times the bisection depths 0, 2, 4, 6, 8, 12,
 * 16, 24 from the same state with every stored threshold cleared, so that
 * the first timed iteration takes the cold search (bracket, bisection,
 * Newton steps; Algorithm 1 Step 2), the only place the depth matters.  The
 * fastest configuration is kept in the handle and returned in *best (may be
 * NULL); the state is restored.  On any failure the starting configuration
 * and state are restored before the status is returned.  Synchronises.  Not
 * offered for sharded problems (MAM_ERR_INVALID_ARG). */
mam_status mam_autotune(mam_problem* h, int32_t iters, mam_kernel_config* best);

/* Measurement support: while enabled, every iteration is launched on its own
 * (no graph replay) between CUDA events on the handle's stream, so that the
 * durations of the column kernel and of the averaging kernel can be read
 * back.  mam_profile_read synchronises, returns the summed milliseconds and
 * the number of iterations timed since the last read, and resets them. */
mam_status mam_profile_enable(mam_problem* h, int32_t enable);
mam_status mam_profile_read(mam_problem* h, double* column_ms, double* average_ms,
                            int64_t* launches);

/* Column update without device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc, such as
 * code whose device memory is owned by another framework's pool (a raw
 * allocation bypasses that pool and may fail once it has reserved the GPU)
 * or latency-critical loops that cannot afford cudaMalloc's implicit
 * synchronisation.  On one measure's plan it computes, for every column s,
 * w = theta_s + 2 d - c_s / rho, pihat_s = Proj_{Delta_R(q_s)}(w) and
 * theta_s <- pihat_s - d (in place), and writes rowsum_out[r] =
 * sum_s theta_rs (FP64).  All pointers are device pointers the caller owns:
 * theta and cost [S][ld] FP32 (column-contiguous, ld >= R), q [S], d [R],
 * rowsum_out [R].  mass_bound must be >= sum_s q_s (it fixes the scale of
 * the integer accumulator).  Work is enqueued on `stream` (NULL = default
 * stream); the call does not synchronise.
 * Failures on the device: the call's only result is rowsum_out, so a column
 * whose threshold search ends with an empty active set (q_s below the FP32
 * resolution of w) or a row sum that overflows the accumulator (mass_bound
 * too small: overflow needs about 4x the true mass and is detected up to
 * about 8x) makes every rowsum_out entry NaN.
 * Scratch: a file-scope device array of 12288 64-bit integers plus one
 * status word (96 KB) that every GPU loading the library keeps until exit;
 * R > 12288 is rejected with MAM_ERR_INVALID_ARG.  The array is cleared at
 * the start of every call, and all calls on a device share it, so calls
 * whose work overlaps on the GPU (different streams, concurrently) race and
 * give wrong row sums.  Every call looks up the array's device address with
 * the caller's device current (a host-side lookup); the first call on a
 * device also loads the library's device code, so make that first call
 * before any stream capture.  Errors go to mam_last_error(NULL). */
mam_status mam_column_update_noalloc(float* theta, const float* cost, const float* q,
                                     const float* d, int32_t R, int32_t ld, int32_t S,
                                     double rho, double mass_bound, double* rowsum_out,
                                     void* stream);

/* Last error message of h, or the thread-local one when h is NULL. */
const char* mam_last_error(const mam_problem* h);

/* Self-test of failure detection: one warp waits, through the bounded
 * mbarrier wait the column kernels use, on a phase that expects two
 * arrivals and receives none.  The wait gives up after limit_us
 * microseconds (1..2000000) and the call returns MAM_ERR_TIMEOUT, the status
 * a real run reports when a device wait runs out; the CUDA context stays
 * usable.  MAM_ERR_STATE if the wait did not run out, MAM_ERR_CUDA on a
 * launch error.  Uses the current device and synchronises it. */
mam_status mam_selftest_wait_timeout(int32_t limit_us);

/* Free everything the handle owns; NULL is allowed. */
void mam_destroy(mam_problem* h);

#ifdef __cplusplus
}
#endif

#endif /* MAM_H_ */
