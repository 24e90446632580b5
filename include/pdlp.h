/*
 * pdlp.h -- C ABI of the B300 restarted-PDHG LP solver.
 *
 * The LP is the one of arXiv 2312.14832, Section 2, Eq. (LP):
 *
 *     min  c'x   s.t.  A x = b,  G x >= h,  l <= x <= u,
 *
 * given stacked as K = [A; G] (rows 0..m1-1 are the equality rows A),
 * q = [b; h], with l_j = -INFINITY / u_j = +INFINITY for absent bounds.
 * The dual is  max q'y + l'lambda^+ - u'lambda^-  s.t.  c - K'y = lambda,
 * y_{m1..m-1} >= 0, lambda in Lambda (the bound-multiplier cone of Section 2).
 *
 * The solver runs restarted PDHG (Section 2, "Restarted PDHG"): the primal
 * step x <- proj_X(x - (eta/omega)(c - K'y)), the dual step
 * y <- proj_Y(y + eta*omega*(q - K(2x_new - x_old))), uniform averaging inside
 * each inner loop, and the KKT_omega-based restart rule of Section 2
 * ("Restart criteria"), with termination by the three relative tests of
 * Section 2 ("Optimality termination criteria").
 *
 * Conventions of every entry point:
 *  - Return value: 0 on success, a negative PDLP_E* code on failure; the text
 *    of the last failure is returned by pdlp_last_error(handle) (or
 *    pdlp_last_error(NULL) for a failed pdlp_setup).  No C++ exception
 *    crosses this boundary.
 *  - A handle is not thread-safe; use one handle per host thread.
 *  - Array arguments are plain pointers.  For pdlp_setup / pdlp_batch_setup
 *    (whose per-LP size arrays are always host arrays) / pdlp_solve /
 *    pdlp_batch_solve / pdlp_get_iterate / pdlp_spmv / pdlp_bound_duals they
 *    are host pointers unless the setup's params.inputs_on_device = 1, in which
 *    case they are device pointers on the current CUDA device.  The library copies what it needs; callers keep
 *    ownership of their arrays and may free them after the call returns.
 *  - All vectors the caller sees are in the caller's (original, unscaled)
 *    row and column order.
 *  - Work runs on a stream owned by the handle; when params.stream is not
 *    NULL that stream is ordered before and after each call.
 */
#ifndef PDLP_B300_H
#define PDLP_B300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* error codes (return values) */
#define PDLP_OK 0
#define PDLP_EINVAL (-1)    /* malformed input: CSR not monotone, column out of range,
                               NaN value, l > u, m1 > m, bad parameter */
#define PDLP_ENOMEM (-2)    /* device or host allocation failed */
#define PDLP_ECUDA (-3)     /* a CUDA runtime call failed (message in pdlp_last_error) */
#define PDLP_ETIMEOUT (-4)  /* a bounded device-side wait gave up (spin limit); the kernel
                               set its error flag and returned, the context stays usable */
#define PDLP_EINTERNAL (-5) /* internal consistency check failed */

/* solve outcome (pdlp_result.status) */
#define PDLP_OPTIMAL 0      /* all three relative tests hold at params.tol */
#define PDLP_ITER_LIMIT 1   /* max_iter reached */
#define PDLP_TIME_LIMIT 2   /* time_limit_s reached */
#define PDLP_NUMERICAL 3    /* a NaN or Inf appeared in the KKT quantities */

/* precision (pdlp_params.precision) */
#define PDLP_FP64 0         /* every iteration in FP64 */
#define PDLP_MIXED 1        /* FP32 SpMVs and vector updates with FP32 iterates; the checks
                               (K x, K'y, KKT, restarts, termination) in FP64 on FP64 copies;
                               FP64 iterations after the switch (refinement).  This
                               precision split is an extension of this library, not the
                               paper's (the paper is FP64 throughout). */

typedef struct pdlp_ctx* pdlp_handle;

typedef struct {
  double tol;            /* epsilon of the three relative tests (default 1e-4)            */
  int64_t max_iter;      /* PDHG iteration limit (default 1e8)                            */
  double time_limit_s;   /* wall-clock limit of pdlp_solve (default +inf)                 */
  int32_t check_every;   /* iterations between restart/termination checks (default 64)    */
  int32_t scaling;       /* 1: Ruiz + Pock-Chambolle scaling at setup (default 0)         */
  double beta_suff;      /* restart condition 1 factor (Section 2; default 0.2)           */
  double beta_nec;       /* restart condition 2 factor (Section 2; default 0.8)           */
  double beta_art;       /* restart condition 3 factor (Section 2; default 0.36)          */
  double step_scale;     /* eta = step_scale / ||K||_2 (default 0.9)                      */
  double omega_theta;    /* primal-weight smoothing at restarts (default 0.5)             */
  int32_t ruiz_iters;    /* Ruiz passes when scaling (default 10)                         */
  int32_t power_iters;   /* power iterations for ||K||_2 (default 100)                    */
  double eta;            /* > 0: fixed step size instead of step_scale/||K||_2 (default 0)*/
  int32_t tile_slots;    /* SpMV work per warp in 32-row slots; 0 = chosen at setup.
                            When tile_slots, tile_chunks and spmv_batch are all 0 and
                            nnz >= 2^20, setup times 16 candidate schedules per layout
                            and keeps the fastest (results then depend on the choice only
                            through the summation order of split rows)                 */
  int32_t inputs_on_device; /* 1: array arguments are device pointers (default 0)        */
  void* stream;          /* cudaStream_t the caller orders with, or NULL                  */
  int32_t log_capacity;  /* per-check records kept on the device (default 4096)          */
  int32_t tile_chunks;   /* at most this many 32-row chunks per SpMV warp task (1..32);
                            0 = chosen at setup                                           */
  int32_t spmv_batch;    /* SpMV slots whose loads are issued together: 4 or 8; 0 = setup */
  int32_t precision;     /* PDLP_FP64 (default) or PDLP_MIXED (single-LP handles only)    */
  double mixed_switch_tol; /* PDLP_MIXED: FP32 iterations until the FP64-measured largest
                            relative error is <= this (or stops improving for 16 checks),
                            then FP64 iterations; 0 = max(tol, 1e-5)                      */
  int32_t cluster_ctas;    /* pdlp_batch_solve: CTAs that share one LP (a thread-block
                              cluster; each keeps x and y in shared memory and owns a
                              slice of the rows and columns): 1..16, or 0 = automatic
                              (the largest power of two <= 16 whose CTAs for the batch
                              come to at most 4 waves of the GPU's resident CTAs, with
                              >= 64 columns of the largest LP per CTA; with the iterates
                              in global memory at most 4 CTAs and one wave; one CTA per
                              LP when the batch fills the GPU)                             */
  int32_t resident;        /* pdlp_batch_solve: where the iterations find their data.
                              0 = automatic; 1 = x, y in shared memory (one replica per
                              CTA), K and K' streamed; 2 = also each CTA's slice of K, K'
                              and of the row and column vectors copied into shared memory
                              when it fits (automatic: when that keeps the CTAs per SM);
                              3 = x, y in global memory, one copy per LP (automatic when
                              x and y of the largest LP do not fit in shared memory)      */
  int32_t step_rule;       /* pdlp_solve: 0 = the constant step eta of Section 2;
                              1 = the adaptive step rule of the cited PDLP paper
                              (Applegate et al. 2021): an attempt with step eta is kept when
                              eta <= (omega |dx|^2 + |dy|^2 / omega) / (2 |dy' K dx|), and
                              the next eta is min((1 - (s+1)^-0.3) eta_max,
                              (1 + (s+1)^-0.6) eta), s = 1 + steps accepted; a rejected
                              attempt leaves the point unchanged (after adaptive_reject_cap
                              rejections in a row the attempt is kept); first eta = 1 / max |K_ij| of the
                              scaled K (or params.eta); averages are weighted by the kept
                              steps' eta; iteration counts (max_iter, check_every, iters)
                              count attempts.  Not with PDLP_MIXED; not for batches.       */
  int32_t engine;          /* pdlp_solve: 0 = automatic (the persistent engine for an LP of at
                              most 2^18 nonzeros whose x and y fit in one CTA's shared
                              memory, FP64 with the constant step and no time limit; the
                              kernels launched per iteration otherwise), 1 = kernels per
                              iteration, 2 = persistent engine (PDLP_EINVAL when the LP does
                              not qualify).  The persistent engine is the batched solver on
                              the handle's own data: one thread-block cluster runs the
                              whole solve in one launch.                                   */
  int64_t batch_tail_iters; /* pdlp_batch_solve: > 0 runs the batch in two stages: every LP
                              stops (resumably, at a check) after this many iterations; the
                              LPs that did not finish then continue in a second launch with
                              teams sized for their number (cluster_ctas 0).  The result is
                              the uninterrupted solve's up to summation order.  0 = one launch */
  int32_t host_layout;     /* setup: 0 = the SELL layouts are built on the device from the
                              caller's arrays (the host only orders rows and columns);
                              1 = built entirely on the host (the reference builder: the
                              same layouts, slower for large inputs)                       */
  int32_t spmv_stage;      /* setup, FP64 products of K and K': how a warp reads its slots'
                              values and column indices.  1 = coalesced global loads;
                              2 / 3 = staged in shared memory by one-dimensional bulk copies
                              (cp.async.bulk, 8 slots per buffer, 2 / 3 buffers per warp),
                              so that the load path serves only the gathers; 0 = chosen by
                              the setup autotuner when it runs (nnz >= 2^20 and no explicit
                              schedule), else 1.  All give bit-identical products for one
                              task plan.  A staged kernel whose bounded wait gives up makes
                              the call return PDLP_ETIMEOUT and the handle unusable.      */
  int32_t batch_tune;      /* pdlp_batch_solve, when cluster_ctas and resident are both 0
                              (automatic) and the batch is FP64: 0 = the first solve of the
                              handle runs the online autotuner and later solves keep its
                              choice; 1 = no tuning (the team-size rule above); 2 = tune
                              again on this solve.  The autotuner times candidates on the
                              solve's own iterations: after a first slice of check_every
                              iterations of every LP (the rule's choice), each candidate
                              runs the next slice of every LP still running as one resumed
                              launch and is scored by stored bytes of the iterations run
                              per second.  Candidates: the rule's team size with each
                              placement that fits (streamed or resident slices; global
                              iterates when x and y do not fit in shared memory), then
                              team sizes doubled while the score improves (or halved when
                              the first doubling loses); at most 8, and only while at
                              least half of the LPs are still running.  The fastest runs
                              the rest.  Results equal the untuned solve's up to
                              summation order.  An FP64 one-stage solve that keeps a choice
                              (or has fixed ones) runs its persistent launch as a CUDA
                              graph.                                                     */
  int32_t mixed_values;    /* PDLP_MIXED, single-LP handles: how the FP32 products read K.
                              0 = automatic: when every entry of the caller's K is +1, -1
                              (or 0), no values are stored for them: each column index
                              carries the entry's sign in its top bit, and the FP32
                              iterations run in the unscaled variables (D_c x, D_r y for
                              K = D_r K0 D_c), where the scaling is a per-row factor
                              D_c^2 (D_r^2) of the step; otherwise FP32 copies of the
                              scaled values.  1 = FP32 value copies always.  2 = sign bits
                              (PDLP_EINVAL when an entry is not +1, -1 or 0).  The FP64
                              checks and the FP64 refinement use the FP64 values in every
                              case.                                                      */
  int32_t adaptive_reject_cap; /* step_rule 1: an attempt is kept after this many rejections
                              in a row (default 64; a safeguard of this implementation, the
                              cited rule has none; 0 keeps every attempt).  Read by
                              pdlp_solve from its params.                                */
} pdlp_params;

typedef struct {
  int32_t status;        /* PDLP_OPTIMAL / ITER_LIMIT / TIME_LIMIT / NUMERICAL             */
  int32_t which;         /* returned point: 0 current iterate, 1 average of the inner loop */
  int64_t iters;         /* PDHG iterations taken (k)                                      */
  int64_t restarts;
  double primal_obj;     /* c'x of the returned point                                      */
  double dual_obj;       /* q'y + l'lambda^+ - u'lambda^- of the returned point            */
  double rel_primal;     /* ||(Ax-b, [h-Gx]^+)|| / (1 + ||q||)                             */
  double rel_dual;       /* ||c - K'y - lambda|| / (1 + ||c||)                             */
  double rel_gap;        /* |dual - primal| / (1 + |dual| + |primal|)                      */
  double kkt_omega;      /* KKT_omega of the returned point on the scaled problem          */
  double omega;          /* final primal weight                                            */
  double eta;            /* step size                                                      */
  double solve_s;        /* host wall time of pdlp_solve                                   */
  double device_ms;      /* device time from the first to the last kernel of the solve     */
  int64_t launches;      /* kernels launched on the device by this solve                  */
  int64_t fp32_iters;    /* PDLP_MIXED: iterations run in FP32 (the rest ran in FP64)     */
  int64_t accepted;      /* steps kept (step_rule 1; equals iters with the constant step) */
} pdlp_result;

/* Per-check record (pdlp_get_log). */
typedef struct {
  int64_t k;             /* iteration count at the check                                   */
  int64_t t;             /* inner-loop length at the check                                 */
  int32_t restart;       /* 0 none, 1 sufficient decay, 2 necessary decay, 3 long loop     */
  int32_t candidate;     /* 0 current iterate, 1 average                                   */
  double omega;          /* primal weight used at this check                               */
  double kkt_cur, kkt_avg, kkt_anchor;
  double rel_primal, rel_dual, rel_gap;  /* of the better of the two points                */
} pdlp_check_record;

/* Static description of the device layout (pdlp_get_info). */
typedef struct {
  int64_t m, n, m1, nnz;
  int64_t slots_K, slots_Kt;   /* 32-wide slots stored for K and K' (nnz plus padding)/32 */
  int64_t tasks_K, tasks_Kt;   /* warp tasks per SpMV                                      */
  int64_t split_chunks_K, split_chunks_Kt;
  int32_t tile_slots_K, tile_slots_Kt;
  int32_t tile_chunks_K, tile_chunks_Kt;
  int32_t spmv_batch_K, spmv_batch_Kt;
  double algorithmic_bytes_per_iter; /* unique-bytes model: 24 nnz + 68 (m + n)         */
  double stored_bytes_per_iter;      /* the same with padding slots counted               */
  double eta, omega0, norm_K;
  int32_t batch_team;          /* batch handles: CTAs per LP of the last pdlp_batch_solve    */
  int32_t batch_resident;      /* batch handles, last launch: 0 replicas, 1 resident slices,
                                  3 iterates in global memory                                 */
  int32_t wide_rows_K;         /* rows of K stored spread over a chunk's lanes (dense rows)   */
  int32_t batch_resumed;       /* batch handles: LPs continued in the second stage of the last
                                  pdlp_batch_solve (batch_tail_iters > 0)                     */
  /* wall time of the setup phases (ms): copy and checks of the input; the host's part of
     the layout (row and column order, chunk shapes; with host_layout = 1 the whole
     layout); the device's part (layout fill, upload, scaling); the SpMV autotuner
     (single-LP handles); the step size and primal weight (power iteration) with the rest
     of the setup */
  double setup_validate_ms, setup_layout_ms, setup_device_ms, setup_tune_ms, setup_step_ms;
  int32_t spmv_stage_K, spmv_stage_Kt;   /* how the FP64 products read the value / index
                                            stream: 1 coalesced loads, 2 / 3 staged in shared
                                            memory by bulk copies (see pdlp_params)        */
  int32_t batch_tuned;         /* batch handles: candidates the last pdlp_batch_solve timed
                                  (0 when it did not tune); the first 8 of them:           */
  int32_t tune_team[8];        /*   CTAs per LP                                            */
  int32_t tune_resident[8];    /*   placement (1 streamed, 2 resident slices, 3 global)    */
  double tune_gbs[8];          /*   score: stored bytes of the iterations run per second,
                                    in GB/s                                                */
  int32_t mixed_values;        /* how the FP32 products read K: 0 FP64 handle (no FP32
                                  products), 1 FP32 value copies, 2 sign bits (pdlp_params) */
} pdlp_info;

/* Fills p with the defaults listed above. */
void pdlp_default_params(pdlp_params* p);

/* Builds a solver handle for the LP (K, c, q, l, u, m1).
 *   m, n     : rows and columns of K (m >= 0, n >= 1), 0 <= m1 <= m.
 *   row_ptr  : int64[m+1], CSR row offsets, row_ptr[0] = 0, nondecreasing.
 *   col_idx  : int32[nnz], column of each entry, 0 <= col < n (nnz = row_ptr[m] < 2^31).
 *   val      : double[nnz], finite.
 *   c, l, u  : double[n]; l_j <= u_j, l_j in R or -INFINITY, u_j in R or +INFINITY.
 *   q        : double[m], finite.
 *   p        : parameters (NULL = defaults).
 * Copies every input (the matrix arrays straight to the device, where the entries are
 * checked and the layouts filled; p->host_layout = 1 builds them on the host instead);
 * builds the length-sorted device layout of K and K', scales
 * (if p->scaling), estimates ||K||_2 and sets eta and the initial primal weight
 * (Section 2 leaves both open: eta = step_scale/||K||_2, omega0 = ||c||/||q||).
 * On success *out owns all device memory of the solver.
 * Errors: PDLP_EINVAL, PDLP_ENOMEM, PDLP_ECUDA; *out is set to NULL on failure. */
int pdlp_setup(pdlp_handle* out, int64_t m, int64_t n, int64_t m1, const int64_t* row_ptr,
               const int32_t* col_idx, const double* val, const double* c, const double* q,
               const double* l, const double* u, const pdlp_params* p);

/* Runs restarted PDHG from (x0, y0) (NULL = 0, projected onto X and Y) with initial
 * primal weight omega0 (<= 0 = the setup value).  tol, max_iter, time_limit_s,
 * check_every and the restart factors are taken from p (NULL = the setup params).
 * Writes the result to *res and the returned point to x_out[n], y_out[m] (either may
 * be NULL).  Each call starts a new solve (iteration count 0).
 * Errors: PDLP_EINVAL (NULL handle, bad parameter), PDLP_ECUDA. */
int pdlp_solve(pdlp_handle h, const pdlp_params* p, const double* x0, const double* y0,
               double omega0, pdlp_result* res, double* x_out, double* y_out);

/* Releases everything the handle owns.  NULL is allowed. */
void pdlp_free(pdlp_handle h);

/* Text of the handle's last error ("" if none); NULL = last failure of pdlp_setup or
 * pdlp_spmv_csr_noalloc on this thread.  The string stays valid until the next call
 * on the handle. */
const char* pdlp_last_error(pdlp_handle h);

/* Copies the solver's state after pdlp_solve: which = 0 current iterate, 1 average of
 * the current inner loop (the current iterate if it is empty), 2 restart anchor
 * z^{n,0}.  Unscaled, original order; x[n], y[m] (either may be NULL). */
int pdlp_get_iterate(pdlp_handle h, int32_t which, double* x, double* y);

/* Iteration counts at which the last solve restarted; returns how many restarts
 * happened (copies at most cap of them), or a negative error code. */
int64_t pdlp_get_restarts(pdlp_handle h, int64_t* iters, int64_t cap);

/* Per-check records of the last solve; returns the number of checks made (copies
 * at most cap, and at most log_capacity were kept), or a negative error code. */
int64_t pdlp_get_log(pdlp_handle h, pdlp_check_record* rec, int64_t cap);

/* out = K in (transpose = 0: in[n], out[m]) or out = K' in (transpose = 1: in[m],
 * out[n]) for the ORIGINAL (unscaled) K, computed by the solver's SpMV kernels on its
 * scaled device copy (in is divided by the scaling on the way in, out multiplied
 * back on the way out; with scaling off the kernels see the input values as given). */
int pdlp_spmv(pdlp_handle h, int32_t transpose, const double* in, double* out);

/* Bound duals lambda = proj_Lambda(c - K'y) of a dual point y (Section 2: Lambda_j is
 * {0}, R^-, R^+ or R as l_j, u_j are infinite or finite), on the original (unscaled)
 * problem; the solver does not return lambda with the point.  y: m doubles, lambda_out:
 * n doubles (both host arrays, or device arrays when the setup's params.inputs_on_device
 * = 1).  Single-LP handles only.
 * Errors: PDLP_EINVAL (NULL pointers, batch handle), PDLP_ECUDA. */
int pdlp_bound_duals(pdlp_handle h, const double* y, double* lambda_out);

/* Layout, step size and byte model of the handle. */
int pdlp_get_info(pdlp_handle h, pdlp_info* info);

/* Runs `iters` plain PDHG iterations (no checks, no restarts) on the handle's current
 * state and returns, through ms_primal / ms_dual (may be NULL), the average device
 * time of one primal kernel (K'y SpMV fused with the primal step) and of one dual
 * kernel (K x SpMV fused with the dual step), each timed with CUDA events recorded
 * on the handle's stream around every launch. */
int pdlp_time_iterations(pdlp_handle h, int64_t iters, double* ms_primal, double* ms_dual);

/* ---------------------------------------------------------------- checkpoint / resume
 * (no counterpart in the paper).  A single-LP FP64 solve that ran the kernels per
 * iteration (engine 1, or engine 0 when the persistent engine was not chosen) can be saved
 * after it returns and continued later, on this handle or on another handle set up from
 * the same LP with the same setup parameters:
 *   pdlp_state_size(h)              bytes of the state of h's last solve (< 0: error code);
 *   pdlp_get_state(h, buf, size)    copies it into the caller's host buffer (size must be
 *                                   pdlp_state_size(h)); opaque, for this build only;
 *   pdlp_solve_resume(h, p, state, size, res, x_out, y_out)
 *                                   loads `state` (host bytes from pdlp_get_state; NULL:
 *                                   continue from h's own last solve), repeats the check that
 *                                   ended it as an ordinary check (restart rule and primal
 *                                   weight of Section 2), then runs check intervals until
 *                                   p->max_iter iterations in total or termination; results as
 *                                   pdlp_solve.  The state holds x, y, their running sums, the
 *                                   restart anchor, K x and the scalar state (k, t, omega, eta,
 *                                   KKT anchors, counters, the adaptive rule's state), the
 *                                   restart iterations and the per-check records.
 * A solve that stopped at an iteration limit that is a multiple of check_every, resumed
 * with the same parameters and a larger max_iter, gives the uninterrupted solve's iterates
 * bit for bit (the same SpMV schedule on both handles).  A solve stopped by its time limit
 * ended with one more (forced) check, so resuming it continues correctly but not bit for
 * bit.
 * Errors: PDLP_EINVAL for batch handles, MIXED handles, a last solve on the persistent
 * engine, engine 2, a buffer of the wrong size, or a state of other LP sizes.  */
int64_t pdlp_state_size(pdlp_handle h);
int pdlp_get_state(pdlp_handle h, void* buf, int64_t size);
int pdlp_solve_resume(pdlp_handle h, const pdlp_params* p, const void* state, int64_t size, pdlp_result* res,
                      double* x_out, double* y_out);

/* ---------------------------------------------------------------- batches
 * Many independent LPs solved by one persistent kernel launch: each team of the launch
 * (one CTA, or a thread-block cluster of up to 16 CTAs that split the LP's rows and
 * columns; params.cluster_ctas) takes LPs from a queue (largest first) and runs the
 * whole restarted PDHG of one LP (power iteration for eta, iterations, checks,
 * restarts, termination).  x and y live in shared memory (a replica per CTA) when
 * (n + m, each rounded up to a multiple of 32) * 8 bytes + 9 KB fits the per-block
 * limit (about 27,000 rows plus columns), else in global memory (one copy per LP);
 * params.resident selects this by hand.  params.precision = PDLP_MIXED runs FP32
 * iterations with FP64 checks, the LPs it leaves unfinished continue in FP64;
 * params.batch_tail_iters moves long-running LPs to a second launch on teams. */

/* Sets up a batch of `count` LPs given back to back:
 *   m[count], n[count], m1[count] : host arrays of each LP's sizes (m1 <= m, n >= 1).
 *   row_ptr : the LPs' CSR row pointers one after the other, each starting at 0
 *             (sum of (m_b + 1) entries);
 *   col_idx, val : their entries one after the other (sum of nnz_b), columns local to the LP;
 *   c, l, u : sum of n_b entries;  q : sum of m_b entries.
 * Scaling (Ruiz + Pock-Chambolle per LP when params.scaling) runs at setup; eta and
 * omega0 are computed per LP inside the solve.  The same handle type as pdlp_setup;
 * free it with pdlp_free.  Single-LP calls on it (pdlp_solve, pdlp_get_iterate,
 * pdlp_time_iterations) return PDLP_EINVAL; pdlp_spmv applies the block-diagonal K.
 * Errors: PDLP_EINVAL (sizes, CSR, bounds), PDLP_ENOMEM, PDLP_ECUDA. */
int pdlp_batch_setup(pdlp_handle* out, int64_t count, const int64_t* m, const int64_t* n, const int64_t* m1,
                     const int64_t* row_ptr, const int32_t* col_idx, const double* val, const double* c,
                     const double* q, const double* l, const double* u, const pdlp_params* p);

/* Solves every LP of the batch from (x0, y0) projected onto X and Y (NULL = 0 for
 * every LP, the cold start) with initial primal weights omega0[count] (NULL or <= 0 =
 * ||c||/||q|| of the LP), using the tolerance, iteration limit, check interval and
 * restart factors of p (NULL = setup params; time_limit_s is not used; precision is the
 * setup's).  x0 (sum n_b)
 * and y0 (sum m_b) are back to back in the caller's order, unscaled.  res[count]
 * receives one result per LP (solve_s and device_ms are those of the whole batch);
 * x_out and y_out (either may be NULL) receive the returned points, back to back. */
int pdlp_batch_solve(pdlp_handle h, const pdlp_params* p, const double* x0, const double* y0, const double* omega0,
                     pdlp_result* res, double* x_out, double* y_out);

/* Iteration counts at which LP `lp` (0 <= lp < count) of the last pdlp_batch_solve
 * restarted (Section 2, restart criteria); the first 256 restarts of each LP are kept.
 * Copies at most cap of them into the host array iters (may be NULL) and returns how
 * many restarts the LP made, or a negative error code (PDLP_EINVAL: not a batch handle,
 * lp out of range, or no solve yet). */
int64_t pdlp_batch_get_restarts(pdlp_handle h, int64_t lp, int64_t* iters, int64_t cap);

/* ---------------------------------------------------------------- dense kernels
 * C[M x N] = A[M x K] * B[N x K]^T (+ bias[N], then max(., 0) if relu) on the tcgen05
 * tensor cores: A and B BF16 row-major (K contiguous) device arrays with 16-byte aligned
 * bases, C FP32 row-major device array, bias FP32 device array or NULL.  M and N
 * multiples of 128, K a multiple of 64.  The operand tiles are copied by the tensor
 * memory accelerator into a shared-memory ring (2 to 6 stages) that one thread refills
 * while another issues the MMAs; a CTA computes one or two 128-row tiles of C against
 * each 128-column tile of B.  Used by the learned warm start (an extension: the paper has
 * no learned component); exposed for testing.  Runs on `stream` (NULL = default) and
 * waits for it; allocates no device memory (its error flag is a device variable of the
 * library).  Errors: PDLP_EINVAL (shapes, alignment), PDLP_ECUDA, PDLP_ETIMEOUT (an
 * mbarrier wait gave up). */
int pdlp_tc_gemm(int32_t M, int32_t N, int32_t K, const void* A, const void* B, float* C, const float* bias,
                 int32_t relu, void* stream);

/* pdlp_tc_gemm with K cut into `splits` slices (>= 1; fewer when K / 64 does not give
 * that many non-empty slices), each computed by its own CTAs into the caller's device
 * array workspace (splits * M * N floats), then added in slice order (+ bias, ReLU) into
 * C.  For products with few 128 x 128 output tiles and a long K.  The MLP uses this path
 * internally.  Errors as pdlp_tc_gemm; PDLP_EINVAL also for splits < 1, or a NULL
 * workspace with splits > 1. */
int pdlp_tc_gemm_split(int32_t M, int32_t N, int32_t K, const void* A, const void* B, float* C, const float* bias,
                       int32_t relu, int32_t splits, float* workspace, void* stream);

/* Self-test of the bounded device waits (no counterpart in the paper): one 128 x 128 x 64
 * tile of pdlp_tc_gemm's kernel (A: 128 x 64 and B: 128 x 64 BF16, C: 128 x 128 FP32,
 * device arrays) with its operand copies withheld, so the MMA thread's first mbarrier
 * wait can only give up after spin_limit polls (>= 1).  The kernel then records the
 * failure, frees its tensor memory and returns; nothing faults and the context stays
 * usable.  Returns PDLP_ETIMEOUT when the wait gave up (the expected outcome), PDLP_OK
 * if it did not, PDLP_EINVAL / PDLP_ECUDA otherwise.  C is not written. */
int pdlp_tc_gemm_wait_selftest(const void* A, const void* B, float* C, int64_t spin_limit, void* stream);

/* ---------------------------------------------------------------- warm-start network
 * A 3-layer MLP for learned warm starts (an extension; the paper has no
 * learned component):  Y = relu(relu(X W1' + b1) W2' + b2) W3' + b3,
 * W1 [hidden x n_in], W2 [hidden x hidden], W3 [n_out x hidden], row-major FP32 masters.
 * Every product runs on the tcgen05 tensor cores with BF16 operands and FP32
 * accumulation (pdlp_tc_gemm's kernel); the BF16 points are X, W1..W3 and the hidden
 * activations.  Training minimises the mean squared error
 *   L = sum over rows r and outputs o of (Y_ro - T_ro)^2 / (2 rows n_out)
 * with AdamW (beta 0.9, 0.999, eps 1e-8, weight decay on the weights only).
 * All arrays of these calls are host arrays; data rows are selected by index. */
typedef struct pdlp_mlp_ctx* pdlp_mlp;

/* hidden: a multiple of 128; max_batch: the most rows one call handles. */
int pdlp_mlp_create(pdlp_mlp* out, int32_t n_in, int32_t hidden, int32_t n_out, int32_t max_batch);
void pdlp_mlp_free(pdlp_mlp h);
const char* pdlp_mlp_last_error(pdlp_mlp h);
/* Sets the parameters (unpadded shapes as above) and clears the optimiser state. */
int pdlp_mlp_set_params(pdlp_mlp h, const float* W1, const float* b1, const float* W2, const float* b2,
                        const float* W3, const float* b3);
int pdlp_mlp_get_params(pdlp_mlp h, float* W1, float* b1, float* W2, float* b2, float* W3, float* b3);
/* Copies a dataset to the device: X [count x n_in], T [count x n_out] (T may be NULL
 * for inference only). */
int pdlp_mlp_load_data(pdlp_mlp h, int64_t count, const float* X, const float* T);
/* Y [rows x n_out] = network(X[idx[r]]), rows <= max_batch. */
int pdlp_mlp_forward(pdlp_mlp h, int32_t rows, const int32_t* idx, float* Y);
/* Loss and gradients of L on the rows idx (no update); any output may be NULL. */
int pdlp_mlp_gradients(pdlp_mlp h, int32_t rows, const int32_t* idx, double* loss, float* gW1, float* gb1,
                       float* gW2, float* gb2, float* gW3, float* gb3);
/* `epochs` passes over the loaded data in minibatches of `batch` rows (order shuffled
 * per epoch from `seed`; a last partial batch is skipped); epoch_loss[epochs] receives
 * the mean minibatch loss, train_ms the device time. */
int pdlp_mlp_train(pdlp_mlp h, int32_t epochs, int32_t batch, float lr, float weight_decay, uint64_t seed,
                   double* epoch_loss, double* train_ms);

/* y = K x for a CSR matrix held in the caller's device memory, with no device memory
 * allocated by the call.  This entry point has no counterpart in the paper; it is for
 * callers that cannot call cudaMalloc at the point where they need the product, for
 * example an application whose device memory is all handed to its own pool allocator,
 * or a latency-bound loop that must not take cudaMalloc's implicit device
 * synchronisation.  It needs no handle.
 *   m, n, nnz : rows, columns and nonzeros of K (m < 2^31, n >= 1).
 *   row_ptr   : int64[m+1] device array, row_ptr[0] = 0, nondecreasing, row_ptr[m] = nnz.
 *   col_idx   : int32[nnz] device array, 0 <= col < n;  val: double[nnz] device array.
 *   x         : double[n] device array;  y: double[m] device array (output, overwritten).
 *               y must not overlap x, row_ptr, col_idx or val: threads write rows of y
 *               while others still read x (y == x is rejected with PDLP_EINVAL).
 *   stream    : cudaStream_t to run on (NULL = the default stream); the call returns
 *               without waiting, y is ready when the stream reaches that point.
 * Scratch: partial sums of rows that cross thread boundaries live in one fixed 8 MiB
 * device array of the library, which every GPU that uses this call keeps until the
 * process exits.  It limits nnz to 22,369,600; larger inputs return PDLP_EINVAL with a
 * message in pdlp_last_error(NULL), before any device work.  The first call on a device
 * looks up that array's device address (with the device current) and keeps it for the
 * device: it belongs to the device's primary context, the one the CUDA runtime uses, so
 * callers must use the runtime's context and must not reset the device
 * (cudaDeviceReset) between calls; make that first call before any stream capture.  Every call on a device shares the array, so calls that
 * overlap on the GPU (different streams, or different host threads) race and give wrong
 * results; the call writes every scratch entry it later reads, so nothing needs clearing.
 * The same 1e-13 relative agreement with pdlp_spmv holds (summation order differs).
 * Cost: each thread reads 64 consecutive nonzeros, so the loads are not coalesced
 * across a warp; a row longer than 64 entries is finished by one thread that adds its
 * ~L/64 run partials one after the other, so a single very long row (L ~ 1e7) makes
 * the call serial in that row.  pdlp_spmv is the fast path for repeated products.
 * Errors: PDLP_EINVAL (sizes, null arrays, y == x), PDLP_ECUDA (no device, launch failure). */
int pdlp_spmv_csr_noalloc(int64_t m, int64_t n, int64_t nnz, const int64_t* row_ptr,
                          const int32_t* col_idx, const double* val, const double* x, double* y,
                          void* stream);

#ifdef __cplusplus
}
#endif
#endif
