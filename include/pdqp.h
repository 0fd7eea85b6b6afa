/*
 * pdqp.h -- C ABI of a GB300 (sm_103a) solver for convex quadratic programs by
 * restarted accelerated primal-dual hybrid gradient (rAPDHG).
 *
 * The method is Algorithm 1 of Lu & Yang, "A Practical and Optimal First-Order
 * Method for Large-Scale Convex Quadratic Programming" (Section 2), run with
 * the practical rules of its Section 6 (PDQP adaptive restart, adaptive step
 * size, primal weight) and the diagonal preconditioning and relative-KKT
 * progress metric of its Section 5.
 *
 * Problem form.  The paper states eq. (1) as  min 1/2 x'Qx + c'x  s.t. Ax <= b
 * and notes (footnote to eq. (1)) that its results extend to other QP forms.
 * This library takes the form
 *
 *     min 1/2 x'Qx + c'x   s.t.  A[0:m_eq]  x  = b[0:m_eq]
 *                                A[m_eq:m] x >= b[m_eq:m]
 *                                l <= x <= u
 *
 * with the saddle function L(x,y) = 1/2 x'Qx + c'x - y'(Ax - b) of eq. (2)
 * (A' = -A, b' = -b), x in [l,u] and y in R^{m_eq} x R_+^{m-m_eq}.
 *
 * Conventions common to every call
 *   - Sparse matrices are CSR: rowptr int32[rows+1] (rowptr[0] = 0,
 *     non-decreasing), col int32[nnz] strictly increasing inside each row and in
 *     [0, cols), values float64[nnz], all finite.  Q is square n x n, symmetric
 *     positive semidefinite and stored in full (both triangles).
 *   - `mem_space` says where the caller's pointers live: PDQP_MEM_HOST (0) for
 *     host memory, PDQP_MEM_DEVICE (1) for device memory of the current CUDA
 *     device (for example a torch CUDA tensor's data_ptr()).
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Every
 *     call enqueues its device work on that stream; calls that return results
 *     to the host synchronise it before returning.
 *   - The library copies everything it is given; the caller keeps ownership of
 *     its arrays and may free them once the call returns.  Outputs are written
 *     into caller-owned buffers.
 *   - Errors are returned as pdqp_status, never thrown; pdqp_last_error()
 *     describes the most recent error of a handle.  A handle is not thread
 *     safe; distinct handles are independent.
 */
#ifndef PDQP_H
#define PDQP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pdqp_problem *pdqp_handle;

typedef enum {
  PDQP_OK = 0,
  PDQP_ERR_INVALID = 1,      /* malformed input (bad CSR, l > u, NaN, m_eq > m, ...) */
  PDQP_ERR_CUDA = 2,         /* a CUDA runtime call failed */
  PDQP_ERR_OOM = 3,          /* device or host allocation failed */
  PDQP_ITER_LIMIT = 10,      /* max_iter reached; the best iterate is returned */
  PDQP_TIME_LIMIT = 11,      /* time_limit reached; the best iterate is returned */
  PDQP_NUMERICAL = 12,       /* NaN or Inf met in the relative KKT error */
  PDQP_DEVICE_TIMEOUT = 13,  /* a bounded device wait gave up */
  /* with options.detect_infeasibility (not in the paper): a certificate was
   * found and is returned in place of the iterate, unscaled, for the original
   * problem.  PRIMAL_INFEASIBLE: y_out holds a Farkas ray y, y_I >= 0, with
   * b'y - sup_{l<=x<=u} (A'y)'x = 1 on the part of A'y the box bounds, the rest
   * of A'y within eps_infeasible; x_out is 0.  DUAL_INFEASIBLE: x_out holds a
   * direction d of the box's recession cone with c'd = -1 and Qd, A_E d and
   * the negative part of A_I d within eps_infeasible; y_out is 0. */
  PDQP_PRIMAL_INFEASIBLE = 14,
  PDQP_DUAL_INFEASIBLE = 15
} pdqp_status;

enum { PDQP_MEM_HOST = 0, PDQP_MEM_DEVICE = 1 };
enum { PDQP_PREC_FP64 = 0, PDQP_PREC_MIXED = 1 };
enum { PDQP_STEP_ADAPTIVE = 0, PDQP_STEP_THEORY = 1 };
enum { PDQP_RESTART_PDQP = 0, PDQP_RESTART_HALVING = 1, PDQP_RESTART_FIXED = 2,
       PDQP_RESTART_NONE = 3 };

typedef struct {
  /* PDQP_PREC_FP64: every step in float64.  PDQP_PREC_MIXED: float32 matrix
   * values, vectors and SpMVs in the iteration; float64 relative-KKT
   * reductions, restart decisions and a float64 residual correction at every
   * restart (not in the paper). */
  int32_t precision;
  /* PDQP_STEP_ADAPTIVE: Section 6 step size eta^{n,k} with primal weight
   * omega (primal step eta/omega, dual step eta*omega).  PDQP_STEP_THEORY:
   * Theorem 1's eta_k = (k+1)/(2(||Q||+K||A||)), tau_k = (k+1)/(2K||A||)
   * with K = fixed_K. */
  int32_t step_rule;
  /* PDQP_RESTART_PDQP: Section 6 conditions (i)-(iii).  _HALVING: Section 5
   * adaptive scheme relKKT(z_bar) <= relKKT(z^{n,0})/2.  _FIXED: after
   * fixed_K inner iterations (taken at the first check with k >= fixed_K).
   * _NONE: never restart. */
  int32_t restart_rule;
  int32_t accelerate;        /* 0: beta_k = theta_k = 1 (plain PDHG, Section 5 "Algorithms") */
  int32_t scaling;           /* Section 5 "Preprocessing" on/off */
  int32_t ruiz_iters;        /* 10 */
  int32_t l2_scaling;        /* 1 */
  int32_t pock_chambolle;    /* 1 (alpha = 1) */
  int32_t fixed_K;           /* restart length for _FIXED and the theory step rule */
  int32_t check_period;      /* iterations between relKKT checks (even; default 64) */
  int64_t max_iter;          /* 200000 (Section 5) */
  double eps;                /* relKKT termination tolerance eq. (terminate); 1e-6 */
  double time_limit;         /* seconds; 3600 (Section 6.1) */
  double beta_suff, beta_nec, beta_art;   /* 0.2, 0.8, 0.36 (Section 6) */
  double pw_theta;           /* 0.2: primal-weight smoothing (Section 6) */
  double eps_zero;           /* 1e-10 */
  double norm_A, norm_Q;     /* > 0: use these spectral norms of the SCALED
                                matrices; <= 0: estimate them by the Lanczos method */
  int32_t norm_iters;        /* Lanczos step limit, 1..512 (default 500) */
  double norm_tol;           /* stop when the largest Ritz value changes by <= this
                                relative (default 1e-6) */
  int32_t spmv_threads;      /* iteration-kernel variant: 256 or 512 threads per row
                                block, 1 = pipelined persistent (cp.async prefetch of
                                the next row block), 2 = a whole chunk of iterations
                                in one launch of a 16-CTA thread-block cluster (8 where
                                16 cannot be resident) with a
                                cluster barrier after each half-step (problems of at
                                most 64 row blocks of A and of P, no row longer than a
                                row block, no low-rank term; else PDQP_ERR_INVALID),
                                3 = family handles (pdqp_create_family; no row longer
                                than a row block, no low-rank term; else
                                PDQP_ERR_INVALID): the iteration vectors interleaved
                                by member, v[j * members + i], one warp per row for 32
                                members, so one matrix entry meets 128 members in one
                                coalesced load,
                                0 = autotuned: 3 for an eligible family handle, else
                                the first full chunk of a handle's first solve in each
                                precision times two rounds of 3 iterations of each
                                eligible variant and keeps the fastest for that
                                precision; the choice is also kept for the process per
                                problem shape, so later handles of the same sizes,
                                nonzeros and row blocks start with it (all variants
                                give bitwise identical iterates) */
  int32_t no_graphs;         /* 0: replay each full chunk of check_period iterations
                                and its check as one captured CUDA graph; 1: launch
                                every kernel directly */
  /* 1: at every check, after the termination and iteration-limit tests, the
   * current and the average iterate's displacement from the epoch's first
   * iterate (projected onto the recession cones of the box and of the dual
   * set) are tested as infeasibility certificates, each to eps_infeasible
   * relative to its own objective term (Farkas value b'y - sup (A'y)'x, or
   * |c'd|); the first that passes ends the solve with PDQP_PRIMAL_INFEASIBLE
   * (tested first) or PDQP_DUAL_INFEASIBLE.  Not in the paper; default 0.
   * Best effort: a problem whose rays do not settle to eps_infeasible ends as
   * without it (iteration limit or numerical error). */
  int32_t detect_infeasibility;
  double eps_infeasible;     /* 1e-8 */
  /* 1: maintained products (Section 2: the updates of Algorithm 1 are
   * linear).  The iteration carries A x and A x_bar of the primal iterate and
   * Q x_bar, A'y and A'y_bar along with the iterates: the dual half-step
   * gathers x^k and forms A x_tilde^k = A x^k + theta_k (A x^k - A x^{k-1}),
   * the primal half-step gathers x^k and y^{k+1} and forms
   * Q x_md^k = (1 - 1/beta_k) Q x_bar^k + Q x^k / beta_k, and a check needs one
   * gather of x for A x and one for Q x (the next iteration starts from those
   * two products) instead of the products of both iterates with A, Q and A'.
   * The iterates equal the default's in exact arithmetic; their rounding
   * differs.  Needs precision PDQP_PREC_FP64, spmv_threads 0 or 256 (the
   * 256-thread row-block kernels run), no low-rank term and no row longer
   * than a row block, and no state loaded by pdqp_set_state: else the solve
   * returns PDQP_ERR_INVALID.  A family handle runs the row-block kernels.
   * pdqp_get_state after such a solve returns PDQP_ERR_INVALID (the state
   * holds no x_md, x_tilde).  Not in the paper; default 0. */
  int32_t maintained_products;
} pdqp_options;

typedef struct {
  int32_t status;            /* pdqp_status of the solve */
  int64_t iterations;        /* total inner iterations */
  int64_t restarts;
  double rel_kkt, r_primal, r_dual, r_gap;   /* of the returned iterate, original problem */
  double primal_obj, dual_obj;
  double seconds;            /* wall time of the call */
  double norm_A, norm_Q;     /* spectral norms used (scaled problem) */
  double omega;              /* final primal weight */
  double setup_seconds;      /* device time of scaling + spectral norms (CUDA events) */
  double iterate_seconds;    /* device time from the first iteration to termination */
  int32_t norm_iters;        /* Lanczos steps taken (0 when the norms were given) */
  int32_t spmv_threads;      /* iteration-kernel variant used after the first chunk */
} pdqp_info;

/* Per-kernel device time of the solver's hot loop, measured with CUDA events
 * recorded on the solve's stream around every launch while profiling is on.
 * kind 0 = dual half-step, 1 = primal half-step, 2 = relKKT check + restart,
 * 3 = the one-launch cluster chunk (spmv_threads 2: both half-steps of a
 * chunk's iterations per launch).  Scaling, norms, start point and output are
 * not timed. */
typedef struct {
  int64_t launches[4];
  double ms[4];              /* summed device milliseconds */
  double bytes[4];           /* algorithmic DRAM bytes of one launch (kinds 0, 1, 3): the
                                mean over the timed launches of the bytes of the instances
                                that were running at each launch (kind 3: both half-steps
                                of every iteration in the launch) */
} pdqp_profile;

/* Fill *opt with the defaults listed above. */
void pdqp_default_options(pdqp_options *opt);

/* Human-readable name of a status code (static string). */
const char *pdqp_status_string(int32_t status);

/* Create a problem handle (Section 1 eq. (1) in the form above).
 * n >= 1 variables, m >= 0 rows of which the first m_eq are equalities.
 * Q_*: CSR of Q (n rows); A_*: CSR of A (m rows; may be NULL when m = 0).
 * c, b, l, u: float64[n], [m], [n], [n]; l may hold -INFINITY and u +INFINITY,
 * l <= u elementwise.  The data are validated, copied to device memory and
 * the transpose of A is built.  Returns PDQP_ERR_INVALID with *out = NULL on
 * malformed input. */
pdqp_status pdqp_create(pdqp_handle *out, int64_t n, int64_t m, int64_t m_eq,
                        const int32_t *Q_rowptr, const int32_t *Q_col, const double *Q_val,
                        const int32_t *A_rowptr, const int32_t *A_col, const double *A_val,
                        const double *c, const double *b, const double *l, const double *u,
                        int32_t mem_space, void *stream);

/* Create one handle holding `count` independent problems of uneven sizes
 * (batching is not in the paper: every instance runs Algorithm 1 with the
 * Section 6 rules on its own, as a standalone solve would), stacked
 * block-diagonally (each instance validated and assembled on the host,
 * on up to 16 threads, then copied to the device; pdqp_create_batch_packed
 * builds the same handle on the device).  Every argument is a host array of
 * `count` entries with the meaning of the pdqp_create argument of the same name
 * (the arrays they point to live in `mem_space`).  pdqp_solve on such a handle
 * solves all instances in the same launches, each with its own step sizes,
 * primal weight, restarts and termination; x0/y0/x_out/y_out are then the
 * instances' vectors concatenated in order, the returned status is the largest
 * status code among the instances and pdqp_batch_info gives each instance's
 * summary. */
pdqp_status pdqp_create_batch(pdqp_handle *out, int32_t count, const int64_t *n, const int64_t *m,
                              const int64_t *m_eq, const int32_t *const *Q_rowptr,
                              const int32_t *const *Q_col, const double *const *Q_val,
                              const int32_t *const *A_rowptr, const int32_t *const *A_col,
                              const double *const *A_val, const double *const *c,
                              const double *const *b, const double *const *l, const double *const *u,
                              int32_t mem_space, void *stream);

/* The handle pdqp_create_batch builds from the same instances (same stacking,
 * row blocks and results; not in the paper), from the batch handed over as one
 * block-diagonal problem: with x_i = n[0] + ... + n[i-1] and y_i = m[0] + ... + m[i-1],
 * instance i owns the variables [x_i, x_i + n[i]) and the rows
 * [y_i, y_i + m[i]) of the stack (N = sum n, M = sum m variables and rows).
 * n, m, m_eq: host arrays of `count` entries, as for pdqp_create_batch.
 * Q_*: CSR of the stacked Q, N rows; A_*: CSR of the stacked A, M rows (may be
 * NULL when M = 0); both with global column indices (the block-diagonal
 * matrix of the instances' matrices), each row's columns inside its own
 * instance's variables.  c, l, u: float64[N]; b: float64[M]; the instances'
 * vectors concatenated.  All ten arrays live in `mem_space`; the library
 * copies them.  Validation, the transpose of A and the stacking run on the
 * device; the host reads only the row pointers (to form the row blocks), so
 * the host cost of a call does not grow with the number of nonzeros.  A
 * column of A with more than 4096 nonzeros sends the call to the host
 * stacking of pdqp_create_batch (same handle).  PDQP_ERR_INVALID with
 * *out = NULL on malformed input, a nonzero outside its row's instance
 * included. */
pdqp_status pdqp_create_batch_packed(pdqp_handle *out, int32_t count, const int64_t *n, const int64_t *m,
                                     const int64_t *m_eq, const int32_t *Q_rowptr, const int32_t *Q_col,
                                     const double *Q_val, const int32_t *A_rowptr, const int32_t *A_col,
                                     const double *A_val, const double *c, const double *b, const double *l,
                                     const double *u, int32_t mem_space, void *stream);

/* Number of instances of a handle (1 for pdqp_create). */
int32_t pdqp_batch_count(pdqp_handle h);

/* One handle for `count` members of a parameterised family (not in the
 * paper; a batch whose members share their structure): every member has
 * the same Q, A, l, u (given once, as for pdqp_create) and its own objective
 * and right-hand side, row i of C [count x n] and of B [count x m] (float64,
 * row-major, in `mem_space`).  The handle is the one pdqp_create_batch would
 * build from the same instances (same stacking, row blocks and results); it
 * is built by replicating the shared structure on the device, so its host
 * cost does not grow with count.  Requires count * (nnz(Q) + nnz(A)) < 2^31. */
pdqp_status pdqp_create_family(pdqp_handle *out, int32_t count, int64_t n, int64_t m, int64_t m_eq,
                               const int32_t *Q_rowptr, const int32_t *Q_col, const double *Q_val,
                               const int32_t *A_rowptr, const int32_t *A_col, const double *A_val, const double *C,
                               const double *B, const double *l, const double *u, int32_t mem_space, void *stream);

/* Per-instance summaries of the last pdqp_solve (infos[count], host). */
pdqp_status pdqp_batch_info(pdqp_handle h, pdqp_info *infos, int32_t count);

/* Add a low-rank term to the objective (not in the paper, whose Q is one sparse
 * matrix): Q_total = Q + F F' with F float32,
 * row-major n x r (1 <= r <= 256), applied as F(F'x) (never formed).  The
 * low-rank term is left out of the scaling norms; D2 scales F's rows. */
pdqp_status pdqp_set_lowrank_Q(pdqp_handle h, int32_t r, const float *F, int32_t mem_space,
                               void *stream);

/* Solve (Algorithm 1 with the Section 6 rules) from (x0, y0) -- NULL means the
 * all-zero start of Section 5 -- writing the returned iterate to x_out[n] and
 * y_out[m] (either may be NULL) and the summary to *info (may be NULL).
 * x0, y0, x_out, y_out live in `mem_space`.  Returns PDQP_OK when relKKT <= eps,
 * PDQP_ITER_LIMIT / PDQP_TIME_LIMIT with the best iterate written, or an
 * error.  Synchronises `stream`. */
pdqp_status pdqp_solve(pdqp_handle h, const pdqp_options *opt, const double *x0, const double *y0,
                       double *x_out, double *y_out, pdqp_info *info, int32_t mem_space,
                       void *stream);

/* Solve `count` separate handles with the same options, one after the other
 * on `stream` (for many small problems, one pdqp_create_batch handle solves
 * them together).  Arrays of per-problem pointers (host arrays of pointers; the
 * pointed-to vectors live in `mem_space`); x0/y0/x_out/y_out may be NULL as a
 * whole or per entry.  infos[count] receives one summary per problem.  Returns
 * the worst status. */
pdqp_status pdqp_solve_batch(int32_t count, const pdqp_handle *hs, const pdqp_options *opt,
                             const double *const *x0, const double *const *y0,
                             double *const *x_out, double *const *y_out, pdqp_info *infos,
                             int32_t mem_space, void *stream);

/* Raw iterate state after the last solve, in original coordinates:
 * x, x_bar (n) and y, y_bar (m) of Algorithm 1 (any pointer may be NULL). */
pdqp_status pdqp_get_iterates(pdqp_handle h, double *x, double *y, double *xbar, double *ybar,
                              int32_t mem_space, void *stream);

/* Complete solver state after the last solve, for checkpoint and resume: the
 * iterates and averages of Algorithm 1, the restart anchor z^{n,0}, and the
 * per-instance scalars of Section 6's rules (primal weight omega, the step
 * size eta, the anchor's relKKT, the previous candidate's relKKT, the epoch
 * and total iteration counters, the restart count, the spectral norms), the
 * preprocessing scaling (Section 5) and the step sizes tabulated for the
 * current check period.  In mixed precision it also holds the float64 base
 * and the float32 deltas and shifted data.
 *
 * buf (HOST memory, caller-owned) receives an opaque blob of this library
 * version; with buf = NULL only *bytes is set to the size needed.  On entry
 * *bytes is the capacity of buf, on return the size written.  Needs a solve
 * on the handle first, one without options.maintained_products (else
 * PDQP_ERR_INVALID); synchronises `stream`.  The blob of a batch handle holds
 * every instance. */
pdqp_status pdqp_get_state(pdqp_handle h, void *buf, size_t *bytes, void *stream);

/* Load a state from pdqp_get_state into a handle of the same problem (the
 * same sizes and nonzero counts; a low-rank term set as before).  The next
 * pdqp_solve on the handle continues from it instead of starting afresh: no
 * preprocessing, norm estimate or initial point (x0 and y0 must be NULL), and
 * an instance that the iteration limit stopped runs on (Section 5's
 * termination test is applied again at its next check).  That solve must use
 * the saved solve's precision, check_period, step, restart and primal-weight
 * options (else PDQP_ERR_INVALID) and a larger max_iter (a total count,
 * including the iterations before the save).  It then follows the trajectory
 * an uninterrupted solve would have taken, bit for bit.  The blob is copied;
 * synchronises `stream`.  Errors: PDQP_ERR_INVALID for a blob of another
 * version or problem, or one shorter than its header says. */
pdqp_status pdqp_set_state(pdqp_handle h, const void *buf, size_t bytes, void *stream);

/* Relative KKT error (Section 5 "Progress metric", equality/bound form) of a
 * caller-given (x, y) on the handle's original problem, computed on the
 * device in float64.  parts[6] (host) receives r_primal, r_dual, r_gap,
 * rel_kkt, primal_obj, dual_obj. */
pdqp_status pdqp_kkt(pdqp_handle h, const double *x, const double *y, double *parts,
                     int32_t mem_space, void *stream);

/* Allocation-free relative KKT error, for callers that cannot allocate device
 * memory once running: real-time control loops (an MPC controller re-solving
 * every few milliseconds must not block on the allocator or synchronise the
 * device) and processes held to a fixed device-memory budget after start-up.
 * The paper has no counterpart; it is a variant of pdqp_kkt that needs no
 * handle and calls no cudaMalloc, cudaFree or allocating library routine.
 *
 * All array arguments are DEVICE pointers owned by the caller: the CSR of Q
 * (n rows, nnz_Q entries), of A (m rows) and of its transpose A' (n rows, the
 * same nnz_A entries, columns sorted), c, b, l, u as in pdqp_create, the point
 * (x[n], y[m]) in original coordinates, and parts[6] which receives r_primal,
 * r_dual, r_gap, rel_kkt, primal_obj, dual_obj.  The work is enqueued on
 * `stream` and the call returns without synchronising.
 *
 * Errors: PDQP_ERR_INVALID for bad sizes, a missing array or an array that is
 * not device (or managed) memory, all before any device work.  The CONTENTS
 * of the CSR arrays are not validated: a decreasing row pointer or a column
 * index out of range (>= n for Q and A, >= m for A') is undefined behaviour.
 * PDQP_ERR_CUDA when an error was already pending on the calling thread (it is
 * left in place and nothing is launched) or a launch of this call failed.
 *
 * Limits: n <= 65536 and m <= 65536; larger problems return PDQP_ERR_INVALID
 * before any device work.  The partial sums live in one 2 MiB array in the
 * library's device image that every GPU loading the library holds until the
 * process exits.  The first call on each device looks up that array's device
 * address (cudaGetSymbolAddress) with the device current; make the first call
 * on a device before any stream capture.  Every call zeroes and reuses the
 * same array, so calls whose device work overlaps (on different streams or
 * from different threads) race on it: order them on one stream. */
pdqp_status pdqp_kkt_noalloc(int64_t n, int64_t m, int64_t m_eq,
                             const int32_t *Q_rowptr, const int32_t *Q_col, const double *Q_val,
                             int64_t nnz_Q,
                             const int32_t *A_rowptr, const int32_t *A_col, const double *A_val,
                             const int32_t *At_rowptr, const int32_t *At_col, const double *At_val,
                             int64_t nnz_A, const double *c, const double *b, const double *l,
                             const double *u, const double *x, const double *y, double *parts,
                             void *stream);

/* Sizes of the handle's problem. */
pdqp_status pdqp_get_sizes(pdqp_handle h, int64_t *n, int64_t *m, int64_t *m_eq,
                           int64_t *nnz_Q, int64_t *nnz_A);

/* Last error message of a handle ("" if none); pdqp_last_error(NULL) gives the
 * last error of a failed pdqp_create on this thread. */
const char *pdqp_last_error(pdqp_handle h);

/* Release all device and host memory of a handle (NULL is a no-op). */
void pdqp_destroy(pdqp_handle h);

/* Turn per-kernel event timing on (resetting the counters) or off. */
pdqp_status pdqp_profile_enable(pdqp_handle h, int32_t on);

/* Read the counters accumulated since profiling was turned on. */
pdqp_status pdqp_profile_read(pdqp_handle h, pdqp_profile *out);

/* Kernel launches the library issued since the process started (for
 * reporting how much GPU work a call did). */
int64_t pdqp_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* PDQP_H */
