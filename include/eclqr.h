/*
 * eclqr.h -- C ABI of the GB300 solver for linear equality-constrained LQR
 * problems, following Sousa-Pinto & Orban, "An Efficient Algorithm for Solving
 * Linear Equality-Constrained LQR Problems" (arXiv 2407.05433).
 *
 * Problem (Sec. 2, eq. problem), for each problem j of a batch:
 *
 *   min  sum_{i<N} 1/2 x_i'Q_i x_i + x_i'M_i u_i + 1/2 u_i'R_i u_i + q_i'x_i + r_i'u_i
 *        + 1/2 x_N'Q_N x_N + q_N'x_N
 *   s.t. x_0 = s_0,   x_{i+1} = A_i x_i + B_i u_i + c_i,
 *        C_i x_i + D_i u_i + d_i = 0 (p_i rows),   E_i x_i + e_i = 0 (q_i rows, i = 0..N).
 *
 * The library runs Algorithm 1: base relations and their associative suffix
 * scan (Sec. 3-4), domain parameterisations (eq. state-param), stage-parallel
 * elimination (Sec. 5), the reduced unconstrained LQR (Sec. 6), recovery
 * (eq. recovery-maps) and multipliers (Sec. 7), all in CUDA kernels for sm_103a.
 *
 * Layout.  All problem arrays are FP64, row-major, packed problem after
 * problem and, inside a problem, stage after stage:
 *   A  N*n*n    B  N*n*m    c  N*n
 *   C  (sum_i p_i)*n   D  (sum_i p_i)*m   d  sum_i p_i      (rows of stage i after stage i-1)
 *   E  (sum_{i<=N} q_i)*n   e  sum_{i<=N} q_i                (stage N = terminal rows)
 *   Q  (N+1)*n*n   qv (N+1)*n          (block N is Q_N, q_N)
 *   M  N*n*m       R  N*m*m     rv N*m
 *   s0 n;  outputs x (N+1)*n, u N*m, lam (N+1)*n, mu sum p_i, eta sum q_i, alpha n.
 * State and control dimensions are uniform inside one problem and may differ
 * between problems; constraint row counts vary per stage and may be zero; rows
 * may be dependent or redundant (Sec. 2).  eclqr_layout() returns the total
 * element count of every array.
 *
 * Ownership.  Descriptor arrays are host memory, read during eclqr_create
 * and eclqr_layout only.  Data, s0 and every output are device pointers owned
 * by the caller; the data must stay unchanged from eclqr_build until the last
 * call that uses the handle.  The handle owns its device workspace (the
 * factors T, Y, Z, the reduced problem, the Riccati factors, the scan slots).
 * Every call is asynchronous on the caller's stream (a cudaStream_t passed as
 * void*; NULL = legacy default stream); a handle serves one stream at a time.
 *
 * Errors.  Return values: ECLQR_OK or a negative ECLQR_E* code for API
 * errors detected on the host (bad arguments, allocation or launch failure).
 * Numerical outcomes are per problem, written asynchronously to the caller's
 * device int32 array status[num_problems] (ECLQR_STATUS_*): the first failure
 * seen for a problem is kept.
 */
#ifndef ECLQR_H
#define ECLQR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define ECLQR_OK 0
#define ECLQR_EINVAL (-1)    /* bad descriptor, option or pointer                  */
#define ECLQR_ENOMEM (-2)    /* device allocation failed                           */
#define ECLQR_ECUDA (-3)     /* a CUDA call or kernel launch failed                */
#define ECLQR_ESTATE (-4)    /* call order violated (e.g. solve before build)      */
#define ECLQR_ETOOBIG (-5)   /* batch larger than the fixed array of eclqr_kkt_residual_noalloc */
#define ECLQR_ESMEM (-6)     /* (n, m, max p_i, max q_i) of a group need more shared memory per task than a CTA holds */

/* per-problem status codes (device array) */
#define ECLQR_STATUS_OK 0
#define ECLQR_STATUS_INFEASIBLE_SUFFIX 1 /* a suffix relation reads 0 = gamma != 0 (Alg. 1)      */
#define ECLQR_STATUS_INFEASIBLE_X0 2     /* s_0 violates H_0 s_0 + h_0 = 0 (eq. initial-feasibility) */
#define ECLQR_STATUS_RANK_INCONSISTENT 3 /* nonzero residual row in Gamma u = -(Phi z + gamma) (Lemma 4 remark) */
#define ECLQR_STATUS_NONCONVEX 4         /* Cholesky of Rbar + Bbar'P Bbar failed (Prop. 6 violated) */
/* 5 is not written: a dual relation (Sec. 7) that reads 0 = gamma != 0 cannot arise
 * in exact arithmetic, since the KKT conditions of a feasible problem with linear
 * equality constraints have a solution.  Where rounding produces one, the row is
 * dropped like a redundant one; the KKT residual and eclqr_refine judge the result. */
#define ECLQR_STATUS_NONFINITE 6         /* a NaN or an infinity in the data, s_0 or an output */

typedef struct eclqr_handle eclqr_handle;

/* Batch structure (host memory). */
typedef struct {
  int32_t num_problems;  /* P >= 1                                                    */
  const int32_t *N;      /* [P] horizons, N_j >= 1                                    */
  const int32_t *n;      /* [P] state dimensions, 1 <= n_j <= ECLQR_MAX_N             */
  const int32_t *m;      /* [P] control dimensions, 1 <= m_j <= ECLQR_MAX_M           */
  const int32_t *p;      /* [sum_j N_j] mixed rows per stage, 0 <= p_i <= ECLQR_MAX_ROWS */
  const int32_t *q;      /* [sum_j (N_j+1)] state-only rows per stage, 0..ECLQR_MAX_ROWS */
} eclqr_desc;

#define ECLQR_MAX_N 32
#define ECLQR_MAX_M 16
#define ECLQR_MAX_ROWS 32
/* Combinations whose largest kernel needs more shared memory than one CTA
 * holds are rejected by eclqr_create with ECLQR_ESMEM.
 * Stage-varying dimensions n_i, m_i (Sec. 2) enter by zero padding to the
 * problem's largest n_i and m_i: zero rows and columns of A_i, B_i, c_i, C_i,
 * D_i, E_i, M_i, q_i, r_i and s_0 at the padded coordinates and identity
 * blocks of Q_i and R_i there.  The padded states stay 0 through the
 * dynamics, the padded controls at their unconstrained minimum 0, and the
 * multipliers of the padded rows are 0; the rest of the solution is that of
 * the unpadded problem. */

/* Problem data (device memory), layout in the header comment. */
typedef struct {
  const double *A, *B, *c;
  const double *C, *D, *d;
  const double *E, *e;
  const double *Q, *M, *R, *qv, *rv;
} eclqr_data;

typedef struct {
  double tau_rank;   /* relative rank cut after row scaling (Sec. 8 items 1-2); default 1e-10 */
  double tau_inc;    /* inconsistency cut on a scaled offset (Sec. 8 item 4); default 1e-8    */
  int32_t refine;    /* refinement passes on the reduced LQR KKT residual; default 2          */
  int32_t chunk;     /* stages per scan chunk; 0 = chosen from N and the SM count: one chunk
                      * per problem when the longest horizon is at most the batch's stages
                      * per SM, else 7 to 64 stages.  A problem that fits one chunk is swept once per
                      * scan, from its terminal element, with no chunk aggregate           */
  int32_t team_warps; /* warps of the CTA that runs one task: 1, 2, 4 or 8 for every kernel;
                       * 0 (default) = per kernel: 4 when a launch has fewer tasks than
                       * SMs; with at least 4 tasks per SM the kernel's measured best for
                       * the group's n (1 for the per-problem sweeps and the small
                       * per-stage kernels, 1 or 4 for the stage elimination, 2 or 8 for
                       * the affine-chain sweep); in between that but at least 2          */
  int32_t scan_skip;  /* 1 (default): take the shortcut of Sec. 6 (complete algorithm and
                       * complexity) where it applies: a problem without state-only or
                       * terminal rows whose every stage's mixed rows leave no row on x_i
                       * once u_i is projected out (Lemma 1, same tolerances) has
                       * X_i = R^n for all i, and its feasible-domain scan is skipped.
                       * 0: always run the scan.  Results are the same either way.       */
  int32_t kkt_refine; /* passes of eclqr_refine, 0..16; default 8.  0 allocates no
                       * refinement workspace and eclqr_refine only computes the residual */
  double refine_tol;  /* eclqr_refine corrects a problem only while its residual exceeds
                       * this; default 5e-10                                              */
  int32_t riccati_fp32; /* 1: mixed precision -- the square-root Riccati sweep of every
                       * problem runs in FP32, everything else in FP64 (the domain scan,
                       * null-space bases and rank decisions, the elimination, rollout,
                       * refinement and multipliers); eclqr_refine then refines in FP64
                       * and redoes in FP64 the problems it leaves above refine_tol.
                       * 0 (default): FP64 throughout                                   */
  int32_t persist;    /* persistent launches of the per-problem sweeps: a fixed number of
                       * CTAs per SM, each taking the next task from a device counter,
                       * longest horizon first (Sec. 6, complexity and depth: the sweeps'
                       * depth is the longest horizon, so it starts first).  0 (default):
                       * 8 CTAs per SM for launches with at least 4 tasks per SM; k in
                       * 1..32: k CTAs per SM for every launch with more than k tasks per
                       * SM; -1: one CTA per task.  Results are the same either way.      */
  int32_t corr_refine; /* refinement passes on the reduced residual inside the corrections
                       * of eclqr_refine, 0..8; -1 (default) = refine.  A correction only
                       * has to shrink the residual that the next pass measures again     */
} eclqr_options;

/* element counts of every packed array (for allocation) */
typedef struct {
  int64_t A, B, c, C, D, d, E, e, Q, M, R, qv, rv, s0;
  int64_t x, u, lam, mu, eta, alpha;
  int64_t stages;    /* sum_j N_j */
} eclqr_layout_info;

/* Fills *opt with the defaults above. */
void eclqr_default_options(eclqr_options *opt);

/* Validates the descriptor and returns array sizes.  Host only. */
int eclqr_layout(const eclqr_desc *desc, eclqr_layout_info *out);

/* Plans the batch and allocates the device workspace (cudaMalloc) on the
 * current device.  opt may be NULL (defaults).  Host-synchronous.  Problems
 * are grouped by (n, m); a group whose n, m, largest p_i and largest q_i need
 * more shared memory in some kernel than a CTA holds is rejected with
 * ECLQR_ESMEM before anything is allocated: first a bound of 219 KB on the
 * dynamic part (no device call), then each kernel's dynamic plus static
 * shared memory against the device's per-CTA limit (n <= 28 fits for any row
 * counts up to ECLQR_MAX_ROWS; n = 32, m = 16 needs max p_i + max q_i <= 46). */
int eclqr_create(const eclqr_desc *desc, const eclqr_options *opt, eclqr_handle **out);

/* Feasible-domain scan and stagewise elimination of Algorithm 1 (Sec. 3-5)
 * plus the coefficient part of the reduced Riccati solve (Sec. 6): everything
 * that does not depend on s_0.  status: device int32[P], overwritten. */
int eclqr_build(eclqr_handle *h, const eclqr_data *data, int32_t *status, void *stream);

/* After eclqr_build: flags (device int32[P]) receives 1 for every problem whose
 * feasible-domain scan the Sec. 6 shortcut skipped (see eclqr_options.scan_skip),
 * 0 otherwise.  Asynchronous on stream.  ECLQR_ESTATE before a build. */
int eclqr_scan_skipped(eclqr_handle *h, int32_t *flags, void *stream);

/* Checks s_0 (eq. initial-feasibility), forms z_0 (eq. reduced-initial), rolls
 * the reduced LQR out with refinement on its KKT residual, and recovers
 * x (N+1)*n and u N*m (eq. recovery-maps).  s0, x, u: device.  status is
 * updated (not cleared). */
int eclqr_solve(eclqr_handle *h, const double *s0, double *x, double *u, int32_t *status,
                void *stream);

/* Multipliers of the original problem (Sec. 7) at the last solve: lambda
 * (N+1)*n with lambda_0 = -alpha, mu, eta, alpha.  x, u: the solve's output.
 * Selects the min-norm representative (min-norm lambda_0, then min-norm
 * lambda_{i+1} given lambda_i, then min-norm (mu_i, eta_i)).  Device pointers. */
int eclqr_multipliers(eclqr_handle *h, const double *x, const double *u, double *lam,
                      double *mu, double *eta, double *alpha, int32_t *status, void *stream);

/* Infinity-norm KKT residual of the original problem (Sec. 9 residual
 * definition): x_0 - s_0, dynamics, equality rows divided by max(1, largest
 * |coefficient|, |offset|) of the row, and stationarity (Sec. 7 sign
 * convention, lambda_0 = -alpha).  resid: device double[P], overwritten.  A NaN
 * anywhere in a row makes that problem's residual NaN (it never passes a
 * comparison with a gate).  Needs a build of the same batch structure; reads
 * the data of the last eclqr_build. */
int eclqr_kkt_residual(eclqr_handle *h, const double *s0, const double *x, const double *u,
                       const double *lam, const double *mu, const double *eta,
                       const double *alpha, double *resid, void *stream);

/* The same residual with its four parts (Sec. 9 residual definition):
 * parts[4 j + 0] initial condition, + 1 dynamics, + 2 normalised equality
 * rows, + 3 stationarity; resid[j] is their maximum.  parts: device
 * double[4 P], overwritten; NULL is ECLQR_EINVAL. */
int eclqr_kkt_residual_parts(eclqr_handle *h, const double *s0, const double *x, const double *u,
                             const double *lam, const double *mu, const double *eta,
                             const double *alpha, double *resid, double *parts, void *stream);

/* Refinement on the original KKT residual (Sec. 8 advises verifying the
 * original residuals; Sec. 5: the reduction is linear in the offsets).  The
 * KKT map F(w) of the problem is affine, so for the point w = (x, u, lam, mu,
 * eta, alpha) with residual rows r = F(w) the correction dw with F(w + dw) = 0
 * solves the same problem with the same matrices and the offsets replaced by
 * r: c' = dynamics rows, d' = mixed rows, e' = state-only rows, q' = state
 * stationarity, r' = control stationarity, s0' = -(x_0 - s_0).  Each pass
 * computes those rows and solves the correction problem in the handle's own
 * workspace (no allocation): through a new build when a primal part of the
 * residual (initial condition, dynamics, equality rows) exceeds
 * opt.refine_tol, otherwise with c' = d' = e' = s0' = 0, homogeneous
 * constraints for which the build's factors serve unchanged (eclqr_set_costs,
 * then solve and multipliers).  It keeps w + dw where the residual is
 * smaller.  A problem takes part in pass k while its status is OK, its
 * residual exceeds opt.refine_tol and every earlier pass at least halved it;
 * the others are left as they are (their kernels return at once).  Up to
 * opt.kkt_refine passes.
 *   In: s0 and the point (the output of eclqr_solve and eclqr_multipliers,
 *   device), status (device int32[P], read only).  Out: the point, improved
 *   in place, and resid (device double[P]): the Sec. 9 residual of the
 *   returned point (the call computes it first, so no eclqr_kkt_residual is
 *   needed before it).
 *   When a pass ran, the offset-dependent parts of the workspace belong to
 *   the last correction: eclqr_solve and eclqr_multipliers return
 *   ECLQR_ESTATE until the next eclqr_build or eclqr_set_costs.
 *   Outside a stream capture the call waits, once per pass, for a 4-byte
 *   flag telling whether any problem takes part, and returns when none does
 *   (so it is host-synchronous); on a capturing stream it records all
 *   opt.kkt_refine passes, whose kernels return at once for the problems
 *   that take no part. */
int eclqr_refine(eclqr_handle *h, const double *s0, double *x, double *u, double *lam, double *mu,
                 double *eta, double *alpha, double *resid, int32_t *status, void *stream);

/* Mixed precision (opt.riccati_fp32 = 1): flags (device int32[P]) receives 1 for
 * every problem whose Riccati sweep eclqr_refine redid in FP64 since the last
 * eclqr_build, 0 for those that kept the FP32 sweep; all 1 when the handle
 * runs in FP64.  Asynchronous on stream.  The paper has no counterpart. */
int eclqr_riccati_fp64_flags(eclqr_handle *h, int32_t *flags, void *stream);

/* Reduced dimensions nbar_i (sum_j (N_j+1)) and mbar_i (sum_j N_j) of the last
 * build, into device int32 arrays. */
int eclqr_reduced_dims(eclqr_handle *h, int32_t *nbar, int32_t *mbar, void *stream);

/* Kernel launches issued through this handle since eclqr_create (host counter,
 * for launch accounting). */
int64_t eclqr_launch_count(const eclqr_handle *h);

/* Measurement hooks (not part of the method).
 * eclqr_time_kernel: when name names one of the library's kernels (e.g.
 * "k_primal_up"), every later launch of that kernel through this handle is
 * bracketed by CUDA events recorded on the launching stream (at most 4096
 * launches are kept); NULL switches it off.  Returns ECLQR_EINVAL for an
 * unknown name.  eclqr_kernel_time reports the launches bracketed since the
 * last eclqr_time_kernel call and their summed duration in milliseconds; it
 * synchronises on the recorded events.
 * eclqr_probe_fp64_peak measures the device's FP64 FMA throughput (TFLOP/s)
 * with a kernel of independent FMA chains on every SM (the roofline
 * denominator for this FP64 path); host-synchronous, allocates 8 MB. */
int eclqr_time_kernel(eclqr_handle *h, const char *name);
int eclqr_kernel_time(eclqr_handle *h, int64_t *launches, double *total_ms);
int eclqr_probe_fp64_peak(double *tflops);

/* Swaps in new linear costs with zero affine offsets on the factors of the
 * last eclqr_build -- the adjoint problem of eclqr_param_grads without a new
 * build.  data: the built problem's matrices (A, B, C, D, E, Q, M, R, same
 * arrays or equal values), new qv and rv, and c, d, e pointing at zeros; the
 * call does not check these preconditions, and with nonzero c, d or e the
 * subsequent solve is wrong.  Zeroes t_i, y_i and cbar_i, recomputes
 * qbar_i = T_i'q_i + Y_i'r_i and rbar_i = Z_i'r_i (eq. reduced-cost-data with
 * t = y = 0) and the square-root Riccati's stage offsets, and sets the
 * Riccati's own offsets to zero, so that the following eclqr_solve starts
 * from z = v = 0 and its first refinement pass (the P-form offset recursion
 * on the stored factors) reaches the new solution, the default second pass
 * adding accuracy.  Asynchronous; the
 * handle then needs eclqr_solve before eclqr_multipliers.  The paper has no
 * counterpart. */
int eclqr_set_costs(eclqr_handle *h, const eclqr_data *data, void *stream);

/* Gradient outputs (device memory): one array per input of eclqr_data plus s0
 * (P x n), each with the packed layout of the corresponding input. */
typedef struct {
  double *A, *B, *c;
  double *C, *D, *d;
  double *E, *e;
  double *Q, *M, *R, *qv, *rv;
  double *s0;
} eclqr_grads;

/* Parameter gradients of a scalar loss l(x, u) by implicit differentiation of
 * the KKT system (problem statement of Sec. 2 with the stationarity equations
 * and multiplier sign convention of Sec. 7; the paper itself has no gradients).
 * (x, u, lam, mu, eta, alpha) is the solution of the problem, (xb, ub, lamb,
 * mub, etab, alphab) the adjoint: the solution of the same problem with the
 * same matrices but offsets q' = -dl/dx, r' = -dl/du, c' = d' = e' = 0 and
 * s0' = 0 (obtained with eclqr_build / eclqr_solve / eclqr_multipliers on
 * that data).  Writes every element of every array of *out:
 *   dA_i = -(lam_{i+1} xb_i' + lamb_{i+1} x_i'), dB_i, dC_i, dD_i, dE_i, dM_i alike;
 *   dQ_i, dR_i symmetrised; dq = -xb, dr = -ub, dc_i = -lamb_{i+1},
 *   dd = -mub, de = -etab, ds0 = alphab.
 * The multipliers enter the result, so where they are not unique (the global
 * constraint Jacobian rank-deficient) neither is the gradient.  Requires a
 * built handle (any data of the same batch structure).  Asynchronous on
 * stream; all pointers device, same layouts as eclqr_multipliers. */
int eclqr_param_grads(eclqr_handle *h, const double *x, const double *u, const double *lam, const double *mu,
                      const double *eta, const double *alpha, const double *xb, const double *ub,
                      const double *lamb, const double *mub, const double *etab, const double *alphab,
                      const eclqr_grads *out, void *stream);

void eclqr_destroy(eclqr_handle *h);
const char *eclqr_strerror(int code);

/* Residual without allocating.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory at the moment they need
 * the check -- real-time control loops that forbid allocation after start-up,
 * or processes whose device memory is fully reserved by another allocator so
 * that cudaMalloc fails.  It computes the same residual as eclqr_kkt_residual,
 * for the batch described by desc and data, with
 * no handle: the per-problem and per-stage descriptors that the handle keeps in
 * its workspace are written instead into one fixed device array of
 * ECLQR_NOALLOC_MAX_PROBLEMS problem and ECLQR_NOALLOC_MAX_STAGES stage records
 * (about 4 MB, held by every GPU that loads the library until the process
 * exits).  The call performs no cudaMalloc, cudaFree or other allocation.
 *   - desc: host memory, as for eclqr_create; data, s0, x, u, lam, mu, eta,
 *     alpha: device, laid out as for eclqr_kkt_residual; resid: device
 *     double[num_problems], zeroed by the call and then written.
 *   - Batches with more than ECLQR_NOALLOC_MAX_PROBLEMS problems or more than
 *     ECLQR_NOALLOC_MAX_STAGES stage records (sum_j (N_j + 1)) are rejected
 *     with ECLQR_ETOOBIG before anything is enqueued.
 *   - The first call on a device looks up the device address of the array
 *     (cudaGetSymbolAddress) with that device current.
 *   - The descriptors reach the device by a copy from a host staging array
 *     that the next call rewrites, so the call cannot be recorded into a CUDA
 *     graph: on a stream that is capturing it returns ECLQR_ESTATE and
 *     enqueues nothing.
 *   - Every call rewrites the array (and a host staging array of the same
 *     size) in full for its batch; calls that overlap -- on the GPU, or from
 *     several host threads -- race and must be serialised by the caller. */
#define ECLQR_NOALLOC_MAX_PROBLEMS 4096
#define ECLQR_NOALLOC_MAX_STAGES 131072
int eclqr_kkt_residual_noalloc(const eclqr_desc *desc, const eclqr_data *data, const double *s0,
                               const double *x, const double *u, const double *lam, const double *mu,
                               const double *eta, const double *alpha, double *resid, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* ECLQR_H */
