/*
 * eclqr_oracle.c -- plain sequential FP64 CPU oracle for the equality-
 * constrained LQR reduction of Sousa-Pinto & Orban, "An Efficient Algorithm
 * for Solving Linear Equality-Constrained LQR Problems" (arXiv 2407.05433).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference against
 * which the CUDA path is checked; it is never linked into, imported by, or
 * called from the product library.  It shares no code, header or constant
 * generator with the CUDA sources.
 *
 * What it computes, in the paper's order (Algorithm 1), one stage at a time:
 *   1. Terminal domain X_N = {E_N x + e_N = 0}, canonicalised            (Sec. 4.1, terminal relation)
 *   2. Backward sweep X_i = R_i o X_{i+1}: the base relation of stage i
 *      (eq. base-system) composed with X_{i+1} (Sec. 3.1) by eliminating
 *      u_i and x_{i+1} together; x_{i+1} is eliminated by substituting the
 *      dynamics, which is the same existential projection (Lemma 1).      (Sec. 4.2, Thm 3)
 *   3. Feasibility of s_0 (eq. initial-feasibility)                       (Sec. 4.2)
 *   4. T_i, t_i, S_i = T_i^T with orthonormal T and min-norm t           (eqs. state-param, left-inverse)
 *   5. Gamma, Phi, gamma -> Z (null basis), Y, y (min-norm)               (eqs. local-control-matrices, Lemma 4)
 *   6. Reduced dynamics, reduced costs, constants kappa                   (Sec. 5.2-5.3)
 *   7. Textbook sequential Riccati on the reduced LQR (cross term kept)   (Sec. 6: "sequential Riccati")
 *   8. Rollout and recovery x = T z + t, u = Y z + Z v + y                (eq. recovery-maps)
 *   9. Multipliers by the sequential variant of Sec. 7: admissible costate
 *      sets propagated right to left, min-norm lambda_0, then forward
 *      substitution choosing the min-norm lambda_{i+1}; min-norm leaf
 *      solves for (mu_i, eta_i), eta_N; alpha = -lambda_0.              (Sec. 7)
 *      A dual relation that reads 0 = gamma != 0 cannot arise in exact
 *      arithmetic (the KKT conditions of a feasible problem with linear
 *      equality constraints always have a solution), so such a row is a
 *      rounding effect: it is dropped like a redundant one and the pass goes
 *      on; the KKT residual and its refinement (step 11) judge the result.
 *  10. KKT residual of the original problem (Sec. 9, residual definition);
 *      a non-finite row makes the residual NaN.
 *  11. Refinement on the original KKT residual (Sec. 8 asks to check the
 *      original residuals; Sec. 5: the reduction is linear in the offsets).
 *      For a point w with residual rows r, the correction dw solves the
 *      same problem with the same matrices and the offsets replaced by r
 *      (c' = dynamics rows, d' = mixed rows, e' = state-only rows,
 *      q' = state stationarity, r' = control stationarity, s0' = -(x_0 - s_0)),
 *      because F(w + dw) = r + K dw for the affine KKT map F.  Pass k runs
 *      when the status is OK and the Sec. 9 residual exceeds refine_tol;
 *      the corrected point replaces w only when its own solve ended with
 *      status OK and its residual is smaller than w's, and the passes go on
 *      only while each one at least halves the residual: where the reduction
 *      itself loses its accuracy, the correction solves lose it as well and
 *      the iteration would diverge, and at the problem's own rounding floor
 *      a pass only trades rounding errors.  When the primal rows of r (x_0,
 *      dynamics, mixed and state-only rows) are all within refine_tol, the
 *      correction takes c' = d' = e' = s0' = 0: the same problem with
 *      homogeneous constraints, whose reduction needs no new offsets.
 *  Inputs with a NaN or an infinity give status ORC_NONFINITE at once.
 *
 * Numerical policy (Sec. 8 asks for one; the paper fixes no constants):
 *   - every projected system is row-scaled to unit 2-norm over its
 *     coefficient columns before any rank test;
 *   - a Householder pivot is accepted when its column norm exceeds
 *     tau_rank * nu, nu = largest column norm of the row-scaled coefficient
 *     matrix;
 *   - a residual row whose coefficients were all rejected is inconsistent
 *     when |offset| > tau_inc * max(1, largest scaled offset);
 *   - relation rows kept after a projection are renormalised to unit norm.
 *
 * Floating point: IEEE double, compiled with -ffp-contract=off.
 * Flops are counted with the standard formulas (Householder step on an
 * r x c block: 4rc; GEMM m x k x n: 2mkn; Cholesky n^3/3; triangular
 * solve n^2 per right-hand side) into a caller-visible counter.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>

/* Mutation hooks for the test suite: building with -DORC_PLANT=k plants one
 * plausible mistake so that the tests can show that some pin fails.  The
 * default build (ORC_PLANT=0) contains none of them. */
#ifndef ORC_PLANT
#define ORC_PLANT 0
#endif

#define ORC_OK 0
#define ORC_INFEASIBLE_SUFFIX 1
#define ORC_INFEASIBLE_X0 2
#define ORC_RANK_INCONSISTENT 3
#define ORC_NONCONVEX 4
/* 5 is retired: a dual relation that reads 0 = gamma != 0 no longer stops
   the multiplier pass (see step 9 below) */
#define ORC_NONFINITE 6
#define ORC_BAD_INPUT 7

static double g_flops = 0.0;
/* flops per phase of Algorithm 1: 0 suffix domains, 1 parameterisation,
   2 stage elimination, 3 Riccati factors, 4 linear passes/rollout/refinement/
   recovery, 5 multipliers, 6 KKT residual, 7 corrections of the refinement on
   the original KKT residual (step 11) */
static double g_phase[8];
static int g_cur = 0;
static int g_in_correction = 0;
/* set around a product that is not counted as work (a product with T_i = I, see step 5) */
static int g_uncounted = 0;
#define ADDF(x)                                                               \
  do {                                                                        \
    if (!g_uncounted) {                                                       \
      double _f = (x);                                                        \
      g_flops += _f;                                                          \
      g_phase[g_in_correction ? 7 : g_cur] += _f;                             \
    }                                                                         \
  } while (0)

/* ------------------------------------------------------------------ */
/* small dense helpers, row-major, explicit leading dimensions          */
/* ------------------------------------------------------------------ */

/* C (m x n) = alpha * op(A) op(B) + beta * C, op = transpose if flag set */
static void gemm(int ta, int tb, int m, int n, int k, double alpha,
                 const double *A, int lda, const double *B, int ldb,
                 double beta, double *C, int ldc) {
  for (int i = 0; i < m; i++)
    for (int j = 0; j < n; j++) {
      double s = 0.0;
      for (int l = 0; l < k; l++) {
        double a = ta ? A[l * lda + i] : A[i * lda + l];
        double b = tb ? B[j * ldb + l] : B[l * ldb + j];
        s += a * b;
      }
      C[i * ldc + j] = alpha * s + (beta == 0.0 ? 0.0 : beta * C[i * ldc + j]);
    }
  ADDF(2.0 * m * n * k);
}

static double *dalloc(size_t n) {
  double *p = (double *)calloc(n ? n : 1, sizeof(double));
  return p;
}

/* ------------------------------------------------------------------ */
/* Lemma 1 realised by ordered column-pivoted Householder row reduction */
/* ------------------------------------------------------------------ */
/*
 * M is r x nc (row-major, ld = nc).  Its columns are, in order:
 * ngroups groups of columns to eliminate (sizes gsz[]), then nkeep kept
 * columns, then one offset column.  The groups are eliminated in order
 * (the eliminated variable is pivoted first, Sec. 8), then the kept columns
 * are reduced to an independent row basis.
 *
 * On return:
 *   grank[g]  = rank found for group g (rows are consumed in order)
 *   *krank    = rank of the kept block
 *   M rows [sum grank, sum grank + krank) hold the kept relation rows
 *   *inconsistent = 1 if a leftover row reads 0 = gamma with gamma != 0
 * The kept rows are also copied, renormalised, into out (krank x (nkeep+1))
 * when out != NULL.
 */
static void project(double *M, int r, int nc, int ngroups, const int *gsz,
                    int nkeep, double tau_rank, double tau_inc, int *grank,
                    int *krank, int *inconsistent, double *out) {
  int ncoef = nc - 1;
  int off = nc - 1;
  /* row scaling */
  for (int i = 0; i < r; i++) {
    double s = 0.0;
    for (int j = 0; j < ncoef; j++) s += M[i * nc + j] * M[i * nc + j];
    s = sqrt(s);
    if (s > 0.0)
      for (int j = 0; j < nc; j++) M[i * nc + j] /= s;
  }
  double nu = 0.0, omega = 1.0;
  for (int j = 0; j < ncoef; j++) {
    double s = 0.0;
    for (int i = 0; i < r; i++) s += M[i * nc + j] * M[i * nc + j];
    if (sqrt(s) > nu) nu = sqrt(s);
  }
  for (int i = 0; i < r; i++)
    if (fabs(M[i * nc + off]) > omega) omega = fabs(M[i * nc + off]);
  double thr = tau_rank * nu;

  char *done = (char *)calloc(nc, 1);
  double *v = dalloc(r);
  int k = 0; /* next pivot row */
  int ntot = ngroups + 1;
  int col0 = 0;
  for (int g = 0; g < ntot; g++) {
    int c0 = col0, c1 = col0 + (g < ngroups ? gsz[g] : nkeep);
    int rk = 0;
    while (k < r) {
      /* pivot: largest remaining column norm over rows [k, r) */
      int piv = -1;
      double best = 0.0;
      for (int j = c0; j < c1; j++) {
        if (done[j]) continue;
        double s = 0.0;
        for (int i = k; i < r; i++) s += M[i * nc + j] * M[i * nc + j];
        s = sqrt(s);
        if (s > best) { best = s; piv = j; }
      }
      if (piv < 0 || best <= thr) break;
      /* Householder reflector from column piv on rows [k, r) */
      double xk = M[k * nc + piv];
      double sg = xk >= 0.0 ? 1.0 : -1.0;
      for (int i = k; i < r; i++) v[i] = M[i * nc + piv];
      v[k] = xk + sg * best;
      double beta = 1.0 / (best * (best + fabs(xk)));
      for (int j = 0; j < nc; j++) {
        if (done[j] || j == piv) continue;
        double w = 0.0;
        for (int i = k; i < r; i++) w += v[i] * M[i * nc + j];
        w *= beta;
        for (int i = k; i < r; i++) M[i * nc + j] -= w * v[i];
      }
      ADDF(4.0 * (r - k) * (nc - k));
      M[k * nc + piv] = -sg * best;
      for (int i = k + 1; i < r; i++) M[i * nc + piv] = 0.0;
      done[piv] = 1;
      k++;
      rk++;
    }
    if (g < ngroups) grank[g] = rk; else *krank = rk;
    col0 = c1;
  }
  *inconsistent = 0;
  for (int i = k; i < r; i++)
    if (fabs(M[i * nc + off]) > tau_inc * omega) *inconsistent = 1;
  if (out) {
    int kr = *krank, k0 = k - kr, kc0 = nc - 1 - nkeep;
    for (int i = 0; i < kr; i++) {
      double s = 0.0;
      for (int j = 0; j < nkeep; j++) s += M[(k0 + i) * nc + kc0 + j] * M[(k0 + i) * nc + kc0 + j];
      s = sqrt(s);
      for (int j = 0; j < nkeep; j++) out[i * (nkeep + 1) + j] = M[(k0 + i) * nc + kc0 + j] / s;
      out[i * (nkeep + 1) + nkeep] = M[(k0 + i) * nc + off] / s;
    }
  }
  free(done);
  free(v);
}

/* ------------------------------------------------------------------ */
/* Null space and minimum-norm solutions of K w = -b                   */
/* ------------------------------------------------------------------ */
/*
 * K is rk x nk.  Computes the column-pivoted Householder QR of K^T
 * (pivoting over the rows of K): K^T Pi = Q R.  rank = number of accepted
 * pivots (tau_rank * largest row norm of K).
 *   Qout (nk x nk, optional): the full orthogonal Q; its last nk - rank
 *       columns are an orthonormal basis of null(K).
 *   For nb right-hand-side columns b (rk x nb, ld nb), writes the
 *   min-norm solutions X (nk x nb) of K X = -b, and returns in *resid the
 *   largest residual of the rows of K that were rejected as dependent,
 *   relative to max(1, |b|_max).
 * Returns the rank.
 */
static int tqr_solve(const double *K, int rk, int nk, double tau_rank,
                     const double *b, int nb, double *X, double *Qout,
                     double *resid) {
  double *W = dalloc((size_t)nk * rk); /* K^T, nk x rk */
  double *Q = dalloc((size_t)nk * nk);
  int *perm = (int *)malloc(sizeof(int) * (rk ? rk : 1));
  double *v = dalloc(nk);
  for (int i = 0; i < nk; i++)
    for (int j = 0; j < rk; j++) W[i * rk + j] = K[j * nk + i];
  for (int i = 0; i < nk; i++) Q[i * nk + i] = 1.0;
  for (int j = 0; j < rk; j++) perm[j] = j;
  double nu = 0.0;
  for (int j = 0; j < rk; j++) {
    double s = 0.0;
    for (int i = 0; i < nk; i++) s += W[i * rk + j] * W[i * rk + j];
    if (sqrt(s) > nu) nu = sqrt(s);
  }
  double thr = tau_rank * nu;
  int rank = 0;
  for (int s = 0; s < rk && s < nk; s++) {
    int piv = -1;
    double best = 0.0;
    for (int j = s; j < rk; j++) {
      double t = 0.0;
      for (int i = s; i < nk; i++) t += W[i * rk + j] * W[i * rk + j];
      t = sqrt(t);
      if (t > best) { best = t; piv = j; }
    }
    if (piv < 0 || best <= thr) break;
    if (piv != s) {
      for (int i = 0; i < nk; i++) {
        double t = W[i * rk + s]; W[i * rk + s] = W[i * rk + piv]; W[i * rk + piv] = t;
      }
      int t = perm[s]; perm[s] = perm[piv]; perm[piv] = t;
    }
    double xk = W[s * rk + s];
    double sg = xk >= 0.0 ? 1.0 : -1.0;
    for (int i = s; i < nk; i++) v[i] = W[i * rk + s];
    v[s] = xk + sg * best;
    double beta = 1.0 / (best * (best + fabs(xk)));
    for (int j = s + 1; j < rk; j++) {
      double w = 0.0;
      for (int i = s; i < nk; i++) w += v[i] * W[i * rk + j];
      w *= beta;
      for (int i = s; i < nk; i++) W[i * rk + j] -= w * v[i];
    }
    W[s * rk + s] = -sg * best;
    for (int i = s + 1; i < nk; i++) W[i * rk + s] = 0.0;
    /* Q <- Q H */
    for (int i = 0; i < nk; i++) {
      double w = 0.0;
      for (int l = s; l < nk; l++) w += Q[i * nk + l] * v[l];
      w *= beta;
      for (int l = s; l < nk; l++) Q[i * nk + l] -= w * v[l];
    }
    ADDF(4.0 * (nk - s) * (rk - s) + 4.0 * nk * (nk - s));
    rank++;
  }
  double rmax = 0.0;
  if (nb > 0) {
    double bmax = 1.0;
    for (int i = 0; i < rk * nb; i++) if (fabs(b[i]) > bmax) bmax = fabs(b[i]);
    double *y = dalloc((size_t)(rank ? rank : 1) * nb);
    /* R11^T y = (Pi^T b)_1, R11 = W[0:rank, 0:rank] upper triangular */
    for (int c = 0; c < nb; c++) {
      for (int i = 0; i < rank; i++) {
        double s = b[perm[i] * nb + c];
        for (int l = 0; l < i; l++) s -= W[l * rk + i] * y[l * nb + c];
        y[i * nb + c] = s / W[i * rk + i];
      }
      /* dependent rows j >= rank: residual b_j - R12^T y (column j of W) */
      for (int j = rank; j < rk; j++) {
        double s = b[perm[j] * nb + c];
        for (int l = 0; l < rank; l++) s -= W[l * rk + j] * y[l * nb + c];
        if (fabs(s) / bmax > rmax) rmax = fabs(s) / bmax;
      }
    }
    ADDF((double)nb * rank * rank + 2.0 * nb * rank * (rk - rank));
    /* X = -Q1 y */
    for (int i = 0; i < nk; i++)
      for (int c = 0; c < nb; c++) {
        double s = 0.0;
        for (int l = 0; l < rank; l++) s += Q[i * nk + l] * y[l * nb + c];
        X[i * nb + c] = -s;
      }
    ADDF(2.0 * nk * rank * nb);
    free(y);
  }
  if (resid) *resid = rmax;
  if (Qout) memcpy(Qout, Q, sizeof(double) * nk * nk);
  free(W); free(Q); free(perm); free(v);
  return rank;
}

/* Cholesky L L^T of an n x n SPD matrix (in place, lower); 0 on success */
static int cholesky(double *Hm, int n) {
  for (int j = 0; j < n; j++) {
    double s = Hm[j * n + j];
    for (int l = 0; l < j; l++) s -= Hm[j * n + l] * Hm[j * n + l];
    if (!(s > 0.0)) return 1;
    double d = sqrt(s);
    Hm[j * n + j] = d;
    for (int i = j + 1; i < n; i++) {
      double t = Hm[i * n + j];
      for (int l = 0; l < j; l++) t -= Hm[i * n + l] * Hm[j * n + l];
      Hm[i * n + j] = t / d;
    }
    for (int i = 0; i < j; i++) Hm[i * n + j] = 0.0;
  }
  ADDF((double)n * n * n / 3.0);
  return 0;
}

/* solve (L L^T) X = Bm in place, Bm is n x nb */
static void chol_solve(const double *L, int n, double *Bm, int nb) {
  for (int c = 0; c < nb; c++) {
    for (int i = 0; i < n; i++) {
      double s = Bm[i * nb + c];
      for (int l = 0; l < i; l++) s -= L[i * n + l] * Bm[l * nb + c];
      Bm[i * nb + c] = s / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; i--) {
      double s = Bm[i * nb + c];
      for (int l = i + 1; l < n; l++) s -= L[l * n + i] * Bm[l * nb + c];
      Bm[i * nb + c] = s / L[i * n + i];
    }
  }
  ADDF(2.0 * n * n * nb);
}

/* ------------------------------------------------------------------ */
/* Problem description (packed, row-major per stage)                    */
/* ------------------------------------------------------------------ */
typedef struct {
  int N, n, m;
  const int *p;      /* [N]   mixed rows per stage            */
  const int *q;      /* [N+1] state-only rows per stage         */
  const double *A;   /* N x n x n */
  const double *B;   /* N x n x m */
  const double *c;   /* N x n */
  const double *C;   /* sum(p) x n */
  const double *D;   /* sum(p) x m */
  const double *d;   /* sum(p) */
  const double *E;   /* sum(q) x n */
  const double *e;   /* sum(q) */
  const double *Q;   /* (N+1) x n x n, last block is Q_N */
  const double *M;   /* N x n x m */
  const double *R;   /* N x m x m */
  const double *qv;  /* (N+1) x n, last is q_N */
  const double *rv;  /* N x m */
  const double *s0;  /* n */
} orc_problem;

/* optional intermediate outputs for tests; any pointer may be NULL */
typedef struct {
  int *nbar;      /* [N+1] reduced state dims            */
  int *mbar;      /* [N]   reduced control dims          */
  int *hrows;     /* [N+1] rows of (H_i, h_i)            */
  double *H;      /* (N+1) x n x (n+1): rows of [H_i | h_i] */
  double *T;      /* (N+1) x n x n, first nbar_i columns  */
  double *t;      /* (N+1) x n */
  double *Y;      /* N x m x n, first nbar_i columns      */
  double *Z;      /* N x m x m, first mbar_i columns      */
  double *y;      /* N x m */
  double *Abar;   /* N x n x n, nbar_{i+1} x nbar_i       */
  double *Bbar;   /* N x n x m, nbar_{i+1} x mbar_i       */
  double *cbar;   /* N x n */
  double *Qbar;   /* (N+1) x n x n                        */
  double *Mbar;   /* N x n x m                            */
  double *Rbar;   /* N x m x m                            */
  double *qbar;   /* (N+1) x n */
  double *rbar;   /* N x m */
  double *kappa;  /* N+1 */
  double *z;      /* (N+1) x n */
  double *v;      /* N x m */
  int *lrows;     /* [N+1] rows of the admissible costate sets */
  double *L;      /* (N+1) x n x (n+1) */
  double *pi;     /* (N+1) x n: reduced costates P_i z_i + p_i (refined) */
  double *UT;     /* (N+1) x n x n: [U_i | T_i] */
} orc_debug;

typedef struct {
  double tau_rank, tau_inc;
  int refine;        /* refinement passes on the reduced LQR KKT residual */
  int kkt_refine;    /* passes of step 11 (refinement on the original KKT residual) */
  double refine_tol; /* step 11 runs a pass only while the residual exceeds this */
} orc_options;

/* ------------------------------------------------------------------ */
/* the solver                                                           */
/* ------------------------------------------------------------------ */
/* one pass of steps 1-9 (Algorithm 1 and Sec. 7) */
static int solve_once(const orc_problem *P, const orc_options *opt, double *x,
                      double *u, double *lam, double *mu, double *eta,
                      double *alpha, int *fail_stage, orc_debug *dbg) {
  const int N = P->N, n = P->n, m = P->m;
  const double tr = opt->tau_rank, ti = opt->tau_inc;
  g_cur = 0;
  *fail_stage = -1;
  int status = ORC_OK;

  /* offsets of the packed constraint rows */
  int *po = (int *)calloc(N + 1, sizeof(int));
  int *qo = (int *)calloc(N + 2, sizeof(int));
  for (int i = 0; i < N; i++) po[i + 1] = po[i] + P->p[i];
  for (int i = 0; i <= N; i++) qo[i + 1] = qo[i] + P->q[i];
  int pmax = 0, qmax = 0;
  for (int i = 0; i < N; i++) if (P->p[i] > pmax) pmax = P->p[i];
  for (int i = 0; i <= N; i++) if (P->q[i] > qmax) qmax = P->q[i];

  const int hld = n + 1;
  double *H = dalloc((size_t)(N + 1) * n * hld);
  int *hr = (int *)calloc(N + 1, sizeof(int));
  double *T = dalloc((size_t)(N + 1) * n * n);
  double *t = dalloc((size_t)(N + 1) * n);
  int *nb = (int *)calloc(N + 1, sizeof(int));
  int *mb = (int *)calloc(N + 1, sizeof(int));
  double *Y = dalloc((size_t)N * m * n), *Z = dalloc((size_t)N * m * (m ? m : 1));
  double *yv = dalloc((size_t)N * (m ? m : 1));
  double *Ab = dalloc((size_t)N * n * n), *Bb = dalloc((size_t)N * n * (m ? m : 1));
  double *cb = dalloc((size_t)N * n);
  double *Qb = dalloc((size_t)(N + 1) * n * n), *Mb = dalloc((size_t)N * n * (m ? m : 1));
  double *Rb = dalloc((size_t)N * (m ? m * m : 1));
  double *qb = dalloc((size_t)(N + 1) * n), *rb = dalloc((size_t)N * (m ? m : 1));
  double *kap = dalloc((size_t)N + 1);
  double *Kg = dalloc((size_t)N * m * n + 1), *kg = dalloc((size_t)N * m + 1);
  double *zz = dalloc((size_t)(N + 1) * n), *vv = dalloc((size_t)N * m + 1);
  double *Ux = dalloc((size_t)(N + 1) * n * n);            /* full Q of H_i^T: [U_i | T_i] */
  int *ur = (int *)calloc(N + 1, sizeof(int));             /* rank of H_i                  */
  double *Pst = dalloc((size_t)(N + 1) * n * n), *pst = dalloc((size_t)(N + 1) * n); /* P_i, p_i */
  double *Lhs = dalloc((size_t)N * m * m), *Hxs = dalloc((size_t)N * m * n);        /* chol(H_uu), H_ux */
  double *pis = dalloc((size_t)(N + 1) * n);                                         /* pi_i = P z + p */

  int rmax = n + pmax + qmax;
  int cmax = m + n + 1;
  double *work = dalloc((size_t)(rmax + 2 * n + m) * (2 * n + m + pmax + qmax + 2));
  int grank[2], krank, inc;

  /* ---- 1. terminal domain X_N (Sec. 4.1) ---- */
  {
    int qN = (ORC_PLANT == 7) ? 0 : P->q[N];
    for (int i = 0; i < qN; i++) {
      for (int j = 0; j < n; j++) work[i * (n + 1) + j] = P->E[(qo[N] + i) * n + j];
      work[i * (n + 1) + n] = P->e[qo[N] + i];
    }
    project(work, qN, n + 1, 0, NULL, n, tr, ti, grank, &krank, &inc, H + (size_t)N * n * hld);
    hr[N] = krank;
    if (inc) { status = ORC_INFEASIBLE_SUFFIX; *fail_stage = N; goto done; }
  }
  /* ---- 2. backward sweep X_i = R_i o X_{i+1} (eq. base-system, Sec. 3.1, Thm 3) ---- */
  for (int i = N - 1; i >= 0; i--) {
    const double *Ai = P->A + (size_t)i * n * n, *Bi = P->B + (size_t)i * n * m;
    const double *ci = P->c + (size_t)i * n;
    const double *Hn = H + (size_t)(i + 1) * n * hld;
    int rn = hr[i + 1], pi = P->p[i], qi = (ORC_PLANT == 9) ? 0 : P->q[i];
    int r = rn + pi + qi;
    /* columns: u (m) | x_i (n) | offset */
    double *Wm = work;
    memset(Wm, 0, sizeof(double) * r * cmax);
    /* H_{i+1}(A x + B u + c) + h_{i+1} = 0 */
    for (int a = 0; a < rn; a++) {
      for (int j = 0; j < m; j++) {
        double s = 0.0;
        for (int l = 0; l < n; l++) s += Hn[a * hld + l] * Bi[l * m + j];
        Wm[a * cmax + j] = s;
      }
      for (int j = 0; j < n; j++) {
        double s = 0.0;
        for (int l = 0; l < n; l++) s += Hn[a * hld + l] * ((ORC_PLANT == 6) ? Ai[j * n + l] : Ai[l * n + j]);
        Wm[a * cmax + m + j] = s;
      }
      double s = (ORC_PLANT == 1) ? 0.0 : Hn[a * hld + n];
      for (int l = 0; l < n; l++) s += Hn[a * hld + l] * ci[l] * ((ORC_PLANT == 2) ? -1.0 : 1.0);
      Wm[a * cmax + m + n] = s;
    }
    ADDF(2.0 * rn * n * (m + n + 1));
    /* C x + D u + d = 0 */
    for (int a = 0; a < pi; a++) {
      int row = rn + a, src = po[i] + a;
      for (int j = 0; j < m; j++) Wm[row * cmax + j] = P->D[(size_t)src * m + j];
      for (int j = 0; j < n; j++) Wm[row * cmax + m + j] = P->C[(size_t)src * n + j];
      Wm[row * cmax + m + n] = P->d[src];
    }
    /* E x + e = 0 */
    for (int a = 0; a < qi; a++) {
      int row = rn + pi + a, src = qo[i] + a;
      for (int j = 0; j < n; j++) Wm[row * cmax + m + j] = P->E[(size_t)src * n + j];
      Wm[row * cmax + m + n] = P->e[src];
    }
    int gs[1] = {m};
    project(Wm, r, cmax, 1, gs, n, tr, ti, grank, &krank, &inc, H + (size_t)i * n * hld);
    hr[i] = krank;
    if (inc) { status = ORC_INFEASIBLE_SUFFIX; *fail_stage = i; goto done; }
  }
  /* ---- 3. feasibility of s_0 (eq. initial-feasibility) ---- */
  {
    double om = 1.0, worst = 0.0;
    for (int a = 0; a < hr[0]; a++) {
      double s = H[a * hld + n];
      if (fabs(s) > om) om = fabs(s);
      for (int l = 0; l < n; l++) s += H[a * hld + l] * P->s0[l];
      if (fabs(s) > worst) worst = fabs(s);
    }
    for (int l = 0; l < n; l++) if (fabs(P->s0[l]) > om) om = fabs(P->s0[l]);
    if (worst > ti * om) { status = ORC_INFEASIBLE_X0; *fail_stage = 0; goto done; }
  }
  /* ---- 4. T_i, t_i (eqs. state-param, left-inverse; S_i = T_i^T) ---- */
  g_cur = 1;
  {
    double *Kb = dalloc((size_t)n * n), *bb = dalloc(n), *Qf = dalloc((size_t)n * n), *tx = dalloc(n);
    for (int i = 0; i <= N; i++) {
      int ri = hr[i];
      for (int a = 0; a < ri; a++) {
        for (int l = 0; l < n; l++) Kb[a * n + l] = H[(size_t)i * n * hld + a * hld + l];
        bb[a] = H[(size_t)i * n * hld + a * hld + n];
      }
      double rs;
      int rk = tqr_solve(Kb, ri, n, tr, bb, 1, tx, Qf, &rs);
      nb[i] = n - rk;
      ur[i] = rk;
      memcpy(Ux + (size_t)i * n * n, Qf, sizeof(double) * n * n);
      for (int l = 0; l < n; l++) {
        t[(size_t)i * n + l] = ri ? tx[l] : 0.0;
        for (int j = 0; j < nb[i]; j++) T[(size_t)i * n * n + l * n + j] = Qf[l * n + rk + j];
      }
    }
    free(Kb); free(bb); free(Qf); free(tx);
  }
  /* ---- 5-6. stage elimination (Sec. 5) ---- */
  g_cur = 2;
  {
    int gr = pmax + n;
    double *Gm = dalloc((size_t)gr * (m ? m : 1));
    double *Rhs = dalloc((size_t)gr * (n + 1));
    double *Sol = dalloc((size_t)(m ? m : 1) * (n + 1));
    double *Qf = dalloc((size_t)(m ? m * m : 1));
    double *AT = dalloc((size_t)n * n), *tmp = dalloc((size_t)n * n), *tmp2 = dalloc((size_t)n * n);
    double *rz = dalloc(m + 1), *qz = dalloc(n), *Mz = dalloc((size_t)n * (m ? m : 1));
    double *RY = dalloc((size_t)(m ? m : 1) * n), *RZ = dalloc((size_t)(m ? m * m : 1)), *Ry = dalloc(m + 1);
    double *BZ = dalloc((size_t)n * m);
    for (int i = 0; i < N; i++) {
      const double *Ai = P->A + (size_t)i * n * n, *Bi = P->B + (size_t)i * n * m;
      const double *ci = P->c + (size_t)i * n;
      const double *Ti = T + (size_t)i * n * n, *ti_ = t + (size_t)i * n;
      const double *Tn = T + (size_t)(i + 1) * n * n, *tn = t + (size_t)(i + 1) * n;
      const double *Hn = H + (size_t)(i + 1) * n * hld;
      int rn = hr[i + 1], pi = P->p[i], ni = nb[i], nn = nb[i + 1];
      int rows = pi + rn;
      /* where the domain has no rows of rank (ur = 0), T = I and t = 0 (eq. state-param): a
         product with T_i or T_{i+1} there is its other factor, which a solver copies, so its
         flops are computed here but not counted as the method's work */
      const int te = ur[i] == 0, tne = ur[i + 1] == 0;
      /* Gamma = [D; H B], [Phi | gamma] = [C T, C t + d; H A T, H (A t + c) + h] */
      for (int a = 0; a < pi; a++) {
        int src = po[i] + a;
        for (int j = 0; j < m; j++) Gm[a * m + j] = P->D[(size_t)src * m + j];
        for (int j = 0; j < ni; j++) {
          double s = 0.0;
          for (int l = 0; l < n; l++) s += P->C[(size_t)src * n + l] * Ti[l * n + j];
          Rhs[a * (n + 1) + j] = s;
        }
        double s = P->d[src];
        for (int l = 0; l < n; l++) s += P->C[(size_t)src * n + l] * ti_[l];
        Rhs[a * (n + 1) + ni] = s;
      }
      if (!te) ADDF(2.0 * pi * n * (ni + 1));
      /* A T and A t + c */
      g_uncounted = te;
      gemm(0, 0, n, ni, n, 1.0, Ai, n, Ti, n, 0.0, AT, n);
      g_uncounted = 0;
      for (int l = 0; l < n; l++) {
        double s = ci[l];
        for (int j = 0; j < n; j++) s += Ai[l * n + j] * ti_[j];
        tmp[l] = s;
      }
      if (!te) ADDF(2.0 * n * n);
      for (int a = 0; a < rn; a++) {
        const double *hrow = Hn + a * hld;
        for (int j = 0; j < m; j++) {
          double s = 0.0;
          for (int l = 0; l < n; l++) s += hrow[l] * Bi[l * m + j];
          Gm[(pi + a) * m + j] = s;
        }
        for (int j = 0; j < ni; j++) {
          double s = 0.0;
          for (int l = 0; l < n; l++) s += hrow[l] * AT[l * n + j];
          Rhs[(pi + a) * (n + 1) + j] = s;
        }
        double s = hrow[n];
        for (int l = 0; l < n; l++) s += hrow[l] * tmp[l];
        Rhs[(pi + a) * (n + 1) + ni] = s;
      }
      ADDF(2.0 * rn * n * (m + ni + 1));
      /* compact Rhs to ld = ni + 1 */
      double *Rc = dalloc((size_t)(rows ? rows : 1) * (ni + 1));
      for (int a = 0; a < rows; a++)
        for (int j = 0; j <= ni; j++) Rc[a * (ni + 1) + j] = Rhs[a * (n + 1) + j];
      double rs = 0.0;
      int rk = tqr_solve(Gm, rows, m, tr, Rc, ni + 1, Sol, Qf, &rs);
      free(Rc);
      if (rs > ti) { status = ORC_RANK_INCONSISTENT; *fail_stage = i; goto done; }
      int mi = m - rk;
      mb[i] = mi;
      double *Yi = Y + (size_t)i * m * n, *Zi = Z + (size_t)i * m * m, *yi = yv + (size_t)i * m;
      for (int a = 0; a < m; a++) {
        for (int j = 0; j < ni; j++) Yi[a * n + j] = Sol[a * (ni + 1) + j];
        yi[a] = Sol[a * (ni + 1) + ni];
        for (int j = 0; j < mi; j++) Zi[a * m + j] = Qf[a * m + rk + j];
      }
      /* reduced dynamics (eq. reduced-dynamics-data), S_{i+1} = T_{i+1}^T */
      double *Abi = Ab + (size_t)i * n * n, *Bbi = Bb + (size_t)i * n * m, *cbi = cb + (size_t)i * n;
      gemm(0, 0, n, ni, m, 1.0, Bi, m, Yi, n, 1.0, AT, n);  /* AT <- A T + B Y */
      g_uncounted = tne;
      gemm(1, 0, nn, ni, n, 1.0, Tn, n, AT, n, 0.0, Abi, n);
      g_uncounted = 0;
      gemm(0, 0, n, mi, m, 1.0, Bi, m, Zi, m, 0.0, BZ, m);       /* B Z */
      g_uncounted = tne;
      gemm(1, 0, nn, mi, n, 1.0, Tn, n, BZ, m, 0.0, Bbi, m);
      g_uncounted = 0;
      for (int l = 0; l < n; l++) {
        double s = tmp[l] - tn[l];       /* A t + c - t_{i+1} */
        for (int j = 0; j < m; j++) s += Bi[l * m + j] * yi[j];
        tmp2[l] = s;
      }
      ADDF(2.0 * n * m);
      g_uncounted = tne;
      gemm(1, 0, nn, 1, n, 1.0, Tn, n, tmp2, 1, 0.0, cbi, 1);
      g_uncounted = 0;
      /* state substitution (eq. state-cost-data) */
      const double *Qi = P->Q + (size_t)i * n * n, *Mi = P->M + (size_t)i * n * m;
      const double *Ri = P->R + (size_t)i * m * m, *qi = P->qv + (size_t)i * n, *ri = P->rv + (size_t)i * m;
      double *Qbi = Qb + (size_t)i * n * n;
      g_uncounted = te;
      gemm(0, 0, n, ni, n, 1.0, Qi, n, Ti, n, 0.0, tmp, n);           /* Q T */
      gemm(1, 0, ni, ni, n, 1.0, Ti, n, tmp, n, 0.0, Qbi, n);          /* Q^z = T^T Q T */
      gemm(1, 0, ni, m, n, 1.0, Ti, n, Mi, m, 0.0, Mz, m);             /* M^z = T^T M */
      g_uncounted = 0;
      for (int l = 0; l < n; l++) {
        double s = qi[l];
        for (int j = 0; j < n; j++) s += Qi[l * n + j] * ti_[j];
        tmp2[l] = s;                                                    /* Q t + q */
      }
      if (!te) ADDF(2.0 * n * n);
      g_uncounted = te;
      gemm(1, 0, ni, 1, n, 1.0, Ti, n, tmp2, 1, 0.0, qz, 1);            /* q^z */
      g_uncounted = 0;
      for (int j = 0; j < m; j++) {
        double s = ri[j];
        for (int l = 0; l < n; l++) s += Mi[l * m + j] * ti_[l];
        rz[j] = s;                                                      /* r^z = M^T t + r */
      }
      if (!te) ADDF(2.0 * n * m);
      /* reduced cost (eq. reduced-cost-data) */
      gemm(0, 0, m, ni, m, 1.0, Ri, m, Yi, n, 0.0, RY, n);             /* R Y */
      gemm(0, 0, m, mi, m, 1.0, Ri, m, Zi, m, 0.0, RZ, m);             /* R Z */
      for (int a = 0; a < m; a++) {
        double s = rz[a];
        for (int j = 0; j < m; j++) s += Ri[a * m + j] * yi[j];
        Ry[a] = s;                                                      /* R y + r^z */
      }
      ADDF(2.0 * m * m);
      /* Qbar = Q^z + M^z Y + Y^T M^z^T + Y^T R Y */
      gemm(0, 0, ni, ni, m, 1.0, Mz, m, Yi, n, 1.0, Qbi, n);
      gemm(1, 1, ni, ni, m, 1.0, Yi, n, Mz, m, 1.0, Qbi, n);
      gemm(1, 0, ni, ni, m, 1.0, Yi, n, RY, n, 1.0, Qbi, n);
      double *Mbi = Mb + (size_t)i * n * m, *Rbi = Rb + (size_t)i * m * m;
      gemm(0, 0, ni, mi, m, 1.0, Mz, m, Zi, m, 0.0, Mbi, m);           /* M^z Z */
      gemm(1, 0, ni, mi, m, 1.0, Yi, n, RZ, m, 1.0, Mbi, m);            /* + Y^T R Z */
      gemm(1, 0, mi, mi, m, 1.0, Zi, m, RZ, m, 0.0, Rbi, m);            /* Z^T R Z */
      double *qbi = qb + (size_t)i * n, *rbi = rb + (size_t)i * m;
      for (int a = 0; a < ni; a++) {
        double s = qz[a];
        for (int j = 0; j < m; j++) s += Mz[a * m + j] * yi[j];
        if (ORC_PLANT != 3)
          for (int j = 0; j < m; j++) s += Yi[j * n + a] * Ry[j];
        qbi[a] = s;
      }
      for (int a = 0; a < mi; a++) {
        double s = 0.0;
        for (int j = 0; j < m; j++) s += Zi[j * m + a] * Ry[j];
        rbi[a] = s;
      }
      ADDF(4.0 * ni * m + 2.0 * mi * m);
      /* kappa_i (eq. stage-constant) */
      {
        double s = 0.0;
        for (int a = 0; a < n; a++) {
          double w = 0.0;
          for (int j = 0; j < n; j++) w += Qi[a * n + j] * ti_[j];
          s += 0.5 * ti_[a] * w + qi[a] * ti_[a];
        }
        for (int a = 0; a < m; a++) {
          double w = 0.0;
          for (int j = 0; j < m; j++) w += Ri[a * m + j] * yi[j];
          s += 0.5 * yi[a] * w + rz[a] * yi[a];
        }
        kap[i] = s;
      }
    }
    /* terminal (eq. terminal-cost-data) */
    {
      const double *QN = P->Q + (size_t)N * n * n, *qN = P->qv + (size_t)N * n;
      const double *TN = T + (size_t)N * n * n, *tN = t + (size_t)N * n;
      int nN = nb[N];
      gemm(0, 0, n, nN, n, 1.0, QN, n, TN, n, 0.0, tmp, n);
      gemm(1, 0, nN, nN, n, 1.0, TN, n, tmp, n, 0.0, Qb + (size_t)N * n * n, n);
      double s = 0.0;
      for (int l = 0; l < n; l++) {
        double w = qN[l];
        for (int j = 0; j < n; j++) w += QN[l * n + j] * tN[j];
        tmp2[l] = w;
        double w2 = 0.0;
        for (int j = 0; j < n; j++) w2 += QN[l * n + j] * tN[j];
        s += 0.5 * tN[l] * w2 + qN[l] * tN[l];
      }
      kap[N] = s;
      gemm(1, 0, nN, 1, n, 1.0, TN, n, tmp2, 1, 0.0, qb + (size_t)N * n, 1);
    }
    free(Gm); free(Rhs); free(Sol); free(Qf); free(AT); free(tmp); free(tmp2);
    free(rz); free(qz); free(Mz); free(RY); free(RZ); free(Ry); free(BZ);
  }
  g_cur = 3;
  /* ---- 7. square-root (information form) Riccati on the reduced LQR ----
   * The paper leaves the unconstrained LQR solver open (Sec. 6).  The textbook
   * recursion P_i = Qbar + Abar'P Abar - H_ux' H_uu^{-1} H_ux cancels large
   * terms when P grows through stretches without control authority, so the
   * value functions are carried in square-root form V_i(z) = 1/2 ||R_i z + s_i||^2
   * (R_i upper triangular): with L L' the Cholesky factor of the stage Hessian
   * [[Qbar, Mbar], [Mbar', Rbar]] (order z, v), the rows
   *     [ L'_v | L'_z | L^{-1}[qbar; rbar] ]     (stage cost)
   *     [ R_{i+1} Bbar | R_{i+1} Abar | R_{i+1} cbar + s_{i+1} ]   (cost to go)
   * over the columns (v | z | 1) are reduced by Householder QR; the first mbar
   * rows give R_vv v + R_vz z + o_v = 0 at the minimiser (K, k), the next nbar
   * rows give R_i, s_i.  P_i = R_i'R_i, H_uu = R_vv'R_vv, H_ux = R_vv'R_vz. */
  {
    double *Rn = dalloc((size_t)n * n), *sn = dalloc(n), *St = dalloc((size_t)(2 * n + m) * (n + m + 1));
    double *Hs = dalloc((size_t)(n + m) * (n + m)), *lv = dalloc(n + m), *vv2 = dalloc(2 * n + m);
    int nN = nb[N];
    /* R_N = chol(Qbar_N)', s_N = R_N^{-T} qbar_N */
    for (int a = 0; a < nN; a++)
      for (int j = 0; j < nN; j++) Hs[a * nN + j] = Qb[(size_t)N * n * n + a * n + j];
    if (nN && cholesky(Hs, nN)) { status = ORC_NONCONVEX; *fail_stage = N; }
    for (int a = 0; a < nN; a++) {
      for (int j = 0; j < nN; j++) Rn[a * n + j] = Hs[j * nN + a];
      double s = qb[(size_t)N * n + a];
      for (int l = 0; l < a; l++) s -= Hs[a * nN + l] * sn[l];
      sn[a] = s / Hs[a * nN + a];
    }
    for (int a = 0; a < nN; a++) {
      for (int j = 0; j < nN; j++) {
        double s = 0.0;
        for (int l = 0; l < nN; l++) s += Rn[l * n + a] * Rn[l * n + j];
        Pst[(size_t)N * n * n + a * n + j] = s;
      }
      pst[(size_t)N * n + a] = qb[(size_t)N * n + a];
    }
    for (int i = N - 1; i >= 0 && status == ORC_OK; i--) {
      int ni = nb[i], nn = nb[i + 1], mi = mb[i];
      int k = ni + mi, rows = k + nn, ld = k + 1;
      const double *Abi = Ab + (size_t)i * n * n, *Bbi = Bb + (size_t)i * n * m, *cbi = cb + (size_t)i * n;
      /* stage Hessian in (z, v) order, Cholesky */
      for (int a = 0; a < k; a++)
        for (int j = 0; j < k; j++) {
          double h;
          if (a < ni && j < ni) h = Qb[(size_t)i * n * n + a * n + j];
          else if (a < ni) h = Mb[(size_t)i * n * m + a * m + (j - ni)];
          else if (j < ni) h = Mb[(size_t)i * n * m + j * m + (a - ni)];
          else h = Rb[(size_t)i * m * m + (a - ni) * m + (j - ni)];
          Hs[a * k + j] = h;
        }
      if (cholesky(Hs, k)) { status = ORC_NONCONVEX; *fail_stage = i; break; }
      /* l = L^{-1} [qbar; rbar] */
      for (int a = 0; a < k; a++) {
        double s = (a < ni) ? qb[(size_t)i * n + a] : rb[(size_t)i * m + (a - ni)];
        for (int l = 0; l < a; l++) s -= Hs[a * k + l] * lv[l];
        lv[a] = s / Hs[a * k + a];
      }
      /* stacked rows, columns (v | z | 1) */
      memset(St, 0, sizeof(double) * rows * ld);
      for (int a = 0; a < k; a++) {
        for (int j = 0; j < ni; j++) St[a * ld + mi + j] = Hs[j * k + a];        /* (L')_{a, z_j} */
        for (int j = 0; j < mi; j++) St[a * ld + j] = Hs[(ni + j) * k + a];     /* (L')_{a, v_j} */
        St[a * ld + k] = lv[a];
      }
      for (int a = 0; a < nn; a++) {
        int row = k + a;
        for (int j = 0; j < mi; j++) {
          double s = 0.0;
          for (int l = 0; l < nn; l++) s += ((ORC_PLANT == 4) ? Rn[l * n + a] : Rn[a * n + l]) * Bbi[l * m + j];
          St[row * ld + j] = s;
        }
        for (int j = 0; j < ni; j++) {
          double s = 0.0;
          for (int l = 0; l < nn; l++) s += ((ORC_PLANT == 4) ? Rn[l * n + a] : Rn[a * n + l]) * Abi[l * n + j];
          St[row * ld + mi + j] = s;
        }
        double s = sn[a];
        for (int l = 0; l < nn; l++) s += Rn[a * n + l] * cbi[l];
        St[row * ld + k] = s;
      }
      ADDF(2.0 * nn * nn * (mi + ni + 1) + (double)k * k * k / 3.0);
      /* Householder QR over the first k columns, no pivoting */
      for (int c = 0; c < k; c++) {
        double nrm = 0.0;
        for (int r = c; r < rows; r++) nrm += St[r * ld + c] * St[r * ld + c];
        nrm = sqrt(nrm);
        if (nrm == 0.0) continue;
        double xk = St[c * ld + c], sg = xk >= 0.0 ? 1.0 : -1.0;
        for (int r = c; r < rows; r++) vv2[r] = St[r * ld + c];
        vv2[c] = xk + sg * nrm;
        double beta = 1.0 / (nrm * (nrm + fabs(xk)));
        for (int j = c + 1; j < ld; j++) {
          double w = 0.0;
          for (int r = c; r < rows; r++) w += vv2[r] * St[r * ld + j];
          w *= beta;
          for (int r = c; r < rows; r++) St[r * ld + j] -= w * vv2[r];
        }
        St[c * ld + c] = -sg * nrm;
        for (int r = c + 1; r < rows; r++) St[r * ld + c] = 0.0;
        ADDF(4.0 * (rows - c) * (ld - c));
      }
      /* K, k: R_vv v = -(R_vz z + o_v) */
      double *Ki = Kg + (size_t)i * m * n, *ki = kg + (size_t)i * m;
      for (int col = 0; col <= ni; col++) {
        /* back substitution for column col of -[R_vz | o_v] */
        for (int a = mi - 1; a >= 0; a--) {
          double s = -St[a * ld + mi + col];
          for (int l = a + 1; l < mi; l++) s -= St[a * ld + l] * ((col < ni) ? Ki[l * n + col] : ki[l]);
          s /= St[a * ld + a];
          if (col < ni) Ki[a * n + col] = s; else ki[a] = s;
        }
      }
      /* H_uu = R_vv'R_vv -> Cholesky factor with positive diagonal; H_ux = R_vv'R_vz */
      double *Lh = Lhs + (size_t)i * m * m, *Hx = Hxs + (size_t)i * m * n;
      for (int a = 0; a < mi; a++) {
        double sga = St[a * ld + a] >= 0.0 ? 1.0 : -1.0;
        for (int j = 0; j < mi; j++) Lh[j * mi + a] = (j >= a) ? sga * St[a * ld + j] : 0.0;
      }
      for (int a = 0; a < mi; a++)
        for (int j = 0; j < ni; j++) {
          double s = 0.0;
          for (int l = 0; l <= a && l < mi; l++) s += St[l * ld + a] * St[l * ld + mi + j];
          Hx[a * n + j] = s;
        }
      /* R_i, s_i and P_i = R_i'R_i */
      for (int a = 0; a < ni; a++) {
        for (int j = 0; j < ni; j++) Rn[a * n + j] = (j >= a) ? St[(mi + a) * ld + mi + j] : 0.0;
        sn[a] = St[(mi + a) * ld + k];
      }
      for (int a = 0; a < ni; a++) {
        for (int j = 0; j < ni; j++) {
          double s = 0.0;
          for (int l = 0; l < ni; l++) s += Rn[l * n + a] * Rn[l * n + j];
          Pst[(size_t)i * n * n + a * n + j] = s;
        }
        double s = 0.0;
        for (int l = 0; l < ni; l++) s += Rn[l * n + a] * sn[l];
        pst[(size_t)i * n + a] = s;                         /* p_i = R_i' s_i */
      }
      ADDF(2.0 * ni * ni * ni + 2.0 * mi * mi * ni);
    }
    free(Rn); free(sn); free(St); free(Hs); free(lv); free(vv2);
    if (status != ORC_OK) goto done;
  }
  g_cur = 4;
  /* ---- 8. linear pass, rollout (eq. reduced-initial) and refinement on the reduced KKT ----
   * lqr_offsets(qb', rb', cb', z0') -> (z, v, pi) solves the reduced LQR with the factors above.
   * Refinement: the residual of the reduced KKT system (reduced dynamics, stationarity in z and
   * v with costates pi) is fed back as offsets of a correction solve with z0' = 0, and the
   * correction is added.  The LQR is linear in its offsets, so each pass contracts the error of
   * the Riccati factors (whose cancellation costs digits when P_i grows large). */
  {
    double *qo_ = dalloc((size_t)(N + 1) * n), *ro_ = dalloc((size_t)N * m), *co_ = dalloc((size_t)N * n);
    double *dz = dalloc((size_t)(N + 1) * n), *dv = dalloc((size_t)N * m), *dpi = dalloc((size_t)(N + 1) * n);
    double *pv = dalloc(n), *w = dalloc(n), *hu = dalloc(m);
    double *xr_ = dalloc(n), *uu_ = dalloc(m), *lh_ = dalloc(n), *ga_ = dalloc(n), *gb_ = dalloc(m);
    memcpy(qo_, qb, sizeof(double) * (N + 1) * n);
    memcpy(ro_, rb, sizeof(double) * N * m);
    memcpy(co_, cb, sizeof(double) * N * n);
    /* z_0 = S_0 (s_0 - t_0), S_0 = T_0^T */
    double *z0 = dalloc(n);
    for (int a = 0; a < nb[0]; a++) {
      double s = 0.0;
      for (int l = 0; l < n; l++) s += T[l * n + a] * (P->s0[l] - t[l]);
      z0[a] = s;
    }
    for (int pass = 0; pass <= opt->refine; pass++) {
      double *Z_ = pass ? dz : zz, *V_ = pass ? dv : vv, *PI_ = pass ? dpi : pis;
      /* linear pass (pass 0 takes p_i, k_i from the square-root recursion) */
      int nN = nb[N];
      if (pass) {
      for (int a = 0; a < nN; a++) pv[a] = qo_[(size_t)N * n + a];
      memcpy(pst + (size_t)N * n, pv, sizeof(double) * n);
      for (int i = N - 1; i >= 0; i--) {
        int ni = nb[i], nn = nb[i + 1], mi = mb[i];
        const double *Abi = Ab + (size_t)i * n * n, *Bbi = Bb + (size_t)i * n * m;
        const double *Pnx = Pst + (size_t)(i + 1) * n * n;
        double *ki = kg + (size_t)i * m;
        for (int a = 0; a < nn; a++) {
          double s = pv[a];
          for (int j = 0; j < nn; j++) s += Pnx[a * n + j] * co_[(size_t)i * n + j];
          w[a] = s;                                       /* P c + p */
        }
        for (int a = 0; a < mi; a++) {
          double s = ro_[(size_t)i * m + a];
          for (int l = 0; l < nn; l++) s += Bbi[l * m + a] * w[l];
          hu[a] = s;                                      /* r + B^T (P c + p) */
        }
        if (mi) chol_solve(Lhs + (size_t)i * m * m, mi, hu, 1);
        for (int a = 0; a < mi; a++) ki[a] = -hu[a];
        for (int a = 0; a < ni; a++) {
          double s = qo_[(size_t)i * n + a];
          for (int l = 0; l < nn; l++) s += Abi[l * n + a] * w[l];
          for (int l = 0; l < mi; l++) s += Hxs[(size_t)i * m * n + l * n + a] * ki[l];
          pv[a] = s;
        }
        memcpy(pst + (size_t)i * n, pv, sizeof(double) * n);
        ADDF(2.0 * nn * nn + 2.0 * mi * nn + 2.0 * ni * (nn + mi));
      }
      }
      /* rollout v = K z + k, z+ = Abar z + Bbar v + cbar; costates pi = P z + p */
      for (int a = 0; a < nb[0]; a++) Z_[a] = pass ? 0.0 : z0[a];
      for (int i = 0; i < N; i++) {
        int ni = nb[i], nn = nb[i + 1], mi = mb[i];
        double *zi = Z_ + (size_t)i * n, *vi = V_ + (size_t)i * m, *zn = Z_ + (size_t)(i + 1) * n;
        for (int a = 0; a < mi; a++) {
          double s = kg[(size_t)i * m + a];
          for (int j = 0; j < ni; j++) s += Kg[(size_t)i * m * n + a * n + j] * zi[j];
          vi[a] = s;
        }
        for (int a = 0; a < nn; a++) {
          double s = (ORC_PLANT == 14) ? 0.0 : co_[(size_t)i * n + a];
          for (int j = 0; j < ni; j++) s += Ab[(size_t)i * n * n + a * n + j] * zi[j];
          for (int j = 0; j < mi; j++) s += Bb[(size_t)i * n * m + a * m + j] * vi[j];
          zn[a] = s;
        }
        ADDF(2.0 * mi * ni + 2.0 * nn * (ni + mi));
      }
      for (int i = 0; i <= N; i++)
        for (int a = 0; a < nb[i]; a++) {
          double s = pst[(size_t)i * n + a];
          for (int j = 0; j < nb[i]; j++) s += Pst[(size_t)i * n * n + a * n + j] * Z_[(size_t)i * n + j];
          PI_[(size_t)i * n + a] = s;
        }
      if (pass) {
        const double sgn = (ORC_PLANT == 11) ? -1.0 : 1.0;
        for (size_t k = 0; k < (size_t)(N + 1) * n; k++) { zz[k] += sgn * dz[k]; pis[k] += sgn * dpi[k]; }
        for (size_t k = 0; k < (size_t)N * m; k++) vv[k] += sgn * dv[k];
      }
      if (pass == opt->refine) break;
      /* residual of the reduced KKT system, evaluated through the original data.
       * Under x_i = T_i z_i + t_i, u_i = Y_i z_i + Z_i v_i + y_i (Thm 5 substitution) the
       * z- and v-gradients of the reduced Lagrangian are T_i'a_i + Y_i'b_i - pi_i and Z_i'b_i,
       * with a_i = g^x_i + A_i' T_{i+1} pi_{i+1} and b_i = g^u_i + B_i' T_{i+1} pi_{i+1}.
       * Forming Qbar z + qbar instead sums terms of size |Y_i|^2, which cancel down to
       * pi_i: where the mixed rows leave D_i ill-conditioned |Y_i| is large and that
       * cancellation, not the solve, sets the accuracy of the multipliers. */
      for (int i = 0; i <= N; i++) {
        int ni = nb[i], nn = (i < N) ? nb[i + 1] : 0, mi = (i < N) ? mb[i] : 0;
        const double *zi = zz + (size_t)i * n, *pii = pis + (size_t)i * n, *Ti = T + (size_t)i * n * n;
        for (int a = 0; a < n; a++) {
          double s = t[(size_t)i * n + a];
          for (int j = 0; j < ni; j++) s += Ti[a * n + j] * zi[j];
          xr_[a] = s;
        }
        if (i < N) {
          const double *Tn = T + (size_t)(i + 1) * n * n, *pn = pis + (size_t)(i + 1) * n;
          for (int a = 0; a < m; a++) {
            double s = yv[(size_t)i * m + a];
            for (int j = 0; j < ni; j++) s += Y[(size_t)i * m * n + a * n + j] * zi[j];
            for (int j = 0; j < mi; j++) s += Z[(size_t)i * m * m + a * m + j] * vv[(size_t)i * m + j];
            uu_[a] = s;
          }
          for (int l = 0; l < n; l++) {
            double s = 0.0;
            for (int j = 0; j < nn; j++) s += Tn[l * n + j] * pn[j];
            lh_[l] = s;                                   /* T_{i+1} pi_{i+1} */
          }
        }
        for (int a = 0; a < n; a++) {
          double s = P->qv[(size_t)i * n + a];
          for (int j = 0; j < n; j++) s += P->Q[(size_t)i * n * n + a * n + j] * xr_[j];
          if (i < N) {
            for (int j = 0; j < m; j++) s += P->M[(size_t)i * n * m + a * m + j] * uu_[j];
            for (int l = 0; l < n; l++) s += P->A[(size_t)i * n * n + l * n + a] * lh_[l];
          }
          ga_[a] = s;
        }
        if (i < N)
          for (int a = 0; a < m; a++) {
            double s = P->rv[(size_t)i * m + a];
            for (int j = 0; j < n; j++) s += P->M[(size_t)i * n * m + j * m + a] * xr_[j];
            for (int j = 0; j < m; j++) s += P->R[(size_t)i * m * m + a * m + j] * uu_[j];
            for (int l = 0; l < n; l++) s += P->B[(size_t)i * n * m + l * m + a] * lh_[l];
            gb_[a] = s;
          }
        for (int a = 0; a < ni; a++) {
          double s = -pii[a];
          for (int l = 0; l < n; l++) s += Ti[l * n + a] * ga_[l];
          if (i < N)
            for (int l = 0; l < m; l++) s += Y[(size_t)i * m * n + l * n + a] * gb_[l];
          qo_[(size_t)i * n + a] = s;
        }
        if (i < N) {
          for (int a = 0; a < mi; a++) {
            double s = 0.0;
            for (int l = 0; l < m; l++) s += Z[(size_t)i * m * m + l * m + a] * gb_[l];
            ro_[(size_t)i * m + a] = s;
          }
          for (int a = 0; a < nn; a++) {
            double s = cb[(size_t)i * n + a] - zz[(size_t)(i + 1) * n + a];
            for (int j = 0; j < ni; j++) s += Ab[(size_t)i * n * n + a * n + j] * zi[j];
            for (int j = 0; j < mi; j++) s += Bb[(size_t)i * n * m + a * m + j] * vv[(size_t)i * m + j];
            co_[(size_t)i * n + a] = s;
          }
        }
        /* products with T_i = I (ur = 0: x = z, the T' part of the z residual) or T_{i+1} = I
           are their other factor: not counted as work (as in step 5) */
        const int tei = ur[i] == 0, ten = i < N && ur[i + 1] == 0;
        ADDF(2.0 * n * ni + 2.0 * m * (ni + mi) + 2.0 * n * nn + 2.0 * n * (2 * n + m) + 2.0 * m * (2 * n + m) +
             2.0 * ni * (n + m) + 2.0 * mi * m + 2.0 * nn * (ni + mi) - (tei ? 4.0 * n * ni : 0.0) -
             (ten ? 2.0 * n * nn : 0.0));
      }
    }
    free(qo_); free(ro_); free(co_); free(dz); free(dv); free(dpi); free(pv); free(w); free(hu); free(z0);
    free(xr_); free(uu_); free(lh_); free(ga_); free(gb_);
  }
  /* recovery (eq. recovery-maps) */
  {
    for (int i = 0; i <= N; i++) {
      int ni = nb[i];
      for (int a = 0; a < n; a++) {
        double s = t[(size_t)i * n + a];
        for (int j = 0; j < ni; j++) s += T[(size_t)i * n * n + a * n + j] * zz[(size_t)i * n + j];
        x[(size_t)i * n + a] = s;
      }
      ADDF(2.0 * n * ni);
    }
    for (int i = 0; i < N; i++) {
      int ni = nb[i], mi = mb[i];
      for (int a = 0; a < m; a++) {
        double s = yv[(size_t)i * m + a];
        for (int j = 0; j < ni; j++) s += Y[(size_t)i * m * n + a * n + j] * zz[(size_t)i * n + j];
        for (int j = 0; j < mi; j++) s += Z[(size_t)i * m * m + a * m + j] * vv[(size_t)i * m + j];
        u[(size_t)i * m + a] = s;
      }
      ADDF(2.0 * m * (ni + mi));
    }
  }
  g_cur = 5;
  /* ---- 9. multipliers (Sec. 7), in the normal coordinates of the domains ----
   * For any KKT multiplier, the chain rule through x = T z + t, u = Y z + Z v + y
   * turns the original Lagrangian into the reduced one with costates
   * T_i^T lambda_i (Thm 5 substitution), so T_i^T lambda_i = pi_i := P_i z_i + p_i,
   * the reduced LQR costate.  Writing lambda_i = T_i pi_i + U_i nu_i, with U_i an
   * orthonormal basis of range(H_i^T), the stationarity equations (eqs.
   * stage-stationarity, terminal-stationarity) restricted to the directions they
   * do not already satisfy are
   *   (a) U_i^T C_i^T mu_i + U_i^T E_i^T eta_i + U_i^T A_i^T U_{i+1} nu_{i+1} - nu_i
   *         + U_i^T (g^x_i + A_i^T T_{i+1} pi_{i+1}) = 0
   *   (b) D_i^T mu_i + B_i^T U_{i+1} nu_{i+1} + (g^u_i + B_i^T T_{i+1} pi_{i+1}) = 0
   *   (N) U_N^T E_N^T eta_N - nu_N + U_N^T g^x_N = 0.
   * These are dual endpoint relations between nu_i and nu_{i+1}; the procedure of
   * Sec. 7 is applied to them: admissible sets right to left by projecting out
   * (mu_i, eta_i) and nu_{i+1}, min-norm nu_0, forward substitution choosing the
   * min-norm nu_{i+1}, then min-norm leaf solves.  Since ||lambda_i||^2 =
   * ||pi_i||^2 + ||nu_i||^2, this is the min-norm-lambda representative of the
   * sequential variant, computed without propagating the tangential part. */
  if (lam) {
    const int lld = n + 1;
    double *Ls = dalloc((size_t)(N + 1) * n * lld);   /* admissible nu-sets [H^nu | h^nu] */
    int *lr = (int *)calloc(N + 1, sizeof(int));
    double *gx = dalloc((size_t)(N + 1) * n), *gu = dalloc((size_t)N * m);
    double *nus = dalloc((size_t)(N + 1) * n);
    double *rx = dalloc((size_t)N * n), *ru = dalloc((size_t)N * m);
    /* objective gradients (eq. objective-gradients) */
    for (int i = 0; i <= N; i++) {
      const double *Qi = P->Q + (size_t)i * n * n, *xi = x + (size_t)i * n;
      for (int a = 0; a < n; a++) {
        double s = P->qv[(size_t)i * n + a];
        for (int j = 0; j < n; j++) s += Qi[a * n + j] * xi[j];
        if (i < N)
          for (int j = 0; j < m; j++) s += P->M[(size_t)i * n * m + a * m + j] * u[(size_t)i * m + j];
        gx[(size_t)i * n + a] = s;
      }
    }
    for (int i = 0; i < N; i++)
      for (int a = 0; a < m; a++) {
        double s = P->rv[(size_t)i * m + a];
        for (int j = 0; j < n; j++) s += P->M[(size_t)i * n * m + j * m + a] * x[(size_t)i * n + j];
        for (int j = 0; j < m; j++) s += P->R[(size_t)i * m * m + a * m + j] * u[(size_t)i * m + j];
        gu[(size_t)i * m + a] = s;
      }
    ADDF(2.0 * (N + 1) * n * (n + m) + 2.0 * N * m * (n + m));
    /* reduced costates pi_i: refined above */
    /* rho^x_i = g^x_i + A_i^T T_{i+1} pi_{i+1}, rho^u_i = g^u_i + B_i^T T_{i+1} pi_{i+1} */
    {
      double *tp = dalloc(n);
      for (int i = 0; i < N; i++) {
        const double *Tn = T + (size_t)(i + 1) * n * n, *pn = pis + (size_t)(i + 1) * n;
        for (int l = 0; l < n; l++) {
          double s = 0.0;
          for (int j = 0; j < nb[i + 1]; j++) s += Tn[l * n + j] * pn[j];
          tp[l] = s;
        }
        for (int a = 0; a < n; a++) {
          double s = gx[(size_t)i * n + a];
          for (int l = 0; l < n; l++) s += P->A[(size_t)i * n * n + l * n + a] * tp[l];
          rx[(size_t)i * n + a] = s;
        }
        for (int a = 0; a < m; a++) {
          double s = gu[(size_t)i * m + a];
          if (ORC_PLANT != 8)
            for (int l = 0; l < n; l++) s += P->B[(size_t)i * n * m + l * m + a] * tp[l];
          ru[(size_t)i * m + a] = s;
        }
      }
      /* T_{i+1} pi_{i+1} with T_{i+1} = I (ur = 0) is pi_{i+1}: not counted (as in step 5) */
      int eye1 = 0;
      for (int i = 0; i < N; i++) eye1 += ur[i + 1] == 0;
      ADDF((double)N * (2.0 * n * n + 2.0 * n * (n + m)) - 2.0 * n * n * eye1);
      free(tp);
    }
    int wr = n + m + n;
    int wc = pmax + qmax + n + n + 1;
    double *Wd = dalloc((size_t)wr * wc);
    double *UA = dalloc((size_t)n * n);   /* U_i^T A_i^T U_{i+1} (r_i x r_{i+1}) */
    double *BU = dalloc((size_t)m * n);   /* B_i^T U_{i+1} (m x r_{i+1}) */
    double *UC = dalloc((size_t)n * (pmax + qmax + 1)); /* U_i^T [C_i^T E_i^T] */
    double *Ux_ = dalloc(n);
    /* stage-i blocks shared by the backward and forward passes */
#define UX(i, l, k) Ux[(size_t)(i) * n * n + (size_t)(l) * n + (k)]
#define STAGE_BLOCKS(i)                                                              \
    do {                                                                             \
      int r0 = ur[i], r1 = ur[(i) + 1], pi = P->p[i], qi = P->q[i];                  \
      const double *Ai = P->A + (size_t)(i) * n * n, *Bi = P->B + (size_t)(i) * n * m; \
      for (int a = 0; a < r0; a++)                                                   \
        for (int b = 0; b < r1; b++) {                                               \
          double s = 0.0;                                                            \
          for (int l = 0; l < n; l++) {                                              \
            double w = 0.0;                                                          \
            for (int k = 0; k < n; k++) w += Ai[k * n + l] * UX((i) + 1, k, b);      \
            s += UX(i, l, a) * w;                                                    \
          }                                                                          \
          UA[a * n + b] = s;                                                         \
        }                                                                            \
      for (int a = 0; a < m; a++)                                                    \
        for (int b = 0; b < r1; b++) {                                               \
          double s = 0.0;                                                            \
          for (int k = 0; k < n; k++) s += Bi[k * m + a] * UX((i) + 1, k, b);        \
          BU[a * n + b] = s;                                                         \
        }                                                                            \
      for (int a = 0; a < r0; a++) {                                                 \
        for (int j = 0; j < pi; j++) {                                               \
          double s = 0.0;                                                            \
          for (int l = 0; l < n; l++) s += UX(i, l, a) * P->C[(size_t)(po[i] + j) * n + l]; \
          UC[a * (pmax + qmax + 1) + j] = s;                                         \
        }                                                                            \
        for (int j = 0; j < qi; j++) {                                               \
          double s = 0.0;                                                            \
          for (int l = 0; l < n; l++) s += UX(i, l, a) * P->E[(size_t)(qo[i] + j) * n + l]; \
          UC[a * (pmax + qmax + 1) + pi + j] = s;                                    \
        }                                                                            \
        double s = 0.0;                                                              \
        for (int l = 0; l < n; l++) s += UX(i, l, a) * rx[(size_t)(i) * n + l];      \
        Ux_[a] = s;                                                                  \
      }                                                                              \
      ADDF(2.0 * r0 * r1 * n * (n + 1) + 2.0 * m * r1 * n + 2.0 * r0 * n * (pi + qi + 1)); \
    } while (0)
    /* terminal relation (N): project eta_N */
    {
      int qN = P->q[N], rN = ur[N];
      int nc = qN + rN + 1;
      memset(Wd, 0, sizeof(double) * (rN ? rN : 1) * nc);
      for (int a = 0; a < rN; a++) {
        for (int j = 0; j < qN; j++) {
          double s = 0.0;
          for (int l = 0; l < n; l++) s += UX(N, l, a) * P->E[(size_t)(qo[N] + j) * n + l];
          Wd[a * nc + j] = s;
        }
        Wd[a * nc + qN + a] = -1.0;
        double s = 0.0;
        for (int l = 0; l < n; l++) s += UX(N, l, a) * gx[(size_t)N * n + l];
        Wd[a * nc + qN + rN] = s;
      }
      int gs[1] = {qN};
      double *outp = dalloc((size_t)(rN ? rN : 1) * (rN + 1));
      project(Wd, rN, nc, 1, gs, rN, tr, ti, grank, &krank, &inc, outp);
      lr[N] = krank;
      for (int a = 0; a < krank; a++)
        for (int b = 0; b <= rN; b++) Ls[(size_t)N * n * lld + a * lld + b] = outp[a * (rN + 1) + b];
      free(outp);
      /* an inconsistent leftover row was dropped (step 9) */
    }
    /* right to left: N_i = D'_i o N_{i+1} */
    for (int i = N - 1; i >= 0; i--) {
      int r0 = ur[i], r1 = ur[i + 1], pi = P->p[i], qi = P->q[i], nw = pi + qi, rn = lr[i + 1];
      STAGE_BLOCKS(i);
      int nc = nw + r1 + r0 + 1;
      int rows = r0 + m + rn;
      memset(Wd, 0, sizeof(double) * (rows ? rows : 1) * nc);
      for (int a = 0; a < r0; a++) {
        for (int j = 0; j < nw; j++) Wd[a * nc + j] = UC[a * (pmax + qmax + 1) + j];
        for (int b = 0; b < r1; b++) Wd[a * nc + nw + b] = UA[a * n + b];
        Wd[a * nc + nw + r1 + a] = (ORC_PLANT == 5) ? 1.0 : -1.0;
        Wd[a * nc + nw + r1 + r0] = Ux_[a];
      }
      for (int a = 0; a < m; a++) {
        int row = r0 + a;
        for (int j = 0; j < pi; j++) Wd[row * nc + j] = P->D[(size_t)(po[i] + j) * m + a];
        for (int b = 0; b < r1; b++) Wd[row * nc + nw + b] = BU[a * n + b];
        Wd[row * nc + nw + r1 + r0] = ru[(size_t)i * m + a];
      }
      for (int a = 0; a < rn; a++) {
        int row = r0 + m + a;
        for (int b = 0; b < r1; b++) Wd[row * nc + nw + b] = Ls[(size_t)(i + 1) * n * lld + a * lld + b];
        Wd[row * nc + nw + r1 + r0] = Ls[(size_t)(i + 1) * n * lld + a * lld + r1];
      }
      int gs[2] = {nw, r1};
      double *outp = dalloc((size_t)(rows ? rows : 1) * (r0 + 1));
      /* with r0 = r1 = 0 nothing is kept (N_i has no coordinates) and the projection only
         finds rows 0 = const, which step 9 drops: a solver skips it, so it is not counted */
      g_uncounted = r0 == 0 && r1 == 0;
      project(Wd, rows, nc, 2, gs, r0, tr, ti, grank, &krank, &inc, outp);
      g_uncounted = 0;
      lr[i] = krank;
      for (int a = 0; a < krank; a++)
        for (int b = 0; b <= r0; b++) Ls[(size_t)i * n * lld + a * lld + b] = outp[a * (r0 + 1) + b];
      free(outp);
      /* an inconsistent leftover row was dropped (step 9) */
    }
    /* root: min-norm nu_0 in N_0 */
    {
      int r0 = ur[0];
      double *Kb = dalloc((size_t)n * n), *bb = dalloc(n), rs;
      for (int a = 0; a < lr[0]; a++) {
        for (int l = 0; l < r0; l++) Kb[a * r0 + l] = Ls[a * lld + l];
        bb[a] = Ls[a * lld + r0];
      }
      for (int l = 0; l < n; l++) nus[l] = 0.0;
      if (lr[0] > 0 && r0 > 0) tqr_solve(Kb, lr[0], r0, tr, bb, 1, nus, NULL, &rs);
      free(Kb); free(bb);
    }
    /* forward substitution (min-norm nu_{i+1}) and leaf solves (min-norm mu_i, eta_i) */
    {
      double *Kb = dalloc((size_t)(n + m + n) * n), *bb = dalloc(n + m + n), rs;
      double *Fl = dalloc((size_t)(n + m) * (pmax + qmax + 1)), *rhs = dalloc(n + m), *wsol = dalloc(pmax + qmax + 1);
      for (int i = 0; i < N; i++) {
        int r0 = ur[i], r1 = ur[i + 1], pi = P->p[i], qi = P->q[i], nw = pi + qi, rn = lr[i + 1];
        STAGE_BLOCKS(i);
        const double *nu0 = nus + (size_t)i * n;
        double *nu1 = nus + (size_t)(i + 1) * n;
        int nc = nw + r1 + 1;
        int rows = r0 + m + rn;
        memset(Wd, 0, sizeof(double) * (rows ? rows : 1) * nc);
        for (int a = 0; a < r0; a++) {
          for (int j = 0; j < nw; j++) Wd[a * nc + j] = UC[a * (pmax + qmax + 1) + j];
          for (int b = 0; b < r1; b++) Wd[a * nc + nw + b] = UA[a * n + b];
          Wd[a * nc + nw + r1] = Ux_[a] + ((ORC_PLANT == 5) ? nu0[a] : -nu0[a]);
        }
        for (int a = 0; a < m; a++) {
          int row = r0 + a;
          for (int j = 0; j < pi; j++) Wd[row * nc + j] = P->D[(size_t)(po[i] + j) * m + a];
          for (int b = 0; b < r1; b++) Wd[row * nc + nw + b] = BU[a * n + b];
          Wd[row * nc + nw + r1] = ru[(size_t)i * m + a];
        }
        for (int a = 0; a < rn; a++) {
          int row = r0 + m + a;
          for (int b = 0; b < r1; b++) Wd[row * nc + nw + b] = Ls[(size_t)(i + 1) * n * lld + a * lld + b];
          Wd[row * nc + nw + r1] = Ls[(size_t)(i + 1) * n * lld + a * lld + r1];
        }
        int gs[1] = {nw};
        double *rel = dalloc((size_t)(rows ? rows : 1) * (r1 + 1));
        project(Wd, rows, nc, 1, gs, r1, tr, ti, grank, &krank, &inc, rel);
        /* an inconsistent leftover row was dropped (step 9) */
        for (int l = 0; l < n; l++) nu1[l] = 0.0;
        if (krank > 0 && r1 > 0) {
          for (int a = 0; a < krank; a++) {
            for (int l = 0; l < r1; l++) Kb[a * r1 + l] = rel[a * (r1 + 1) + l];
            bb[a] = rel[a * (r1 + 1) + r1];
          }
          tqr_solve(Kb, krank, r1, tr, bb, 1, nu1, NULL, &rs);
        }
        free(rel);
        /* leaf: [[U^T C^T, U^T E^T]; [D^T, 0]] w = -rhs */
        if (nw > 0) {
          for (int a = 0; a < r0; a++) {
            for (int j = 0; j < nw; j++) Fl[a * nw + j] = UC[a * (pmax + qmax + 1) + j];
            double s = Ux_[a] + ((ORC_PLANT == 5) ? nu0[a] : -nu0[a]);
            for (int b = 0; b < r1; b++) s += UA[a * n + b] * nu1[b];
            rhs[a] = s;
          }
          for (int a = 0; a < m; a++) {
            for (int j = 0; j < pi; j++) Fl[(r0 + a) * nw + j] = P->D[(size_t)(po[i] + j) * m + a];
            for (int j = 0; j < qi; j++) Fl[(r0 + a) * nw + pi + j] = 0.0;
            double s = ru[(size_t)i * m + a];
            if (ORC_PLANT != 12)
              for (int b = 0; b < r1; b++) s += BU[a * n + b] * nu1[b];
            rhs[r0 + a] = s;
          }
          ADDF(2.0 * (r0 + m) * r1);
          tqr_solve(Fl, r0 + m, nw, tr, rhs, 1, wsol, NULL, &rs);
          for (int j = 0; j < pi; j++) mu[po[i] + j] = wsol[j];
          for (int j = 0; j < qi; j++) eta[qo[i] + j] = wsol[pi + j];
        }
      }
      /* terminal leaf: U_N^T E_N^T eta_N = nu_N - U_N^T g_N */
      if (status == ORC_OK && P->q[N] > 0) {
        int qN = P->q[N], rN = ur[N];
        for (int a = 0; a < rN; a++) {
          double s = 0.0;
          for (int j = 0; j < qN; j++) {
            double w = 0.0;
            for (int l = 0; l < n; l++) w += UX(N, l, a) * P->E[(size_t)(qo[N] + j) * n + l];
            Fl[a * qN + j] = w;
          }
          for (int l = 0; l < n; l++) s += UX(N, l, a) * gx[(size_t)N * n + l];
          rhs[a] = (ORC_PLANT == 13) ? s + nus[(size_t)N * n + a] : s - nus[(size_t)N * n + a];
        }
        for (int j = 0; j < qN; j++) wsol[j] = 0.0;
        if (rN > 0) tqr_solve(Fl, rN, qN, tr, rhs, 1, wsol, NULL, &rs);
        for (int j = 0; j < qN; j++) eta[qo[N] + j] = wsol[j];
      }
      free(Kb); free(bb); free(Fl); free(rhs); free(wsol);
    }
    /* lambda_i = T_i pi_i + U_i nu_i ; alpha = -lambda_0 */
    if (status == ORC_OK) {
      for (int i = 0; i <= N; i++)
        for (int l = 0; l < n; l++) {
          double s = 0.0;
          for (int j = 0; j < nb[i]; j++) s += T[(size_t)i * n * n + l * n + j] * pis[(size_t)i * n + j];
          for (int a = 0; a < ur[i]; a++) s += UX(i, l, a) * nus[(size_t)i * n + a];
          lam[(size_t)i * n + l] = s;
        }
      /* lambda_i = pi_i where T_i = I and nu_i has no coordinates (ur = 0): not counted */
      int eye0 = 0;
      for (int i = 0; i <= N; i++) eye0 += ur[i] == 0;
      ADDF(2.0 * (N + 1) * n * n - 2.0 * n * n * eye0);
      for (int l = 0; l < n; l++) alpha[l] = -lam[l];
    }
#undef STAGE_BLOCKS
#undef UX
    if (dbg && dbg->lrows) memcpy(dbg->lrows, lr, sizeof(int) * (N + 1));
    if (dbg && dbg->L) memcpy(dbg->L, Ls, sizeof(double) * (N + 1) * n * lld);
    free(Ls); free(lr); free(gx); free(gu); free(Wd); free(nus); free(rx); free(ru);
    free(UA); free(BU); free(UC); free(Ux_);
  }

done:
  if (dbg) {
    if (dbg->nbar) memcpy(dbg->nbar, nb, sizeof(int) * (N + 1));
    if (dbg->mbar) memcpy(dbg->mbar, mb, sizeof(int) * N);
    if (dbg->hrows) memcpy(dbg->hrows, hr, sizeof(int) * (N + 1));
    if (dbg->H) memcpy(dbg->H, H, sizeof(double) * (N + 1) * n * hld);
    if (dbg->T) memcpy(dbg->T, T, sizeof(double) * (N + 1) * n * n);
    if (dbg->t) memcpy(dbg->t, t, sizeof(double) * (N + 1) * n);
    if (dbg->Y) memcpy(dbg->Y, Y, sizeof(double) * N * m * n);
    if (dbg->Z) memcpy(dbg->Z, Z, sizeof(double) * N * m * m);
    if (dbg->y) memcpy(dbg->y, yv, sizeof(double) * N * m);
    if (dbg->Abar) memcpy(dbg->Abar, Ab, sizeof(double) * N * n * n);
    if (dbg->Bbar) memcpy(dbg->Bbar, Bb, sizeof(double) * N * n * m);
    if (dbg->cbar) memcpy(dbg->cbar, cb, sizeof(double) * N * n);
    if (dbg->Qbar) memcpy(dbg->Qbar, Qb, sizeof(double) * (N + 1) * n * n);
    if (dbg->Mbar) memcpy(dbg->Mbar, Mb, sizeof(double) * N * n * m);
    if (dbg->Rbar) memcpy(dbg->Rbar, Rb, sizeof(double) * N * m * m);
    if (dbg->qbar) memcpy(dbg->qbar, qb, sizeof(double) * (N + 1) * n);
    if (dbg->rbar) memcpy(dbg->rbar, rb, sizeof(double) * N * m);
    if (dbg->kappa) memcpy(dbg->kappa, kap, sizeof(double) * (N + 1));
    if (dbg->z) memcpy(dbg->z, zz, sizeof(double) * (N + 1) * n);
    if (dbg->pi) memcpy(dbg->pi, pis, sizeof(double) * (N + 1) * n);
    if (dbg->UT) memcpy(dbg->UT, Ux, sizeof(double) * (N + 1) * n * n);
    if (dbg->v) memcpy(dbg->v, vv, sizeof(double) * N * m);
  }
  free(po); free(qo); free(H); free(hr); free(T); free(t); free(nb); free(mb);
  free(Y); free(Z); free(yv); free(Ab); free(Bb); free(cb); free(Qb); free(Mb); free(Rb);
  free(qb); free(rb); free(kap); free(Kg); free(kg); free(zz); free(vv); free(work);
  free(Ux); free(ur); free(Pst); free(pst); free(Lhs); free(Hxs); free(pis);
  return status;
}

/* ------------------------------------------------------------------ */
/* KKT residual of the original problem (Sec. 9 residual definition)    */
/* ------------------------------------------------------------------ */
/* The larger of a and b; NaN when either is NaN (fmax would drop it). */
static double nanmax(double a, double b) { return (a > b || a != a) ? a : b; }

/*
 * Residual rows of the KKT system at (x, u, lam, mu, eta, alpha), in the
 * layout of the problem's offsets (Sec. 7 sign convention, lambda_0 = -alpha):
 *   rs0 (n)          x_0 - s_0
 *   rc  (N x n)      A_i x_i + B_i u_i + c_i - x_{i+1}
 *   rd  (sum p)      C_i x_i + D_i u_i + d_i
 *   re  (sum q)      E_i x_i + e_i
 *   rq  ((N+1) x n)  Q_i x_i + M_i u_i + q_i + A_i' lam_{i+1} - lam_i + C_i' mu_i + E_i' eta_i
 *                    (stage 0: + alpha for - lam_0; stage N: Q_N x_N + q_N - lam_N + E_N' eta_N)
 *   rr  (N x m)      M_i' x_i + R_i u_i + r_i + B_i' lam_{i+1} + D_i' mu_i
 */
static void kkt_rows(const orc_problem *P, const double *x, const double *u, const double *lam,
                     const double *mu, const double *eta, const double *alpha, double *rs0, double *rc,
                     double *rd, double *re, double *rq, double *rr) {
  const int N = P->N, n = P->n, m = P->m;
  int po = 0, qo = 0;
  for (int a = 0; a < n; a++) rs0[a] = x[a] - P->s0[a];
  for (int i = 0; i <= N; i++) {
    const double *xi = x + (size_t)i * n, *li = lam + (size_t)i * n;
    int pi = i < N ? P->p[i] : 0, qi = P->q[i];
    if (i < N) {
      const double *Ai = P->A + (size_t)i * n * n, *Bi = P->B + (size_t)i * n * m;
      const double *ui = u + (size_t)i * m, *xn = x + (size_t)(i + 1) * n, *ln = lam + (size_t)(i + 1) * n;
      for (int a = 0; a < n; a++) {
        double s = P->c[(size_t)i * n + a] - xn[a];
        for (int j = 0; j < n; j++) s += Ai[a * n + j] * xi[j];
        for (int j = 0; j < m; j++) s += Bi[a * m + j] * ui[j];
        rc[(size_t)i * n + a] = s;
      }
      for (int k = 0; k < pi; k++) {
        const double *Ck = P->C + (size_t)(po + k) * n, *Dk = P->D + (size_t)(po + k) * m;
        double s = P->d[po + k];
        for (int j = 0; j < n; j++) s += Ck[j] * xi[j];
        for (int j = 0; j < m; j++) s += Dk[j] * ui[j];
        rd[po + k] = s;
      }
      for (int a = 0; a < m; a++) {
        double s = P->rv[(size_t)i * m + a];
        for (int j = 0; j < n; j++) s += P->M[(size_t)i * n * m + j * m + a] * xi[j];
        for (int j = 0; j < m; j++) s += P->R[(size_t)i * m * m + a * m + j] * ui[j];
        for (int j = 0; j < n; j++) s += Bi[j * m + a] * ln[j];
        for (int k = 0; k < pi; k++) s += P->D[(size_t)(po + k) * m + a] * mu[po + k];
        rr[(size_t)i * m + a] = s;
      }
      for (int a = 0; a < n; a++) {
        double s = P->qv[(size_t)i * n + a];
        for (int j = 0; j < n; j++) s += P->Q[(size_t)i * n * n + a * n + j] * xi[j];
        for (int j = 0; j < m; j++) s += P->M[(size_t)i * n * m + a * m + j] * ui[j];
        s += (i == 0) ? alpha[a] : -li[a];
        for (int j = 0; j < n; j++) s += Ai[j * n + a] * ln[j];
        for (int k = 0; k < pi; k++) s += P->C[(size_t)(po + k) * n + a] * mu[po + k];
        for (int k = 0; k < qi; k++) s += P->E[(size_t)(qo + k) * n + a] * eta[qo + k];
        rq[(size_t)i * n + a] = s;
      }
    } else {
      for (int a = 0; a < n; a++) {
        double s = P->qv[(size_t)N * n + a] - li[a];
        for (int j = 0; j < n; j++) s += P->Q[(size_t)N * n * n + a * n + j] * xi[j];
        for (int k = 0; k < qi; k++) s += P->E[(size_t)(qo + k) * n + a] * eta[qo + k];
        rq[(size_t)N * n + a] = s;
      }
    }
    for (int k = 0; k < qi; k++) {
      const double *Ek = P->E + (size_t)(qo + k) * n;
      double s = P->e[qo + k];
      for (int j = 0; j < n; j++) s += Ek[j] * xi[j];
      re[qo + k] = s;
    }
    po += pi;
    qo += qi;
  }
}

static void row_counts(const orc_problem *P, int *ptot, int *qtot) {
  int a = 0, b = 0;
  for (int i = 0; i < P->N; i++) a += P->p[i];
  for (int i = 0; i <= P->N; i++) b += P->q[i];
  *ptot = a;
  *qtot = b;
}

/*
 * Infinity norm over: x_0 - s_0; dynamics; mixed and state-only rows, each
 * divided by max(1, largest |coefficient|, |offset|) of its row; stationarity
 * (unnormalised).  parts = {initial, dynamics, equalities, stationarity}.
 * Any non-finite row makes the result (and its part) NaN.
 */
double orc_kkt_residual(const orc_problem *P, const double *x, const double *u,
                        const double *lam, const double *mu, const double *eta,
                        const double *alpha, double *parts) {
  const int N = P->N, n = P->n, m = P->m;
  int pt, qt;
  row_counts(P, &pt, &qt);
  double *rs0 = dalloc(n), *rc = dalloc((size_t)N * n), *rd = dalloc(pt + 1), *re = dalloc(qt + 1);
  double *rq = dalloc((size_t)(N + 1) * n), *rr = dalloc((size_t)N * m);
  kkt_rows(P, x, u, lam, mu, eta, alpha, rs0, rc, rd, re, rq, rr);
  double r0 = 0.0, r1 = 0.0, r2 = 0.0, r3 = 0.0;
  for (int a = 0; a < n; a++) r0 = nanmax(r0, fabs(rs0[a]));
  for (size_t k = 0; k < (size_t)N * n; k++) r1 = nanmax(r1, fabs(rc[k]));
  for (int k = 0; k < pt; k++) {
    const double *Ck = P->C + (size_t)k * n, *Dk = P->D + (size_t)k * m;
    double sc = nanmax(1.0, fabs(P->d[k]));
    for (int j = 0; j < n; j++) sc = nanmax(sc, fabs(Ck[j]));
    for (int j = 0; j < m; j++) sc = nanmax(sc, fabs(Dk[j]));
    r2 = nanmax(r2, fabs(rd[k]) / ((ORC_PLANT == 10) ? 1.0 : sc));
  }
  for (int k = 0; k < qt; k++) {
    const double *Ek = P->E + (size_t)k * n;
    double sc = nanmax(1.0, fabs(P->e[k]));
    for (int j = 0; j < n; j++) sc = nanmax(sc, fabs(Ek[j]));
    r2 = nanmax(r2, fabs(re[k]) / sc);
  }
  for (size_t k = 0; k < (size_t)(N + 1) * n; k++) r3 = nanmax(r3, fabs(rq[k]));
  for (size_t k = 0; k < (size_t)N * m; k++) r3 = nanmax(r3, fabs(rr[k]));
  free(rs0); free(rc); free(rd); free(re); free(rq); free(rr);
  if (parts) { parts[0] = r0; parts[1] = r1; parts[2] = r2; parts[3] = r3; }
  return nanmax(nanmax(r0, r1), nanmax(r2, r3));
}

/* ------------------------------------------------------------------ */
/* Entry point: steps 1-9, then the refinement of step 11               */
/* ------------------------------------------------------------------ */
static int finite_all(const double *a, size_t k) {
  for (size_t i = 0; i < k; i++)
    if (!isfinite(a[i])) return 0;
  return 1;
}

static int inputs_finite(const orc_problem *P) {
  const size_t N = P->N, n = P->n, m = P->m;
  int pt, qt;
  row_counts(P, &pt, &qt);
  return finite_all(P->A, N * n * n) && finite_all(P->B, N * n * m) && finite_all(P->c, N * n) &&
         finite_all(P->C, (size_t)pt * n) && finite_all(P->D, (size_t)pt * m) && finite_all(P->d, pt) &&
         finite_all(P->E, (size_t)qt * n) && finite_all(P->e, qt) && finite_all(P->Q, (N + 1) * n * n) &&
         finite_all(P->M, N * n * m) && finite_all(P->R, N * m * m) && finite_all(P->qv, (N + 1) * n) &&
         finite_all(P->rv, N * m) && finite_all(P->s0, n);
}

int orc_solve(const orc_problem *P, const orc_options *opt, double *x,
              double *u, double *lam, double *mu, double *eta,
              double *alpha, int *fail_stage, double *flops, orc_debug *dbg) {
  const int N = P->N, n = P->n, m = P->m;
  if (N < 1 || n < 1 || m < 1) return ORC_BAD_INPUT;
  g_flops = 0.0;
  for (int k = 0; k < 8; k++) g_phase[k] = 0.0;
  g_in_correction = 0;
  *fail_stage = -1;
  if (flops) *flops = 0.0;
  if (!inputs_finite(P)) return ORC_NONFINITE;
  int status = solve_once(P, opt, x, u, lam, mu, eta, alpha, fail_stage, dbg);
  int pt, qt;
  row_counts(P, &pt, &qt);
  if (status == ORC_OK &&
      !(finite_all(x, (size_t)(N + 1) * n) && finite_all(u, (size_t)N * m) &&
        (!lam || (finite_all(lam, (size_t)(N + 1) * n) && finite_all(mu, pt) && finite_all(eta, qt) &&
                  finite_all(alpha, n)))))
    status = ORC_NONFINITE;
  if (lam && status == ORC_OK && opt->kkt_refine > 0) {
    g_in_correction = 1;
    orc_problem C = *P;
    double *rs0 = dalloc(n), *rc = dalloc((size_t)N * n), *rd = dalloc(pt + 1), *re = dalloc(qt + 1);
    double *rq = dalloc((size_t)(N + 1) * n), *rr = dalloc((size_t)N * m), *s0c = dalloc(n);
    double *dx = dalloc((size_t)(N + 1) * n), *du = dalloc((size_t)N * m), *dl = dalloc((size_t)(N + 1) * n);
    double *dmu = dalloc(pt + 1), *deta = dalloc(qt + 1), *dal = dalloc(n);
    C.c = rc; C.d = rd; C.e = re; C.qv = rq; C.rv = rr; C.s0 = s0c;
    for (int k = 0; k < opt->kkt_refine; k++) {
      const double res = orc_kkt_residual(P, x, u, lam, mu, eta, alpha, NULL);
      if (!(res > opt->refine_tol)) break;
      double parts[4];
      orc_kkt_residual(P, x, u, lam, mu, eta, alpha, parts);
      kkt_rows(P, x, u, lam, mu, eta, alpha, rs0, rc, rd, re, rq, rr);
      for (int a = 0; a < n; a++) s0c[a] = -rs0[a];
      if (nanmax(parts[0], nanmax(parts[1], parts[2])) <= opt->refine_tol) {
        /* primal rows within the tolerance: homogeneous constraints */
        for (int a = 0; a < n; a++) s0c[a] = 0.0;
        for (size_t j = 0; j < (size_t)N * n; j++) rc[j] = 0.0;
        for (int j = 0; j < pt; j++) rd[j] = 0.0;
        for (int j = 0; j < qt; j++) re[j] = 0.0;
      }
      int fs;
      const int st = solve_once(&C, opt, dx, du, dl, dmu, deta, dal, &fs, NULL);
      if (st != ORC_OK) break;
      /* trial point w + dw, kept only when its residual is smaller (a
         correction from a solve that lost its accuracy is refused) */
      const double sg = (ORC_PLANT == 16) ? -1.0 : 1.0;
      for (size_t j = 0; j < (size_t)(N + 1) * n; j++) { dx[j] = x[j] + sg * dx[j]; dl[j] += lam[j]; }
      for (size_t j = 0; j < (size_t)N * m; j++) du[j] += u[j];
      for (int j = 0; j < pt; j++) dmu[j] = ((ORC_PLANT == 15) ? 0.0 : dmu[j]) + mu[j];
      for (int j = 0; j < qt; j++) deta[j] += eta[j];
      for (int j = 0; j < n; j++) dal[j] += alpha[j];
      const double trial = orc_kkt_residual(P, dx, du, dl, dmu, deta, dal, NULL);
      if (!(trial < res)) break;
      memcpy(x, dx, sizeof(double) * (N + 1) * n);
      memcpy(lam, dl, sizeof(double) * (N + 1) * n);
      memcpy(u, du, sizeof(double) * N * m);
      memcpy(mu, dmu, sizeof(double) * pt);
      memcpy(eta, deta, sizeof(double) * qt);
      memcpy(alpha, dal, sizeof(double) * n);
      if (!(trial < 0.5 * res)) break;
    }
    free(rs0); free(rc); free(rd); free(re); free(rq); free(rr); free(s0c);
    free(dx); free(du); free(dl); free(dmu); free(deta); free(dal);
    g_in_correction = 0;
  }
  if (flops) *flops = g_flops;
  return status;
}

/* exported helpers so tests can exercise Lemma 1 and the null-space solve
   on their own, against independent numpy computations */
/* flops of the last orc_solve per phase (see g_phase) */
void orc_phase_flops(double *out) {
  for (int k = 0; k < 8; k++) out[k] = g_phase[k];
}

int orc_project(double *M, int r, int nc, int ngroups, const int *gsz, int nkeep,
                double tau_rank, double tau_inc, int *grank, int *krank, double *out) {
  int inc = 0;
  project(M, r, nc, ngroups, gsz, nkeep, tau_rank, tau_inc, grank, krank, &inc, out);
  return inc;
}

int orc_tqr_solve(const double *K, int rk, int nk, double tau_rank, const double *b,
                  int nb, double *X, double *Q, double *resid) {
  return tqr_solve(K, rk, nk, tau_rank, b, nb, X, Q, resid);
}
