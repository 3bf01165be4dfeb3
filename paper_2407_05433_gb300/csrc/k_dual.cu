// k_dual.cu -- multiplier recovery (Sec. 7) and the KKT residual (Sec. 9).
//
// For every KKT multiplier the chain rule through x = T z + t, u = Y z + Z v + y
// turns the original Lagrangian into the reduced one with costates
// T_i' lambda_i, so T_i' lambda_i = pi_i = P_i z_i + p_i, the reduced LQR
// costate from the solve.  Writing lambda_i = T_i pi_i + U_i nu_i (U_i an
// orthonormal basis of range(H_i')), the stationarity equations (eqs.
// stage-stationarity, terminal-stationarity) that are not already satisfied
// read
//   (a) U_i'C_i' mu_i + U_i'E_i' eta_i + U_i'A_i'U_{i+1} nu_{i+1} - nu_i + U_i' rho^x_i = 0
//   (b) D_i' mu_i + B_i'U_{i+1} nu_{i+1} + rho^u_i = 0
//   (N) U_N'E_N' eta_N - nu_N + U_N' g^x_N = 0
// with rho^x_i = g^x_i + A_i'T_{i+1} pi_{i+1}, rho^u_i = g^u_i + B_i'T_{i+1} pi_{i+1}.
// These are dual endpoint relations between nu_i and nu_{i+1}: projecting out
// (mu_i, eta_i) (Lemma 1) and contracting them is the procedure of Sec. 7.
// Admissible sets come from a chunked suffix scan (same kernels as the primal
// scan); the representative is the min-norm nu_0, then the min-norm nu_{i+1}
// given nu_i (an affine map, expanded by a forward affine scan), then min-norm
// leaf solves for (mu_i, eta_i).  Since ||lambda_i||^2 = ||pi_i||^2 + ||nu_i||^2
// this is the min-norm representative of the sequential variant of Sec. 7,
// without propagating the tangential part of lambda through the horizon.
// A dual relation that reads 0 = gamma != 0 cannot arise in exact arithmetic
// (the KKT conditions of a feasible problem with linear equality constraints
// have a solution); where rounding produces one, the projection drops the row
// like a redundant one and the pass goes on, leaving the judgement to the KKT
// residual and the refinement on it (eclqr_refine).
#include "kernels.cuh"

namespace eclqr {

__host__ int smem_dual_stage(int n, int m) { return n * n + 4 * n + m + 8; }
// Down-sweep scratch for the forward maps (Wt, Qf, X, Ys, tq, perm), in doubles.
// It is live only between the two projections of a stage, when M is dead, so
// it sits inside M whenever it fits there.
__host__ __device__ inline int dual_solve_scratch(int n, int rows) {
  return n * rows + n * n + n * (n + 1) + rows * (n + 1) + 4 * n + rows;
}
__host__ int smem_dual_sweep(int n, int m, int pmax, int qmax) {
  const int rows = 3 * n + m, ldm = pmax + qmax + 3 * n + 1, ldr = 2 * n + 1;
  const int base = 2 * n * ldr + rows * ldm + rows * ldr + rows + 2 * ldm;
  const int solve = dual_solve_scratch(n, rows);
  return base + (solve <= rows * ldm ? 0 : solve) + 16;
}
__host__ int smem_dual_leaf(int n, int m, int wmax) {
  int w = wmax, rows = n + m;
  return rows * w + rows + w * rows + w * w + w + rows + 2 * (rows + w) + rows + 16;
}

// ---------------------------------------------------------------- per-stage blocks
__global__ void __launch_bounds__(256, 3) k_dual_stage(Group g, const double *x, const double *u, int per_task) {
  for_stages(g, [&](const int s) {
    const StageInfo S = g.st[s];
    const ProbInfo &P = g.prob[S.prob];
    if (skipped_by_mask(g, S.prob)) return;
    const int n = g.n, m = g.m, tid = team_rank(), i = S.i;
    double *ws = stage_ws(g, s);
    const int *wi = stage_wi(g, s);
    const int r0 = wi[SI_UR];
    const double *U = ws + g.ws.UT;  // first r0 columns, ld n
    const double *xi = x + P.ox + (size_t)i * n;
    const double *Q = g.Q + P.oQ + (size_t)i * n * n, *q = g.qv + P.oqv + (size_t)i * n;
    const int ldc = g.pmax + g.qmax + 1;
    double *sm = team_smem(per_task);
    double *X = sm, *gx = X + n * n, *tp = gx + n, *rx = tp + n, *gu = rx + n;
    if (i == P.N) {
      for (int a = tid; a < n; a += TEAM) {
        double v = q[a];
        for (int j = 0; j < n; j++) v = fma(Q[a * n + j], xi[j], v);
        gx[a] = v;
      }
      tsync();
      for (int a = tid; a < r0; a += TEAM) {
        double v = 0.0;
        for (int l = 0; l < n; l++) v = fma(U[l * n + a], gx[l], v);
        ws[g.ws.Ux + a] = v;
      }
      for (int idx = tid; idx < r0 * S.q; idx += TEAM) {
        int a = idx / S.q, j = idx - a * S.q;
        double v = 0.0;
        for (int l = 0; l < n; l++) v = fma(U[l * n + a], g.E[P.oE + (size_t)(S.qrow + j) * n + l], v);
        ws[g.ws.UC + a * ldc + j] = v;
      }
      return;
    }
    const double *A = g.A + P.oA + (size_t)i * n * n, *B = g.B + P.oB + (size_t)i * n * m;
    const double *Mm = g.M + P.oM + (size_t)i * n * m, *R = g.R + P.oR + (size_t)i * m * m;
    const double *r = g.rv + P.orv + (size_t)i * m, *ui = u + P.ou + (size_t)i * m;
    const double *wn = stage_ws(g, s + 1);
    const int *win = stage_wi(g, s + 1);
    const int r1 = win[SI_UR], nb1 = n - r1;
    const double *U1 = wn + g.ws.UT, *T1 = wn + g.ws.UT + r1, *pi1 = wn + g.ws.pi;
    // objective gradients (eq. objective-gradients) and T_{i+1} pi_{i+1}
    const bool tne = win[SI_TEYE] != 0;  // T_{i+1} = I: T_{i+1} pi_{i+1} = pi_{i+1}
    for (int a = tid; a < n; a += TEAM) {
      double v = q[a];
      for (int j = 0; j < n; j++) v = fma(Q[a * n + j], xi[j], v);
      for (int j = 0; j < m; j++) v = fma(Mm[a * m + j], ui[j], v);
      gx[a] = v;
      double t = 0.0;
      if (tne) t = pi1[a];
      else
        for (int j = 0; j < nb1; j++) t = fma(T1[a * n + j], pi1[j], t);
      tp[a] = t;
    }
    for (int a = tid; a < m; a += TEAM) {
      double v = r[a];
      for (int j = 0; j < n; j++) v = fma(Mm[j * m + a], xi[j], v);
      for (int j = 0; j < m; j++) v = fma(R[a * m + j], ui[j], v);
      gu[a] = v;
    }
    tsync();
    for (int a = tid; a < n; a += TEAM) {
      double v = gx[a];
      for (int l = 0; l < n; l++) v = fma(A[l * n + a], tp[l], v);
      rx[a] = v;
    }
    for (int a = tid; a < m; a += TEAM) {
      double v = gu[a];
      for (int l = 0; l < n; l++) v = fma(B[l * m + a], tp[l], v);
      ws[g.ws.ru + a] = v;
    }
    // X = A' U_{i+1} (n x r1)
    for (int idx = tid; idx < n * r1; idx += TEAM) {
      int l = idx / r1, b = idx - l * r1;
      double v = 0.0;
      for (int k = 0; k < n; k++) v = fma(A[k * n + l], U1[k * n + b], v);
      X[l * n + b] = v;
    }
    tsync();
    wgemm<true, false>(r0, r1, n, 1.0, U, n, X, n, 0.0, ws + g.ws.UA, n);   // U' A' U1
    for (int idx = tid; idx < m * r1; idx += TEAM) {
      int a = idx / r1, b = idx - a * r1;
      double v = 0.0;
      for (int k = 0; k < n; k++) v = fma(B[k * m + a], U1[k * n + b], v);
      ws[g.ws.BU + a * n + b] = v;                                         // B' U1
    }
    for (int idx = tid; idx < r0 * (S.p + S.q); idx += TEAM) {
      int a = idx / (S.p + S.q), j = idx - a * (S.p + S.q);
      const double *row = (j < S.p) ? g.C + P.oC + (size_t)(S.prow + j) * n : g.E + P.oE + (size_t)(S.qrow + j - S.p) * n;
      double v = 0.0;
      for (int l = 0; l < n; l++) v = fma(U[l * n + a], row[l], v);
      ws[g.ws.UC + a * ldc + j] = v;                                       // U' [C' E']
    }
    for (int a = tid; a < r0; a += TEAM) {
      double v = 0.0;
      for (int l = 0; l < n; l++) v = fma(U[l * n + a], rx[l], v);
      ws[g.ws.Ux + a] = v;                                                 // U' rho^x
    }
  });
}

// rows (a) and (b) of stage s into M (ld ldm) at row 0, with the column
// layout  mu,eta (w) | nu_{i+1} (r1) | nu_i (r0) | [extra zero block (ext)] | 1.
// Returns the number of rows written (r0 + m).
__device__ int dual_stage_rows(const Group &g, int s, double *M, int ldm, int ext) {
  const int n = g.n, m = g.m, tid = team_rank();
  const StageInfo S = g.st[s];
  const ProbInfo &P = g.prob[S.prob];
  const double *ws = stage_ws(g, s);
  const int r0 = stage_wi(g, s)[SI_UR], r1 = stage_wi(g, s + 1)[SI_UR];
  const int w = S.p + S.q, ldc = g.pmax + g.qmax + 1;
  const int rows = r0 + m;
  for (int idx = tid; idx < rows * ldm; idx += TEAM) {
    int r = idx / ldm, j = idx - r * ldm;
    double val = 0.0;
    if (r < r0) {
      if (j < w) val = ws[g.ws.UC + r * ldc + j];
      else if (j < w + r1) val = ws[g.ws.UA + r * n + (j - w)];
      else if (j == w + r1 + r) val = -1.0;
      else if (j == ldm - 1) val = ws[g.ws.Ux + r];
    } else {
      const int a = r - r0;
      if (j < S.p) val = g.D[P.oD + (size_t)(S.prow + j) * m + a];
      else if (j >= w && j < w + r1) val = ws[g.ws.BU + a * n + (j - w)];
      else if (j == ldm - 1) val = ws[g.ws.ru + a];
    }
    M[idx] = val;
  }
  (void)ext;
  tsync();
  return rows;
}

// ---------------------------------------------------------------- terminal relation on nu_N
__global__ void k_dual_terminal(Group g, int per_task) {
  const int t = team_task();
  if (t >= g.nprob) return;
  const ProbInfo &P = g.prob[t];
  if (skipped_by_mask(g, t)) return;
  const int n = g.n, tid = team_rank();
  const int s = P.st0 + P.N;
  const StageInfo S = g.st[s];
  double *ws = stage_ws(g, s);
  int *wi = stage_wi(g, s);
  const int rN = wi[SI_UR], qN = S.q, ldc = g.pmax + g.qmax + 1;
  const int ldm = qN + rN + 1;
  double *sm = team_smem(per_task);
  double *M = sm, *out = M + n * ldm, *scr = out + n * (n + 1);
  for (int idx = tid; idx < rN * ldm; idx += TEAM) {
    int r = idx / ldm, j = idx - r * ldm;
    double val = 0.0;
    if (j < qN) val = ws[g.ws.UC + r * ldc + j];
    else if (j == qN + r) val = -1.0;
    else if (j == ldm - 1) val = ws[g.ws.Ux + r];
    M[idx] = val;
  }
  tsync();
  const int gs[1] = {qN};
  ProjResult pr = wproject(M, ldm, rN, 1, gs, rN, g.tau_rank, g.tau_inc, out, rN + 1, scr);
  double *NH = ws + g.ws.NH;
  const int slot = P.ch0 + P.nch, ldr = 2 * n + 1;
  double *cs = g.CS[0] + (size_t)slot * g.cs_stride;
  for (int idx = tid; idx < pr.krank * (rN + 1); idx += TEAM) {
    int r = idx / (rN + 1), j = idx - r * (rN + 1);
    NH[r * (n + 1) + j] = out[idx];
    cs[r * ldr + j] = out[idx];
  }
  if (tid == 0) {
    wi[SI_NUROWS] = pr.krank;
    int *cm = g.CI[0] + (size_t)slot * CI_STRIDE;
    cm[CI_ROWS] = pr.krank; cm[CI_NA] = rN; cm[CI_NB] = 0;
  }
}

// ---------------------------------------------------------------- chunk up-sweep on (nu_a, nu_b)
__global__ void k_dual_up(Group g, int per_task) {
  const int t = team_task();
  if (t >= g.nslot) return;
  const ChunkInfo ci = g.chunk[t];
  const ProbInfo &P = g.prob[ci.prob];
  if (skipped_by_mask(g, ci.prob)) return;
  if (ci.c >= P.nch) return;
  const int n = g.n, m = g.m, tid = team_rank();
  if (P.nch == 1) {  // one chunk: k_dual_down starts from the terminal set alone
    if (tid == 0) {
      int *cm = g.CI[0] + (size_t)t * CI_STRIDE;
      cm[CI_ROWS] = 0; cm[CI_NA] = 0; cm[CI_NB] = 0;
    }
    return;
  }
  const int a = ci.c * P.L, b = min(a + P.L, P.N);
  const int rb = stage_wi(g, P.st0 + b)[SI_UR];
  const int ldr = 2 * n + 1;
  const int ldm_max = g.pmax + g.qmax + 3 * n + 1, rows_max = 3 * n + m;
  double *sm = team_smem(per_task);
  double *Rel = sm, *M = Rel + 2 * n * ldr, *scr = M + rows_max * ldm_max;
  // identity on (nu_b', nu_b)
  for (int idx = tid; idx < rb * ldr; idx += TEAM) {
    int i = idx / ldr, j = idx - i * ldr;
    Rel[idx] = (j == i) ? 1.0 : ((j == rb + i) ? -1.0 : 0.0);
  }
  tsync();
  int rr = rb;
  for (int i = b - 1; i >= a; --i) {
    const int s = P.st0 + i;
    const StageInfo S = g.st[s];
    const int r0 = stage_wi(g, s)[SI_UR], r1 = stage_wi(g, s + 1)[SI_UR], w = S.p + S.q;
    // columns: mu,eta | nu_{i+1} | nu_i | nu_b | 1
    const int ldm = w + r1 + r0 + rb + 1;
    int rows = dual_stage_rows(g, s, M, ldm, rb);
    // the stage rows were written with offset column ldm - 1 and a zero nu_b block
    for (int idx = tid; idx < rr * ldm; idx += TEAM) {
      int r = idx / ldm, j = idx - r * ldm;
      const double *row = Rel + r * ldr;  // [L (r1) | R (rb) | l]
      double val = 0.0;
      if (j >= w && j < w + r1) val = row[j - w];
      else if (j >= w + r1 + r0 && j < w + r1 + r0 + rb) val = row[r1 + (j - w - r1 - r0)];
      else if (j == ldm - 1) val = row[r1 + rb];
      M[(rows + r) * ldm + j] = val;
    }
    tsync();
    const int gs[2] = {w, r1};
    ProjResult pr = wproject(M, ldm, rows + rr, 2, gs, r0 + rb, g.tau_rank, g.tau_inc, Rel, ldr, scr);
    rr = pr.krank;
    tsync();
  }
  double *cs = g.CS[0] + (size_t)t * g.cs_stride;
  for (int idx = tid; idx < rr * ldr; idx += TEAM) cs[idx] = Rel[idx];
  if (tid == 0) {
    int *cm = g.CI[0] + (size_t)t * CI_STRIDE;
    cm[CI_ROWS] = rr; cm[CI_NA] = stage_wi(g, P.st0 + a)[SI_UR]; cm[CI_NB] = rb;
  }
}

// ---------------------------------------------------------------- chunk down-sweep: sets N_i and forward maps
__global__ void k_dual_down(Group g, int fin, int per_task) {
  const int t = team_task();
  if (t >= g.nslot) return;
  const ChunkInfo ci = g.chunk[t];
  const ProbInfo &P = g.prob[ci.prob];
  if (skipped_by_mask(g, ci.prob)) return;
  if (ci.c >= P.nch) return;
  const int n = g.n, m = g.m, tid = team_rank();
  const int a = ci.c * P.L, b = min(a + P.L, P.N);
  const int ldr = 2 * n + 1;
  const int ldm_max = g.pmax + g.qmax + 3 * n + 1, rows_max = 3 * n + m;
  double *sm = team_smem(per_task);
  double *Ns = sm;                          // n x (2n+1): current set on nu_{i+1}
  double *M = Ns + 2 * n * ldr;             // rows_max x ldm_max
  double *K = M + rows_max * ldm_max;       // rows_max x (2n+1): rows after eliminating mu,eta
  double *scr = K + rows_max * ldr;         // projection scratch
  // forward-map scratch: inside M (dead between the two projections) when it fits
  double *Wt = (dual_solve_scratch(n, rows_max) <= rows_max * ldm_max) ? M : scr + rows_max + 2 * ldm_max;  // n x rows
  double *Qf = Wt + n * rows_max;           // n x n
  double *X = Qf + n * n;                   // n x (n+1)
  double *Ys = X + n * (n + 1);             // rows x (n+1)
  double *tq = Ys + rows_max * (n + 1);     // 4n (wtqr needs r1 + max(r1, rows) <= 3n)
  int *perm = (int *)(tq + 4 * n);
  // N_b after the scan: unary relation in slot t + 1
  {
    const double *src = g.CS[fin] + (size_t)(t + 1) * g.cs_stride;
    const int rows = g.CI[fin][(size_t)(t + 1) * CI_STRIDE + CI_ROWS];
    for (int idx = tid; idx < rows * ldr; idx += TEAM) Ns[idx] = src[idx];
    tsync();
    if (b == P.N) { /* stage N's set was stored by k_dual_terminal */ }
    int rr = rows;
    for (int i = b - 1; i >= a; --i) {
      const int s = P.st0 + i;
      const StageInfo S = g.st[s];
      double *ws = stage_ws(g, s);
      const int r0 = stage_wi(g, s)[SI_UR], r1 = stage_wi(g, s + 1)[SI_UR], w = S.p + S.q;
      if (r0 == 0 && r1 == 0) {
        // nu_i and nu_{i+1} have no coordinates (X_i = X_{i+1} = R^n): no forward map, and
        // eliminating (mu, eta) leaves only rows 0 = const, which the relation drops as
        // redundant or (from rounding) inconsistent, so N_i has no rows
        rr = 0;
        if (tid == 0) stage_wi(g, s)[SI_NUROWS] = 0;
        continue;
      }
      const int ldm = w + r1 + r0 + 1;
      int rows2 = dual_stage_rows(g, s, M, ldm, 0);
      for (int idx = tid; idx < rr * ldm; idx += TEAM) {
        int r = idx / ldm, j = idx - r * ldm;
        const double *row = Ns + r * ldr;  // [H (r1) | h]
        double val = 0.0;
        if (j >= w && j < w + r1) val = row[j - w];
        else if (j == ldm - 1) val = row[r1];
        M[(rows2 + r) * ldm + j] = val;
      }
      tsync();
      // eliminate (mu, eta): rows [Kn (r1) | L (r0) | l]
      const int gs1[1] = {w};
      ProjResult p1 = wproject(M, ldm, rows2 + rr, 1, gs1, r1 + r0, g.tau_rank, g.tau_inc, K, ldr, scr);
      const int kr = p1.krank;
      // forward map: nu_{i+1} = -Kn^+ (L nu_i + l)
      double *Pnu = ws + g.ws.Pnu, *pnu = ws + g.ws.pnu;
      {
        const int rank = wtqr(K, ldr, kr, r1, g.tau_rank, Wt, (kr > 0 ? kr : 1), Qf, n, perm, tq);
        wtqr_solve(Wt, (kr > 0 ? kr : 1), Qf, n, perm, kr, r1, rank, K + r1, ldr, r0 + 1, X, n + 1, Ys, n + 1);
        for (int idx = tid; idx < r1 * (r0 + 1); idx += TEAM) {
          int r = idx / (r0 + 1), j = idx - r * (r0 + 1);
          if (j < r0) Pnu[r * n + j] = X[r * (n + 1) + j]; else pnu[r] = X[r * (n + 1) + j];
        }
        tsync();  // X may live inside M, which is rewritten next
      }
      // N_i: project nu_{i+1} out of the same rows
      for (int idx = tid; idx < kr * (r1 + r0 + 1); idx += TEAM) {
        int r = idx / (r1 + r0 + 1), j = idx - r * (r1 + r0 + 1);
        M[idx] = K[r * ldr + j];
      }
      tsync();
      const int gs2[1] = {r1};
      ProjResult p2 = wproject(M, r1 + r0 + 1, kr, 1, gs2, r0, g.tau_rank, g.tau_inc, Ns, ldr, scr);
      rr = p2.krank;
      double *NH = ws + g.ws.NH;
      for (int idx = tid; idx < rr * (r0 + 1); idx += TEAM) {
        int r = idx / (r0 + 1), j = idx - r * (r0 + 1);
        NH[r * (n + 1) + j] = Ns[r * ldr + j];
      }
      if (tid == 0) stage_wi(g, s)[SI_NUROWS] = rr;
      tsync();
    }
  }
}

// ---------------------------------------------------------------- root: min-norm nu_0 in N_0
__global__ void k_dual_root(Group g, int per_task) {
  const int t = team_task();
  if (t >= g.nprob) return;
  const ProbInfo &P = g.prob[t];
  if (skipped_by_mask(g, t)) return;
  const int n = g.n, tid = team_rank();
  const int s = P.st0;
  double *ws = stage_ws(g, s);
  const int r0 = stage_wi(g, s)[SI_UR], rr = stage_wi(g, s)[SI_NUROWS];
  double *sm = team_smem(per_task);
  double *Hs = sm, *hb = Hs + n * (n + 1), *Wt = hb + n, *Qf = Wt + n * n, *X = Qf + n * n, *Ys = X + n;
  double *tq = Ys + n;
  int *perm = (int *)(tq + 4 * n);
  const double *NH = ws + g.ws.NH;
  for (int idx = tid; idx < rr * (n + 1); idx += TEAM) Hs[idx] = NH[idx];
  for (int r = tid; r < rr; r += TEAM) hb[r] = NH[r * (n + 1) + r0];
  tsync();
  const int rank = wtqr(Hs, n + 1, rr, r0, g.tau_rank, Wt, (rr > 0 ? rr : 1), Qf, n, perm, tq);
  wtqr_solve(Wt, (rr > 0 ? rr : 1), Qf, n, perm, rr, r0, rank, hb, 1, 1, X, 1, Ys, 1);
  for (int a = tid; a < n; a += TEAM) ws[g.ws.nu + a] = (a < r0) ? X[a] : 0.0;
}

// ---------------------------------------------------------------- leaves: mu_i, eta_i, lambda_i, alpha, eta_N
__global__ void __launch_bounds__(256, 4) k_dual_leaf(Group g, double *lam, double *mu, double *eta, double *alpha, int per_task) {
  for_stages(g, [&](const int s) {
    const StageInfo S = g.st[s];
    const ProbInfo &P = g.prob[S.prob];
    if (skipped_by_mask(g, S.prob)) return;
    const int n = g.n, m = g.m, tid = team_rank(), i = S.i;
    const double *ws = stage_ws(g, s);
    const int r0 = stage_wi(g, s)[SI_UR], nb = n - r0;
    const int ldc = g.pmax + g.qmax + 1;
    const double *nu0 = ws + g.ws.nu;
    // lambda_i = T_i pi_i + U_i nu_i
    const double *UT = ws + g.ws.UT, *pi = ws + g.ws.pi;
    bool bad = false;
    const bool te = stage_wi(g, s)[SI_TEYE] != 0;  // T_i = I, no nu_i: lambda_i = pi_i
    for (int a = tid; a < n; a += TEAM) {
      double v = 0.0;
      if (te) {
        v = pi[a];
      } else {
        for (int j = 0; j < r0; j++) v = fma(UT[a * n + j], nu0[j], v);
        for (int j = 0; j < nb; j++) v = fma(UT[a * n + r0 + j], pi[j], v);
      }
      lam[P.olam + (size_t)i * n + a] = v;
      if (i == 0) alpha[P.oalpha + a] = -v;
      bad = bad || !isfinite(v);
    }
    if (__syncthreads_or(bad) && tid == 0) set_status(g, S.prob, ST_NONFINITE);
    const int w = (i < P.N) ? S.p + S.q : S.q;
    if (w == 0) return;
    double *sm = team_smem(per_task);
    const int wmax = g.wmax, rmax = n + m;
    double *F = sm, *rhs = F + rmax * wmax, *Wt = rhs + rmax, *Qf = Wt + wmax * rmax, *X = Qf + wmax * wmax;
    double *Ys = X + wmax, *tq = Ys + rmax;
    int *perm = (int *)(tq + 2 * (rmax + wmax));
    int rows;
    if (i < P.N) {
      const double *wn = stage_ws(g, s + 1);
      const int r1 = stage_wi(g, s + 1)[SI_UR];
      const double *nu1 = wn + g.ws.nu;
      rows = r0 + m;
      for (int idx = tid; idx < rows * w; idx += TEAM) {
        int r = idx / w, j = idx - r * w;
        double val;
        if (r < r0) val = ws[g.ws.UC + r * ldc + j];
        else val = (j < S.p) ? g.D[P.oD + (size_t)(S.prow + j) * m + (r - r0)] : 0.0;
        F[idx] = val;
      }
      for (int r = tid; r < rows; r += TEAM) {
        double v;
        if (r < r0) {
          v = ws[g.ws.Ux + r] - nu0[r];
          for (int b = 0; b < r1; b++) v = fma(ws[g.ws.UA + r * n + b], nu1[b], v);
        } else {
          v = ws[g.ws.ru + (r - r0)];
          for (int b = 0; b < r1; b++) v = fma(ws[g.ws.BU + (r - r0) * n + b], nu1[b], v);
        }
        rhs[r] = v;
      }
    } else {
      rows = r0;
      for (int idx = tid; idx < rows * w; idx += TEAM) {
        int r = idx / w, j = idx - r * w;
        F[idx] = ws[g.ws.UC + r * ldc + j];
      }
      for (int r = tid; r < rows; r += TEAM) rhs[r] = ws[g.ws.Ux + r] - nu0[r];
    }
    tsync();
    const int rank = wtqr(F, w, rows, w, g.tau_rank, Wt, (rows > 0 ? rows : 1), Qf, wmax, perm, tq);
    wtqr_solve(Wt, (rows > 0 ? rows : 1), Qf, wmax, perm, rows, w, rank, rhs, 1, 1, X, 1, Ys, 1);
    bad = false;
    if (i < P.N) {
      for (int j = tid; j < S.p; j += TEAM) mu[P.omu + S.prow + j] = X[j];
      for (int j = tid; j < S.q; j += TEAM) eta[P.oeta + S.qrow + j] = X[S.p + j];
    } else {
      for (int j = tid; j < S.q; j += TEAM) eta[P.oeta + S.qrow + j] = X[j];
    }
    for (int j = tid; j < w; j += TEAM) bad = bad || !isfinite(X[j]);
    if (__syncthreads_or(bad) && tid == 0) set_status(g, S.prob, ST_NONFINITE);
  });
}

// ---------------------------------------------------------------- KKT residual (Sec. 9 definition)
// Values reduced here are magnitudes or NaN.  The bit pattern of a non-negative
// double orders like its value, and a positive NaN's pattern is above +inf's, so
// an integer maximum over the patterns is a maximum that keeps NaN (fmax drops it).
__device__ __forceinline__ double nanmax(double a, double b) { return (a > b || a != a) ? a : b; }

__device__ __forceinline__ double team_max_keep_nan(double v) {
  __shared__ long long red_bits[32];
  long long k = __double_as_longlong(fabs(v));
#pragma unroll
  for (int o = 16; o; o >>= 1) k = max(k, __shfl_xor_sync(kFull, k, o));
  if ((threadIdx.x & 31) == 0) red_bits[threadIdx.x >> 5] = k;
  __syncthreads();
  long long r = red_bits[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); w++) r = max(r, red_bits[w]);
  __syncthreads();
  return __longlong_as_double(r);
}

__device__ __forceinline__ void atomic_max_nonneg(double *addr, double v) {
  atomicMax((unsigned long long *)addr, (unsigned long long)__double_as_longlong(v));
}

// One stage of the residual rows (Sec. 7 sign convention, lambda_0 = -alpha):
//   x_0 - s_0;  A x + B u + c - x';  C x + D u + d;  E x + e;
//   Q x + M u + q + A' lam' - lam + C' mu + E' eta;  M' x + R u + r + B' lam' + D' mu
// (stage N: Q_N x_N + q_N - lam_N + E_N' eta_N).  With rows set, the rows are
// written in the layout of the offsets they replace in a correction problem
// (c, d, e, qv, rv, and s0 = -(x_0 - s_0)); with resid set, the Sec. 9 norm
// (equality rows divided by max(1, largest |coefficient|, |offset|)) is reduced
// into resid[id] and, with parts set, into parts[4 id + k] for k = initial,
// dynamics, equalities, stationarity.  Any NaN in a row reaches the norm.
// v + sum_j a[j sa] x[j], in order; unrolled by two, so that the residual kernel needs
// under 80 registers a thread and 25 one-warp CTAs fit an SM (16 at 128 registers)
__device__ __forceinline__ double kkt_dot(double v, const double *a, int sa, const double *x, int len) {
#pragma unroll 2
  for (int j = 0; j < len; j++) v = fma(a[(size_t)j * sa], x[j], v);
  return v;
}

__global__ void __launch_bounds__(256, 3) k_kkt(Group g, const double *s0, const double *x, const double *u, const double *lam,
                      const double *mu, const double *eta, const double *alpha, KktRows rows, double *resid,
                      double *parts) {
  for_stages(g, [&](const int s) {
    const StageInfo S = g.st[s];
    const ProbInfo &P = g.prob[S.prob];
    if (skipped_by_mask(g, S.prob)) return;
    const int n = g.n, m = g.m, tid = team_rank(), i = S.i;
    const bool wr = rows.c != nullptr;
    const double *xi = x + P.ox + (size_t)i * n, *li = lam + P.olam + (size_t)i * n;
    const double *Q = g.Q + P.oQ + (size_t)i * n * n, *q = g.qv + P.oqv + (size_t)i * n;
    double r0 = 0.0, r1 = 0.0, r2 = 0.0, r3 = 0.0;
    if (i == 0)
      for (int a = tid; a < n; a += TEAM) {
        const double v = xi[a] - s0[P.os0 + a];
        r0 = nanmax(r0, fabs(v));
        if (wr) rows.s0[P.os0 + a] = -v;
      }
    // state-only rows, normalised
    for (int k = tid; k < S.q; k += TEAM) {
      const double *Ek = g.E + P.oE + (size_t)(S.qrow + k) * n;
      double e = g.e[P.oe + S.qrow + k], v = e, sc = nanmax(1.0, fabs(e));
#pragma unroll 2
      for (int j = 0; j < n; j++) { v = fma(Ek[j], xi[j], v); sc = nanmax(sc, fabs(Ek[j])); }
      r2 = nanmax(r2, fabs(v) / sc);
      if (wr) rows.e[P.oe + S.qrow + k] = v;
    }
    const double *etai = eta + P.oeta + S.qrow;
    if (i < P.N) {
      const double *A = g.A + P.oA + (size_t)i * n * n, *B = g.B + P.oB + (size_t)i * n * m;
      const double *c = g.c + P.oc + (size_t)i * n;
      const double *Mm = g.M + P.oM + (size_t)i * n * m, *R = g.R + P.oR + (size_t)i * m * m;
      const double *rv = g.rv + P.orv + (size_t)i * m;
      const double *ui = u + P.ou + (size_t)i * m, *xn = x + P.ox + (size_t)(i + 1) * n;
      const double *ln = lam + P.olam + (size_t)(i + 1) * n, *mui = mu + P.omu + S.prow;
      for (int a = tid; a < n; a += TEAM) {
        const double v = kkt_dot(kkt_dot(c[a] - xn[a], A + a * n, 1, xi, n), B + a * m, 1, ui, m);
        r1 = nanmax(r1, fabs(v));
        if (wr) rows.c[P.oc + (size_t)i * n + a] = v;
      }
      for (int k = tid; k < S.p; k += TEAM) {
        const double *Ck = g.C + P.oC + (size_t)(S.prow + k) * n, *Dk = g.D + P.oD + (size_t)(S.prow + k) * m;
        double dd = g.d[P.od + S.prow + k], v = dd, sc = nanmax(1.0, fabs(dd));
#pragma unroll 2
        for (int j = 0; j < n; j++) { v = fma(Ck[j], xi[j], v); sc = nanmax(sc, fabs(Ck[j])); }
#pragma unroll 2
        for (int j = 0; j < m; j++) { v = fma(Dk[j], ui[j], v); sc = nanmax(sc, fabs(Dk[j])); }
        r2 = nanmax(r2, fabs(v) / sc);
        if (wr) rows.d[P.od + S.prow + k] = v;
      }
      for (int a = tid; a < m; a += TEAM) {
        double v = kkt_dot(rv[a], Mm + a, m, xi, n);
        v = kkt_dot(v, R + a * m, 1, ui, m);
        v = kkt_dot(v, B + a, m, ln, n);
        v = kkt_dot(v, g.D + P.oD + (size_t)S.prow * m + a, m, mui, S.p);
        r3 = nanmax(r3, fabs(v));
        if (wr) rows.rv[P.orv + (size_t)i * m + a] = v;
      }
      for (int a = tid; a < n; a += TEAM) {
        double v = kkt_dot(q[a] + ((i == 0) ? alpha[P.oalpha + a] : -li[a]), Q + a * n, 1, xi, n);
        v = kkt_dot(v, Mm + a * m, 1, ui, m);
        v = kkt_dot(v, A + a, n, ln, n);
        v = kkt_dot(v, g.C + P.oC + (size_t)S.prow * n + a, n, mui, S.p);
        v = kkt_dot(v, g.E + P.oE + (size_t)S.qrow * n + a, n, etai, S.q);
        r3 = nanmax(r3, fabs(v));
        if (wr) rows.qv[P.oqv + (size_t)i * n + a] = v;
      }
    } else {
      for (int a = tid; a < n; a += TEAM) {
        double v = kkt_dot(q[a] - li[a], Q + a * n, 1, xi, n);
        v = kkt_dot(v, g.E + P.oE + (size_t)S.qrow * n + a, n, etai, S.q);
        r3 = nanmax(r3, fabs(v));
        if (wr) rows.qv[P.oqv + (size_t)i * n + a] = v;
      }
    }
    if (resid == nullptr) return;
    if (parts != nullptr) {
      r0 = team_max_keep_nan(r0);
      r1 = team_max_keep_nan(r1);
      r2 = team_max_keep_nan(r2);
      r3 = team_max_keep_nan(r3);
      if (tid == 0) {
        double *pp = parts + 4 * (size_t)P.id;
        atomic_max_nonneg(pp + 0, r0);
        atomic_max_nonneg(pp + 1, r1);
        atomic_max_nonneg(pp + 2, r2);
        atomic_max_nonneg(pp + 3, r3);
        atomic_max_nonneg(resid + P.id, nanmax(nanmax(r0, r1), nanmax(r2, r3)));
      }
    } else {
      const double r = team_max_keep_nan(nanmax(nanmax(r0, r1), nanmax(r2, r3)));
      if (tid == 0) atomic_max_nonneg(resid + P.id, r);
    }
  });
}

}  // namespace eclqr
