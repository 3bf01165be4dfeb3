// k_primal.cu -- feasible-domain scan (Sec. 3-4) and stage-parallel
// elimination (Sec. 5) on sm_103a.  One CTA per task; small matrices live in
// the task's shared-memory window.
//
// Scan schedule.  A problem's stages are cut into chunks of L stages.  Each
// chunk first composes its own base relations (eq. base-system) into one
// relation between its endpoint states (up-sweep, k_primal_up); the chunk
// relations and the terminal relation (eq. terminal-relation) are then
// combined by a log-depth suffix scan over chunks (k_rel_level, one launch
// per level, Prop. 1 licensing the reparenthesisation); finally every chunk
// walks back from the suffix domain at its right end and produces every
// X_i = {H_i x + h_i = 0} inside it (down-sweep, k_primal_down).  Composing a
// base relation with a relation on (x_{i+1}, x_b) eliminates u_i and x_{i+1}
// together: x_{i+1} is fixed by the dynamics, so substituting it is the same
// existential projection (Lemma 1) as stacking eq. composition-matrix.
#include "kernels.cuh"

namespace eclqr {

// ----------------------------------------------------------- shared memory sizes (doubles per task)
__host__ int smem_primal_sweep(int n, int m, int pmax, int qmax) {
  int rows = 2 * n + pmax + qmax, ldm = m + 2 * n + 1;
  return 2 * n * (2 * n + 1) + rows * ldm + rows + 2 * ldm + 8;
}
// k_primal_stage: the output rows, the stage's own rows and wproject's scratch
__host__ int smem_primal_stage(int n, int m, int wmax) {
  const int rows = wmax, ldm = m + n + 1;
  return n * (n + 1) + rows * ldm + 2 * ldm + rows + ldm / 2 + 16;
}
__host__ int smem_rel_level(int n, int pmax, int qmax) {
  int nmax = n;  // relation endpoint dimensions never exceed n
  int rows = 4 * nmax, ldm = 3 * nmax + 1;
  (void)pmax; (void)qmax;
  return rows * ldm + rows + 2 * ldm + 8;
}
__host__ int smem_scan_check(int n, int m, int pmax) {
  const int ld = m + n + 1;
  return pmax * ld + 2 * ld + pmax + ld / 2 + 8;
}
__host__ int smem_param(int n) { return n * (n + 1) + n * n + n * n + n + n + 4 * n + 8 + n; }
// k_elim's shared memory: the blocks live through the whole stage (A T, Q_m, Y, the
// vectors, the QR scratch and permutation) and one region that three phases use in
// turn: Lemma 4's solve (Gamma, then [Phi | gamma] in the same block once the QR has
// copied Gamma; the factor, the solution and the solve's scratch), the substitution
// products, and the bordered stage Hessian.  H_{i+1} is read where it lies in the
// workspace.
__host__ __device__ inline int elim_vec(int n, int m, int pmax) {
  const int rows = pmax + n;
  // A t + c, c_v, Q t + q, q^z (n each); r^z, R y + r^z, y (m each); the QR's scratch
  // (m + max(m, rows)); the permutation (rows ints)
  return 4 * n + 4 * m + (m > rows ? m : rows) + (rows + 1) / 2 + 2;
}
__host__ __device__ inline int elim_union(int n, int m, int pmax) {
  const int rows = pmax + n;
  const int gr = rows * m > rows * (n + 1) ? rows * m : rows * (n + 1);
  const int ab = gr + m * rows + 2 * m * (n + 1);
  const int c = n * n + 3 * n * m + m * m;
  const int d = (n + m + 1) * (n + m + 1);
  return ab > c ? (ab > d ? ab : d) : (c > d ? c : d);
}
__host__ int smem_elim(int n, int m, int pmax) {
  return n * n + m * m + n * m + elim_vec(n, m, pmax) + elim_union(n, m, pmax) + 8;
}

// ----------------------------------------------------------- shortcut test (Sec. 6)
// For a problem the host found eligible (no state-only or terminal rows,
// p_i <= m), stage i keeps X_i = R^n only if projecting u_i out of its mixed
// rows [D_i | C_i | d_i] (Lemma 1, the scan's tolerance policy) leaves no row
// on x_i.  A stage that leaves one marks the problem as needing the scan.
__global__ void k_scan_check(Group g, int per_task) {
  const int s = team_task();
  if (s >= g.nstage) return;
  const StageInfo S = g.st[s];
  const ProbInfo &P = g.prob[S.prob];
  if (skipped_by_mask(g, S.prob)) return;
  if (!P.skip_ok || S.i >= P.N || S.p == 0) return;
  const int n = g.n, m = g.m, tid = team_rank(), ld = m + n + 1;
  double *sm = team_smem(per_task);
  double *M = sm, *scr = M + g.pmax * ld;
  for (int idx = tid; idx < S.p * ld; idx += TEAM) {
    const int r = idx / ld, j = idx - r * ld;
    const size_t row = S.prow + r;
    M[idx] = (j < m) ? g.D[P.oD + row * m + j]
                     : ((j < m + n) ? g.C[P.oC + row * n + (j - m)] : g.d[P.od + row]);
  }
  tsync();
  const int gs[1] = {m};
  const ProjResult pr = wproject(M, ld, S.p, 1, gs, n, g.tau_rank, g.tau_inc, nullptr, 0, scr);
  if (tid == 0 && (pr.krank > 0 || pr.inconsistent)) g.need_scan[S.prob] = 1;
}

// flags[P.id] = 1 where the shortcut skipped the problem's scan
__global__ void k_skip_flags(Group g, int32_t *flags) {
  const int t = team_task();
  if (t < g.nprob && team_rank() == 0) flags[g.prob[t].id] = scan_skipped(g, t) ? 1 : 0;
}

// ----------------------------------------------------------- terminal domain X_N
__global__ void k_terminal(Group g, int per_task) {
  const int t = team_task();
  if (t >= g.nprob) return;
  const ProbInfo &P = g.prob[t];
  if (skipped_by_mask(g, t)) return;
  const int n = g.n, tid = team_rank();
  const int s = P.st0 + P.N;
  if (scan_skipped(g, t)) {  // X_N = R^n: no terminal rows
    if (tid == 0) stage_wi(g, s)[SI_HROWS] = 0;
    return;
  }
  const StageInfo S = g.st[s];
  double *sm = team_smem(per_task);
  const int ld = n + 1;
  double *M = sm, *scr = sm + g.qmax * ld;
  for (int idx = tid; idx < S.q * ld; idx += TEAM) {
    int i = idx / ld, j = idx - i * ld;
    M[idx] = (j < n) ? g.E[P.oE + (size_t)(S.qrow + i) * n + j] : g.e[P.oe + S.qrow + i];
  }
  tsync();
  double *H = stage_ws(g, s) + g.ws.H;
  ProjResult r = wproject(M, ld, S.q, 0, nullptr, n, g.tau_rank, g.tau_inc, H, ld, scr);
  // terminal element of the chunk scan: unary relation on x_N
  const int slot = P.ch0 + P.nch;
  double *cs = g.CS[0] + (size_t)slot * g.cs_stride;
  const int ldr = 2 * n + 1;
  for (int idx = tid; idx < r.krank * ld; idx += TEAM) {
    int i = idx / ld, j = idx - i * ld;
    cs[i * ldr + j] = H[i * ld + j];
  }
  if (tid == 0) {
    stage_wi(g, s)[SI_HROWS] = r.krank;
    int *ci = g.CI[0] + (size_t)slot * CI_STRIDE;
    ci[CI_ROWS] = r.krank; ci[CI_NA] = n; ci[CI_NB] = 0;
    if (r.inconsistent) set_status(g, t, ST_INFEASIBLE_SUFFIX);
  }
}

// ----------------------------------------------------------- chunk up-sweep
// Relation on (x_i, x_b) built from stage b-1 down to a.  Columns of the
// projected system: u_i (m) | x_i (n) | x_b (n) | 1.
__global__ void k_primal_up(Group g, int per_task) {
  const int t = team_task();
  if (t >= g.nslot) return;
  const ChunkInfo ci = g.chunk[t];
  const ProbInfo &P = g.prob[ci.prob];
  if (skipped_by_mask(g, ci.prob)) return;
  if (ci.c >= P.nch || scan_skipped(g, ci.prob)) return;
  const int n = g.n, m = g.m, tid = team_rank();
  if (P.nch == 1) {
    // one chunk: its down-sweep starts from the terminal slot and reads no
    // aggregate, so the slot gets an empty relation that the levels copy
    if (tid == 0) {
      int *cm = g.CI[0] + (size_t)t * CI_STRIDE;
      cm[CI_ROWS] = 0; cm[CI_NA] = n; cm[CI_NB] = 0;
    }
    return;
  }
  const int a = ci.c * P.L, b = min(a + P.L, P.N);
  double *sm = team_smem(per_task);
  const int ldr = 2 * n + 1, ldm = m + 2 * n + 1;
  const int rows_max = 2 * n + g.pmax + g.qmax;
  double *Rel = sm, *M = Rel + 2 * n * ldr, *scr = M + rows_max * ldm;
  // identity relation x_{b}' - x_b = 0 on (x_{b}', x_b)
  for (int idx = tid; idx < n * ldr; idx += TEAM) {
    int i = idx / ldr, j = idx - i * ldr;
    Rel[idx] = (j == i) ? 1.0 : ((j == n + i) ? -1.0 : 0.0);
  }
  tsync();
  int rr = n;
  for (int i = b - 1; i >= a; --i) {
    const StageInfo S = g.st[P.st0 + i];
    const double *A = g.A + P.oA + (size_t)i * n * n, *B = g.B + P.oB + (size_t)i * n * m;
    const double *c = g.c + P.oc + (size_t)i * n;
    // [L B | L A | R | L c + l]
    wgemm<false, false>(rr, m, n, 1.0, Rel, ldr, B, m, 0.0, M, ldm);
    wgemm<false, false>(rr, n, n, 1.0, Rel, ldr, A, n, 0.0, M + m, ldm);
    for (int idx = tid; idx < rr * (n + 1); idx += TEAM) {
      int r = idx / (n + 1), j = idx - r * (n + 1);
      if (j < n) {
        M[r * ldm + m + n + j] = Rel[r * ldr + n + j];
      } else {
        double s0 = Rel[r * ldr + 2 * n];
        for (int l = 0; l < n; l++) s0 = fma(Rel[r * ldr + l], c[l], s0);
        M[r * ldm + m + 2 * n] = s0;
      }
    }
    // [D | C | 0 | d] and [0 | E | 0 | e]
    for (int idx = tid; idx < (S.p + S.q) * ldm; idx += TEAM) {
      int r = idx / ldm, j = idx - r * ldm;
      double val = 0.0;
      if (r < S.p) {
        const size_t row = S.prow + r;
        if (j < m) val = g.D[P.oD + row * m + j];
        else if (j < m + n) val = g.C[P.oC + row * n + (j - m)];
        else if (j == m + 2 * n) val = g.d[P.od + row];
      } else {
        const size_t row = S.qrow + (r - S.p);
        if (j >= m && j < m + n) val = g.E[P.oE + row * n + (j - m)];
        else if (j == m + 2 * n) val = g.e[P.oe + row];
      }
      M[(rr + r) * ldm + j] = val;
    }
    tsync();
    const int gs[1] = {m};
    ProjResult pr = wproject(M, ldm, rr + S.p + S.q, 1, gs, 2 * n, g.tau_rank, g.tau_inc, Rel, ldr, scr);
    rr = pr.krank;
    if (pr.inconsistent && tid == 0) set_status(g, ci.prob, ST_INFEASIBLE_SUFFIX);
    tsync();
  }
  double *cs = g.CS[0] + (size_t)t * g.cs_stride;
  for (int idx = tid; idx < rr * ldr; idx += TEAM) cs[idx] = Rel[idx];
  if (tid == 0) {
    int *cm = g.CI[0] + (size_t)t * CI_STRIDE;
    cm[CI_ROWS] = rr; cm[CI_NA] = n; cm[CI_NB] = n;
  }
}

// ----------------------------------------------------------- one level of the chunk suffix scan
// slot t <- slot t o slot t+d when both belong to the same problem, else copied.
// Works for any endpoint dimensions recorded in the slot ints (primal and dual).
__global__ void k_rel_level(Group g, int src, int d, int fail_code, int per_task) {
  const int t = team_task();
  if (t >= g.nslot) return;
  const ChunkInfo ci = g.chunk[t];
  const ProbInfo &P = g.prob[ci.prob];
  if (skipped_by_mask(g, ci.prob)) return;
  if (fail_code == ST_INFEASIBLE_SUFFIX && scan_skipped(g, ci.prob)) return;  // primal scan skipped
  const int tid = team_rank();
  const int ldr = 2 * g.n + 1;
  const double *S1 = g.CS[src] + (size_t)t * g.cs_stride;
  const int *I1 = g.CI[src] + (size_t)t * CI_STRIDE;
  double *Dst = g.CS[src ^ 1] + (size_t)t * g.cs_stride;
  int *J = g.CI[src ^ 1] + (size_t)t * CI_STRIDE;
  const int r1 = I1[CI_ROWS], na = I1[CI_NA], nb = I1[CI_NB];
  if (ci.c + d > P.nch || nb == 0) {
    for (int idx = tid; idx < r1 * ldr; idx += TEAM) Dst[idx] = S1[idx];
    if (tid == 0) { J[CI_ROWS] = r1; J[CI_NA] = na; J[CI_NB] = nb; }
    return;
  }
  const double *S2 = g.CS[src] + (size_t)(t + d) * g.cs_stride;
  const int *I2 = g.CI[src] + (size_t)(t + d) * CI_STRIDE;
  const int r2 = I2[CI_ROWS], nd = I2[CI_NB];
  double *sm = team_smem(per_task);
  const int ldm = nb + na + nd + 1;
  double *M = sm, *scr = sm + (r1 + r2) * ldm;
  // columns: b | a | d | 1
  for (int idx = tid; idx < (r1 + r2) * ldm; idx += TEAM) {
    int r = idx / ldm, j = idx - r * ldm;
    double val = 0.0;
    if (r < r1) {
      const double *row = S1 + r * ldr;      // [L1 (a) | R1 (b) | l1]
      if (j < nb) val = row[na + j];
      else if (j < nb + na) val = row[j - nb];
      else if (j == ldm - 1) val = row[na + nb];
    } else {
      const double *row = S2 + (r - r1) * ldr;  // [L2 (b) | R2 (d) | l2]
      if (j < nb) val = row[j];
      else if (j >= nb + na && j < nb + na + nd) val = row[nb + (j - nb - na)];
      else if (j == ldm - 1) val = row[nb + nd];
    }
    M[idx] = val;
  }
  tsync();
  const int gs[1] = {nb};
  ProjResult pr = wproject(M, ldm, r1 + r2, 1, gs, na + nd, g.tau_rank, g.tau_inc, Dst, ldr, scr);
  if (tid == 0) {
    J[CI_ROWS] = pr.krank; J[CI_NA] = na; J[CI_NB] = nd;
    if (pr.inconsistent && fail_code != ST_OK) set_status(g, ci.prob, fail_code);
  }
}

// ----------------------------------------------------------- chunk down-sweep: every X_i
// One stage of the down-sweep: from X_{i+1} = {H x + h = 0} (rows rr of Hs),
// project u_i out of [H B | H A | H c + h] stacked with the stage's own rows;
// Hs receives X_i.  Returns its row count.
__device__ int primal_down_stage(const Group &g, const ProbInfo &P, int i, double *Hs, int rr, double *M,
                                 double *scr, int *inconsistent) {
  const int n = g.n, m = g.m, tid = team_rank();
  const int ldh = n + 1, ldm = m + n + 1;
  const StageInfo S = g.st[P.st0 + i];
  const double *A = g.A + P.oA + (size_t)i * n * n, *B = g.B + P.oB + (size_t)i * n * m;
  const double *c = g.c + P.oc + (size_t)i * n;
  wgemm<false, false>(rr, m, n, 1.0, Hs, ldh, B, m, 0.0, M, ldm);
  wgemm<false, false>(rr, n, n, 1.0, Hs, ldh, A, n, 0.0, M + m, ldm);
  for (int r = tid; r < rr; r += TEAM) {
    double s0 = Hs[r * ldh + n];
    for (int l = 0; l < n; l++) s0 = fma(Hs[r * ldh + l], c[l], s0);
    M[r * ldm + m + n] = s0;
  }
  for (int idx = tid; idx < (S.p + S.q) * ldm; idx += TEAM) {
    int r = idx / ldm, j = idx - r * ldm;
    double val = 0.0;
    if (r < S.p) {
      const size_t row = S.prow + r;
      if (j < m) val = g.D[P.oD + row * m + j];
      else if (j < m + n) val = g.C[P.oC + row * n + (j - m)];
      else val = g.d[P.od + row];
    } else {
      const size_t row = S.qrow + (r - S.p);
      if (j >= m && j < m + n) val = g.E[P.oE + row * n + (j - m)];
      else if (j == m + n) val = g.e[P.oe + row];
    }
    M[(rr + r) * ldm + j] = val;
  }
  tsync();
  const int gs[1] = {m};
  const ProjResult pr = wproject(M, ldm, rr + S.p + S.q, 1, gs, n, g.tau_rank, g.tau_inc, Hs, ldh, scr);
  *inconsistent = pr.inconsistent;
  return pr.krank;
}

// Every chunk but the last first re-sweeps the next chunk's stages from the
// same scan value that chunk starts from.  The set it reaches at its own end
// is then the one the next chunk computes and stores for that stage, bit for
// bit, instead of the scan's composition of the same set: the two agree only
// up to rounding, and a stage whose domain was derived from one set while the
// next stage's basis comes from the other leaves U_b'(A T + B Y) at that
// rounding level, which the multipliers of Sec. 7 multiply by |nu_b|.
// The stage's own rows (mixed and state-only) projected onto x_i, for every stage at
// once: the down-sweep's step at a stage whose successor domain X_{i+1} is the whole
// space (no rows) is this projection, the same call on the same matrix, so the sweep
// takes the stored result there instead of computing it on its sequential chain.
__global__ void k_primal_stage(Group g, int per_task) {
  for_stages(g, [&](const int s) {
    const StageInfo S = g.st[s];
    const ProbInfo &P = g.prob[S.prob];
    if (skipped_by_mask(g, S.prob)) return;
    if (S.i >= P.N || scan_skipped(g, S.prob)) return;
    const int n = g.n, m = g.m, tid = team_rank();
    const int ldh = n + 1, ldm = m + n + 1;
    double *sm = team_smem(per_task);
    double *Hs = sm, *M = Hs + n * ldh, *scr = M + g.wmax * ldm;
    int inc = 0;
    const int rr = primal_down_stage(g, P, S.i, Hs, 0, M, scr, &inc);
    double *Hp = stage_ws(g, s) + g.ws.Hpre;
    for (int idx = tid; idx < rr * ldh; idx += TEAM) Hp[idx] = Hs[idx];
    if (tid == 0) {
      int *wi = stage_wi(g, s);
      wi[SI_PRE] = rr;
      wi[SI_PREINC] = inc;
    }
  });
}

static __device__ void primal_down_task(const Group &g, int fin, int t, int per_task);
__global__ void k_primal_down(Group g, int fin, int per_task, int *queue) {
  for_tasks(g.nslot, queue, [&](int t) { primal_down_task(g, fin, t, per_task); });
}

static __device__ void primal_down_task(const Group &g, int fin, int t, int per_task) {
  if (t >= g.nslot) return;
  const ChunkInfo ci = g.chunk[t];
  const ProbInfo &P = g.prob[ci.prob];
  if (skipped_by_mask(g, ci.prob)) return;
  if (ci.c >= P.nch) return;
  const int n = g.n, m = g.m, tid = team_rank();
  const int a = ci.c * P.L, b = min(a + P.L, P.N);
  if (scan_skipped(g, ci.prob)) {  // X_i = R^n: no rows
    for (int i = a + tid; i < b; i += TEAM) stage_wi(g, P.st0 + i)[SI_HROWS] = 0;
    return;
  }
  const bool resweep = ci.c + 1 < P.nch;
  const int start = resweep ? min(b + P.L, P.N) : b;
  double *sm = team_smem(per_task);
  const int ldh = n + 1, ldr = 2 * n + 1, ldm = m + n + 1;
  const int rows_max = n + g.pmax + g.qmax;
  double *Hs = sm, *M = Hs + n * ldh, *scr = M + rows_max * ldm;
  // X at `start` from the scan (unary relation held by the slot after the chunk that ends there)
  const int src = resweep ? t + 2 : t + 1;
  const double *xb = g.CS[fin] + (size_t)src * g.cs_stride;
  int rr = g.CI[fin][(size_t)src * CI_STRIDE + CI_ROWS];
  for (int idx = tid; idx < rr * ldh; idx += TEAM) {
    int i = idx / ldh, j = idx - i * ldh;
    Hs[idx] = xb[i * ldr + j];
  }
  tsync();
  for (int i = start - 1; i >= a; --i) {
    int inc = 0;
    if (rr == 0) {  // X_{i+1} = R^n: the stage's own projection, formed by k_primal_stage
      const int *wi = stage_wi(g, P.st0 + i);
      const double *Hp = stage_ws(g, P.st0 + i) + g.ws.Hpre;
      rr = wi[SI_PRE];
      inc = wi[SI_PREINC];
      for (int idx = tid; idx < rr * ldh; idx += TEAM) Hs[idx] = Hp[idx];
      tsync();
    } else {
      rr = primal_down_stage(g, P, i, Hs, rr, M, scr, &inc);
    }
    if (i >= b) continue;  // the next chunk's stage: stored by that chunk
    const int s = P.st0 + i;
    double *H = stage_ws(g, s) + g.ws.H;
    for (int idx = tid; idx < rr * ldh; idx += TEAM) H[idx] = Hs[idx];
    if (tid == 0) {
      stage_wi(g, s)[SI_HROWS] = rr;
      if (inc) set_status(g, ci.prob, ST_INFEASIBLE_SUFFIX);
    }
    tsync();
  }
}

// ----------------------------------------------------------- T_i, t_i, U_i (eq. state-param)
// QR of H_i^T: Q = [U_i | T_i], U_i spans range(H_i^T), T_i = orthonormal basis
// of null(H_i); t_i = min-norm solution of H_i t = -h_i; S_i = T_i^T.
__global__ void k_param(Group g, int per_task) {
  for_stages(g, [&](const int s) {
    const StageInfo S = g.st[s];
    const ProbInfo &P = g.prob[S.prob];
    if (skipped_by_mask(g, S.prob)) return;
    const int n = g.n, tid = team_rank();
    double *ws = stage_ws(g, s);
    int *wi = stage_wi(g, s);
    const int r = wi[SI_HROWS];
    double *sm = team_smem(per_task);
    double *Hs = sm, *Wt = Hs + n * (n + 1), *Qf = Wt + n * n, *hb = Qf + n * n, *X = hb + n;
    double *scr = X + n;
    int *perm = (int *)(scr + 4 * n);
    const double *H = ws + g.ws.H;
    for (int idx = tid; idx < r * (n + 1); idx += TEAM) Hs[idx] = H[idx];
    for (int i = tid; i < r; i += TEAM) hb[i] = H[i * (n + 1) + n];
    tsync();
    const int rank = wtqr(Hs, n + 1, r, n, g.tau_rank, Wt, (r > 0 ? r : 1), Qf, n, perm, scr);
    double *Ys = scr + 2 * n;  // rank x 1
    wtqr_solve(Wt, (r > 0 ? r : 1), Qf, n, perm, r, n, rank, hb, 1, 1, X, 1, Ys, 1);
    double *UT = ws + g.ws.UT, *tt = ws + g.ws.t;
    // T = I and t = 0 exactly (compared as bit patterns, on the integer pipe; a zero of
    // either sign counts as zero): the stage elimination then skips its products with T_i,
    // whose results are the factors themselves
    bool eye = true;
    for (int idx = tid; idx < n * n; idx += TEAM) {
      UT[idx] = Qf[idx];
      const long long b = __double_as_longlong(Qf[idx]);
      eye = eye && ((idx / n) * (n + 1) == idx ? b == __double_as_longlong(1.0) : (b << 1) == 0);
    }
    for (int i = tid; i < n; i += TEAM) {
      tt[i] = X[i];
      eye = eye && (__double_as_longlong(X[i]) << 1) == 0;
    }
    eye = __syncthreads_and(eye) != 0;
    if (tid == 0) { wi[SI_UR] = rank; wi[SI_NBAR] = n - rank; wi[SI_TEYE] = (rank == 0 && eye) ? 1 : 0; }
    tsync();
    if (S.i == P.N) {
      // terminal cost (eq. terminal-cost-data): Qbar_N = T' Q_N T, qbar_N = T'(Q_N t + q_N)
      const int nb = n - rank;
      const double *QN = g.Q + P.oQ + (size_t)P.N * n * n, *qN = g.qv + P.oqv + (size_t)P.N * n;
      double *QT = Wt;  // n x nb (reuse)
      double *T = Qf + rank;  // columns rank.. of Qf, ld n
      wgemm<false, false>(n, nb, n, 1.0, QN, n, T, n, 0.0, QT, n);
      wgemm<true, false>(nb, nb, n, 1.0, T, n, QT, n, 0.0, ws + g.ws.Qb, n);
      for (int l = tid; l < n; l += TEAM) {
        double s0 = qN[l];
        for (int j = 0; j < n; j++) s0 = fma(QN[l * n + j], X[j], s0);
        Hs[l] = s0;
      }
      tsync();
      wgemm<true, false>(nb, 1, n, 1.0, T, n, Hs, 1, 0.0, ws + g.ws.qb, 1);
    }
  });
}

// ----------------------------------------------------------- stage elimination (Sec. 5)
// at most 64 registers a thread: with four-warp teams (n >= 16) 80 registers left 6 CTAs
// per SM where 64 leave 8 (n = 16: 40 ms against 45 over the group)
__global__ void __launch_bounds__(256, 4) k_elim(Group g, int per_task) {
  for_stages(g, [&](const int s) {
    const StageInfo S = g.st[s];
    const ProbInfo &P = g.prob[S.prob];
    if (skipped_by_mask(g, S.prob)) return;
    if (S.i >= P.N) return;
    const int n = g.n, m = g.m, tid = team_rank(), i = S.i;
    double *ws = stage_ws(g, s), *wn = stage_ws(g, s + 1);
    int *wi = stage_wi(g, s), *win = stage_wi(g, s + 1);
    const int ur = wi[SI_UR], nb = n - ur, ur1 = win[SI_UR], nn = n - ur1, r1 = win[SI_HROWS];
    const int rows = S.p + r1;
    // T_i = I, t_i = 0 (te) and T_{i+1} = I, t_{i+1} = 0 (tne): a product with T is then its other
    // factor, bit for bit up to the sign of zeros, and is copied instead of computed
    const bool te = wi[SI_TEYE] != 0, tne = win[SI_TEYE] != 0;
    const double *A = g.A + P.oA + (size_t)i * n * n, *B = g.B + P.oB + (size_t)i * n * m;
    const double *c = g.c + P.oc + (size_t)i * n;
    const double *Q = g.Q + P.oQ + (size_t)i * n * n, *Mm = g.M + P.oM + (size_t)i * n * m;
    const double *R = g.R + P.oR + (size_t)i * m * m;
    const double *q = g.qv + P.oqv + (size_t)i * n, *r = g.rv + P.orv + (size_t)i * m;
    const double *T = ws + g.ws.UT + ur, *t = ws + g.ws.t;        // ld n
    const double *Tn = wn + g.ws.UT + ur1, *tn = wn + g.ws.t;     // ld n
    const double *Hn = wn + g.ws.H;                                 // ld n + 1
    double *sm = team_smem(per_task);
    const int rmax = g.pmax + n;
    // live through the stage
    double *AT = sm;                       // n x n (ld n)
    double *Qm = AT + n * n;               // m x m: Q of Gamma' (Z = its last columns)
    double *Yw = Qm + m * m;               // m x n  (ld n): Y
    double *vec = Yw + n * m;              // elim_vec doubles
    double *Atc = vec, *cv = Atc + n, *Qtq = cv + n, *qz = Qtq + n, *rz = qz + n, *Ry = rz + m;
    double *ys = Ry + m, *scr = ys + m;    // the QR's scratch: m + max(m, rmax)
    int *perm = (int *)(scr + m + (m > rmax ? m : rmax));
    double *U = vec + elim_vec(n, m, g.pmax);  // the phases' region
    // Lemma 4's solve
    const int gr = rmax * m > rmax * (n + 1) ? rmax * m : rmax * (n + 1);
    double *Gm = U;                        // rmax x m: Gamma, copied into Wt by the QR
    double *Rh = U;                        // rmax x (n+1): [Phi | gamma], formed after the QR
    double *Wt = U + gr;                   // m x rmax
    double *Sol = Wt + m * rmax;           // m x (n+1)
    double *X1 = Sol + m * (n + 1);        // m x (n+1) scratch for the min-norm solve
    // the substitution products
    double *QT = U;                        // n x n: Q T, read only by Q^z
    double *X2 = QT;                       // n x n: M^z Y, after Q^z
    double *Mz = QT + n * n;               // n x m
    double *RY = Mz + n * m;               // m x n
    double *BZ = RY + n * m;               // n x m
    double *RZ = BZ + n * m;               // m x m
    // A T, A t + c
    if (te) {
      for (int idx = tid; idx < n * n; idx += TEAM) AT[idx] = A[idx];
      for (int l = tid; l < n; l += TEAM) Atc[l] = c[l];
    } else {
      wgemm<false, false>(n, nb, n, 1.0, A, n, T, n, 0.0, AT, n);
      for (int l = tid; l < n; l += TEAM) {
        double s0 = c[l];
        for (int j = 0; j < n; j++) s0 = fma(A[l * n + j], t[j], s0);
        Atc[l] = s0;
      }
    }
    // Gamma = [D; Hn B]
    for (int idx = tid; idx < S.p * m; idx += TEAM) {
      int a = idx / m, j = idx - a * m;
      Gm[a * m + j] = g.D[P.oD + (size_t)(S.prow + a) * m + j];
    }
    wgemm<false, false>(r1, m, n, 1.0, Hn, n + 1, B, m, 0.0, Gm + S.p * m, m);
    // Lemma 4: Z = null(Gamma), [Y | y] = -Gamma^- [Phi | gamma] (min norm)
    // the small form only: this kernel runs many CTAs to an SM, and the large form's
    // registers and static scratch would cost it occupancy
    const int rank = wtqr_small(Gm, m, rows, m, g.tau_rank, Wt, (rows > 0 ? rows : 1), Qm, m, perm, scr);
    // [Phi | gamma] = [C T | C t + d; Hn A T | Hn (A t + c) + hn], in Gamma's block (the QR
    // has copied Gamma into Wt)
    for (int idx = tid; idx < S.p * (nb + 1); idx += TEAM) {
      int a = idx / (nb + 1), j = idx - a * (nb + 1);
      const double *Cr = g.C + P.oC + (size_t)(S.prow + a) * n;
      double s0 = 0.0;
      if (te) {
        s0 = (j < nb) ? Cr[j] : g.d[P.od + S.prow + a];
      } else if (j < nb) {
        for (int l = 0; l < n; l++) s0 = fma(Cr[l], T[l * n + j], s0);
      } else {
        s0 = g.d[P.od + S.prow + a];
        for (int l = 0; l < n; l++) s0 = fma(Cr[l], t[l], s0);
      }
      Rh[a * (nb + 1) + j] = s0;
    }
    for (int idx = tid; idx < r1 * (nb + 1); idx += TEAM) {
      int a = idx / (nb + 1), j = idx - a * (nb + 1);
      const double *hr = Hn + a * (n + 1);
      double s0 = 0.0;
      if (j < nb) {
        for (int l = 0; l < n; l++) s0 = fma(hr[l], AT[l * n + j], s0);
      } else {
        s0 = hr[n];
        for (int l = 0; l < n; l++) s0 = fma(hr[l], Atc[l], s0);
      }
      Rh[(S.p + a) * (nb + 1) + j] = s0;
    }
    tsync();
    const double rs = wtqr_solve(Wt, (rows > 0 ? rows : 1), Qm, m, perm, rows, m, rank, Rh, nb + 1, nb + 1,
                                 Sol, nb + 1, X1, nb + 1);
    if (tid == 0 && rs > g.tau_inc) set_status(g, S.prob, ST_RANK_INCONSISTENT);
    const int mb = m - rank;
    const double *Z = Qm + rank;  // ld m
    // Y (m x nb, ld n), y (m)
    for (int idx = tid; idx < m * nb; idx += TEAM) {
      int a = idx / nb, j = idx - a * nb;
      Yw[a * n + j] = Sol[a * (nb + 1) + j];
    }
    for (int a = tid; a < m; a += TEAM) ys[a] = Sol[a * (nb + 1) + nb];
    tsync();
    // reduced dynamics (eq. reduced-dynamics-data), S_{i+1} = T_{i+1}^T
    wgemm<false, false>(n, nb, m, 1.0, B, m, Yw, n, 1.0, AT, n);            // A T + B Y
    if (!tne) wgemm<true, false>(nn, nb, n, 1.0, Tn, n, AT, n, 0.0, ws + g.ws.Ab, n);
    wgemm<false, false>(n, mb, m, 1.0, B, m, Z, m, 0.0, BZ, m);             // B Z
    if (!tne) wgemm<true, false>(nn, mb, n, 1.0, Tn, n, BZ, m, 0.0, ws + g.ws.Bb, m);
    for (int l = tid; l < n; l += TEAM) {
      double s0 = Atc[l] - tn[l];
      for (int j = 0; j < m; j++) s0 = fma(B[l * m + j], ys[j], s0);
      cv[l] = s0;
    }
    tsync();
    if (tne) {  // Abar = A T + B Y, Bbar = B Z, cbar = c_v
      for (int idx = tid; idx < n * nb; idx += TEAM) {
        const int a = idx / nb, j = idx - a * nb;
        ws[g.ws.Ab + a * n + j] = AT[a * n + j];
      }
      for (int idx = tid; idx < n * mb; idx += TEAM) {
        const int a = idx / mb, j = idx - a * mb;
        ws[g.ws.Bb + a * m + j] = BZ[a * m + j];
      }
      for (int l = tid; l < n; l += TEAM) ws[g.ws.cb + l] = cv[l];
    } else {
      wgemm<true, false>(nn, 1, n, 1.0, Tn, n, cv, 1, 0.0, ws + g.ws.cb, 1);
    }
    // state substitution (eq. state-cost-data)
    double *Qb = ws + g.ws.Qb, *Mb = ws + g.ws.Mb, *Rb = ws + g.ws.Rb;
    if (te) {  // Q^z = Q, M^z = M, q^z = q, r^z = r
      for (int idx = tid; idx < n * n; idx += TEAM) Qb[idx] = Q[idx];
      for (int idx = tid; idx < n * m; idx += TEAM) Mz[idx] = Mm[idx];
      for (int l = tid; l < n; l += TEAM) qz[l] = q[l];
      for (int a = tid; a < m; a += TEAM) rz[a] = r[a];
      tsync();
    } else {
      wgemm<false, false>(n, nb, n, 1.0, Q, n, T, n, 0.0, QT, n);             // Q T
      wgemm<true, false>(nb, nb, n, 1.0, T, n, QT, n, 0.0, Qb, n);            // Q^z
      wgemm<true, false>(nb, m, n, 1.0, T, n, Mm, m, 0.0, Mz, m);             // M^z
      for (int l = tid; l < n; l += TEAM) {
        double s0 = q[l];
        for (int j = 0; j < n; j++) s0 = fma(Q[l * n + j], t[j], s0);
        Qtq[l] = s0;
      }
      for (int a = tid; a < m; a += TEAM) {
        double s0 = r[a];
        for (int l = 0; l < n; l++) s0 = fma(Mm[l * m + a], t[l], s0);
        rz[a] = s0;                                                           // r^z
      }
      tsync();
      wgemm<true, false>(nb, 1, n, 1.0, T, n, Qtq, 1, 0.0, qz, 1);            // q^z
    }
    // reduced cost (eq. reduced-cost-data)
    wgemm<false, false>(m, nb, m, 1.0, R, m, Yw, n, 0.0, RY, n);            // R Y
    wgemm<false, false>(m, mb, m, 1.0, R, m, Z, m, 0.0, RZ, m);             // R Z
    for (int a = tid; a < m; a += TEAM) {
      double s0 = rz[a];
      for (int j = 0; j < m; j++) s0 = fma(R[a * m + j], ys[j], s0);
      Ry[a] = s0;                                                           // R y + r^z
    }
    tsync();
    wgemm<false, false>(nb, nb, m, 1.0, Mz, m, Yw, n, 0.0, X2, n);          // M^z Y
    for (int idx = tid; idx < nb * nb; idx += TEAM) {
      int a = idx / nb, j = idx - a * nb;
      Qb[a * n + j] += X2[a * n + j] + X2[j * n + a];
    }
    tsync();
    wgemm<true, false>(nb, nb, m, 1.0, Yw, n, RY, n, 1.0, Qb, n);           // + Y' R Y
    wgemm<false, false>(nb, mb, m, 1.0, Mz, m, Z, m, 0.0, Mb, m);           // M^z Z
    wgemm<true, false>(nb, mb, m, 1.0, Yw, n, RZ, m, 1.0, Mb, m);           // + Y' R Z
    wgemm<true, false>(mb, mb, m, 1.0, Z, m, RZ, m, 0.0, Rb, m);            // Z' R Z
    double *qb = ws + g.ws.qb, *rb = ws + g.ws.rb;
    for (int a = tid; a < nb; a += TEAM) {
      double s0 = qz[a];
      for (int j = 0; j < m; j++) s0 = fma(Mz[a * m + j], ys[j], s0);
      for (int j = 0; j < m; j++) s0 = fma(Yw[j * n + a], Ry[j], s0);
      qb[a] = s0;
    }
    for (int a = tid; a < mb; a += TEAM) {
      double s0 = 0.0;
      for (int j = 0; j < m; j++) s0 = fma(Z[j * m + a], Ry[j], s0);
      rb[a] = s0;
    }
    // Y, Z, y for recovery (eq. recovery-maps)
    double *Yo = ws + g.ws.Y, *Zo = ws + g.ws.Z, *yo = ws + g.ws.y;
    for (int idx = tid; idx < m * n; idx += TEAM) Yo[idx] = Yw[idx];
    for (int idx = tid; idx < m * m; idx += TEAM) {
      int a = idx / m, j = idx - a * m;
      Zo[idx] = (j < mb) ? Z[a * m + j] : 0.0;
    }
    for (int a = tid; a < m; a += TEAM) yo[a] = ys[a];
    if (tid == 0) wi[SI_MBAR] = mb;
    tsync();
    // square root of the reduced stage Hessian [[Qbar, Mbar], [Mbar', Rbar]] (order z, v):
    // L L' = H, stored as L' (upper) with l = L^{-1} [qbar; rbar], for the square-root LQR
    {
      // stage Hessian in the order (v, z) -- the column order of the Riccati's QR, so that L'
      // is upper triangular there -- bordered by g = [rbar; qbar]
      const int kh = nb + mb, ldh = n + m, ldH = kh + 1;
      double *Hh = U;  // the phases' region: everything else there is dead
      for (int idx = tid; idx < (kh + 1) * kh; idx += TEAM) {
        int a = idx / kh, j = idx - a * kh;
        double h;
        if (a == kh) h = (j < mb) ? rb[j] : qb[j - mb];
        else if (a < mb && j < mb) h = Rb[a * m + j];
        else if (a < mb) h = Mb[(j - mb) * m + a];
        else if (j < mb) h = Mb[(a - mb) * m + j];
        else h = Qb[(a - mb) * n + (j - mb)];
        Hh[a * ldH + j] = h;
      }
      tsync();
      int fail = 0;
      if (tid < 32) fail = wchol_bordered(Hh, ldH, kh);
      fail = __syncthreads_or(fail);
      if (fail && tid == 0) set_status(g, S.prob, ST_NONCONVEX);
      double *LT = ws + g.ws.LT, *lt = ws + g.ws.lt;
      for (int idx = tid; idx < kh * kh; idx += TEAM) {
        int a = idx / kh, j = idx - a * kh;
        LT[a * ldh + j] = (j >= a) ? Hh[j * ldH + a] : 0.0;
      }
      for (int a = tid; a < kh; a += TEAM) lt[a] = Hh[kh * ldH + a];  // L^{-1} [rbar; qbar]
    }
  });
}

}  // namespace eclqr
