// k_lqr.cu -- the reduced unconstrained LQR (Sec. 6) and the recovery maps
// (eq. recovery-maps) on sm_103a.
//
// Riccati factors.  The paper obtains log depth from an associative LQR scan
// [ref-AS-LQR].  Here the scan elements are conditional costs V(z_a | z_b) of
// a chunk kept in square-root form, as "cost relations": constraint rows that
// hold exactly (states z_b reachable from z_a) and least-squares cost rows on
// (z_a, z_b).  Composition eliminates the shared state by equality-constrained
// least squares (wlse_elim: orthogonal and pivoted), so value functions whose
// Hessians grow without bound through stretches without control authority
// turn into constraints instead of cancelling.  Chunks compose their own
// stages, a log-depth scan over chunks gives V at every chunk boundary, and
// each chunk then runs the square-root Riccati recursion inward, storing P_i,
// K_i, the Cholesky factor of Rbar + Bbar'P Bbar and Phi_i = Abar + Bbar K_i.
//
// Linear passes.  With those factors the remaining recursions are affine
// chains: p_i = Phi_i' (P_{i+1} c_i + p_{i+1}) + q_i + K_i' r_i backwards and
// z_{i+1} = Phi_i z_i + Bbar k_i + c_i forwards.  They run as chunked affine
// scans (k_aff_*), also used for the refinement passes on the reduced KKT
// residual and for the forward costate expansion of Sec. 7.
#include "kernels.cuh"

namespace eclqr {

__host__ int smem_lqr_up(int n, int m) {
  const int ldr = 2 * n + 1, rows = 5 * n + m, ldm = m + 2 * n + 1;
  return 2 * (2 * n) * ldr + rows * ldm + 2 * rows + 2 * (ldm + rows) + m + 16;
}
__host__ int smem_lqr_level(int n) {
  const int rows = 8 * n, ldm = 3 * n + 1;
  return rows * ldm + 2 * rows + 2 * (ldm + rows) + n + 16;
}
// V, the stacked rows, and the reflector's two vectors; the FP32 sweep's blocks (the same
// ones in floats, its gains and the stage data) fit in the same bytes
__host__ int smem_riccati(int n, int m) {
  const int rows = 2 * n + m, ld = n + m + 1;
  return n * (n + 1) + rows * ld + rows + ld + 8;
}
__host__ int smem_riccati_finish(int n, int m) { return m * (n + m + 1) + n * (n + 1) + m * (n + 1) + 8; }
__host__ int smem_aff(int n, int m) { return 2 * (n * n + n) + n * n + 5 * n + 2 * m + 8; }

// Cost-relation slot layout (ld 2n + 1): constraint rows at 0 (CI_ROWS of them),
// cost rows at offset 2n (2n + 1) (CI_ROWS2 of them); CI_NA / CI_NB are the
// endpoint dimensions, CI_NB = 0 marks a value function (unary, cost only).
__device__ __forceinline__ double *crel_cost(double *slot, int n) { return slot + 2 * n * (2 * n + 1); }

// ----------------------------------------------------------- chunk conditional costs
// Up-sweep over stages b-1 .. a of the conditional cost V(z_i | z_b): a cost
// relation on (z_i, z_b).  Stage i substitutes the reduced dynamics
// z_{i+1} = Abar z_i + Bbar v + cbar into the rows on (z_{i+1}, z_b), stacks the
// stage cost rows L'[z; v] + l and eliminates v (wlse_elim).
__global__ void k_lqr_up(Group g, int per_task) {
  const int t = team_task();
  if (t >= g.nslot) return;
  const ChunkInfo ci = g.chunk[t];
  const ProbInfo &P = g.prob[ci.prob];
  if (skipped_by_mask(g, ci.prob)) return;
  const int n = g.n, m = g.m, tid = team_rank();
  const int ldr = 2 * n + 1;
  double *slot = g.CS[0] + (size_t)t * g.cs_stride;
  int *cm = g.CI[0] + (size_t)t * CI_STRIDE;
  double *sm = team_smem(per_task);
  if (ci.c == P.nch) {
    // terminal value: rows [L' | L^{-1} qbar_N], L L' = Qbar_N (eq. terminal-cost-data)
    const int sN = P.st0 + P.N;
    const double *ws = stage_ws(g, sN);
    const int nN = stage_wi(g, sN)[SI_NBAR];
    double *Hh = sm, *l = sm + n * n;
    for (int idx = tid; idx < nN * nN; idx += TEAM) {
      int a = idx / nN, j = idx - a * nN;
      Hh[idx] = ws[g.ws.Qb + a * n + j];
    }
    tsync();
    const int fail = wcholesky(Hh, nN, nN);
    if (tid == 0) {
      for (int a = 0; a < nN; a++) {
        double s0 = ws[g.ws.qb + a];
        for (int k = 0; k < a; k++) s0 = fma(-Hh[a * nN + k], l[k], s0);
        l[a] = s0 / Hh[a * nN + a];
      }
    }
    tsync();
    double *cost = crel_cost(slot, n);
    for (int idx = tid; idx < nN * (nN + 1); idx += TEAM) {
      int a = idx / (nN + 1), j = idx - a * (nN + 1);
      cost[a * ldr + j] = (j < nN) ? Hh[j * nN + a] : l[a];
    }
    if (tid == 0) {
      cm[CI_ROWS] = 0; cm[CI_NA] = nN; cm[CI_NB] = 0; cm[CI_ROWS2] = nN;
      if (fail) set_status(g, ci.prob, ST_NONCONVEX);
    }
    return;
  }
  if (P.nch == 1) {  // one chunk: k_riccati_down starts from the terminal value alone
    if (tid == 0) { cm[CI_ROWS] = 0; cm[CI_NA] = 0; cm[CI_NB] = 0; cm[CI_ROWS2] = 0; }
    return;
  }
  const int a = ci.c * P.L, b = min(a + P.L, P.N);
  const int nbz = stage_wi(g, P.st0 + b)[SI_NBAR];
  const int rows_max = 5 * n + m, ldm_max = m + 2 * n + 1;
  double *Cons = sm, *Cost = Cons + 2 * n * ldr, *M = Cost + 2 * n * ldr, *scr = M + rows_max * ldm_max;
  // z_b' = z_b on (z_b', z_b)
  for (int idx = tid; idx < nbz * ldr; idx += TEAM) {
    int i = idx / ldr, j = idx - i * ldr;
    Cons[idx] = (j == i) ? 1.0 : ((j == nbz + i) ? -1.0 : 0.0);
  }
  tsync();
  int rc = nbz, rq = 0;
  int fail = 0;
  for (int i = b - 1; i >= a; --i) {
    const int s = P.st0 + i;
    const double *ws = stage_ws(g, s);
    const int *wi = stage_wi(g, s);
    const int nx = wi[SI_NBAR], mu = wi[SI_MBAR], n1 = stage_wi(g, s + 1)[SI_NBAR];
    const int ldm = mu + nx + nbz + 1, kh = nx + mu;
    const double *Ab = ws + g.ws.Ab, *Bb = ws + g.ws.Bb, *cb = ws + g.ws.cb, *LT = ws + g.ws.LT, *lt = ws + g.ws.lt;
    // columns v (mu) | z_i (nx) | z_b (nbz) | 1
    // rows: constraints (rc) then stage cost (kh) then old cost (rq)
    const int rtot = rc + kh + rq;
    for (int idx = tid; idx < rtot * ldm; idx += TEAM) {
      int r = idx / ldm, j = idx - r * ldm;
      double val = 0.0;
      if (r < rc || r >= rc + kh) {
        const double *row = (r < rc) ? Cons + r * ldr : Cost + (r - rc - kh) * ldr;  // [K1 (n1) | Kb (nbz) | k]
        if (j < mu) {
          for (int l = 0; l < n1; l++) val = fma(row[l], Bb[l * m + j], val);
        } else if (j < mu + nx) {
          for (int l = 0; l < n1; l++) val = fma(row[l], Ab[l * n + (j - mu)], val);
        } else if (j < mu + nx + nbz) {
          val = row[n1 + (j - mu - nx)];
        } else {
          val = row[n1 + nbz];
          for (int l = 0; l < n1; l++) val = fma(row[l], cb[l], val);
        }
      } else {
        const int q = r - rc;  // stage cost row q of L' (columns v then z, as here)
        if (j < mu + nx) val = LT[q * (n + m) + j];
        else if (j == ldm - 1) val = lt[q];
      }
      M[idx] = val;
    }
    tsync();
    LseResult lr = wlse_elim(M, ldm, rc, kh + rq, mu, nx + nbz, g.tau_rank, g.tau_inc, Cons, Cost, ldr, scr);
    rc = lr.kc;
    rq = lr.kq;
    fail |= lr.inconsistent;
  }
  for (int idx = tid; idx < rc * ldr; idx += TEAM) slot[idx] = Cons[idx];
  double *cost = crel_cost(slot, n);
  for (int idx = tid; idx < rq * ldr; idx += TEAM) cost[idx] = Cost[idx];
  if (tid == 0) {
    cm[CI_ROWS] = rc; cm[CI_NA] = stage_wi(g, P.st0 + a)[SI_NBAR]; cm[CI_NB] = nbz; cm[CI_ROWS2] = rq;
    if (fail) set_status(g, ci.prob, ST_NONCONVEX);
  }
}

// One level of the chunk suffix scan on cost relations: slot t <- slot t o slot t + d,
// eliminating the shared state (wlse_elim); a value on the right gives a value.
__global__ void k_lqr_level(Group g, int src, int d, int per_task) {
  const int t = team_task();
  if (t >= g.nslot) return;
  const ChunkInfo ci = g.chunk[t];
  const ProbInfo &P = g.prob[ci.prob];
  if (skipped_by_mask(g, ci.prob)) return;
  const int n = g.n, tid = team_rank(), ldr = 2 * n + 1;
  double *S1 = g.CS[src] + (size_t)t * g.cs_stride;
  const int *I1 = g.CI[src] + (size_t)t * CI_STRIDE;
  double *Dst = g.CS[src ^ 1] + (size_t)t * g.cs_stride;
  int *J = g.CI[src ^ 1] + (size_t)t * CI_STRIDE;
  const int rc1 = I1[CI_ROWS], na = I1[CI_NA], nm = I1[CI_NB], rq1 = I1[CI_ROWS2];
  if (ci.c + d > P.nch || nm == 0) {
    for (int idx = tid; idx < rc1 * ldr; idx += TEAM) Dst[idx] = S1[idx];
    for (int idx = tid; idx < rq1 * ldr; idx += TEAM) crel_cost(Dst, n)[idx] = crel_cost(S1, n)[idx];
    if (tid == 0) { J[CI_ROWS] = rc1; J[CI_NA] = na; J[CI_NB] = nm; J[CI_ROWS2] = rq1; }
    return;
  }
  double *S2 = g.CS[src] + (size_t)(t + d) * g.cs_stride;
  const int *I2 = g.CI[src] + (size_t)(t + d) * CI_STRIDE;
  const int rc2 = I2[CI_ROWS], nb = I2[CI_NB], rq2 = I2[CI_ROWS2];
  double *sm = team_smem(per_task);
  const int ldm = nm + na + nb + 1;
  const int rc = rc1 + rc2, rq = rq1 + rq2;
  double *M = sm, *scr = sm + (rc + rq) * ldm;
  // columns z_m | z_a | z_b | 1 ; rows: constraints of e1, e2, then costs of e1, e2
  for (int idx = tid; idx < (rc + rq) * ldm; idx += TEAM) {
    int r = idx / ldm, j = idx - r * ldm;
    bool left;
    const double *row;
    if (r < rc1) { left = true; row = S1 + r * ldr; }
    else if (r < rc) { left = false; row = S2 + (r - rc1) * ldr; }
    else if (r < rc + rq1) { left = true; row = crel_cost(S1, n) + (r - rc) * ldr; }
    else { left = false; row = crel_cost(S2, n) + (r - rc - rq1) * ldr; }
    double val = 0.0;
    if (left) {          // [z_a (na) | z_m (nm) | 1]
      if (j < nm) val = row[na + j];
      else if (j < nm + na) val = row[j - nm];
      else if (j == ldm - 1) val = row[na + nm];
    } else {             // [z_m (nm) | z_b (nb) | 1]
      if (j < nm) val = row[j];
      else if (j >= nm + na && j < nm + na + nb) val = row[nm + (j - nm - na)];
      else if (j == ldm - 1) val = row[nm + nb];
    }
    M[idx] = val;
  }
  tsync();
  LseResult lr = wlse_elim(M, ldm, rc, rq, nm, na + nb, g.tau_rank, g.tau_inc, Dst, crel_cost(Dst, n), ldr, scr);
  if (tid == 0) {
    J[CI_ROWS] = lr.kc; J[CI_NA] = na; J[CI_NB] = nb; J[CI_ROWS2] = lr.kq;
    if (lr.inconsistent) set_status(g, ci.prob, ST_NONCONVEX);
  }
}

// ----------------------------------------------------------- chunk down-sweep: square-root Riccati
// From V_b = 1/2 ||C z_b + c||^2 (the scan's value at the chunk end), each stage
// stacks [L'_v | L'_z | l] and [C Bbar | C Abar | C cbar + c] over (v | z | 1) and
// triangularises them by Householder QR: R_vv v + R_vz z + o_v = 0 at the
// minimiser (K, k) and V_i = 1/2 ||R_i z + s_i||^2 with R_i upper triangular,
// rows signed so that its diagonal is positive.  The sweep carries only V from
// stage to stage; it stores the minimiser's rows (R_vv | R_vz | o_v) and
// [R_i | s_i] (in the slots of P_i, p_i), and k_riccati_finish forms the
// factors from them for every stage at once, off the sequential chain.
static __device__ void riccati_task(const Group &g, int fin, int t, int per_task);
__global__ void k_riccati_down(Group g, int fin, int per_task, int *queue) {
  for_tasks(g.nslot, queue, [&](int t) { riccati_task(g, fin, t, per_task); });
}

static __device__ void riccati_task(const Group &g, int fin, int t, int per_task) {
  if (t >= g.nslot) return;
  const ChunkInfo ci = g.chunk[t];
  const ProbInfo &P = g.prob[ci.prob];
  if (skipped_by_mask(g, ci.prob)) return;
  if (g.fp64 != nullptr && g.fp64[P.id] == 0) return;  // mixed precision: k_riccati_down_f32 sweeps it
  if (ci.c >= P.nch) return;
  const int n = g.n, m = g.m, tid = team_rank();
  const int a = ci.c * P.L, b = min(a + P.L, P.N);
  // every chunk but the last re-sweeps the next chunk's stages from the same scan value, so that the
  // value function it starts from is, bit for bit, the one the next chunk computes at their boundary
  const bool resweep = ci.c + 1 < P.nch;
  const int start = resweep ? min(b + P.L, P.N) : b;
  const int ldr = 2 * n + 1;
  double *sm = team_smem(per_task);
  const int rows_max = 2 * n + m, ldst = n + m + 1;
  double *V = sm, *St = V + n * (n + 1), *v = St + rows_max * ldst, *w = v + rows_max;
  // V_b, rows signed to a positive diagonal
  int rv;
  {
    const int slot = resweep ? t + 2 : t + 1;
    const double *src = crel_cost(g.CS[fin] + (size_t)slot * g.cs_stride, n);
    const int *I = g.CI[fin] + (size_t)slot * CI_STRIDE;
    const int nbz = I[CI_NA];
    rv = I[CI_ROWS2];
    for (int idx = tid; idx < rv * (nbz + 1); idx += TEAM) {
      int r = idx / (nbz + 1), j = idx - r * (nbz + 1);
      const double sg = (src[r * ldr + r] >= 0.0) ? 1.0 : -1.0;
      V[r * (n + 1) + j] = sg * src[r * ldr + j];
    }
    tsync();
    if (b == P.N) {  // P_N = C'C, p_N = C'c
      double *wsN = stage_ws(g, P.st0 + b);
      for (int idx = tid; idx < nbz * (nbz + 1); idx += TEAM) {
        int r = idx / (nbz + 1), j = idx - r * (nbz + 1);
        double s0 = 0.0;
        for (int l = 0; l < rv; l++) s0 = fma(V[l * (n + 1) + r], V[l * (n + 1) + j], s0);
        if (j < nbz) wsN[g.ws.P + r * n + j] = s0; else wsN[g.ws.p + r] = s0;
      }
    }
  }
  for (int i = start - 1; i >= a; --i) {
    const bool store = i < b;  // the next chunk's stages are stored by that chunk
    const int s = P.st0 + i;
    double *ws = stage_ws(g, s);
    int *wi = stage_wi(g, s);
    const int nx = wi[SI_NBAR], mu = wi[SI_MBAR], n1 = stage_wi(g, s + 1)[SI_NBAR];
    const int kh = nx + mu, ld = kh + 1;
    const double *Ab = ws + g.ws.Ab, *Bb = ws + g.ws.Bb, *cb = ws + g.ws.cb, *LT = ws + g.ws.LT, *lt = ws + g.ws.lt;
    // value rows [V Bbar | V Abar | V cbar + s] at St rows kh .. kh + rv - 1; after the first
    // stage V = [R_{i+1} | s_{i+1}] with R_{i+1} upper triangular (exact zeros below its
    // diagonal), so row r's products start at column r
    for (int idx = tid; idx < rv * ld; idx += TEAM) {
      int r = idx / ld, j = idx - r * ld;
      const double *row = V + r * (n + 1);
      const int l0 = (i < start - 1) ? r : 0;
      double val = 0.0;
      if (j < mu) {
        for (int l = l0; l < n1; l++) val = fma(row[l], Bb[l * m + j], val);
      } else if (j < kh) {
        for (int l = l0; l < n1; l++) val = fma(row[l], Ab[l * n + (j - mu)], val);
      } else {
        val = row[n1];
        for (int l = l0; l < n1; l++) val = fma(row[l], cb[l], val);
      }
      St[(kh + r) * ld + j] = val;
    }
    // QR of [L' l; value rows] with L' (columns v, z) upper triangular: the reflector of
    // column k has entries only in row k of L' and in the value rows, so step k works on
    // those rv + 1 rows alone.  Row k of L' is loaded into the slot right above the value
    // rows (St row kh - 1), and the finished row moves to St row k before the next load.
    // The next row of L' is read from global memory into registers before the current step
    // runs (thread tid holds columns tid and tid + TEAM, kh + 1 <= 2 TEAM), so its latency
    // hides behind the step.
    double nxt[2];
    for (int q = 0; q < 2; q++) {
      const int j = tid + q * TEAM;
      nxt[q] = (j <= kh && kh > 0) ? ((j < kh) ? LT[j] : lt[0]) : 0.0;
    }
    for (int k = 0; k < kh; k++) {
      double *W = St + (kh - 1) * ld;
      for (int q = 0; q < 2; q++) {
        const int j = tid + q * TEAM;
        if (j > kh) continue;
        if (k > 0 && j >= k - 1) St[(k - 1) * ld + j] = W[j];
        if (j >= k) W[j] = nxt[q];
      }
      tsync();
      if (k + 1 < kh)
        for (int q = 0; q < 2; q++) {
          const int j = tid + q * TEAM;
          if (j >= k + 1 && j <= kh) nxt[q] = (j < kh) ? LT[(k + 1) * (n + m) + j] : lt[k + 1];
        }
      HHLayout L = hh_layout(kh + 1 - k, rv + 1);
      hh_core(W, ld, 0, rv + 1, k, nullptr, k, kh + 1 - k, L, v, w, 0.0);
    }
    // sign the z rows to a positive diagonal (rows mu .. kh - 1), on the integer pipe: a row
    // whose diagonal is below zero (sign bit set, not -0, not NaN) has every sign bit flipped
    for (int idx = tid; idx < nx * ld; idx += TEAM) {
      int r = mu + idx / ld, j = idx - (idx / ld) * ld;
      const long long db = __double_as_longlong(St[r * ld + r]);
      const bool neg = db < 0 && (db & 0x7fffffffffffffffll) != 0 && (db & 0x7fffffffffffffffll) <= 0x7ff0000000000000ll;
      if (neg && j != r) St[r * ld + j] = __longlong_as_double(__double_as_longlong(St[r * ld + j]) ^ (1ll << 63));
    }
    tsync();
    for (int r = mu + tid; r < kh; r += TEAM)
      St[r * ld + r] = __longlong_as_double(__double_as_longlong(St[r * ld + r]) & 0x7fffffffffffffffll);
    tsync();
    // the minimiser's rows (R_vv | R_vz | o_v) for k_riccati_finish, and the new value rows
    // [R_i | s_i], kept here and stored in the slots of P_i, p_i (ld n + 1)
    if (store) {
      double *Rv = ws + g.ws.Rv;
      for (int idx = tid; idx < mu * ld; idx += TEAM) {
        int r = idx / ld, j = idx - r * ld;
        Rv[r * (n + m + 1) + j] = St[r * ld + j];
      }
    }
    for (int idx = tid; idx < nx * (nx + 1); idx += TEAM) {
      int r = idx / (nx + 1), c = idx - r * (nx + 1);
      V[r * (n + 1) + c] = (c < nx) ? ((c >= r) ? St[(mu + r) * ld + mu + c] : 0.0) : St[(mu + r) * ld + kh];
    }
    tsync();
    rv = nx;
    if (store)
      for (int idx = tid; idx < nx * (nx + 1); idx += TEAM) {
        int r = idx / (nx + 1), c = idx - r * (nx + 1);
        ws[g.ws.P + r * (n + 1) + c] = V[r * (n + 1) + c];
      }
  }
}

// ----------------------------------------------------------- Riccati factors, every stage at once
// For each stage i < N that the sweep stored (FP64 sweeps only): from the
// minimiser's rows, R_vv [K | k] = -[R_vz | o_v] by back substitution, the
// Cholesky factor of H_uu = R_vv'R_vv (R_vv' with rows signed to a positive
// diagonal), Phi = Abar + Bbar K (the closed-loop map of the affine chains), and
// from [R_i | s_i], P_i = R_i'R_i and p_i = R_i's_i, which replace it.
__global__ void k_riccati_finish(Group g, int per_task) {
  for_stages(g, [&](const int s) {
    const StageInfo S = g.st[s];
    const ProbInfo &P = g.prob[S.prob];
    if (skipped_by_mask(g, S.prob)) return;
    if (S.i >= P.N) return;
    if (g.fp64 != nullptr && g.fp64[P.id] == 0) return;  // k_riccati_down_f32 stored this problem's factors
    const int n = g.n, m = g.m, tid = team_rank();
    double *ws = stage_ws(g, s);
    const int *wi = stage_wi(g, s);
    const int nx = wi[SI_NBAR], mu = wi[SI_MBAR], n1 = stage_wi(g, s + 1)[SI_NBAR];
    const int ldr = n + m + 1;
    double *sm = team_smem(per_task);
    double *R = sm, *V = R + m * ldr, *Kt = V + n * (n + 1);
    const double *Rv = ws + g.ws.Rv, *Ab = ws + g.ws.Ab, *Bb = ws + g.ws.Bb;
    for (int idx = tid; idx < mu * (nx + mu + 1); idx += TEAM) {
      int r = idx / (nx + mu + 1), j = idx - r * (nx + mu + 1);
      R[r * ldr + j] = Rv[r * ldr + j];
    }
    for (int idx = tid; idx < nx * (nx + 1); idx += TEAM) {
      int r = idx / (nx + 1), c = idx - r * (nx + 1);
      V[r * (n + 1) + c] = ws[g.ws.P + r * (n + 1) + c];
    }
    tsync();
    // K, k:  R_vv [K | k] = -[R_vz | o_v]
    for (int c = tid; c <= nx; c += TEAM) {
      for (int r = mu - 1; r >= 0; r--) {
        double s0 = -R[r * ldr + mu + c];
        for (int l = r + 1; l < mu; l++) s0 = fma(-R[r * ldr + l], Kt[l * (n + 1) + c], s0);
        Kt[r * (n + 1) + c] = s0 / R[r * ldr + r];
      }
    }
    for (int idx = tid; idx < nx * (nx + 1); idx += TEAM) {
      int r = idx / (nx + 1), c = idx - r * (nx + 1);
      double s0 = 0.0;
      for (int l = 0; l <= r && l < nx; l++) s0 = fma(V[l * (n + 1) + r], V[l * (n + 1) + c], s0);
      if (c < nx) ws[g.ws.P + r * n + c] = s0; else ws[g.ws.p + r] = s0;
    }
    for (int idx = tid; idx < mu * mu; idx += TEAM) {
      int r = idx / mu, j = idx - r * mu;
      double sg = R[j * ldr + j] >= 0.0 ? 1.0 : -1.0;
      ws[g.ws.Lh + r * m + j] = (j <= r) ? sg * R[j * ldr + r] : 0.0;
    }
    tsync();
    for (int idx = tid; idx < mu * (nx + 1); idx += TEAM) {
      int r = idx / (nx + 1), c = idx - r * (nx + 1);
      if (c < nx) ws[g.ws.K + r * n + c] = Kt[r * (n + 1) + c]; else ws[g.ws.k + r] = Kt[r * (n + 1) + c];
    }
    for (int idx = tid; idx < n1 * nx; idx += TEAM) {
      int r = idx / nx, c = idx - r * nx;
      double s0 = Ab[r * n + c];
      for (int l = 0; l < mu; l++) s0 = fma(Bb[r * m + l], Kt[l * (n + 1) + c], s0);
      ws[g.ws.Phi + r * n + c] = s0;
    }
  });
}

// ----------------------------------------------------------- affine chain scans
// Per-stage maps by mode (d_i = dimension of the chained vector at stage i):
//   AFF_ROLL  forward  z_{i+1} = Phi_i z_i + Bbar k_i + cbar_i        -> z
//   AFF_CROLL forward  dz_{i+1} = Phi_i dz_i + Bbar k'_i + rc_i       -> dz (k' held in dv)
//   AFF_PLIN  backward p'_i = Phi_i' p'_{i+1} + rq_i + K_i' rr_i + Phi_i' P_{i+1} rc_i, the
//             refinement's linear pass for the offsets (rq, rr, rc)                  -> pp
//   AFF_NU    forward  nu_{i+1} = Pnu_i nu_i + pnu_i                  -> nu
enum { AFF_ROLL = 0, AFF_CROLL = 1, AFF_PLIN = 2, AFF_NU = 3 };

__device__ __forceinline__ int aff_dim(const Group &g, int s, int mode) {
  return (mode == AFF_NU) ? stage_wi(g, s)[SI_UR] : stage_wi(g, s)[SI_NBAR];
}
__device__ __forceinline__ bool aff_forward(int mode) { return mode != AFF_PLIN; }
__device__ __forceinline__ int aff_out(const Group &g, int mode) {
  return mode == AFF_ROLL ? g.ws.z : mode == AFF_CROLL ? g.ws.dz : mode == AFF_PLIN ? g.ws.pp : g.ws.nu;
}

// map of stage i: y_out = G y_in + gv.  Forward: in = stage i, out = stage i+1;
// backward: in = stage i+1, out = stage i.  G (dout x din, ld n) and gv into smem.
__device__ void aff_stage_map(const Group &g, int s, int mode, double *G, double *gv, double *tmp) {
  const int n = g.n, m = g.m, tid = team_rank();
  const double *ws = stage_ws(g, s), *wn = stage_ws(g, s + 1);
  const int *wi = stage_wi(g, s);
  if (mode == AFF_NU) {
    const int din = wi[SI_UR], dout = stage_wi(g, s + 1)[SI_UR];
    for (int idx = tid; idx < dout * din; idx += TEAM) {
      int i = idx / din, j = idx - i * din;
      G[i * n + j] = ws[g.ws.Pnu + i * n + j];
    }
    for (int i = tid; i < dout; i += TEAM) gv[i] = ws[g.ws.pnu + i];
    tsync();
    return;
  }
  const int nx = wi[SI_NBAR], ny = stage_wi(g, s + 1)[SI_NBAR], mu = wi[SI_MBAR];
  const double *Phi = ws + g.ws.Phi, *Bb = ws + g.ws.Bb;
  if (mode == AFF_ROLL || mode == AFF_CROLL) {
    const double *kk = ws + (mode == AFF_ROLL ? g.ws.k : g.ws.dv);
    const double *cc = ws + (mode == AFF_ROLL ? g.ws.cb : g.ws.rc);
    for (int idx = tid; idx < ny * nx; idx += TEAM) {
      int i = idx / nx, j = idx - i * nx;
      G[i * n + j] = Phi[i * n + j];
    }
    for (int i = tid; i < ny; i += TEAM) {
      double s0 = cc[i];
      for (int l = 0; l < mu; l++) s0 = fma(Bb[i * m + l], kk[l], s0);
      gv[i] = s0;
    }
    tsync();
    return;
  }
  // AFF_PLIN: G = Phi' (nx x ny), gv = rq + K' rr + Phi' (P_{i+1} rc)
  const double *K = ws + g.ws.K, *Pn = wn + g.ws.P, *rc = ws + g.ws.rc;
  for (int b = tid; b < ny; b += TEAM) {
    double s0 = 0.0;
    for (int l = 0; l < ny; l++) s0 = fma(Pn[b * n + l], rc[l], s0);
    tmp[b] = s0;
  }
  for (int idx = tid; idx < nx * ny; idx += TEAM) {
    int i = idx / ny, j = idx - i * ny;
    G[i * n + j] = Phi[j * n + i];
  }
  tsync();
  for (int i = tid; i < nx; i += TEAM) {
    double s0 = ws[g.ws.rq + i];
    for (int l = 0; l < mu; l++) s0 = fma(K[l * n + i], ws[g.ws.rr + l], s0);
    for (int b = 0; b < ny; b++) s0 = fma(Phi[b * n + i], tmp[b], s0);
    gv[i] = s0;
  }
  tsync();
}

// The offsets of every stage's map, stage-parallel, before a chain sweeps
// them (ws.gv; the same arithmetic as aff_stage_map): ROLL cbar + Bbar k,
// CROLL rc + Bbar k', PLIN rq + K' rr + Phi' P_{i+1} rc.  NU reads pnu.
__global__ void k_aff_prep(Group g, int mode, int per_task) {
  for_stages(g, [&](const int s) {
    const StageInfo S = g.st[s];
    const ProbInfo &P = g.prob[S.prob];
    if (skipped_by_mask(g, S.prob)) return;
    if (S.i >= P.N || mode == AFF_NU) return;
    const int n = g.n, m = g.m, tid = team_rank();
    double *ws = stage_ws(g, s);
    const double *wn = stage_ws(g, s + 1);
    const int *wi = stage_wi(g, s);
    const int nx = wi[SI_NBAR], ny = stage_wi(g, s + 1)[SI_NBAR], mu = wi[SI_MBAR];
    const double *Phi = ws + g.ws.Phi, *Bb = ws + g.ws.Bb;
    double *gv = ws + g.ws.gv;
    if (mode == AFF_ROLL || mode == AFF_CROLL) {
      const double *kk = ws + (mode == AFF_ROLL ? g.ws.k : g.ws.dv);
      const double *cc = ws + (mode == AFF_ROLL ? g.ws.cb : g.ws.rc);
      for (int i = tid; i < ny; i += TEAM) {
        double s0 = cc[i];
        for (int l = 0; l < mu; l++) s0 = fma(Bb[i * m + l], kk[l], s0);
        gv[i] = s0;
      }
      return;
    }
    double *tmp = team_smem(per_task);  // P_{i+1} rc (ny)
    const double *K = ws + g.ws.K, *Pn = wn + g.ws.P, *rc = ws + g.ws.rc;
    for (int b = tid; b < ny; b += TEAM) {
      double s0 = 0.0;
      for (int l = 0; l < ny; l++) s0 = fma(Pn[b * n + l], rc[l], s0);
      tmp[b] = s0;
    }
    tsync();
    for (int i = tid; i < nx; i += TEAM) {
      double s0 = ws[g.ws.rq + i];
      for (int l = 0; l < mu; l++) s0 = fma(K[l * n + i], ws[g.ws.rr + l], s0);
      for (int b = 0; b < ny; b++) s0 = fma(Phi[b * n + i], tmp[b], s0);
      gv[i] = s0;
    }
  });
}

// chunk aggregates; also the boundary value slot (forward: slot 0 of the
// problem holds y_0, backward: slot nch holds y_N).
__global__ void k_aff_up(Group g, int mode, int per_task) {
  const int t = team_task();
  if (t >= g.nslot) return;
  const ChunkInfo ci = g.chunk[t];
  const ProbInfo &P = g.prob[ci.prob];
  if (skipped_by_mask(g, ci.prob)) return;
  const int n = g.n, tid = team_rank();
  const bool fwd = aff_forward(mode);
  double *cs0 = g.CS[0];
  if (ci.c == P.nch) {
    // boundary value
    const int s = fwd ? P.st0 : P.st0 + P.N;
    const int slot = fwd ? P.ch0 : P.ch0 + P.nch;
    const int dim = aff_dim(g, s, mode);
    double *gv = cs0 + (size_t)slot * g.cs_stride + n * n;
    const double *src = stage_ws(g, s);
    for (int i = tid; i < dim; i += TEAM) {
      double v;
      if (mode == AFF_ROLL) v = src[g.ws.z + i];
      else if (mode == AFF_CROLL) v = 0.0;
      else if (mode == AFF_PLIN) v = src[g.ws.rq + i];  // p'_N = rq_N
      else v = src[g.ws.nu + i];
      gv[i] = v;
    }
    if (tid == 0) {
      int *cm = g.CI[0] + (size_t)slot * CI_STRIDE;
      cm[CI_ROWS] = 1; cm[CI_NA] = dim; cm[CI_NB] = 0;
    }
    return;
  }
  const int slot = fwd ? P.ch0 + ci.c + 1 : P.ch0 + ci.c;
  if (P.nch == 1) {
    // one chunk: k_aff_down starts from the boundary value, so the chunk's map is not
    // composed; an empty map (no rows, no dimensions) ends the level at once
    if (tid == 0) {
      int *cm = g.CI[0] + (size_t)slot * CI_STRIDE;
      cm[CI_ROWS] = 0; cm[CI_NA] = 0; cm[CI_NB] = 0;
    }
    return;
  }
  const int a = ci.c * P.L, b = min(a + P.L, P.N);
  double *sm = team_smem(per_task);
  double *Gm = sm, *gm = Gm + n * n, *Gs = gm + n, *gs = Gs + n * n, *Tm = gs + n, *tmp = Tm + n * n;
  const int d0 = fwd ? aff_dim(g, P.st0 + a, mode) : aff_dim(g, P.st0 + b, mode);
  for (int idx = tid; idx < n * n; idx += TEAM) {
    int i = idx / n, j = idx - i * n;
    Gm[idx] = (i == j) ? 1.0 : 0.0;
  }
  for (int i = tid; i < n; i += TEAM) gm[i] = 0.0;
  tsync();
  int dcur = d0;  // rows of the aggregate (current output dimension)
  for (int k = 0; k < b - a; k++) {
    const int i = fwd ? a + k : b - 1 - k;
    const int s = P.st0 + i;
    aff_stage_map(g, s, mode, Gs, gs, tmp);
    const int dout = fwd ? aff_dim(g, s + 1, mode) : aff_dim(g, s, mode);
    // Tm = Gs Gm (dout x d0), tmp = Gs gm + gs
    wgemm<false, false>(dout, d0, dcur, 1.0, Gs, n, Gm, n, 0.0, Tm, n);
    for (int r = tid; r < dout; r += TEAM) {
      double s0 = gs[r];
      for (int l = 0; l < dcur; l++) s0 = fma(Gs[r * n + l], gm[l], s0);
      tmp[r] = s0;
    }
    tsync();
    for (int idx = tid; idx < dout * d0; idx += TEAM) {
      int r = idx / d0, j = idx - r * d0;
      Gm[r * n + j] = Tm[r * n + j];
    }
    for (int r = tid; r < dout; r += TEAM) gm[r] = tmp[r];
    tsync();
    dcur = dout;
  }
  double *cs = cs0 + (size_t)slot * g.cs_stride;
  for (int idx = tid; idx < n * n; idx += TEAM) cs[idx] = Gm[idx];
  for (int i = tid; i < n; i += TEAM) cs[n * n + i] = gm[i];
  if (tid == 0) {
    int *cm = g.CI[0] + (size_t)slot * CI_STRIDE;
    cm[CI_ROWS] = 0; cm[CI_NA] = d0; cm[CI_NB] = dcur;
  }
}

// One level of a radix-4 Kogge-Stone scan over the chunk slots of an affine
// chain.  Before the level with stride d every slot holds the composition of
// the d slots ending at it; it composes that with the slots at distances d,
// 2d and 3d in the scan direction (each holding the d slots before the
// previous one), so after the levels d = 1, 4, 16, ... every slot holds its
// inclusive prefix.  A value (a boundary vector, CI_ROWS == 1) ends the
// composition.  The four-way level halves the launches of a radix-2 scan;
// the chain elements are small (n x n), so the level is launch-bound.
__global__ void k_aff_level(Group g, int src, int d, int fwd, int per_task) {
  const int t = team_task();
  if (t >= g.nslot) return;
  const ChunkInfo ci = g.chunk[t];
  const ProbInfo &P = g.prob[ci.prob];
  if (skipped_by_mask(g, ci.prob)) return;
  const int n = g.n, tid = team_rank(), sz = n * n + n;
  const int j = t - P.ch0;  // slot index 0..nch
  const double *S0 = g.CS[src] + (size_t)t * g.cs_stride;
  const int *I1 = g.CI[src] + (size_t)t * CI_STRIDE;
  double *Dst = g.CS[src ^ 1] + (size_t)t * g.cs_stride;
  int *J = g.CI[src ^ 1] + (size_t)t * CI_STRIDE;
  int rows = I1[CI_ROWS], na = I1[CI_NA], nb = I1[CI_NB];
  double *sm = team_smem(per_task);
  double *acc = sm, *oth = acc + sz, *Tm = oth + sz, *tv = Tm + n * n;
  for (int idx = tid; idx < sz; idx += TEAM) acc[idx] = S0[idx];
  tsync();
  for (int q = 1; q <= 3 && rows != 1; q++) {
    const int j2 = fwd ? j - q * d : j + q * d;
    if (j2 < 0 || j2 > P.nch) break;
    const int t2 = P.ch0 + j2;
    const double *S2 = g.CS[src] + (size_t)t2 * g.cs_stride;
    const int *I2 = g.CI[src] + (size_t)t2 * CI_STRIDE;
    const int rows2 = I2[CI_ROWS], na2 = I2[CI_NA];
    for (int idx = tid; idx < sz; idx += TEAM) oth[idx] = S2[idx];
    tsync();
    if (rows2 == 1) {
      // value: y = G v + g, dimension nb
      for (int r = tid; r < nb; r += TEAM) {
        double s0 = acc[n * n + r];
        for (int l = 0; l < na2; l++) s0 = fma(acc[r * n + l], oth[n * n + l], s0);
        tv[r] = s0;
      }
      tsync();
      for (int r = tid; r < nb; r += TEAM) acc[n * n + r] = tv[r];
      rows = 1;
      na = nb;
      nb = 0;
    } else {
      // (G G2, G g2 + g): input dimension na2, output nb
      wgemm<false, false>(nb, na2, na, 1.0, acc, n, oth, n, 0.0, Tm, n);
      for (int r = tid; r < nb; r += TEAM) {
        double s0 = acc[n * n + r];
        for (int l = 0; l < na; l++) s0 = fma(acc[r * n + l], oth[n * n + l], s0);
        tv[r] = s0;
      }
      tsync();
      for (int idx = tid; idx < nb * na2; idx += TEAM) {
        const int r = idx / na2, c = idx - r * na2;
        acc[r * n + c] = Tm[r * n + c];
      }
      for (int r = tid; r < nb; r += TEAM) acc[n * n + r] = tv[r];
      rows = 0;
      na = na2;
    }
    tsync();
  }
  for (int idx = tid; idx < sz; idx += TEAM) Dst[idx] = acc[idx];
  if (tid == 0) { J[CI_ROWS] = rows; J[CI_NA] = na; J[CI_NB] = nb; }
}

// The chain of one chunk: y_out = G_i y_in + gv_i stage after stage, G_i = Phi_i
// (ROLL, CROLL), Phi_i' (PLIN, backward) or Pnu_i (NU), gv_i from k_aff_prep (pnu
// for NU).  Each output row is a dot product split over seg lanes (seg a power of
// two with seg * n <= the team), so its dependent chain is about n / seg FMAs and
// log2(seg) shuffle additions; the lanes load the next stage's G and gv into
// registers while the current stage runs, and y alternates between two buffers,
// one barrier per stage.
__global__ void k_aff_down(Group g, int mode, int fin, int per_task) {
  const int t = team_task();
  if (t >= g.nslot) return;
  const ChunkInfo ci = g.chunk[t];
  const ProbInfo &P = g.prob[ci.prob];
  if (skipped_by_mask(g, ci.prob)) return;
  if (ci.c >= P.nch) return;
  const int n = g.n, tid = team_rank();
  const bool fwd = aff_forward(mode), tr = mode == AFF_PLIN;
  const int a = ci.c * P.L, b = min(a + P.L, P.N);
  const int off = aff_out(g, mode);
  const int goff = mode == AFF_NU ? g.ws.Pnu : g.ws.Phi, voff = mode == AFF_NU ? g.ws.pnu : g.ws.gv;
  double *sm = team_smem(per_task);
  double *ya = sm, *yb = ya + n;
  int seg = 8;
  while (seg > 1 && seg * n > TEAM) seg >>= 1;
  const int q = tid & (seg - 1), row = tid / seg;  // this lane's row and column offset
  // boundary value after the scan: forward slot (ch0 + c) = y_a; backward slot (ch0 + c + 1) = y_b
  const int slot = fwd ? P.ch0 + ci.c : P.ch0 + ci.c + 1;
  const double *sv = g.CS[fin] + (size_t)slot * g.cs_stride + n * n;
  int dcur = fwd ? aff_dim(g, P.st0 + a, mode) : aff_dim(g, P.st0 + b, mode);
  for (int i = tid; i < n; i += TEAM) ya[i] = (i < dcur) ? sv[i] : 0.0;
  // stage k of the sweep (k = 0 .. b - a - 1): its stage, and its output dimension
  auto stage_of = [&](int k) { return P.st0 + (fwd ? a + k : b - 1 - k); };
  auto dout_of = [&](int s) { return fwd ? aff_dim(g, s + 1, mode) : aff_dim(g, s, mode); };
  // registers: this lane's entries of G (columns q, q + seg, q + 2 seg, q + 3 seg) and gv
  constexpr int KP = 4;
  double gr[KP], gvr = 0.0;
  auto load = [&](int s, int din, int dout, double *gx, double &gvx) {
    const double *G = stage_ws(g, s) + goff;
#pragma unroll
    for (int k = 0; k < KP; k++) {
      const int l = q + k * seg;
      gx[k] = (row < dout && l < din) ? (tr ? G[l * n + row] : G[row * n + l]) : 0.0;
    }
    gvx = (row < dout && q == 0) ? stage_ws(g, s)[voff + row] : 0.0;
  };
  const int steps = b - a;
  if (!fwd && b == P.N) {
    double *o = stage_ws(g, P.st0 + b) + off;
    for (int r = tid; r < n; r += TEAM) o[r] = (r < dcur) ? ya[r] : 0.0;
  }
  int s = steps > 0 ? stage_of(0) : 0;
  int dout = steps > 0 ? dout_of(s) : 0;
  // the output dimension of the next stage, read one stage ahead of its map's entries so
  // that the two global reads do not follow each other on the chain
  int dpre = steps > 1 ? dout_of(stage_of(1)) : 0;
  if (steps > 0) load(s, dcur, dout, gr, gvr);
  tsync();
  for (int k = 0; k < steps; k++) {
    if (fwd) {  // the value of stage s is the chain's input
      double *o = stage_ws(g, s) + off;
      for (int r = tid; r < n; r += TEAM) o[r] = (r < dcur) ? ya[r] : 0.0;
    }
    // next stage's entries, in flight while this stage runs
    double gn[KP], gvn = 0.0;
    int sn = s, dn = 0;
    if (k + 1 < steps) {
      sn = stage_of(k + 1);
      dn = dpre;
      load(sn, dout, dn, gn, gvn);
      if (k + 2 < steps) dpre = dout_of(stage_of(k + 2));
    }
    double acc = 0.0;
#pragma unroll
    for (int kk = 0; kk < KP; kk++) {
      const int l = q + kk * seg;
      if (l < dcur) acc = fma(gr[kk], ya[l], acc);
    }
    if (row < dout) {  // columns beyond the registers (teams too small for seg = 8)
      const double *G = stage_ws(g, s) + goff;
      for (int l = q + KP * seg; l < dcur; l += seg) acc = fma(tr ? G[l * n + row] : G[row * n + l], ya[l], acc);
    }
    for (int o = seg >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
    if (q == 0 && row < dout) yb[row] = gvr + acc;
    tsync();
    double *tmp = ya; ya = yb; yb = tmp;
    if (!fwd) {  // the chain's output is the value of stage s
      double *o = stage_ws(g, s) + off;
      for (int r = tid; r < n; r += TEAM) o[r] = (r < dout) ? ya[r] : 0.0;
    }
    dcur = dout;
    s = sn;
    dout = dn;
#pragma unroll
    for (int kk = 0; kk < KP; kk++) gr[kk] = gn[kk];
    gvr = gvn;
  }
  if (fwd && b == P.N) {
    double *o = stage_ws(g, P.st0 + b) + off;
    for (int r = tid; r < n; r += TEAM) o[r] = (r < dcur) ? ya[r] : 0.0;
  }
}

// ----------------------------------------------------------- stage-parallel helpers of the solve
// z_0 = T_0'(s_0 - t_0) and the check H_0 s_0 + h_0 = 0 (eqs. initial-feasibility, reduced-initial)
__global__ void k_solve_init(Group g, const double *s0) {
  const int t = team_task();
  if (t >= g.nprob) return;
  const ProbInfo &P = g.prob[t];
  if (skipped_by_mask(g, t)) return;
  const int n = g.n, tid = team_rank();
  const int s = P.st0;
  double *ws = stage_ws(g, s);
  const int *wi = stage_wi(g, s);
  const int r = wi[SI_HROWS], ur = wi[SI_UR], nb = n - ur;
  const double *x0 = s0 + P.os0;
  const double *H = ws + g.ws.H, *T = ws + g.ws.UT + ur, *tt = ws + g.ws.t;
  double worst = 0.0, om = 0.0;
  for (int a = tid; a < r; a += TEAM) {
    double v = H[a * (n + 1) + n];
    om = fmax(om, fabs(v));
    for (int l = 0; l < n; l++) v = fma(H[a * (n + 1) + l], x0[l], v);
    worst = fmax(worst, fabs(v));
  }
  bool bad = false;
  for (int l = tid; l < n; l += TEAM) {
    om = fmax(om, fabs(x0[l]));
    bad = bad || !isfinite(x0[l]);
  }
  if (__syncthreads_or(bad)) {
    if (tid == 0) set_status(g, t, ST_NONFINITE);
  }
  worst = team_max(worst);
  om = fmax(1.0, team_max(om));
  if (tid == 0 && worst > g.tau_inc * om) set_status(g, t, ST_INFEASIBLE_X0);
  for (int a = tid; a < n; a += TEAM) {
    double v = 0.0;
    if (a < nb)
      for (int l = 0; l < n; l++) v = fma(T[l * n + a], x0[l] - tt[l], v);
    ws[g.ws.z + a] = v;
  }
}

// pass 0: v_i = K z + k, pi_i = P z + p.  correction passes: dv = K dz + k', dpi = P dz + p',
// then z += dz, v += dv, pi += dpi.
__global__ void k_post_roll(Group g, int corr) {
  for_stages(g, [&](const int s) {
    const StageInfo S = g.st[s];
    const ProbInfo &P = g.prob[S.prob];
    if (skipped_by_mask(g, S.prob)) return;
    const int n = g.n, m = g.m, tid = team_rank();
    double *ws = stage_ws(g, s);
    const int *wi = stage_wi(g, s);
    const int nx = wi[SI_NBAR], mu = (S.i < P.N) ? wi[SI_MBAR] : 0;
    const double *zz = ws + (corr ? g.ws.dz : g.ws.z);
    const double *kk = ws + (corr ? g.ws.dv : g.ws.k);
    const double *pp = ws + (corr ? g.ws.pp : g.ws.p);
    // v (or dv) -- computed into registers of the lanes then written
    double myv = 0.0, mypi = 0.0;
    const int r = tid;
    if (r < mu) {
      myv = kk[r];
      for (int l = 0; l < nx; l++) myv = fma(ws[g.ws.K + r * n + l], zz[l], myv);
    }
    if (r < nx) {
      mypi = pp[r];
      for (int l = 0; l < nx; l++) mypi = fma(ws[g.ws.P + r * n + l], zz[l], mypi);
    }
    tsync();
    if (!corr) {
      if (r < m) ws[g.ws.v + r] = (r < mu) ? myv : 0.0;
      if (r < n) ws[g.ws.pi + r] = (r < nx) ? mypi : 0.0;
    } else {
      if (r < mu) ws[g.ws.v + r] += myv;
      if (r < nx) { ws[g.ws.pi + r] += mypi; ws[g.ws.z + r] += zz[r]; }
    }
  });
}

// Residual of the reduced KKT system, evaluated through the original data.
// Under x_i = T z + t, u_i = Y z + Z v + y (Thm 5 substitution), with
// a = g^x + A'T_{i+1}pi_{i+1} and b = g^u + B'T_{i+1}pi_{i+1} at that point,
// the z-rows are T'a + Y'b - pi, the v-rows Z'b, and the costate rows
// cbar + Abar z + Bbar v - z_{i+1}.  Forming Qbar z + qbar instead would sum
// terms of size |Y|^2 that cancel down to pi: where the mixed rows leave D_i
// ill-conditioned |Y| is large, and that cancellation would set the accuracy
// of the costates and so of the multipliers.  Per task: 3n + 2m doubles.
__global__ void k_resid(Group g, int per_task) {
  for_stages(g, [&](const int s) {
    const StageInfo S = g.st[s];
    const ProbInfo &P = g.prob[S.prob];
    if (skipped_by_mask(g, S.prob)) return;
    const int n = g.n, m = g.m, tid = team_rank(), i = S.i;
    double *ws = stage_ws(g, s);
    const int *wi = stage_wi(g, s);
    const bool last = i == P.N;
    const double *wn = last ? ws : stage_ws(g, s + 1);
    const int nx = wi[SI_NBAR], mu = last ? 0 : wi[SI_MBAR], ny = last ? 0 : stage_wi(g, s + 1)[SI_NBAR];
    const int ur = wi[SI_UR], ur1 = last ? 0 : stage_wi(g, s + 1)[SI_UR];
    const double *z = ws + g.ws.z, *v = ws + g.ws.v, *pi = ws + g.ws.pi, *pin = wn + g.ws.pi, *zn = wn + g.ws.z;
    const double *T = ws + g.ws.UT + ur, *Tn = wn + g.ws.UT + ur1;
    const double *Y = ws + g.ws.Y, *Z = ws + g.ws.Z, *Ab = ws + g.ws.Ab, *Bb = ws + g.ws.Bb;
    double *sm = team_smem(per_task);
    double *xs = sm, *us = xs + n, *lh = us + m, *ga = lh + n, *gb = ga + n;
    // T_i = I, t_i = 0 (te) or T_{i+1} = I (tne): the products with them are their other factor
    const bool te = wi[SI_TEYE] != 0, tne = !last && stage_wi(g, s + 1)[SI_TEYE] != 0;
    for (int a = tid; a < n; a += TEAM) {
      double s0 = ws[g.ws.t + a];
      if (te) s0 = z[a];
      else
        for (int j = 0; j < nx; j++) s0 = fma(T[a * n + j], z[j], s0);
      xs[a] = s0;
    }
    if (!last) {
      for (int a = tid; a < m; a += TEAM) {
        double s0 = ws[g.ws.y + a];
        for (int j = 0; j < nx; j++) s0 = fma(Y[a * n + j], z[j], s0);
        for (int j = 0; j < mu; j++) s0 = fma(Z[a * m + j], v[j], s0);
        us[a] = s0;
      }
      for (int l = tid; l < n; l += TEAM) {
        double s0 = 0.0;
        if (tne) s0 = pin[l];
        else
          for (int j = 0; j < ny; j++) s0 = fma(Tn[l * n + j], pin[j], s0);
        lh[l] = s0;                                               // T_{i+1} pi_{i+1}
      }
    }
    tsync();
    const double *Q = g.Q + P.oQ + (size_t)i * n * n, *q = g.qv + P.oqv + (size_t)i * n;
    const double *A = g.A + P.oA + (size_t)i * n * n, *B = g.B + P.oB + (size_t)i * n * m;
    const double *Mm = g.M + P.oM + (size_t)i * n * m, *R = g.R + P.oR + (size_t)i * m * m;
    const double *rv = g.rv + P.orv + (size_t)i * m;
    for (int a = tid; a < n; a += TEAM) {
      double s0 = q[a];
      for (int j = 0; j < n; j++) s0 = fma(Q[a * n + j], xs[j], s0);
      if (!last) {
        for (int j = 0; j < m; j++) s0 = fma(Mm[a * m + j], us[j], s0);
        for (int l = 0; l < n; l++) s0 = fma(A[l * n + a], lh[l], s0);
      }
      ga[a] = s0;
    }
    if (!last)
      for (int a = tid; a < m; a += TEAM) {
        double s0 = rv[a];
        for (int j = 0; j < n; j++) s0 = fma(Mm[j * m + a], xs[j], s0);
        for (int j = 0; j < m; j++) s0 = fma(R[a * m + j], us[j], s0);
        for (int l = 0; l < n; l++) s0 = fma(B[l * m + a], lh[l], s0);
        gb[a] = s0;
      }
    tsync();
    for (int r = tid; r < nx; r += TEAM) {
      double s0 = -pi[r];
      if (te) s0 = ga[r] - pi[r];
      else
        for (int l = 0; l < n; l++) s0 = fma(T[l * n + r], ga[l], s0);
      if (!last)
        for (int l = 0; l < m; l++) s0 = fma(Y[l * n + r], gb[l], s0);
      ws[g.ws.rq + r] = s0;
    }
    for (int r = tid; r < mu; r += TEAM) {
      double s0 = 0.0;
      for (int l = 0; l < m; l++) s0 = fma(Z[l * m + r], gb[l], s0);
      ws[g.ws.rr + r] = s0;
    }
    for (int r = tid; r < ny; r += TEAM) {
      double s0 = ws[g.ws.cb + r] - zn[r];
      for (int l = 0; l < nx; l++) s0 = fma(Ab[r * n + l], z[l], s0);
      for (int l = 0; l < mu; l++) s0 = fma(Bb[r * m + l], v[l], s0);
      ws[g.ws.rc + r] = s0;
    }
  });
}

// Correction controls of a refinement pass: with w = P_{i+1} rc_i + p'_{i+1},
// k'_i = -H_uu^{-1} (rr_i + Bbar' w) through the Cholesky factor of H_uu (-> dv).
__global__ void k_pcorr(Group g, int per_task) {
  for_stages(g, [&](const int s) {
    const StageInfo S = g.st[s];
    const ProbInfo &P = g.prob[S.prob];
    if (skipped_by_mask(g, S.prob)) return;
    if (S.i >= P.N) return;
    const int n = g.n, m = g.m, tid = team_rank();
    double *ws = stage_ws(g, s);
    const double *wn = stage_ws(g, s + 1);
    const int mu = stage_wi(g, s)[SI_MBAR], ny = stage_wi(g, s + 1)[SI_NBAR];
    double *sm = team_smem(per_task);
    double *w = sm, *hu = sm + n, *Ls = hu + m;  // Ls: chol(H_uu), mu x mu (ld m)
    const double *Pn = wn + g.ws.P, *ppn = wn + g.ws.pp, *rc = ws + g.ws.rc, *Bb = ws + g.ws.Bb;
    for (int idx = tid; idx < mu * mu; idx += TEAM) {
      const int a = idx / mu, l = idx - a * mu;
      Ls[a * m + l] = ws[g.ws.Lh + a * m + l];
    }
    for (int b = tid; b < ny; b += TEAM) {
      double s0 = ppn[b];
      for (int l = 0; l < ny; l++) s0 = fma(Pn[b * n + l], rc[l], s0);
      w[b] = s0;
    }
    tsync();
    for (int a = tid; a < mu; a += TEAM) {
      double s0 = ws[g.ws.rr + a];
      for (int b = 0; b < ny; b++) s0 = fma(Bb[b * m + a], w[b], s0);
      hu[a] = s0;
    }
    tsync();
    // dv = -H_uu^{-1} hu with H_uu = L L' (L = Ls, lower): forward then backward
    // substitution by the first warp, lane a holding row a (mu <= 16), column by column
    if (tid < 32) {
      const int a = tid;
      double x = (a < mu) ? hu[a] : 0.0;
      for (int l = 0; l < mu; l++) {
        const double xl = __shfl_sync(kFull, x, l) / Ls[l * m + l];
        if (a == l) x = xl;
        else if (a > l && a < mu) x = fma(-Ls[a * m + l], xl, x);
      }
      for (int l = mu - 1; l >= 0; l--) {
        const double xl = __shfl_sync(kFull, x, l) / Ls[l * m + l];
        if (a == l) x = xl;
        else if (a < l) x = fma(-Ls[l * m + a], xl, x);
      }
      if (a < mu) ws[g.ws.dv + a] = -x;
    }
  });
}

// x_i = T z + t, u_i = Y z + Z v + y (eq. recovery-maps)
__global__ void k_recover(Group g, double *x, double *u) {
  for_stages(g, [&](const int s) {
    const StageInfo S = g.st[s];
    const ProbInfo &P = g.prob[S.prob];
    if (skipped_by_mask(g, S.prob)) return;
    const int n = g.n, m = g.m, tid = team_rank();
    const double *ws = stage_ws(g, s);
    const int *wi = stage_wi(g, s);
    const int ur = wi[SI_UR], nb = n - ur;
    const double *T = ws + g.ws.UT + ur, *z = ws + g.ws.z;
    bool bad = false;
    for (int a = tid; a < n; a += TEAM) {
      double v = ws[g.ws.t + a];
      for (int j = 0; j < nb; j++) v = fma(T[a * n + j], z[j], v);
      x[P.ox + (size_t)S.i * n + a] = v;
      bad = bad || !isfinite(v);
    }
    if (S.i < P.N) {
      const int mb = wi[SI_MBAR];
      const double *Y = ws + g.ws.Y, *Z = ws + g.ws.Z, *vv = ws + g.ws.v;
      for (int a = tid; a < m; a += TEAM) {
        double v = ws[g.ws.y + a];
        for (int j = 0; j < nb; j++) v = fma(Y[a * n + j], z[j], v);
        for (int j = 0; j < mb; j++) v = fma(Z[a * m + j], vv[j], v);
        u[P.ou + (size_t)S.i * m + a] = v;
        bad = bad || !isfinite(v);
      }
    }
    if (__syncthreads_or(bad) && tid == 0) set_status(g, S.prob, ST_NONFINITE);
  });
}

}  // namespace eclqr

namespace eclqr {
// reduced dimensions into batch-ordered arrays: nbar has N_j + 1 entries per
// problem, mbar N_j entries (the prefix of N_j + 1 minus one per earlier problem)
__global__ void k_dims(Group g, int *nbar, int *mbar) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.nstage) return;
  const StageInfo S = g.st[s];
  const ProbInfo &P = g.prob[S.prob];
  if (skipped_by_mask(g, S.prob)) return;
  const int *wi = stage_wi(g, s);
  nbar[P.ost + S.i] = wi[SI_NBAR];
  if (S.i < P.N) mbar[P.ost - P.id + S.i] = wi[SI_MBAR];
}
}  // namespace eclqr
