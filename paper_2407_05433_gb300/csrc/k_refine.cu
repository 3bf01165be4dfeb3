// k_refine.cu -- refinement on the original KKT residual, and the check of the
// problem data for NaN and infinities.
//
// The KKT map F(w) of the problem (Sec. 2 problem, Sec. 7 stationarity and
// sign convention) is affine in w = (x, u, lambda, mu, eta, alpha), and the
// reduction is linear in the offsets (Sec. 5).  So for a point w with
// residual rows r = F(w), the correction dw with F(w + dw) = 0 is the solution
// of the same problem with the same matrices and the offsets replaced by the
// rows of r (k_kkt writes them in that layout).  eclqr_refine runs that solve
// through the same kernels as the first one, masked to the problems whose
// Sec. 9 residual still exceeds the tolerance, and keeps the corrected point
// only where its residual is smaller (Sec. 8 advises checking the original
// residuals).
#include "kernels.cuh"

namespace eclqr {

// Status NONFINITE for every stage whose data hold a NaN or an infinity.
__global__ void k_check_inputs(Group g) {
  const int s = team_task();
  if (s >= g.nstage) return;
  const StageInfo S = g.st[s];
  const ProbInfo &P = g.prob[S.prob];
  if (skipped_by_mask(g, S.prob)) return;
  const int n = g.n, m = g.m, tid = team_rank(), i = S.i;
  bool bad = false;
  auto scan = [&](const double *a, long long k) {
    for (long long j = tid; j < k; j += TEAM) bad = bad || !isfinite(a[j]);
  };
  scan(g.Q + P.oQ + (size_t)i * n * n, (long long)n * n);
  scan(g.qv + P.oqv + (size_t)i * n, n);
  scan(g.E + P.oE + (size_t)S.qrow * n, (long long)S.q * n);
  scan(g.e + P.oe + S.qrow, S.q);
  if (i < P.N) {
    scan(g.A + P.oA + (size_t)i * n * n, (long long)n * n);
    scan(g.B + P.oB + (size_t)i * n * m, (long long)n * m);
    scan(g.c + P.oc + (size_t)i * n, n);
    scan(g.C + P.oC + (size_t)S.prow * n, (long long)S.p * n);
    scan(g.D + P.oD + (size_t)S.prow * m, (long long)S.p * m);
    scan(g.d + P.od + S.prow, S.p);
    scan(g.M + P.oM + (size_t)i * n * m, (long long)n * m);
    scan(g.R + P.oR + (size_t)i * m * m, (long long)m * m);
    scan(g.rv + P.orv + (size_t)i * m, m);
  }
  if (__syncthreads_or(bad) && tid == 0) set_status(g, S.prob, ST_NONFINITE);
}

// Per problem, before a pass: it runs when the previous pass kept its correction
// and halved the residual (or this is the first pass), the status is OK and the
// residual exceeds tol (a NaN residual does not); the pass's status and trial
// residual start at 0.  A problem whose primal parts (initial condition,
// dynamics, equality rows) are within tol takes the correction with homogeneous
// constraints (full[id] = 0), which reuses the build's offset-free factors;
// the others rebuild on the residual rows (full[id] = 1).  *any is set when some
// problem takes part.
__global__ void k_refine_prep(Group g, const int32_t *status, const double *resid, const double *parts,
                              RefineMasks mk, int32_t *cstatus, double *tresid, double *tparts, double tol, int first,
                              int *any) {
  const int t = team_task();
  if (t >= g.nprob || team_rank() != 0) return;
  const int id = g.prob[t].id;
  const bool prev = first ? true : mk.active[id] != 0;
  const bool on = prev && status[id] == ST_OK && resid[id] > tol;
  const double *pp = parts + 4 * (size_t)id;
  const bool full = on && !(pp[0] <= tol && pp[1] <= tol && pp[2] <= tol);
  mk.active[id] = on ? 1 : 0;
  mk.full[id] = full ? 1 : 0;
  mk.cheap[id] = (on && !full) ? 1 : 0;
  cstatus[id] = ST_OK;
  tresid[id] = 0.0;
  for (int k = 0; k < 4; k++) tparts[4 * (size_t)id + k] = 0.0;
  if (on) *any = 1;
}

// Per problem, after k_refine_prep: the stages of the problems in each of the
// pass's masks (active, full, cheap) are appended to that mask's list (lists +
// f * nstage, length counts[f], zero before the launch), so that the pass's
// per-stage kernels visit those stages only.  The order of the stages in a list
// does not matter: every stage's work is independent of the others'.
__global__ void k_stage_lists(Group g, RefineMasks mk, int *lists, int *counts) {
  const int t = team_task();
  if (t >= g.nprob || threadIdx.x >= 32) return;  // one warp per problem
  const ProbInfo &P = g.prob[t];
  const int lane = threadIdx.x, ns = P.N + 1;
  const int *flags[3] = {mk.active, mk.full, mk.cheap};
  for (int f = 0; f < 3; f++) {
    if (!flags[f][P.id]) continue;  // uniform
    int base = 0;
    if (lane == 0) base = atomicAdd(counts + f, ns);
    base = __shfl_sync(kFull, base, 0);
    for (int k = lane; k < ns; k += 32) lists[(size_t)f * g.nstage + base + k] = P.st0 + k;
  }
}

// After the correction solve: a problem whose correction ended with a status
// other than OK keeps its point and stops refining.
__global__ void k_refine_gate(Group g, const int32_t *cstatus, int *active) {
  const int t = team_task();
  if (t >= g.nprob || team_rank() != 0) return;
  const int id = g.prob[t].id;
  if (active[id] && cstatus[id] != ST_OK) active[id] = 0;
}

// The parts of the residual at the trial point replace the point's where the
// trial point is kept (k_refine_post decides with the same comparison).
__global__ void k_refine_parts(Group g, const int *active, double *parts, const double *tparts,
                               const double *resid, const double *tresid) {
  const int t = team_task();
  if (t >= g.nprob || team_rank() != 0) return;
  const int id = g.prob[t].id;
  if (active[id] && tresid[id] < resid[id])
    for (int k = 0; k < 4; k++) parts[4 * (size_t)id + k] = tparts[4 * (size_t)id + k];
}

// t = w + t for one stage's blocks (t holds the correction on entry).
__global__ void k_refine_trial(Group g, Sol w, SolMut t) {
  for_stages(g, [&](const int s) {
    const StageInfo S = g.st[s];
    const ProbInfo &P = g.prob[S.prob];
    if (skipped_by_mask(g, S.prob)) return;
    const int n = g.n, m = g.m, tid = team_rank(), i = S.i;
    for (int a = tid; a < n; a += TEAM) {
      const size_t o = P.ox + (size_t)i * n + a;
      t.x[o] += w.x[o];
      t.lam[o] += w.lam[o];
    }
    if (i < P.N) {
      for (int a = tid; a < m; a += TEAM) t.u[P.ou + (size_t)i * m + a] += w.u[P.ou + (size_t)i * m + a];
      for (int k = tid; k < S.p; k += TEAM) t.mu[P.omu + S.prow + k] += w.mu[P.omu + S.prow + k];
    }
    for (int k = tid; k < S.q; k += TEAM) t.eta[P.oeta + S.qrow + k] += w.eta[P.oeta + S.qrow + k];
    if (i == 0)
      for (int a = tid; a < n; a += TEAM) t.alpha[P.oalpha + a] += w.alpha[P.oalpha + a];
  });
}

// Copies the trial point over the solution where its residual is smaller.
__global__ void k_refine_accept(Group g, Sol t, double *x, double *u, double *lam, double *mu, double *eta,
                                double *alpha, const double *resid, const double *tresid) {
  for_stages(g, [&](const int s) {
    const StageInfo S = g.st[s];
    const ProbInfo &P = g.prob[S.prob];
    if (skipped_by_mask(g, S.prob)) return;
    if (!(tresid[P.id] < resid[P.id])) return;
    const int n = g.n, m = g.m, tid = team_rank(), i = S.i;
    for (int a = tid; a < n; a += TEAM) {
      const size_t o = P.ox + (size_t)i * n + a;
      x[o] = t.x[o];
      lam[o] = t.lam[o];
    }
    if (i < P.N) {
      for (int a = tid; a < m; a += TEAM) u[P.ou + (size_t)i * m + a] = t.u[P.ou + (size_t)i * m + a];
      for (int k = tid; k < S.p; k += TEAM) mu[P.omu + S.prow + k] = t.mu[P.omu + S.prow + k];
    }
    for (int k = tid; k < S.q; k += TEAM) eta[P.oeta + S.qrow + k] = t.eta[P.oeta + S.qrow + k];
    if (i == 0)
      for (int a = tid; a < n; a += TEAM) alpha[P.oalpha + a] = t.alpha[P.oalpha + a];
  });
}

// Per problem, after the accept: the residual of the kept point; the passes go
// on while each one at least halves it (at the problem's rounding floor a pass
// only trades rounding errors).
__global__ void k_refine_post(Group g, double *resid, const double *tresid, int *active) {
  const int t = team_task();
  if (t >= g.nprob || team_rank() != 0) return;
  const int id = g.prob[t].id;
  if (!active[id]) return;
  const double old = resid[id], now = tresid[id];
  if (now < old) resid[id] = now;
  if (!(now < 0.5 * old)) active[id] = 0;
}

// Mixed precision, after the passes: a problem whose status is OK but whose
// residual is still above tol (or NaN) is redone with its Riccati sweep in FP64
// (fp64 flag 1); its residual and parts restart from zero for the new point.
__global__ void k_rescue_prep(Group g, const int32_t *status, double *resid, double *parts, int *fp64, int *active,
                              double tol, int *any) {
  const int t = team_task();
  if (t >= g.nprob || team_rank() != 0) return;
  const int id = g.prob[t].id;
  const bool on = status[id] == ST_OK && fp64[id] == 0 && !(resid[id] <= tol);
  active[id] = on ? 1 : 0;
  if (!on) return;
  fp64[id] = 1;
  resid[id] = 0.0;
  for (int k = 0; k < 4; k++) parts[4 * (size_t)id + k] = 0.0;
  *any = 1;
}

}  // namespace eclqr
