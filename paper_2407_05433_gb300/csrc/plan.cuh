// plan.cuh -- batch plan shared by the kernels and the host orchestration.
//
// A batch is split into groups of problems with equal (n, m).  Inside a
// group every stage owns a fixed-stride workspace slot (doubles) and a few
// ints; every problem owns nch + 1 chunk slots (nch scan chunks plus the
// terminal element), double-buffered for the log-depth chunk scans.
#pragma once
#include <stdint.h>
#include "la.cuh"

namespace eclqr {

struct ProbInfo {
  int N;        // horizon
  int L;        // stages per chunk
  int nch;      // number of chunks, ceil(N / L)
  int ch0;      // first chunk slot of this problem (nch + 1 slots)
  int st0;      // first stage slot (N + 1 slots: stages 0..N)
  int id;       // index in the batch (status, residual)
  long long oA, oB, oc, oC, oD, od, oE, oe, oQ, oM, oR, oqv, orv;  // element offsets of the problem's data
  long long os0, ox, ou, olam, omu, oeta, oalpha;                // element offsets of s0 and outputs
  long long ost;  // sum over earlier problems of (N + 1): batch stage offset
  int skip_ok;    // no state-only or terminal rows, p_i <= m, shortcut enabled: the scan may be skipped
};

struct StageInfo {
  int prob;     // problem index inside the group
  int i;        // stage index 0..N
  int p, q;     // mixed / state-only rows
  int prow, qrow;  // first row of this stage in the problem's C/D/d and E/e blocks
};

struct ChunkInfo {
  int prob;     // problem index inside the group
  int c;        // chunk index 0..nch (nch = terminal element)
};

// ---- per-stage workspace layout (offsets in doubles) ----
struct WsLayout {
  int H, UT, t, Y, Z, y, Ab, Bb, cb, Qb, Mb, Rb, qb, rb;
  int P, p, K, k, Lh, Phi;
  int z, v, pi, dz, dv, dpi, rq, rr, rc, pp;
  int nu, NH, Pnu, pnu, UA, BU, UC, Ux, ru;
  int LT, lt;   // Cholesky factor L' of the reduced stage Hessian in the order (v, z), upper
                // triangular (L L' = [Rbar Mbar'; Mbar Qbar]), and L^{-1} [rbar; qbar]
  int Rv;       // the Riccati QR's rows of the minimiser, (R_vv | R_vz | o_v), ld n + m + 1
  int gv;       // offset of the affine chain's stage map (k_aff_prep), n
  int Hpre;     // the stage's own rows projected onto x_i (k_primal_stage), n x (n + 1)
  int stride;
};

__host__ __device__ inline WsLayout make_ws_layout(int n, int m, int pmax, int qmax) {
  WsLayout L;
  int o = 0;
  auto take = [&](int sz) { int r = o; o += sz; return r; };
  L.H = take(n * (n + 1));
  L.UT = take(n * n);
  L.t = take(n);
  L.Y = take(m * n);
  L.Z = take(m * m);
  L.y = take(m);
  L.Ab = take(n * n);
  L.Bb = take(n * m);
  L.cb = take(n);
  L.Qb = take(n * n);
  L.Mb = take(n * m);
  L.Rb = take(m * m);
  L.qb = take(n);
  L.rb = take(m);
  L.P = take(n * n);
  L.p = take(n);
  L.K = take(m * n);
  L.k = take(m);
  L.Lh = take(m * m);
  L.Phi = take(n * n);
  L.z = take(n);
  L.v = take(m);
  L.pi = take(n);
  L.dz = take(n);
  L.dv = take(m);
  L.dpi = take(n);
  L.rq = take(n);
  L.rr = take(m);
  L.rc = take(n);
  L.pp = take(n);
  L.nu = take(n);
  L.NH = take(n * (n + 1));
  L.Pnu = take(n * n);
  L.pnu = take(n);
  L.UA = take(n * n);
  L.BU = take(m * n);
  L.UC = take(n * (pmax + qmax + 1));
  L.Ux = take(n);
  L.ru = take(m);
  L.LT = take((n + m) * (n + m));
  L.lt = take(n + m);
  L.Rv = take(m * (n + m + 1));
  L.gv = take(n);
  L.Hpre = take(n * (n + 1));
  L.stride = (o + 3) & ~3;
  return L;
}

// per-stage ints
// SI_TEYE: 1 when T_i is the identity and t_i = 0, bit for bit (X_i = R^n);
// SI_PRE, SI_PREINC: rows and inconsistency of the stage's own rows projected onto x_i
enum { SI_HROWS = 0, SI_UR = 1, SI_NBAR = 2, SI_MBAR = 3, SI_NUROWS = 4, SI_TEYE = 5, SI_PRE = 6, SI_PREINC = 7,
       SI_STRIDE = 8 };
// per-chunk-slot ints: rows, left dim, right dim (0 = unary/value)
enum { CI_ROWS = 0, CI_NA = 1, CI_NB = 2, CI_ROWS2 = 3, CI_STRIDE = 4 };

struct Group {
  int n, m, pmax, qmax;
  int wmax;  // the most rows of one stage: p_i + q_i for i < N, q_N at N
  int nprob, nstage, nslot;
  const ProbInfo *prob;
  const StageInfo *st;
  const ChunkInfo *chunk;
  // problem data (device, batch-global packed arrays)
  const double *A, *B, *c, *C, *D, *d, *E, *e, *Q, *M, *R, *qv, *rv;
  // workspace
  WsLayout ws;
  double *W;      // nstage * ws.stride
  int *WI;        // nstage * SI_STRIDE
  double *CS[2];  // nslot * cs_stride
  int *CI[2];     // nslot * CI_STRIDE
  int cs_stride;
  double *CR;     // nslot * cr_stride: per-slot scan results kept across kernels
  int cr_stride;
  int *status;    // batch-global, indexed by ProbInfo::id
  int *need_scan; // per problem: 1 once a stage leaves rows on x_i (set by k_scan_check)
  const int *active;  // batch-global, indexed by ProbInfo::id; when set, every kernel skips
                      // the tasks of problems whose entry is 0 (refinement passes)
  const int *fp64;    // mixed precision: batch-global flags, 1 = this problem's Riccati sweep in
                      // FP64, 0 = in FP32; null = every sweep in FP64
  const int *slist;   // when set, the per-stage kernels run only the stages slist[0 .. *scount)
  const int *scount;  // (a refinement pass's problems), each CTA looping over them
  double tau_rank, tau_inc;
};

// a primal-dual solution (device pointers, batch-packed as in the ABI) and gradient outputs
struct Sol {
  const double *x, *u, *lam, *mu, *eta, *alpha;
};
struct SolMut {
  double *x, *u, *lam, *mu, *eta, *alpha;
};
// the per-problem masks of a refinement pass (batch-global, indexed by ProbInfo::id):
// taking part, with a rebuild on the residual rows, with homogeneous constraints
struct RefineMasks {
  int *active, *full, *cheap;
};
// residual rows of the KKT system, written where a correction problem keeps the
// offsets they replace (any pointer null: rows not written)
struct KktRows {
  double *c, *d, *e, *qv, *rv, *s0;
};
struct GradOut {
  double *A, *B, *c, *C, *D, *d, *E, *e, *Q, *M, *R, *qv, *rv, *s0;
};

__device__ __forceinline__ void set_status(const Group &g, int prob, int code) {
  atomicCAS(g.status + g.prob[prob].id, 0, code);
}

// true when a refinement pass leaves this problem (group-local index) alone
__device__ __forceinline__ bool skipped_by_mask(const Group &g, int prob) {
  return g.active != nullptr && g.active[g.prob[prob].id] == 0;
}

__device__ __forceinline__ bool all_finite(const double *a, int k) {
  bool ok = true;
  for (int j = 0; j < k; j++) ok = ok && isfinite(a[j]);
  return ok;
}

// Sec. 6 shortcut: X_i = R^n for every stage of the problem, so its
// feasible-domain scan is skipped and every H_i has no rows.
__device__ __forceinline__ bool scan_skipped(const Group &g, int prob) {
  return g.prob[prob].skip_ok && !g.need_scan[prob];
}

__device__ __forceinline__ double *stage_ws(const Group &g, int s) { return g.W + (size_t)s * g.ws.stride; }
__device__ __forceinline__ int *stage_wi(const Group &g, int s) { return g.WI + (size_t)s * SI_STRIDE; }

// One task per CTA: the task index, and the task's shared-memory window (the
// whole dynamic allocation).
__device__ __forceinline__ int team_task() { return blockIdx.x; }

extern __shared__ double g_smem[];
__device__ __forceinline__ double *team_smem(int /*per_task*/) { return g_smem; }

// Runs body(s) for the stages of a per-stage launch: the CTA's own stage (one CTA per
// stage), or, when the group carries a stage list, the listed stages
// blockIdx.x, blockIdx.x + gridDim.x, ... in turn, with a barrier between them so
// that a stage's shared memory is free before the next one writes it.
template <typename F>
__device__ __forceinline__ void for_stages(const Group &g, F body) {
  if (g.slist == nullptr) {
    const int s = team_task();
    if (s < g.nstage) body(s);
    return;
  }
  const int cnt = *g.scount;
  for (int t = blockIdx.x; t < cnt; t += gridDim.x) {
    body(g.slist[t]);
    __syncthreads();
  }
}

// Runs body(t) for the tasks [0, ntasks) of a launch.  queue null: the CTA's own
// task.  Otherwise the launch is persistent: each CTA takes the next task index
// from the counter *queue (zero before the launch) until none is left, so the
// tasks start in index order -- longest horizon first, as the plan orders the
// problems -- and an SM that finishes early takes more work.
template <typename F>
__device__ __forceinline__ void for_tasks(int ntasks, int *queue, F body) {
  if (queue == nullptr) {
    body(team_task());
    return;
  }
  __shared__ int next;
  for (;;) {
    if (threadIdx.x == 0) next = atomicAdd(queue, 1);
    __syncthreads();
    const int t = next;
    __syncthreads();  // every thread has read next before thread 0 takes the following task
    if (t >= ntasks) return;
    body(t);
  }
}

// status codes (mirror include/eclqr.h)
enum {
  ST_OK = 0, ST_INFEASIBLE_SUFFIX = 1, ST_INFEASIBLE_X0 = 2, ST_RANK_INCONSISTENT = 3,
  ST_NONCONVEX = 4, ST_NONFINITE = 6
};

}  // namespace eclqr
