// api.cu -- host orchestration behind the C ABI of include/eclqr.h.
//
// eclqr_create plans the batch (groups of equal (n, m), stage and chunk
// descriptors, workspace layout) and allocates one device block per group.
// The other calls only enqueue kernels on the caller's stream, with no
// allocation; the only host synchronisation is eclqr_refine's check, outside
// a stream capture, whether another refinement pass has work.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "../../include/eclqr.h"
#include "kernels.cuh"

using namespace eclqr;

namespace {

// dynamic shared memory per task: the 227 KB opt-in limit less room for the
// static scratch of the team reductions and the Householder core (< 8 KB)
constexpr int kMaxSmemBytes = 219 * 1024;
constexpr int kTeamWarps = 4;  // default team: one warp per SM sub-partition
constexpr int kManyTasksPerSm = 4;  // a launch with at least this many tasks per SM takes the table's team
constexpr int kPersistCtasPerSm = 8;  // default CTAs per SM of a persistent launch
constexpr int kListCtasPerSm = 32;    // CTAs per SM of a per-stage launch over a stage list

struct GroupHost {
  Group g;
  cudaStream_t s = nullptr;     // the group's own stream when the batch has several groups
  cudaEvent_t done = nullptr;   // records the end of the group's work on s
  int maxnch = 0;
  int levels = 0;
  bool any_skip = false;  // some problem of the group may take the Sec. 6 shortcut
  void *dmem = nullptr;
  int *queue = nullptr;  // device counter of the group's persistent launches (in dmem)
  int *slists = nullptr; // a refinement pass's stage lists (active, full, cheap), 3 x nstage (in dmem)
  int *scounts = nullptr;  // their lengths (3)
  std::vector<int> ids;  // batch indices of the problems in this group
};

int ilog2ceil(int x) {
  int k = 0;
  while ((1 << k) < x) k++;
  return k;
}

}  // namespace

struct eclqr_handle {
  int P = 0;
  eclqr_options opt;
  eclqr_layout_info lay;
  std::vector<GroupHost> groups;
  long long launches = 0;
  bool built = false, solved = false;
  int device = 0;
  // optional event bracket around one kernel (measurement hook)
  const void *timed = nullptr;
  std::vector<cudaEvent_t> ev;
  int nev = 0;
  cudaEvent_t fork = nullptr;   // the caller's stream position the group streams start from
  // refinement on the original KKT residual (eclqr_refine): correction offsets, trial
  // point, per-problem pass status, trial residual and mask, in one allocation
  void *rmem = nullptr;
  KktRows rows{};
  SolMut trial{};
  int32_t *cstatus = nullptr;
  double *tresid = nullptr;
  RefineMasks mk{};
  double *parts = nullptr, *tparts = nullptr;  // residual parts of the point and of the trial point
  double *zeros = nullptr;  // offsets of the corrections with homogeneous constraints
  int *any = nullptr;       // device: some problem takes part in the pass
  int *fp64 = nullptr;      // mixed precision: per-problem flags of the Riccati sweep's precision
  int *any_host = nullptr;  // pinned host copy of it
  bool stale = false;  // the offset-dependent factors are a correction's (after eclqr_refine)
  int sms = 152;       // SMs of the handle's device
};

namespace {

// Team size of one launch of a kernel on a group with state dimension n.
// opt.team_warps != 0 fixes it for every kernel.  Otherwise a launch with fewer
// tasks than SMs takes four warps, one per SM sub-partition, so that one task
// spreads over the SM; one with at least kManyTasksPerSm tasks per SM takes the
// kernel's entry below, and one in between the entry but at least two warps.  There the SM is filled by many tasks at once, and an FP64 warp
// instruction costs its sub-partition the same time whatever its active lanes,
// so the sequential per-problem sweeps and the small per-stage kernels run
// fastest as one warp per task: one warp forms each reflector's scalars, each
// reduction and each triangular solve once, where four warps would each repeat
// them, and needs no CTA barrier.  The entries are the fastest team measured per
// kernel and state dimension on the 4096-problem uneven batch (each (n, m) group
// alone, about seven problems per SM).  For example the Riccati sweep takes 247
// ms over the four groups with one warp per problem against 320 ms with four
// (at n = 24, 86 ms with two warps against 93 with one); the affine chains take
// 4 ms with two warps at n = 8 against 7 with eight, but 7 ms with eight at
// n = 24 against 11 with two; the chunk up-sweeps of the long horizon (65536
// stages in 1024 chunks) take 27 ms with two warps per chunk against 37 with one;
// the stage elimination takes 14 ms with one warp at n = 8 against 29 ms with
// four, but 86 ms with four at n = 24 against 120 ms with one, where its stage
// matrices fill four warps.
int team_for(const eclqr_handle *h, const void *kern, int ntasks, int n) {
  if (h->opt.team_warps != 0) return h->opt.team_warps;
  if (ntasks < h->sms) return kTeamWarps;
  // warps below n_from, and from n_from up
  static const struct { const void *fn; int warps, n_from, warps_from; } table[] = {
      {(const void *)k_riccati_down, 1, 24, 2},  {(const void *)k_riccati_down_f32, 1, 0, 1},
      {(const void *)k_riccati_finish, 1, 0, 1}, {(const void *)k_elim, 1, 16, 4},
      {(const void *)k_primal_down, 1, 24, 2},   {(const void *)k_dual_down, 1, 0, 1},
      {(const void *)k_primal_stage, 1, 24, 2},
      {(const void *)k_aff_down, 2, 24, 8},      {(const void *)k_dual_leaf, 1, 0, 1},
      {(const void *)k_aff_prep, 1, 0, 1},       {(const void *)k_stage_lists, 1, 0, 1},
      {(const void *)k_dual_stage, 2, 0, 2},     {(const void *)k_param, 1, 0, 1},
      {(const void *)k_resid, 1, 0, 1},          {(const void *)k_pcorr, 1, 0, 1},
      {(const void *)k_kkt, 1, 0, 1},            {(const void *)k_post_roll, 1, 0, 1},
      {(const void *)k_recover, 1, 0, 1},        {(const void *)k_check_inputs, 1, 0, 1},
      {(const void *)k_refine_trial, 1, 0, 1},   {(const void *)k_refine_accept, 1, 0, 1},
      {(const void *)k_refine_prep, 1, 0, 1},    {(const void *)k_refine_gate, 1, 0, 1},
      {(const void *)k_refine_parts, 1, 0, 1},   {(const void *)k_refine_post, 1, 0, 1},
      {(const void *)k_rescue_prep, 1, 0, 1},    {(const void *)k_scan_check, 1, 0, 1},
      {(const void *)k_terminal, 1, 0, 1},       {(const void *)k_dual_terminal, 1, 0, 1},
      {(const void *)k_lqr_up, 2, 0, 2},         {(const void *)k_primal_up, 1, 0, 1},
      {(const void *)k_dual_up, 2, 0, 2}};
  const bool many = ntasks >= kManyTasksPerSm * h->sms;
  for (const auto &e : table)
    if (e.fn == kern) {
      const int w = n >= e.n_from ? e.warps_from : e.warps;
      // one to four tasks per SM: a one-warp entry takes two warps (256 problems of 256
      // stages, n = 16: 37 ms with two, 42 with one, 49 with four)
      return many ? w : std::max(w, 2);
    }
  return kTeamWarps;
}

// the state dimension of the group a launch works on (every kernel's first argument)
inline int group_n(const Group &g) { return g.n; }
template <typename A0, typename... Rest>
int group_n(const A0 &a0, const Rest &...) {
  return group_n(a0);
}

// grid CTAs (teams of team_for warps, chosen for ntasks tasks), with per_task
// doubles of dynamic shared memory
template <typename... KArgs, typename... Args>
int launch_grid(eclqr_handle *h, void (*kern)(KArgs...), int ntasks, int grid, int per_task, cudaStream_t st,
                Args... args) {
  if (ntasks <= 0) return ECLQR_OK;
  const size_t smem = (size_t)per_task * sizeof(double);
  if (smem > (size_t)kMaxSmemBytes) return ECLQR_EINVAL;
  // without the opt-in, dynamic plus static shared memory is capped at 48 KB;
  // the kernels' static scratch stays below 16 KB
  if (smem > 32 * 1024) {
    if (cudaFuncSetAttribute((const void *)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return ECLQR_ECUDA;
  }
  const bool timed = h->timed == (const void *)kern && h->nev + 2 <= (int)h->ev.size();
  if (timed) cudaEventRecord(h->ev[h->nev], st);
  kern<<<grid, 32 * team_for(h, (const void *)kern, ntasks, group_n(args...)), smem, st>>>(args...);
  if (timed) {
    cudaEventRecord(h->ev[h->nev + 1], st);
    h->nev += 2;
  }
  h->launches++;
  return cudaPeekAtLastError() == cudaSuccess ? ECLQR_OK : ECLQR_ECUDA;
}

// the per-stage kernels written with for_stages, which can run over a stage list
bool stage_list_kernel(const void *kern) {
  static const void *const table[] = {
      (const void *)k_kkt,        (const void *)k_param,         (const void *)k_elim,
      (const void *)k_riccati_finish, (const void *)k_aff_prep,  (const void *)k_post_roll,
      (const void *)k_resid,      (const void *)k_pcorr,         (const void *)k_recover,
      (const void *)k_dual_stage, (const void *)k_dual_leaf,     (const void *)k_set_costs,
      (const void *)k_refine_trial, (const void *)k_refine_accept, (const void *)k_primal_stage};
  for (const void *k : table)
    if (k == kern) return true;
  return false;
}
inline const int *group_slist(const Group &g) { return g.slist; }
template <typename A0, typename... Rest>
const int *group_slist(const A0 &a0, const Rest &...) {
  return group_slist(a0);
}

// one CTA per task; a per-stage kernel on a group with a stage list takes
// kListCtasPerSm CTAs per SM (at most one per stage) that loop over the list
template <typename... KArgs, typename... Args>
int launch(eclqr_handle *h, void (*kern)(KArgs...), int ntasks, int per_task, cudaStream_t st, Args... args) {
  int grid = ntasks;
  if (group_slist(args...) != nullptr && stage_list_kernel((const void *)kern))
    grid = std::min(ntasks, kListCtasPerSm * h->sms);
  return launch_grid(h, kern, ntasks, grid, per_task, st, args...);
}

// A per-problem sweep as a persistent launch: per_sm CTAs per SM take the tasks
// from the group's counter in index order (longest horizon first), so an SM that
// finishes its problems early takes more instead of idling while the longest
// sweeps end.  opt.persist = 0 does this for launches with at least
// kManyTasksPerSm tasks per SM, with kPersistCtasPerSm CTAs per SM; k > 0 for
// every launch with more than k tasks per SM; -1 never.  Otherwise one CTA per
// task.  The kernel's last argument is the counter, or null.
template <typename... KArgs, typename... Args>
int launch_sweep(eclqr_handle *h, int *queue, void (*kern)(KArgs...), int ntasks, int per_task, cudaStream_t st,
                 Args... args) {
  if (ntasks <= 0) return ECLQR_OK;
  const int per_sm = h->opt.persist == 0 ? kPersistCtasPerSm : h->opt.persist;
  const bool many = h->opt.persist != 0 || ntasks >= kManyTasksPerSm * h->sms;
  if (h->opt.persist == -1 || !many || ntasks <= per_sm * h->sms)
    return launch(h, kern, ntasks, per_task, st, args..., (int *)nullptr);
  if (cudaMemsetAsync(queue, 0, sizeof(int), st) != cudaSuccess) return ECLQR_ECUDA;
  return launch_grid(h, kern, ntasks, per_sm * h->sms, per_task, st, args..., queue);
}

#define TRY(x)                 \
  do {                         \
    int _rc = (x);             \
    if (_rc != ECLQR_OK) return _rc; \
  } while (0)

// Groups of different (n, m) share no data: with more than one group, each
// runs on its own stream, forked from the caller's stream and joined back
// into it, so that small groups fill the SMs a large group leaves idle.
int fork_groups(eclqr_handle *h, cudaStream_t st) {
  if (h->groups.size() < 2) return ECLQR_OK;
  if (cudaEventRecord(h->fork, st) != cudaSuccess) return ECLQR_ECUDA;
  for (auto &gh : h->groups)
    if (cudaStreamWaitEvent(gh.s, h->fork, 0) != cudaSuccess) return ECLQR_ECUDA;
  return ECLQR_OK;
}
cudaStream_t group_stream(const eclqr_handle *h, const GroupHost &gh, cudaStream_t st) {
  return h->groups.size() < 2 ? st : gh.s;
}
int join_groups(eclqr_handle *h, cudaStream_t st) {
  if (h->groups.size() < 2) return ECLQR_OK;
  for (auto &gh : h->groups) {
    if (cudaEventRecord(gh.done, gh.s) != cudaSuccess) return ECLQR_ECUDA;
    if (cudaStreamWaitEvent(st, gh.done, 0) != cudaSuccess) return ECLQR_ECUDA;
  }
  return ECLQR_OK;
}

int validate(const eclqr_desc *d) {
  if (!d || d->num_problems < 1 || !d->N || !d->n || !d->m || !d->p || !d->q) return ECLQR_EINVAL;
  long long ps = 0, qs = 0;
  for (int j = 0; j < d->num_problems; j++) {
    if (d->N[j] < 1 || d->n[j] < 1 || d->n[j] > ECLQR_MAX_N || d->m[j] < 1 || d->m[j] > ECLQR_MAX_M)
      return ECLQR_EINVAL;
    for (int i = 0; i < d->N[j]; i++)
      if (d->p[ps + i] < 0 || d->p[ps + i] > ECLQR_MAX_ROWS) return ECLQR_EINVAL;
    for (int i = 0; i <= d->N[j]; i++)
      if (d->q[qs + i] < 0 || d->q[qs + i] > ECLQR_MAX_ROWS) return ECLQR_EINVAL;
    ps += d->N[j];
    qs += d->N[j] + 1;
  }
  return ECLQR_OK;
}

}  // namespace

namespace {
// eight independent FMA chains per thread: throughput, not latency, bound
__global__ void k_fp64_probe(double *out, int iters, double a, double b) {
  double x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; i++) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
}  // namespace

extern "C" {

int eclqr_probe_fp64_peak(double *tflops) {
  if (!tflops) return ECLQR_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ECLQR_ECUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * 8, threads = 256, iters = 4096;
  double *buf = nullptr;
  if (cudaMalloc(&buf, sizeof(double) * (size_t)blocks * threads) != cudaSuccess) return ECLQR_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_fp64_probe<<<blocks, threads>>>(buf, 64, 1.0000001, 1e-9);
  float best = 1e30f;
  for (int rep = 0; rep < 3; rep++) {
    cudaEventRecord(e0);
    k_fp64_probe<<<blocks, threads>>>(buf, iters, 1.0000001, 1e-9);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    best = std::min(best, ms);
  }
  const cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (err != cudaSuccess) return ECLQR_ECUDA;
  *tflops = 2.0 * 8.0 * iters * (double)blocks * threads / (best * 1e-3) / 1e12;
  return ECLQR_OK;
}

void eclqr_default_options(eclqr_options *opt) {
  if (!opt) return;
  opt->tau_rank = 1e-10;
  opt->tau_inc = 1e-8;
  opt->refine = 2;
  opt->chunk = 0;
  opt->team_warps = 0;
  opt->scan_skip = 1;
  opt->kkt_refine = 8;
  opt->refine_tol = 5e-10;
  opt->riccati_fp32 = 0;
  opt->persist = 0;
  opt->corr_refine = -1;
}

int eclqr_layout(const eclqr_desc *d, eclqr_layout_info *out) {
  if (!out) return ECLQR_EINVAL;
  TRY(validate(d));
  eclqr_layout_info L;
  std::memset(&L, 0, sizeof(L));
  long long ps = 0, qs = 0;
  for (int j = 0; j < d->num_problems; j++) {
    const long long N = d->N[j], n = d->n[j], m = d->m[j];
    long long Pj = 0, Qj = 0;
    for (int i = 0; i < N; i++) Pj += d->p[ps + i];
    for (int i = 0; i <= N; i++) Qj += d->q[qs + i];
    ps += N;
    qs += N + 1;
    L.A += N * n * n; L.B += N * n * m; L.c += N * n;
    L.C += Pj * n; L.D += Pj * m; L.d += Pj;
    L.E += Qj * n; L.e += Qj;
    L.Q += (N + 1) * n * n; L.M += N * n * m; L.R += N * m * m; L.qv += (N + 1) * n; L.rv += N * m;
    L.s0 += n; L.x += (N + 1) * n; L.u += N * m; L.lam += (N + 1) * n; L.mu += Pj; L.eta += Qj; L.alpha += n;
    L.stages += N;
  }
  *out = L;
  return ECLQR_OK;
}

int eclqr_create(const eclqr_desc *d, const eclqr_options *opt, eclqr_handle **out) {
  if (!out) return ECLQR_EINVAL;
  *out = nullptr;
  TRY(validate(d));
  eclqr_handle *h = new (std::nothrow) eclqr_handle();
  if (!h) return ECLQR_ENOMEM;
  eclqr_default_options(&h->opt);
  if (opt) h->opt = *opt;
  const int tw = h->opt.team_warps;
  if (h->opt.refine < 0 || h->opt.refine > 8 || h->opt.chunk < 0 || !(h->opt.tau_rank > 0) || !(h->opt.tau_inc > 0) ||
      !(tw == 0 || tw == 1 || tw == 2 || tw == 4 || tw == 8) || !(h->opt.scan_skip == 0 || h->opt.scan_skip == 1) ||
      h->opt.kkt_refine < 0 || h->opt.kkt_refine > 16 || !(h->opt.refine_tol >= 0) ||
      !(h->opt.riccati_fp32 == 0 || h->opt.riccati_fp32 == 1) || h->opt.persist < -1 || h->opt.persist > 32 ||
      h->opt.corr_refine < -1 || h->opt.corr_refine > 8) {
    delete h;
    return ECLQR_EINVAL;
  }
  eclqr_layout(d, &h->lay);
  h->P = d->num_problems;
  cudaGetDevice(&h->device);
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  h->sms = sms;

  // batch offsets of every problem
  const int P = d->num_problems;
  std::vector<ProbInfo> pinfo(P);
  std::vector<long long> pstage(P + 1, 0), qstage(P + 1, 0);
  {
    long long oA = 0, oB = 0, oc = 0, oC = 0, oD = 0, od = 0, oE = 0, oe = 0, oQ = 0, oM = 0, oR = 0, oqv = 0,
              orv = 0, os0 = 0, ox = 0, ou = 0, olam = 0, omu = 0, oeta = 0, oal = 0;
    for (int j = 0; j < P; j++) {
      const long long N = d->N[j], n = d->n[j], m = d->m[j];
      pstage[j + 1] = pstage[j] + N;
      qstage[j + 1] = qstage[j] + N + 1;
      long long Pj = 0, Qj = 0;
      for (long long i = 0; i < N; i++) Pj += d->p[pstage[j] + i];
      for (long long i = 0; i <= N; i++) Qj += d->q[qstage[j] + i];
      ProbInfo &pi = pinfo[j];
      std::memset(&pi, 0, sizeof(pi));
      pi.N = (int)N;
      pi.id = j;
      pi.oA = oA; pi.oB = oB; pi.oc = oc; pi.oC = oC; pi.oD = oD; pi.od = od; pi.oE = oE; pi.oe = oe;
      pi.oQ = oQ; pi.oM = oM; pi.oR = oR; pi.oqv = oqv; pi.orv = orv;
      pi.os0 = os0; pi.ox = ox; pi.ou = ou; pi.olam = olam; pi.omu = omu; pi.oeta = oeta; pi.oalpha = oal;
      pi.ost = qstage[j];
      oA += N * n * n; oB += N * n * m; oc += N * n; oC += Pj * n; oD += Pj * m; od += Pj; oE += Qj * n; oe += Qj;
      oQ += (N + 1) * n * n; oM += N * n * m; oR += N * m * m; oqv += (N + 1) * n; orv += N * m;
      os0 += n; ox += (N + 1) * n; ou += N * m; olam += (N + 1) * n; omu += Pj; oeta += Qj; oal += n;
    }
  }
  // groups of equal (n, m)
  std::map<std::pair<int, int>, std::vector<int>> by_dims;
  for (int j = 0; j < P; j++) by_dims[{d->n[j], d->m[j]}].push_back(j);
  long long total_stages = h->lay.stages;
  int nmax = 1;  // the longest horizon of the batch
  for (int j = 0; j < P; j++) nmax = std::max(nmax, d->N[j]);
  for (auto &kv : by_dims) {
    GroupHost gh;
    Group &g = gh.g;
    std::memset(&g, 0, sizeof(g));
    g.n = kv.first.first;
    g.m = kv.first.second;
    gh.ids = kv.second;
    // longest horizons first: the tasks of a launch are issued in this order, so the
    // longest sweeps start in the first wave instead of finishing alone in the last
    std::stable_sort(gh.ids.begin(), gh.ids.end(), [&](int a, int b) { return d->N[a] > d->N[b]; });
    int pmax = 0, qmax = 0, wmax = 0;
    for (int j : gh.ids) {
      for (long long i = 0; i < d->N[j]; i++) {
        pmax = std::max(pmax, d->p[pstage[j] + i]);
        wmax = std::max(wmax, d->p[pstage[j] + i] + d->q[qstage[j] + i]);
      }
      for (long long i = 0; i <= d->N[j]; i++) qmax = std::max(qmax, d->q[qstage[j] + i]);
      wmax = std::max(wmax, d->q[qstage[j] + d->N[j]]);
    }
    g.pmax = pmax;
    g.qmax = qmax;
    g.wmax = wmax;
    // every kernel's shared memory must fit one task (one CTA)
    {
      const int n = g.n, m = g.m;
      const int need = std::max({smem_primal_sweep(n, m, pmax, qmax), smem_rel_level(n, pmax, qmax), smem_param(n),
                                 smem_elim(n, m, pmax), smem_lqr_up(n, m), smem_lqr_level(n), smem_riccati(n, m),
                                 smem_riccati_finish(n, m),
                                 smem_aff(n, m), smem_dual_stage(n, m), smem_dual_sweep(n, m, pmax, qmax),
                                 smem_dual_leaf(n, m, wmax), smem_scan_check(n, m, pmax)});
      if ((size_t)need * sizeof(double) > (size_t)kMaxSmemBytes) {
        for (auto &x : h->groups) cudaFree(x.dmem);
        delete h;
        return ECLQR_ESMEM;
      }
      // exact test: each kernel's dynamic request plus its static scratch against the
      // device's per-CTA limit (the bound above leaves the static part out)
      const int sw = smem_primal_sweep(n, m, pmax, qmax), sl = smem_rel_level(n, pmax, qmax), sa = smem_aff(n, m);
      const int sdw = smem_dual_sweep(n, m, pmax, qmax);
      const struct { const void *fn; int dyn; } kk[] = {
          {(const void *)k_scan_check, smem_scan_check(n, m, pmax)}, {(const void *)k_terminal, sw},
          {(const void *)k_primal_up, sw}, {(const void *)k_primal_down, sw}, {(const void *)k_primal_stage, smem_primal_stage(n, m, wmax)}, {(const void *)k_rel_level, sl},
          {(const void *)k_param, smem_param(n)}, {(const void *)k_elim, smem_elim(n, m, pmax)},
          {(const void *)k_lqr_up, smem_lqr_up(n, m)}, {(const void *)k_lqr_level, smem_lqr_level(n)},
          {(const void *)k_riccati_down, smem_riccati(n, m)},
          {(const void *)k_riccati_finish, smem_riccati_finish(n, m)}, {(const void *)k_aff_up, sa},
          {(const void *)k_aff_level, sa}, {(const void *)k_aff_down, sa}, {(const void *)k_resid, 3 * n + 2 * m},
          {(const void *)k_pcorr, n + m + m * m}, {(const void *)k_dual_stage, smem_dual_stage(n, m)},
          {(const void *)k_dual_terminal, sdw}, {(const void *)k_dual_up, sdw}, {(const void *)k_dual_down, sdw},
          {(const void *)k_dual_root, sdw}, {(const void *)k_dual_leaf, smem_dual_leaf(n, m, wmax)}};
      int optin = 0;
      int rc = (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device) == cudaSuccess)
                   ? ECLQR_OK : ECLQR_ECUDA;
      for (const auto &k : kk) {
        if (rc != ECLQR_OK) break;
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, k.fn) != cudaSuccess) rc = ECLQR_ECUDA;
        else if ((size_t)k.dyn * sizeof(double) + fa.sharedSizeBytes > (size_t)optin) rc = ECLQR_ESMEM;
      }
      if (rc != ECLQR_OK) {
        for (auto &x : h->groups) cudaFree(x.dmem);
        delete h;
        return rc;
      }
    }
    std::vector<ProbInfo> gp;
    std::vector<StageInfo> gs;
    std::vector<ChunkInfo> gc;
    gh.any_skip = false;
    for (int j : gh.ids) {
      ProbInfo pi = pinfo[j];
      int L = h->opt.chunk;
      if (L <= 0 && (long long)nmax * sms <= total_stages) {
        // the longest horizon is at most the stages per SM: one chunk per problem.  Its
        // sweeps then run without chunk aggregates, scan levels or next-chunk re-sweeps,
        // the least work, and no problem's sequential sweep outlasts an SM's share of the
        // batch (256 problems of 256 stages: 37 ms against 83 ms chunked).
        L = std::max(1, pi.N);
      } else if (L <= 0) {
        // enough chunks to give every SM work, but never shorter than 7 stages: shorter
        // chunks place more boundaries, and where a boundary meets an ill-conditioned
        // stage the refinement needs more than its default passes (on the degenerate
        // n = 12 instance 6-stage chunks miss the 1e-9 gate after two).  A 1024-stage
        // problem then runs as 147 chunks, one CTA each, on a 152-SM GB300.
        long long target = std::max<long long>(1, total_stages / (2LL * sms));
        L = (int)std::min<long long>(64, std::max<long long>(7, target));
        L = std::max(1, std::min(L, pi.N));
      }
      pi.L = L;
      pi.nch = (pi.N + L - 1) / L;
      pi.ch0 = (int)gc.size();
      pi.st0 = (int)gs.size();
      const int local = (int)gp.size();
      int prow = 0, qrow = 0;
      // Sec. 6 shortcut: eligible when no stage has state-only or terminal rows and
      // every D_i could have full row rank (p_i <= m); k_scan_check decides the rest
      pi.skip_ok = h->opt.scan_skip ? 1 : 0;
      for (int i = 0; i <= pi.N; i++) {
        StageInfo si;
        si.prob = local;
        si.i = i;
        si.p = (i < pi.N) ? d->p[pstage[j] + i] : 0;
        si.q = d->q[qstage[j] + i];
        si.prow = prow;
        si.qrow = qrow;
        if (si.q > 0 || si.p > g.m) pi.skip_ok = 0;
        prow += si.p;
        qrow += si.q;
        gs.push_back(si);
      }
      for (int c = 0; c <= pi.nch; c++) gc.push_back(ChunkInfo{local, c});
      gh.maxnch = std::max(gh.maxnch, pi.nch);
      gh.any_skip = gh.any_skip || pi.skip_ok;
      gp.push_back(pi);
    }
    g.nprob = (int)gp.size();
    g.nstage = (int)gs.size();
    g.nslot = (int)gc.size();
    gh.levels = ilog2ceil(gh.maxnch + 1);
    g.ws = make_ws_layout(g.n, g.m, pmax, qmax);
    g.cs_stride = ((8 * g.n * g.n + 4 * g.n) + 3) & ~3;  // cost relations: 2n constraint + 2n cost rows
    g.cr_stride = 0;
    g.tau_rank = h->opt.tau_rank;
    g.tau_inc = h->opt.tau_inc;
    // one allocation: descriptors, stage workspace, chunk slots
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t r = off; off += (bytes + 255) & ~size_t(255); return r; };
    size_t o_prob = take(sizeof(ProbInfo) * gp.size()), o_st = take(sizeof(StageInfo) * gs.size()),
           o_ch = take(sizeof(ChunkInfo) * gc.size());
    size_t o_W = take(sizeof(double) * (size_t)g.ws.stride * g.nstage);
    size_t o_WI = take(sizeof(int) * (size_t)SI_STRIDE * g.nstage);
    size_t o_CS0 = take(sizeof(double) * (size_t)g.cs_stride * g.nslot);
    size_t o_CS1 = take(sizeof(double) * (size_t)g.cs_stride * g.nslot);
    size_t o_CI0 = take(sizeof(int) * CI_STRIDE * g.nslot), o_CI1 = take(sizeof(int) * CI_STRIDE * g.nslot);
    size_t o_need = take(sizeof(int) * (size_t)g.nprob), o_queue = take(sizeof(int));
    size_t o_sl = take(sizeof(int) * 3 * (size_t)g.nstage), o_sc = take(sizeof(int) * 3);
    if (cudaMalloc(&gh.dmem, off) != cudaSuccess) {
      for (auto &x : h->groups) cudaFree(x.dmem);
      delete h;
      return ECLQR_ENOMEM;
    }
    char *base = (char *)gh.dmem;
    if (cudaMemset(base, 0, off) != cudaSuccess ||
        cudaMemcpy(base + o_prob, gp.data(), sizeof(ProbInfo) * gp.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(base + o_st, gs.data(), sizeof(StageInfo) * gs.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(base + o_ch, gc.data(), sizeof(ChunkInfo) * gc.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaFree(gh.dmem);
      eclqr_destroy(h);  // the groups planned so far
      return ECLQR_ECUDA;
    }
    g.prob = (const ProbInfo *)(base + o_prob);
    g.st = (const StageInfo *)(base + o_st);
    g.chunk = (const ChunkInfo *)(base + o_ch);
    g.W = (double *)(base + o_W);
    g.WI = (int *)(base + o_WI);
    g.CS[0] = (double *)(base + o_CS0);
    g.CS[1] = (double *)(base + o_CS1);
    g.CI[0] = (int *)(base + o_CI0);
    g.CI[1] = (int *)(base + o_CI1);
    g.need_scan = (int *)(base + o_need);
    gh.queue = (int *)(base + o_queue);
    gh.slists = (int *)(base + o_sl);
    gh.scounts = (int *)(base + o_sc);
    h->groups.push_back(gh);
  }
  if (h->opt.kkt_refine > 0) {
    const eclqr_layout_info &L = h->lay;
    size_t off = 0;
    auto take = [&](size_t elems, size_t esz) { size_t r = off; off += (std::max<size_t>(elems, 1) * esz + 255) & ~size_t(255); return r; };
    const size_t o_c = take(L.c, 8), o_d = take(L.d, 8), o_e = take(L.e, 8), o_qv = take(L.qv, 8),
                 o_rv = take(L.rv, 8), o_s0 = take(L.s0, 8), o_x = take(L.x, 8), o_u = take(L.u, 8),
                 o_lam = take(L.lam, 8), o_mu = take(L.mu, 8), o_eta = take(L.eta, 8), o_al = take(L.alpha, 8),
                 o_cs = take(P, 4), o_tr = take(P, 8), o_ac = take(P, 4), o_any = take(1, 4),
                 o_fu = take(P, 4), o_ch = take(P, 4), o_pa = take(4 * (size_t)P, 8), o_tp = take(4 * (size_t)P, 8),
                 o_z = take(std::max({L.c, L.d, L.e, L.s0}), 8);
    if (cudaMalloc(&h->rmem, off) != cudaSuccess || cudaMemset(h->rmem, 0, off) != cudaSuccess) {
      eclqr_destroy(h);
      return ECLQR_ENOMEM;
    }
    char *b = (char *)h->rmem;
    h->rows = KktRows{(double *)(b + o_c), (double *)(b + o_d), (double *)(b + o_e), (double *)(b + o_qv),
                      (double *)(b + o_rv), (double *)(b + o_s0)};
    h->trial = SolMut{(double *)(b + o_x), (double *)(b + o_u), (double *)(b + o_lam), (double *)(b + o_mu),
                      (double *)(b + o_eta), (double *)(b + o_al)};
    h->cstatus = (int32_t *)(b + o_cs);
    h->tresid = (double *)(b + o_tr);
    h->mk = RefineMasks{(int *)(b + o_ac), (int *)(b + o_fu), (int *)(b + o_ch)};
    h->parts = (double *)(b + o_pa);
    h->tparts = (double *)(b + o_tp);
    h->zeros = (double *)(b + o_z);
    h->any = (int *)(b + o_any);
    if (cudaMallocHost(&h->any_host, sizeof(int)) != cudaSuccess) {
      h->any_host = nullptr;
      eclqr_destroy(h);
      return ECLQR_ENOMEM;
    }
  }
  if (h->opt.riccati_fp32 && cudaMalloc(&h->fp64, sizeof(int) * (size_t)P) != cudaSuccess) {
    h->fp64 = nullptr;
    eclqr_destroy(h);
    return ECLQR_ENOMEM;
  }
  if (h->groups.size() > 1) {
    bool ok = cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming) == cudaSuccess;
    for (auto &gh : h->groups) {
      ok = ok && cudaStreamCreateWithFlags(&gh.s, cudaStreamNonBlocking) == cudaSuccess;
      ok = ok && cudaEventCreateWithFlags(&gh.done, cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) {
      eclqr_destroy(h);
      return ECLQR_ECUDA;
    }
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    eclqr_destroy(h);
    return ECLQR_ECUDA;
  }
  *out = h;
  return ECLQR_OK;
}

}  // extern "C"

namespace {

// Algorithm 1 up to the Riccati factors (Sec. 3-6) for one group, with the data,
// status and mask that g carries.  scan_check: run the Sec. 6 shortcut's test
// and the check of the data for NaN (the first build of a data set; correction
// problems have the same matrices and reuse its flags).
int run_build(eclqr_handle *h, GroupHost &gh, const Group &g, cudaStream_t gst, bool first) {
  const int n = g.n, m = g.m, pm = g.pmax, qm = g.qmax;
  const int sw = smem_primal_sweep(n, m, pm, qm), sl = smem_rel_level(n, pm, qm);
  if (first) {
    TRY(launch(h, k_check_inputs, g.nstage, 0, gst, g));
    if (gh.any_skip) {
      if (cudaMemsetAsync(g.need_scan, 0, sizeof(int) * g.nprob, gst) != cudaSuccess) return ECLQR_ECUDA;
      const int sk = smem_scan_check(n, m, pm);
      TRY(launch(h, k_scan_check, g.nstage, sk, gst, g, sk));
    }
  }
  TRY(launch(h, k_terminal, g.nprob, sw, gst, g, sw));
  TRY(launch(h, k_primal_up, g.nslot, sw, gst, g, sw));
  int src = 0;
  for (int k = 0; k < gh.levels; k++, src ^= 1)
    TRY(launch(h, k_rel_level, g.nslot, sl, gst, g, src, 1 << k, (int)ST_INFEASIBLE_SUFFIX, sl));
  const int sps = smem_primal_stage(n, m, g.wmax);
  TRY(launch(h, k_primal_stage, g.nstage, sps, gst, g, sps));
  TRY(launch_sweep(h, gh.queue, k_primal_down, g.nslot, sw, gst, g, src, sw));
  const int sp = smem_param(n), se = smem_elim(n, m, pm);
  TRY(launch(h, k_param, g.nstage, sp, gst, g, sp));
  TRY(launch(h, k_elim, g.nstage, se, gst, g, se));
  const int su = smem_lqr_up(n, m), slv = smem_lqr_level(n), sr = smem_riccati(n, m);
  TRY(launch(h, k_lqr_up, g.nslot, su, gst, g, su));
  src = 0;
  for (int k = 0; k < gh.levels; k++, src ^= 1) TRY(launch(h, k_lqr_level, g.nslot, slv, gst, g, src, 1 << k, slv));
  TRY(launch_sweep(h, gh.queue, k_riccati_down, g.nslot, sr, gst, g, src, sr));
  if (g.fp64) TRY(launch(h, k_riccati_down_f32, g.nslot, sr, gst, g, src, sr));
  const int sf = smem_riccati_finish(n, m);
  TRY(launch(h, k_riccati_finish, g.nstage, sf, gst, g, sf));
  return ECLQR_OK;
}

int aff_scan(eclqr_handle *h, const GroupHost &gh, const Group &g, int mode, cudaStream_t st) {
  const int sa = smem_aff(g.n, g.m);
  const int fwd = (mode == AFF_PLIN_) ? 0 : 1;
  TRY(launch(h, k_aff_prep, g.nstage, g.n + 8, st, g, mode, g.n + 8));
  TRY(launch(h, k_aff_up, g.nslot, sa, st, g, mode, sa));
  int src = 0;
  // radix-4 levels: strides 1, 4, 16, ... until they cover every slot
  for (int d = 1; d < gh.maxnch + 1; d *= 4, src ^= 1) TRY(launch(h, k_aff_level, g.nslot, sa, st, g, src, d, fwd, sa));
  TRY(launch(h, k_aff_down, g.nslot, sa, st, g, mode, src, sa));
  return ECLQR_OK;
}

// rollout with refinement on the reduced residual, and recovery (Sec. 6, eq. recovery-maps)
int run_solve(eclqr_handle *h, const GroupHost &gh, const Group &g, cudaStream_t gst, const double *s0, double *x,
              double *u, int refine_passes) {
  TRY(launch(h, k_solve_init, g.nprob, 0, gst, g, s0));
  TRY(aff_scan(h, gh, g, AFF_ROLL_, gst));
  TRY(launch(h, k_post_roll, g.nstage, 0, gst, g, 0));
  for (int r = 0; r < refine_passes; r++) {
    const int sres = 3 * g.n + 2 * g.m;
    TRY(launch(h, k_resid, g.nstage, sres, gst, g, sres));
    TRY(aff_scan(h, gh, g, AFF_PLIN_, gst));
    const int sc = g.n + g.m + g.m * g.m;
    TRY(launch(h, k_pcorr, g.nstage, sc, gst, g, sc));
    TRY(aff_scan(h, gh, g, AFF_CROLL_, gst));
    TRY(launch(h, k_post_roll, g.nstage, 0, gst, g, 1));
  }
  TRY(launch(h, k_recover, g.nstage, 0, gst, g, x, u));
  return ECLQR_OK;
}

// multipliers (Sec. 7)
int run_mult(eclqr_handle *h, const GroupHost &gh, const Group &g, cudaStream_t gst, const double *x, const double *u,
             double *lam, double *mu, double *eta, double *alpha) {
  const int n = g.n, m = g.m, pm = g.pmax, qm = g.qmax;
  const int sd = smem_dual_stage(n, m), sw = smem_dual_sweep(n, m, pm, qm), sl = smem_rel_level(n, pm, qm);
  const int sf = smem_dual_leaf(n, m, g.wmax);
  TRY(launch(h, k_dual_stage, g.nstage, sd, gst, g, x, u, sd));
  TRY(launch(h, k_dual_terminal, g.nprob, sw, gst, g, sw));
  TRY(launch(h, k_dual_up, g.nslot, sw, gst, g, sw));
  int src = 0;
  for (int k = 0; k < gh.levels; k++, src ^= 1)
    TRY(launch(h, k_rel_level, g.nslot, sl, gst, g, src, 1 << k, (int)ST_OK, sl));
  TRY(launch(h, k_dual_down, g.nslot, sw, gst, g, src, sw));
  TRY(launch(h, k_dual_root, g.nprob, sw, gst, g, sw));
  TRY(aff_scan(h, gh, g, AFF_NU_, gst));
  TRY(launch(h, k_dual_leaf, g.nstage, sf, gst, g, lam, mu, eta, alpha, sf));
  return ECLQR_OK;
}

void set_data(Group &g, const eclqr_data *data) {
  g.A = data->A; g.B = data->B; g.c = data->c; g.C = data->C; g.D = data->D; g.d = data->d;
  g.E = data->E; g.e = data->e; g.Q = data->Q; g.M = data->M; g.R = data->R; g.qv = data->qv; g.rv = data->rv;
}

}  // namespace

extern "C" {

int eclqr_build(eclqr_handle *h, const eclqr_data *data, int32_t *status, void *stream) {
  if (!h || !data || !status) return ECLQR_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(status, 0, sizeof(int32_t) * h->P, st) != cudaSuccess) return ECLQR_ECUDA;
  // mixed precision: every problem starts with its Riccati sweep in FP32
  if (h->fp64 && cudaMemsetAsync(h->fp64, 0, sizeof(int) * h->P, st) != cudaSuccess) return ECLQR_ECUDA;
  TRY(fork_groups(h, st));
  for (auto &gh : h->groups) {
    set_data(gh.g, data);
    gh.g.status = status;
    gh.g.active = nullptr;
    gh.g.fp64 = h->fp64;
    TRY(run_build(h, gh, gh.g, group_stream(h, gh, st), true));
  }
  TRY(join_groups(h, st));
  h->built = true;
  h->solved = false;
  h->stale = false;
  return ECLQR_OK;
}

int eclqr_solve(eclqr_handle *h, const double *s0, double *x, double *u, int32_t *status, void *stream) {
  if (!h || !s0 || !x || !u || !status) return ECLQR_EINVAL;
  if (!h->built || h->stale) return ECLQR_ESTATE;
  cudaStream_t st = (cudaStream_t)stream;
  TRY(fork_groups(h, st));
  for (auto &gh : h->groups) {
    gh.g.status = status;
    TRY(run_solve(h, gh, gh.g, group_stream(h, gh, st), s0, x, u, h->opt.refine));
  }
  TRY(join_groups(h, st));
  h->solved = true;
  return ECLQR_OK;
}

int eclqr_multipliers(eclqr_handle *h, const double *x, const double *u, double *lam, double *mu, double *eta,
                      double *alpha, int32_t *status, void *stream) {
  if (!h || !x || !u || !lam || !alpha || !status) return ECLQR_EINVAL;
  if (h->lay.mu > 0 && !mu) return ECLQR_EINVAL;
  if (h->lay.eta > 0 && !eta) return ECLQR_EINVAL;
  if (!h->solved) return ECLQR_ESTATE;
  cudaStream_t st = (cudaStream_t)stream;
  TRY(fork_groups(h, st));
  for (auto &gh : h->groups) {
    gh.g.status = status;
    TRY(run_mult(h, gh, gh.g, group_stream(h, gh, st), x, u, lam, mu, eta, alpha));
  }
  TRY(join_groups(h, st));
  return ECLQR_OK;
}

namespace {
int residual(eclqr_handle *h, const double *s0, const double *x, const double *u, const double *lam,
             const double *mu, const double *eta, const double *alpha, double *resid, double *parts, void *stream) {
  if (!h || !s0 || !x || !u || !lam || !alpha || !resid) return ECLQR_EINVAL;
  if (h->lay.mu > 0 && !mu) return ECLQR_EINVAL;
  if (h->lay.eta > 0 && !eta) return ECLQR_EINVAL;
  if (!h->built) return ECLQR_ESTATE;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(resid, 0, sizeof(double) * h->P, st) != cudaSuccess) return ECLQR_ECUDA;
  if (parts && cudaMemsetAsync(parts, 0, sizeof(double) * 4 * h->P, st) != cudaSuccess) return ECLQR_ECUDA;
  TRY(fork_groups(h, st));
  for (auto &gh : h->groups) {
    Group g = gh.g;
    g.active = nullptr;
    TRY(launch(h, k_kkt, g.nstage, 0, group_stream(h, gh, st), g, s0, x, u, lam, mu, eta, alpha, KktRows{},
               resid, parts));
  }
  TRY(join_groups(h, st));
  return ECLQR_OK;
}
}  // namespace

int eclqr_kkt_residual(eclqr_handle *h, const double *s0, const double *x, const double *u, const double *lam,
                       const double *mu, const double *eta, const double *alpha, double *resid, void *stream) {
  return residual(h, s0, x, u, lam, mu, eta, alpha, resid, nullptr, stream);
}

int eclqr_kkt_residual_parts(eclqr_handle *h, const double *s0, const double *x, const double *u, const double *lam,
                             const double *mu, const double *eta, const double *alpha, double *resid, double *parts,
                             void *stream) {
  if (!parts) return ECLQR_EINVAL;
  return residual(h, s0, x, u, lam, mu, eta, alpha, resid, parts, stream);
}

int eclqr_refine(eclqr_handle *h, const double *s0, double *x, double *u, double *lam, double *mu, double *eta,
                 double *alpha, double *resid, int32_t *status, void *stream) {
  if (!h || !s0 || !x || !u || !lam || !alpha || !resid || !status) return ECLQR_EINVAL;
  if (h->lay.mu > 0 && !mu) return ECLQR_EINVAL;
  if (h->lay.eta > 0 && !eta) return ECLQR_EINVAL;
  if (!h->built || h->stale) return ECLQR_ESTATE;
  TRY(residual(h, s0, x, u, lam, mu, eta, alpha, resid, h->opt.kkt_refine > 0 ? h->parts : nullptr, stream));
  if (h->opt.kkt_refine == 0) return ECLQR_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const Sol w{x, u, lam, mu, eta, alpha};
  const SolMut &t = h->trial;
  const Sol tc{t.x, t.u, t.lam, t.mu, t.eta, t.alpha};
  const RefineMasks mk = h->mk;
  const int corr = h->opt.corr_refine < 0 ? h->opt.refine : h->opt.corr_refine;
  // outside a stream capture the passes stop as soon as no problem takes part (one 4-byte read
  // back per pass); a captured sequence holds every pass, whose kernels return at once for
  // problems that take no part
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return ECLQR_ECUDA;
  const bool eager = cap == cudaStreamCaptureStatusNone;
  bool corrected = false;
  // up to opt.kkt_refine passes; first = 1 starts every problem afresh, 0 continues the problems
  // that mk.active marks
  auto passes = [&](int first) -> int {
  for (int k = 0; k < h->opt.kkt_refine; k++) {
    if (cudaMemsetAsync(h->any, 0, sizeof(int), st) != cudaSuccess) return ECLQR_ECUDA;
    TRY(fork_groups(h, st));
    for (auto &gh : h->groups) {
      Group gu = gh.g;  // unmasked, for the per-problem bookkeeping
      gu.active = nullptr;
      TRY(launch(h, k_refine_prep, gu.nprob, 0, group_stream(h, gh, st), gu, (const int32_t *)status,
                 (const double *)resid, (const double *)h->parts, mk, h->cstatus, h->tresid, h->tparts, h->opt.refine_tol,
                 k == 0 ? first : 0, h->any));
    }
    if (eager) {
      TRY(join_groups(h, st));
      if (cudaMemcpyAsync(h->any_host, h->any, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        return ECLQR_ECUDA;
      if (*h->any_host == 0) break;
      TRY(fork_groups(h, st));
    }
    corrected = true;
    for (auto &gh : h->groups) {
      const cudaStream_t gst = group_stream(h, gh, st);
      Group gu = gh.g;
      gu.active = nullptr;
      // the stages of the problems that take part, of those that rebuild and of those that
      // take the cheap correction: the pass's per-stage kernels visit only those
      if (cudaMemsetAsync(gh.scounts, 0, 3 * sizeof(int), gst) != cudaSuccess) return ECLQR_ECUDA;
      TRY(launch(h, k_stage_lists, gu.nprob, 0, gst, gu, mk, gh.slists, gh.scounts));
      Group g = gh.g;  // the problem's data, masked to the problems that take part
      g.active = mk.active;
      g.status = h->cstatus;
      g.slist = gh.slists;
      g.scount = gh.scounts;
      // residual rows of the point, in the layout of the offsets they replace
      TRY(launch(h, k_kkt, g.nstage, 0, gst, g, s0, (const double *)x, (const double *)u, (const double *)lam,
                 (const double *)mu, (const double *)eta, (const double *)alpha, h->rows, (double *)nullptr,
                 (double *)nullptr));
      // primal rows above the tolerance: the same matrices with the residual rows as offsets,
      // through a new build
      Group gf = g;
      gf.active = mk.full;
      gf.slist = gh.slists + gu.nstage;
      gf.scount = gh.scounts + 1;
      gf.c = h->rows.c; gf.d = h->rows.d; gf.e = h->rows.e; gf.qv = h->rows.qv; gf.rv = h->rows.rv;
      TRY(run_build(h, gh, gf, gst, false));
      TRY(run_solve(h, gh, gf, gst, h->rows.s0, t.x, t.u, corr));
      TRY(run_mult(h, gh, gf, gst, t.x, t.u, t.lam, t.mu, t.eta, t.alpha));
      // primal rows within it: homogeneous constraints, so the build's factors serve as they
      // are and only the linear costs change (as for the adjoint, eclqr_set_costs)
      Group gz = g;
      gz.active = mk.cheap;
      gz.slist = gh.slists + 2 * (size_t)gu.nstage;
      gz.scount = gh.scounts + 2;
      gz.c = h->zeros; gz.d = h->zeros; gz.e = h->zeros; gz.qv = h->rows.qv; gz.rv = h->rows.rv;
      TRY(launch(h, k_set_costs, gz.nstage, smem_set_costs(gz.n, gz.m), gst, gz, smem_set_costs(gz.n, gz.m)));
      TRY(run_solve(h, gh, gz, gst, h->zeros, t.x, t.u, corr));
      TRY(run_mult(h, gh, gz, gst, t.x, t.u, t.lam, t.mu, t.eta, t.alpha));
      // trial point w + dw, its residual, and the choice
      TRY(launch(h, k_refine_gate, gu.nprob, 0, gst, gu, (const int32_t *)h->cstatus, mk.active));
      TRY(launch(h, k_refine_trial, g.nstage, 0, gst, g, w, t));
      TRY(launch(h, k_kkt, g.nstage, 0, gst, g, s0, tc.x, tc.u, tc.lam, tc.mu, tc.eta, tc.alpha, KktRows{},
                 h->tresid, h->tparts));
      TRY(launch(h, k_refine_accept, g.nstage, 0, gst, g, tc, x, u, lam, mu, eta, alpha, (const double *)resid,
                 (const double *)h->tresid));
      TRY(launch(h, k_refine_parts, gu.nprob, 0, gst, gu, (const int *)mk.active, h->parts,
                 (const double *)h->tparts, (const double *)resid, (const double *)h->tresid));
      TRY(launch(h, k_refine_post, gu.nprob, 0, gst, gu, resid, (const double *)h->tresid, mk.active));
    }
    TRY(join_groups(h, st));
  }
  return ECLQR_OK;
  };
  TRY(passes(1));
  if (h->fp64) {
    // mixed precision: the problems still above the tolerance are redone with their Riccati
    // sweep in FP64 (build, solve, multipliers, residual), then refined again
    if (cudaMemsetAsync(h->any, 0, sizeof(int), st) != cudaSuccess) return ECLQR_ECUDA;
    TRY(fork_groups(h, st));
    for (auto &gh : h->groups) {
      Group gu = gh.g;
      gu.active = nullptr;
      TRY(launch(h, k_rescue_prep, gu.nprob, 0, group_stream(h, gh, st), gu, (const int32_t *)status, resid, h->parts,
                 h->fp64, mk.active, h->opt.refine_tol, h->any));
    }
    bool work = true;
    if (eager) {
      TRY(join_groups(h, st));
      if (cudaMemcpyAsync(h->any_host, h->any, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        return ECLQR_ECUDA;
      work = *h->any_host != 0;
      if (work) TRY(fork_groups(h, st));
    }
    if (work) {
      corrected = true;
      for (auto &gh : h->groups) {
        const cudaStream_t gst = group_stream(h, gh, st);
        Group g = gh.g;  // the problem's own data, masked to the rescued problems
        g.active = mk.active;
        g.status = status;
        TRY(run_build(h, gh, g, gst, false));
        TRY(run_solve(h, gh, g, gst, s0, x, u, h->opt.refine));
        TRY(run_mult(h, gh, g, gst, x, u, lam, mu, eta, alpha));
        TRY(launch(h, k_kkt, g.nstage, 0, gst, g, s0, (const double *)x, (const double *)u, (const double *)lam,
                   (const double *)mu, (const double *)eta, (const double *)alpha, KktRows{}, resid, h->parts));
      }
      TRY(join_groups(h, st));
      TRY(passes(0));
    }
  }
  if (corrected) {
    h->stale = true;
    h->solved = false;
  }
  return ECLQR_OK;
}

int eclqr_set_costs(eclqr_handle *h, const eclqr_data *data, void *stream) {
  if (!h || !data) return ECLQR_EINVAL;
  if (!h->built) return ECLQR_ESTATE;
  cudaStream_t st = (cudaStream_t)stream;
  TRY(fork_groups(h, st));
  for (auto &gh : h->groups) {
    Group &g = gh.g;
    g.A = data->A; g.B = data->B; g.c = data->c; g.C = data->C; g.D = data->D; g.d = data->d;
    g.E = data->E; g.e = data->e; g.Q = data->Q; g.M = data->M; g.R = data->R; g.qv = data->qv; g.rv = data->rv;
    g.active = nullptr;
    TRY(launch(h, k_set_costs, g.nstage, smem_set_costs(g.n, g.m), group_stream(h, gh, st), g, smem_set_costs(g.n, g.m)));
  }
  TRY(join_groups(h, st));
  h->solved = false;
  h->stale = false;
  return ECLQR_OK;
}

int eclqr_param_grads(eclqr_handle *h, const double *x, const double *u, const double *lam, const double *mu,
                      const double *eta, const double *alpha, const double *xb, const double *ub,
                      const double *lamb, const double *mub, const double *etab, const double *alphab,
                      const eclqr_grads *out, void *stream) {
  if (!h || !x || !u || !lam || !alpha || !xb || !ub || !lamb || !alphab || !out) return ECLQR_EINVAL;
  if (h->lay.mu > 0 && (!mu || !mub || !out->C || !out->D || !out->d)) return ECLQR_EINVAL;
  if (h->lay.eta > 0 && (!eta || !etab || !out->E || !out->e)) return ECLQR_EINVAL;
  if (!out->A || !out->B || !out->c || !out->Q || !out->M || !out->R || !out->qv || !out->rv || !out->s0)
    return ECLQR_EINVAL;
  if (!h->built) return ECLQR_ESTATE;
  cudaStream_t st = (cudaStream_t)stream;
  const Sol w{x, u, lam, mu, eta, alpha}, wb{xb, ub, lamb, mub, etab, alphab};
  const GradOut o{out->A, out->B, out->c, out->C, out->D, out->d, out->E, out->e,
                  out->Q, out->M, out->R, out->qv, out->rv, out->s0};
  TRY(fork_groups(h, st));
  for (auto &gh : h->groups) TRY(launch(h, k_param_grads, gh.g.nstage, 0, group_stream(h, gh, st), gh.g, w, wb, o));
  TRY(join_groups(h, st));
  return ECLQR_OK;
}

int eclqr_reduced_dims(eclqr_handle *h, int32_t *nbar, int32_t *mbar, void *stream) {
  if (!h || !nbar || !mbar) return ECLQR_EINVAL;
  if (!h->built) return ECLQR_ESTATE;
  cudaStream_t st = (cudaStream_t)stream;
  for (auto &gh : h->groups) {
    const int blocks = (gh.g.nstage + 255) / 256;
    k_dims<<<blocks, 256, 0, st>>>(gh.g, nbar, mbar);
    h->launches++;
    if (cudaPeekAtLastError() != cudaSuccess) return ECLQR_ECUDA;
  }
  return ECLQR_OK;
}

int eclqr_scan_skipped(eclqr_handle *h, int32_t *flags, void *stream) {
  if (!h || !flags) return ECLQR_EINVAL;
  if (!h->built) return ECLQR_ESTATE;
  cudaStream_t st = (cudaStream_t)stream;
  TRY(fork_groups(h, st));
  for (auto &gh : h->groups) TRY(launch(h, k_skip_flags, gh.g.nprob, 0, group_stream(h, gh, st), gh.g, flags));
  TRY(join_groups(h, st));
  return ECLQR_OK;
}

int64_t eclqr_launch_count(const eclqr_handle *h) { return h ? h->launches : 0; }

int eclqr_riccati_fp64_flags(eclqr_handle *h, int32_t *flags, void *stream) {
  if (!h || !flags) return ECLQR_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (!h->fp64) {
    // FP64 throughout: every sweep in FP64
    std::vector<int32_t> ones(h->P, 1);
    return cudaMemcpyAsync(flags, ones.data(), sizeof(int32_t) * h->P, cudaMemcpyHostToDevice, st) == cudaSuccess &&
                   cudaStreamSynchronize(st) == cudaSuccess
               ? ECLQR_OK
               : ECLQR_ECUDA;
  }
  return cudaMemcpyAsync(flags, h->fp64, sizeof(int32_t) * h->P, cudaMemcpyDeviceToDevice, st) == cudaSuccess
             ? ECLQR_OK
             : ECLQR_ECUDA;
}

void eclqr_destroy(eclqr_handle *h) {
  if (!h) return;
  for (auto &gh : h->groups) {
    cudaFree(gh.dmem);
    if (gh.s) cudaStreamDestroy(gh.s);
    if (gh.done) cudaEventDestroy(gh.done);
  }
  if (h->fork) cudaEventDestroy(h->fork);
  if (h->rmem) cudaFree(h->rmem);
  if (h->any_host) cudaFreeHost(h->any_host);
  if (h->fp64) cudaFree(h->fp64);
  for (auto e : h->ev) cudaEventDestroy(e);
  delete h;
}

int eclqr_time_kernel(eclqr_handle *h, const char *name) {
  if (!h) return ECLQR_EINVAL;
  h->nev = 0;
  if (!name) {
    h->timed = nullptr;
    return ECLQR_OK;
  }
  static const struct { const char *name; const void *fn; } table[] = {
      {"k_scan_check", (const void *)k_scan_check}, {"k_terminal", (const void *)k_terminal}, {"k_primal_up", (const void *)k_primal_up},
      {"k_rel_level", (const void *)k_rel_level}, {"k_primal_down", (const void *)k_primal_down}, {"k_primal_stage", (const void *)k_primal_stage},
      {"k_param", (const void *)k_param}, {"k_elim", (const void *)k_elim},
      {"k_lqr_up", (const void *)k_lqr_up}, {"k_lqr_level", (const void *)k_lqr_level},
      {"k_riccati_down", (const void *)k_riccati_down}, {"k_riccati_finish", (const void *)k_riccati_finish},
      {"k_aff_up", (const void *)k_aff_up},
      {"k_aff_level", (const void *)k_aff_level}, {"k_aff_down", (const void *)k_aff_down},
      {"k_aff_prep", (const void *)k_aff_prep},
      {"k_solve_init", (const void *)k_solve_init}, {"k_post_roll", (const void *)k_post_roll},
      {"k_resid", (const void *)k_resid}, {"k_pcorr", (const void *)k_pcorr},
      {"k_recover", (const void *)k_recover}, {"k_dual_stage", (const void *)k_dual_stage},
      {"k_dual_terminal", (const void *)k_dual_terminal}, {"k_dual_up", (const void *)k_dual_up},
      {"k_dual_down", (const void *)k_dual_down}, {"k_dual_root", (const void *)k_dual_root},
      {"k_dual_leaf", (const void *)k_dual_leaf}, {"k_kkt", (const void *)k_kkt},
      {"k_param_grads", (const void *)k_param_grads}, {"k_set_costs", (const void *)k_set_costs},
      {"k_check_inputs", (const void *)k_check_inputs}, {"k_refine_prep", (const void *)k_refine_prep},
      {"k_refine_gate", (const void *)k_refine_gate}, {"k_refine_trial", (const void *)k_refine_trial},
      {"k_refine_accept", (const void *)k_refine_accept}, {"k_refine_post", (const void *)k_refine_post},
      {"k_refine_parts", (const void *)k_refine_parts}, {"k_rescue_prep", (const void *)k_rescue_prep},
      {"k_riccati_down_f32", (const void *)k_riccati_down_f32}};
  for (const auto &e : table)
    if (std::strcmp(e.name, name) == 0) {
      if (h->ev.empty()) {
        h->ev.resize(2 * 4096);
        for (auto &x : h->ev)
          if (cudaEventCreate(&x) != cudaSuccess) return ECLQR_ECUDA;
      }
      h->timed = e.fn;
      return ECLQR_OK;
    }
  return ECLQR_EINVAL;
}

int eclqr_kernel_time(eclqr_handle *h, int64_t *launches, double *total_ms) {
  if (!h || !launches || !total_ms) return ECLQR_EINVAL;
  double t = 0.0;
  for (int k = 0; k + 1 < h->nev; k += 2) {
    float ms = 0.f;
    if (cudaEventSynchronize(h->ev[k + 1]) != cudaSuccess) return ECLQR_ECUDA;
    if (cudaEventElapsedTime(&ms, h->ev[k], h->ev[k + 1]) != cudaSuccess) return ECLQR_ECUDA;
    t += ms;
  }
  *launches = h->nev / 2;
  *total_ms = t;
  return ECLQR_OK;
}

const char *eclqr_strerror(int code) {
  switch (code) {
    case ECLQR_OK: return "ok";
    case ECLQR_EINVAL: return "invalid argument";
    case ECLQR_ENOMEM: return "device allocation failed";
    case ECLQR_ECUDA: return "CUDA error";
    case ECLQR_ESTATE: return "call out of order";
    case ECLQR_ETOOBIG: return "batch exceeds the fixed array of eclqr_kkt_residual_noalloc";
    case ECLQR_ESMEM: return "dimensions need more shared memory per task than a CTA can hold";
    default: return "unknown error";
  }
}

}  // extern "C"
