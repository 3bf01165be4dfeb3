// noalloc.cu -- eclqr_kkt_residual_noalloc: the KKT residual of
// eclqr_kkt_residual for callers that cannot allocate device memory.
//
// The residual kernel reads per-problem and per-stage descriptors (offsets of
// every block in the packed arrays).  The handle-based path keeps them in the
// workspace eclqr_create allocates; here they live in one fixed device array
// declared below, filled from a fixed host staging array of the same size, so
// the call performs no cudaMalloc, cudaFree or other allocation.
#include <cuda_runtime.h>

#include <cstring>

#include "../../include/eclqr.h"
#include "kernels.cuh"

using namespace eclqr;

namespace {

constexpr size_t kProbBytes = sizeof(ProbInfo) * ECLQR_NOALLOC_MAX_PROBLEMS;
constexpr size_t kScratchBytes = kProbBytes + sizeof(StageInfo) * ECLQR_NOALLOC_MAX_STAGES;

// The scratch: every GPU that loads the library holds these bytes until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// host staging copy of the descriptors (static: no host heap either)
static unsigned char h_noalloc_stage[kScratchBytes];

// device address of g_noalloc_scratch, looked up once per device
constexpr int kMaxDevices = 64;
static void *d_noalloc_scratch[kMaxDevices];

}  // namespace

extern "C" int eclqr_kkt_residual_noalloc(const eclqr_desc *d, const eclqr_data *data, const double *s0,
                                          const double *x, const double *u, const double *lam, const double *mu,
                                          const double *eta, const double *alpha, double *resid, void *stream) {
  if (!d || !data || !s0 || !x || !u || !lam || !alpha || !resid) return ECLQR_EINVAL;
  eclqr_layout_info lay;
  int rc = eclqr_layout(d, &lay);
  if (rc != ECLQR_OK) return rc;
  if (lay.mu > 0 && !mu) return ECLQR_EINVAL;
  if (lay.eta > 0 && !eta) return ECLQR_EINVAL;
  const int P = d->num_problems;
  if (P > ECLQR_NOALLOC_MAX_PROBLEMS || lay.stages + P > ECLQR_NOALLOC_MAX_STAGES) return ECLQR_ETOOBIG;
  cudaStream_t st = (cudaStream_t)stream;
  // the descriptors reach the device by a copy from the host staging array, which
  // the next call rewrites: a captured copy would replay whatever it then holds
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return ECLQR_ECUDA;
  if (cap != cudaStreamCaptureStatusNone) return ECLQR_ESTATE;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ECLQR_ECUDA;
  if (!d_noalloc_scratch[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return ECLQR_ECUDA;
    d_noalloc_scratch[dev] = p;
  }
  unsigned char *dbase = (unsigned char *)d_noalloc_scratch[dev];
  if (cudaMemsetAsync(resid, 0, sizeof(double) * P, st) != cudaSuccess) return ECLQR_ECUDA;

  // descriptors: all problems, then their stages grouped by (n, m) as the kernel expects
  ProbInfo *hp = (ProbInfo *)h_noalloc_stage;
  StageInfo *hs = (StageInfo *)(h_noalloc_stage + kProbBytes);
  long long oA = 0, oB = 0, oc = 0, oC = 0, oD = 0, od = 0, oE = 0, oe = 0, oQ = 0, oM = 0, oR = 0, oqv = 0, orv = 0,
            os0 = 0, ox = 0, ou = 0, olam = 0, omu = 0, oeta = 0, oal = 0, ps = 0, qs = 0;
  for (int j = 0; j < P; j++) {
    const long long N = d->N[j], n = d->n[j], m = d->m[j];
    long long Pj = 0, Qj = 0;
    for (long long i = 0; i < N; i++) Pj += d->p[ps + i];
    for (long long i = 0; i <= N; i++) Qj += d->q[qs + i];
    ProbInfo &pi = hp[j];
    std::memset(&pi, 0, sizeof(pi));
    pi.N = (int)N;
    pi.id = j;
    pi.oA = oA; pi.oB = oB; pi.oc = oc; pi.oC = oC; pi.oD = oD; pi.od = od; pi.oE = oE; pi.oe = oe;
    pi.oQ = oQ; pi.oM = oM; pi.oR = oR; pi.oqv = oqv; pi.orv = orv;
    pi.os0 = os0; pi.ox = ox; pi.ou = ou; pi.olam = olam; pi.omu = omu; pi.oeta = oeta; pi.oalpha = oal;
    pi.ost = qs;
    oA += N * n * n; oB += N * n * m; oc += N * n; oC += Pj * n; oD += Pj * m; od += Pj; oE += Qj * n; oe += Qj;
    oQ += (N + 1) * n * n; oM += N * n * m; oR += N * m * m; oqv += (N + 1) * n; orv += N * m;
    os0 += n; ox += (N + 1) * n; ou += N * m; olam += (N + 1) * n; omu += Pj; oeta += Qj; oal += n;
    ps += N;
    qs += N + 1;
  }
  // one launch per distinct (n, m); each group's stage records occupy their own range
  long long sbase = 0;
  struct Launch { int n, m; long long s0, ns; } launches[ECLQR_MAX_N * ECLQR_MAX_M];
  int nl = 0;
  for (int j0 = 0; j0 < P; j0++) {
    bool seen = false;
    for (int j = 0; j < j0 && !seen; j++) seen = d->n[j] == d->n[j0] && d->m[j] == d->m[j0];
    if (seen) continue;
    const long long start = sbase;
    long long qoff = 0, poff = 0;
    for (int j = 0; j < P; j++) {
      const int N = d->N[j];
      if (d->n[j] == d->n[j0] && d->m[j] == d->m[j0]) {
        int prow = 0, qrow = 0;
        for (int i = 0; i <= N; i++) {
          StageInfo &si = hs[sbase++];
          si.prob = j;
          si.i = i;
          si.p = (i < N) ? d->p[poff + i] : 0;
          si.q = d->q[qoff + i];
          si.prow = prow;
          si.qrow = qrow;
          prow += si.p;
          qrow += si.q;
        }
      }
      poff += N;
      qoff += N + 1;
    }
    launches[nl++] = Launch{d->n[j0], d->m[j0], start, sbase - start};
  }
  // pageable copies: each returns once the staging array has been read, so the
  // next call may overwrite it; the device array is shared by every call
  if (cudaMemcpyAsync(dbase, h_noalloc_stage, sizeof(ProbInfo) * (size_t)P, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return ECLQR_ECUDA;
  if (cudaMemcpyAsync(dbase + kProbBytes, h_noalloc_stage + kProbBytes, sizeof(StageInfo) * (size_t)sbase,
                      cudaMemcpyHostToDevice, st) != cudaSuccess)
    return ECLQR_ECUDA;
  for (int k = 0; k < nl; k++) {
    Group g;
    std::memset(&g, 0, sizeof(g));
    g.n = launches[k].n;
    g.m = launches[k].m;
    g.nprob = P;
    g.nstage = (int)launches[k].ns;
    g.prob = (const ProbInfo *)dbase;
    g.st = (const StageInfo *)(dbase + kProbBytes) + launches[k].s0;
    g.A = data->A; g.B = data->B; g.c = data->c; g.C = data->C; g.D = data->D; g.d = data->d;
    g.E = data->E; g.e = data->e; g.Q = data->Q; g.M = data->M; g.R = data->R; g.qv = data->qv; g.rv = data->rv;
    k_kkt<<<g.nstage, 128, 0, st>>>(g, s0, x, u, lam, mu, eta, alpha, KktRows{}, resid, nullptr);
    if (cudaPeekAtLastError() != cudaSuccess) return ECLQR_ECUDA;
  }
  return ECLQR_OK;
}
