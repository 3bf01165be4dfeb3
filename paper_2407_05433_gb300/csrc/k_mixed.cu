// k_mixed.cu -- the square-root Riccati sweep in FP32 (mixed-precision mode).
//
// Same recursion as k_riccati_down (Sec. 6, square-root cost rows; the stage
// factor L' upper triangular in the QR's column order (v, z)), with every
// product, reflector and triangular solve in FP32 and the stored factors (P, p,
// K, k, chol(H_uu), Phi) widened to FP64.  The rank-revealing parts of the
// method -- the domain scan, the null-space bases T, Z, the particular solutions
// t, y and every rank decision -- stay FP64 in the other kernels.  The factors
// carry FP32 rounding; the rollout, the reduced refinement and the refinement on
// the original KKT residual run in FP64 through the original data, so their
// fixed point is the FP64 solution wherever the iteration contracts, and
// eclqr_refine redoes in FP64 the problems where it does not.
//
// A problem takes this kernel when the group's fp64 flags say so (flag 0); the
// FP64 kernel takes the others.  On this GPU an FP32 warp instruction costs the
// pipe about one sixty-fourth of an FP64 one, and its dependent latency is a
// few cycles instead of about 65.
#include "kernels.cuh"

namespace eclqr {

__device__ __forceinline__ bool riccati_fp32(const Group &g, int prob) {
  return g.fp64 != nullptr && g.fp64[g.prob[prob].id] == 0;
}

// One Householder step in FP32 on rows [0, r) of W (ld) for column k, applied
// to columns [k, c): column k becomes (-sign(x) |x|, 0, ..., 0).  Every thread
// forms the pivot column's norm itself (r FP32 FMAs), so the dot products, the
// reflector vector v (scratch of r floats) and the coefficients wj (scratch of
// c floats) come out of one pass, and the update of all columns, column k
// included, out of a second: two barriers.  Called by the whole team.
__device__ void hh_step_f32(float *W, int ld, int r, int k, int c, float *v, float *wj) {
  const int tid = team_rank();
  float dp = 0.f;
  for (int i = 0; i < r; i++) dp = fmaf(W[i * ld + k], W[i * ld + k], dp);
  const float xk = W[k];
  if (!(dp > 0.f)) return;  // uniform
  const float nrm = sqrtf(dp);
  const float shift = (xk >= 0.f) ? nrm : -nrm;
  const float vk = xk + shift;
  const float beta = 1.f / (nrm * (nrm + fabsf(xk)));
  // w_j = beta v'W_j = beta (x'W_j + shift W_0j)
  for (int j = k + 1 + tid; j < c; j += TEAM) {
    float acc = 0.f;
    for (int i = 0; i < r; i++) acc = fmaf(W[i * ld + k], W[i * ld + j], acc);
    wj[j] = beta * fmaf(shift, W[j], acc);
  }
  for (int i = tid; i < r; i += TEAM) v[i] = (i == 0) ? vk : W[i * ld + k];
  tsync();
  const int nc = c - k;
  for (int idx = tid; idx < r * nc; idx += TEAM) {
    const int i = idx / nc, j = k + (idx - i * nc);
    W[i * ld + j] = (j == k) ? ((i == 0) ? -shift : 0.f) : fmaf(-wj[j], v[i], W[i * ld + j]);
  }
  tsync();
}

__global__ void k_riccati_down_f32(Group g, int fin, int per_task) {
  const int t = team_task();
  if (t >= g.nslot) return;
  const ChunkInfo ci = g.chunk[t];
  const ProbInfo &P = g.prob[ci.prob];
  if (skipped_by_mask(g, ci.prob)) return;
  if (!riccati_fp32(g, ci.prob)) return;
  if (ci.c >= P.nch) return;
  const int n = g.n, m = g.m, tid = team_rank();
  const int a = ci.c * P.L, b = min(a + P.L, P.N);
  const bool resweep = ci.c + 1 < P.nch;
  const int start = resweep ? min(b + P.L, P.N) : b;
  const int ldr = 2 * n + 1;
  float *sm = (float *)team_smem(per_task);
  const int rows_max = 2 * n + m, ldst = n + m + 1;
  float *V = sm, *St = V + n * (n + 1), *v = St + rows_max * ldst, *wj = v + rows_max;
  float *Kt = wj + ldst;          // m x (n + 1)
  float *Af = Kt + m * (n + 1);   // stage data converted once per stage: Abar (n1 x nx, ld n),
  float *Bf = Af + n * n;         // Bbar (n1 x mu, ld m), cbar (n1)
  float *cf = Bf + n * m;
  int rv;
  {
    const int slot = resweep ? t + 2 : t + 1;
    const double *src = g.CS[fin] + (size_t)slot * g.cs_stride + 2 * n * ldr;  // cost rows of the slot
    const int *I = g.CI[fin] + (size_t)slot * CI_STRIDE;
    const int nbz = I[CI_NA];
    rv = I[CI_ROWS2];
    for (int idx = tid; idx < rv * (nbz + 1); idx += TEAM) {
      int r = idx / (nbz + 1), j = idx - r * (nbz + 1);
      const double sg = (src[r * ldr + r] >= 0.0) ? 1.0 : -1.0;
      V[r * (n + 1) + j] = (float)(sg * src[r * ldr + j]);
    }
    tsync();
    if (b == P.N) {  // P_N = C'C, p_N = C'c
      double *wsN = stage_ws(g, P.st0 + b);
      for (int idx = tid; idx < nbz * (nbz + 1); idx += TEAM) {
        int r = idx / (nbz + 1), j = idx - r * (nbz + 1);
        float s0 = 0.f;
        for (int l = 0; l < rv; l++) s0 = fmaf(V[l * (n + 1) + r], V[l * (n + 1) + j], s0);
        if (j < nbz) wsN[g.ws.P + r * n + j] = s0; else wsN[g.ws.p + r] = s0;
      }
    }
  }
  for (int i = start - 1; i >= a; --i) {
    const bool store = i < b;
    const int s = P.st0 + i;
    double *ws = stage_ws(g, s);
    const int *wi = stage_wi(g, s);
    const int nx = wi[SI_NBAR], mu = wi[SI_MBAR], n1 = stage_wi(g, s + 1)[SI_NBAR];
    const int kh = nx + mu, ld = kh + 1;
    const double *Ab = ws + g.ws.Ab, *Bb = ws + g.ws.Bb, *cb = ws + g.ws.cb, *LT = ws + g.ws.LT, *lt = ws + g.ws.lt;
    for (int idx = tid; idx < n1 * nx; idx += TEAM) {
      int r = idx / nx, c = idx - r * nx;
      Af[r * n + c] = (float)Ab[r * n + c];
    }
    for (int idx = tid; idx < n1 * mu; idx += TEAM) {
      int r = idx / mu, c = idx - r * mu;
      Bf[r * m + c] = (float)Bb[r * m + c];
    }
    for (int r = tid; r < n1; r += TEAM) cf[r] = (float)cb[r];
    tsync();
    // value rows [V Bbar | V Abar | V cbar + s] at St rows kh .. kh + rv - 1
    for (int idx = tid; idx < rv * ld; idx += TEAM) {
      int r = idx / ld, j = idx - r * ld;
      const float *row = V + r * (n + 1);
      float val = 0.f;
      if (j < mu) {
        for (int l = 0; l < n1; l++) val = fmaf(row[l], Bf[l * m + j], val);
      } else if (j < kh) {
        for (int l = 0; l < n1; l++) val = fmaf(row[l], Af[l * n + (j - mu)], val);
      } else {
        val = row[n1];
        for (int l = 0; l < n1; l++) val = fmaf(row[l], cf[l], val);
      }
      St[(kh + r) * ld + j] = val;
    }
    // QR of [L' l; value rows], L' upper triangular: step k on row k of L' and the value rows
    // next row of L' prefetched into registers while the current step runs (kh + 1 <= 2 TEAM)
    float nxt[2];
    for (int q = 0; q < 2; q++) {
      const int j = tid + q * TEAM;
      nxt[q] = (j <= kh && kh > 0) ? (float)((j < kh) ? LT[j] : lt[0]) : 0.f;
    }
    for (int k = 0; k < kh; k++) {
      float *W = St + (kh - 1) * ld;
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
          if (j >= k + 1 && j <= kh) nxt[q] = (float)((j < kh) ? LT[(k + 1) * (n + m) + j] : lt[k + 1]);
        }
      hh_step_f32(W, ld, rv + 1, k, kh + 1, v, wj);
    }
    for (int idx = tid; idx < nx * ld; idx += TEAM) {
      int r = mu + idx / ld, j = idx % ld;
      if (St[r * ld + r] < 0.f && j != r) St[r * ld + j] = -St[r * ld + j];
    }
    tsync();
    for (int r = mu + tid; r < kh; r += TEAM) St[r * ld + r] = fabsf(St[r * ld + r]);
    tsync();
    // K, k:  R_vv [K | k] = -[R_vz | o_v]
    for (int c = tid; c <= nx; c += TEAM) {
      for (int r = mu - 1; r >= 0; r--) {
        float s0 = -St[r * ld + mu + c];
        for (int l = r + 1; l < mu; l++) s0 = fmaf(-St[r * ld + l], Kt[l * (n + 1) + c], s0);
        Kt[r * (n + 1) + c] = s0 / St[r * ld + r];
      }
    }
    tsync();
    if (store) {
      for (int idx = tid; idx < mu * (nx + 1); idx += TEAM) {
        int r = idx / (nx + 1), c = idx - r * (nx + 1);
        if (c < nx) ws[g.ws.K + r * n + c] = Kt[r * (n + 1) + c]; else ws[g.ws.k + r] = Kt[r * (n + 1) + c];
      }
      for (int idx = tid; idx < mu * mu; idx += TEAM) {
        int r = idx / mu, j = idx - r * mu;
        float sg = St[j * ld + j] >= 0.f ? 1.f : -1.f;
        ws[g.ws.Lh + r * m + j] = (j <= r) ? sg * St[j * ld + r] : 0.0;
      }
      for (int idx = tid; idx < n1 * nx; idx += TEAM) {
        int r = idx / nx, c = idx - r * nx;
        float s0 = Af[r * n + c];
        for (int l = 0; l < mu; l++) s0 = fmaf(Bf[r * m + l], Kt[l * (n + 1) + c], s0);
        ws[g.ws.Phi + r * n + c] = s0;
      }
    }
    tsync();
    for (int idx = tid; idx < nx * (nx + 1); idx += TEAM) {
      int r = idx / (nx + 1), c = idx - r * (nx + 1);
      V[r * (n + 1) + c] = (c < nx) ? ((c >= r) ? St[(mu + r) * ld + mu + c] : 0.f) : St[(mu + r) * ld + kh];
    }
    tsync();
    rv = nx;
    for (int idx = tid; idx < nx * (nx + 1); idx += TEAM) {
      int r = idx / (nx + 1), c = idx - r * (nx + 1);
      float s0 = 0.f;
      for (int l = 0; l <= r && l < nx; l++) s0 = fmaf(V[l * (n + 1) + r], V[l * (n + 1) + c], s0);
      if (!store) continue;
      if (c < nx) ws[g.ws.P + r * n + c] = s0; else ws[g.ws.p + r] = s0;
    }
    tsync();
  }
}

}  // namespace eclqr
