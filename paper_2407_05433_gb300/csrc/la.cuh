// la.cuh -- FP64 dense linear algebra on small matrices held in shared
// memory, executed by a team: all threads of one CTA work on one task.  Every
// routine is called by the whole team, converged; matrices are row-major with
// explicit leading dimensions.
//
// Cost model on sm_103a: an FP64 instruction occupies its SM sub-partition's
// FP64 pipe for the whole warp whatever its active mask, and each of the four
// sub-partitions has its own pipe.  A team of four warps therefore has four
// times the FP64 issue rate of one warp; loops hand each thread an independent
// output element (element-parallel updates, thread-per-column dot products)
// instead of reducing across threads wherever possible.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace eclqr {

constexpr unsigned kFull = 0xffffffffu;

// rank of the calling thread in its team, the team size, and the team barrier
__device__ __forceinline__ int team_rank() { return threadIdx.x; }
#define TEAM ((int)blockDim.x)
__device__ __forceinline__ void tsync() { __syncthreads(); }

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// arg-max over non-negative values; ties resolve to the lowest index.  The
// bit pattern of a non-negative double orders like the value, so the
// comparison runs on the integer pipe.
__device__ __forceinline__ void warp_argmax(long long &key, int &idx) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    long long k2 = __shfl_xor_sync(kFull, key, o);
    int i2 = __shfl_xor_sync(kFull, idx, o);
    if (k2 > key || (k2 == key && i2 < idx)) { key = k2; idx = i2; }
  }
}

// Team reductions: warp shuffles, then one partial per warp through shared
// memory.  The trailing barrier lets the next reduction reuse the slots.
__device__ __forceinline__ double team_max(double v) {
  __shared__ double red_max[32];
  v = warp_max(v);
  if ((threadIdx.x & 31) == 0) red_max[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = red_max[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); w++) r = fmax(r, red_max[w]);
  __syncthreads();
  return r;
}

__device__ __forceinline__ double team_sum(double v) {
  __shared__ double red_sum[32];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red_sum[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = red_sum[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); w++) r += red_sum[w];
  __syncthreads();
  return r;
}

__device__ __forceinline__ void team_argmax(double v, int idx, double &bv, int &bi) {
  __shared__ long long red_key[32];
  __shared__ int red_idx[32];
  long long key = __double_as_longlong(v);
  warp_argmax(key, idx);
  if ((threadIdx.x & 31) == 0) {
    red_key[threadIdx.x >> 5] = key;
    red_idx[threadIdx.x >> 5] = idx;
  }
  __syncthreads();
  key = red_key[0];
  idx = red_idx[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); w++) {
    const long long k2 = red_key[w];
    const int i2 = red_idx[w];
    if (k2 > key || (k2 == key && i2 < idx)) { key = k2; idx = i2; }
  }
  __syncthreads();
  bv = __longlong_as_double(key);
  bi = idx;
}

__device__ __forceinline__ void wzero(double *p, int n) {
  for (int i = team_rank(); i < n; i += TEAM) p[i] = 0.0;
  tsync();
}

__device__ __forceinline__ void wcopy(double *dst, int ldd, const double *src, int lds, int rows,
                                      int cols) {
  for (int idx = team_rank(); idx < rows * cols; idx += TEAM) {
    int i = idx / cols, j = idx - i * cols;
    dst[i * ldd + j] = src[i * lds + j];
  }
  tsync();
}

// C (m x n) = alpha * op(A) op(B) + beta * C; op(A) is m x k, op(B) is k x n.
// C must not alias A or B.
template <bool TA, bool TB>
static __device__ void wgemm(int m, int n, int k, double alpha, const double *A, int lda, const double *B,
                      int ldb, double beta, double *C, int ldc) {
  for (int idx = team_rank(); idx < m * n; idx += TEAM) {
    int i = idx / n, j = idx - i * n;
    double s0 = 0.0, s1 = 0.0;
    int l = 0;
    for (; l + 1 < k; l += 2) {
      double a0 = TA ? A[l * lda + i] : A[i * lda + l];
      double a1 = TA ? A[(l + 1) * lda + i] : A[i * lda + l + 1];
      double b0 = TB ? B[j * ldb + l] : B[l * ldb + j];
      double b1 = TB ? B[j * ldb + l + 1] : B[(l + 1) * ldb + j];
      s0 = fma(a0, b0, s0);
      s1 = fma(a1, b1, s1);
    }
    if (l < k) {
      double a0 = TA ? A[l * lda + i] : A[i * lda + l];
      double b0 = TB ? B[j * ldb + l] : B[l * ldb + j];
      s0 = fma(a0, b0, s0);
    }
    double s = alpha * (s0 + s1);
    C[i * ldc + j] = (beta == 0.0) ? s : fma(beta, C[i * ldc + j], s);
  }
  tsync();
}

// ---------------------------------------------------------------------------
// Householder core shared by the factorizations below.
//
// Per-CTA static scratch: one partial dot product per thread, and for column
// pivoting the running squared norms of the candidate columns with their
// values at the last exact evaluation.  Sized for teams of up to kMaxTeam
// threads and matrices of up to kMaxCols columns (the header's dimension
// limits keep every factored matrix below 3 * 32 + 64 + 1 columns).
// ---------------------------------------------------------------------------
constexpr int kMaxTeam = 256;
constexpr int kMaxCols = 192;
__device__ __forceinline__ double *hh_part() {
  __shared__ double part[kMaxTeam];
  return part;
}
__device__ __forceinline__ double *hh_norms() {
  __shared__ double norms[2 * kMaxCols];
  return norms;
}

// Reflector H = I - beta v v' from column piv on rows [r0, r1) (nrm = the
// column's 2-norm there, > 0), applied to the columns of [c0, c1) that are not
// done and are not piv; column piv becomes (-sign(x_k) nrm, 0, ..., 0).  v
// (indexed by row) keeps the reflector, beta = 1 / (nrm |v[r0]|).  The dot
// products v'M_j are split over the team by column and by row segment, so a
// column of R rows costs about R * columns / TEAM FMAs per thread.
static __device__ void whouse_apply(double *M, int ld, int r0, int r1, int piv, int c0, int c1, const int *done,
                                    double *v, double *w, double nrm) {
  const int tid = team_rank(), T = TEAM;
  double *part = hh_part();
  const double xk = M[r0 * ld + piv];
  const double sg = xk >= 0.0 ? 1.0 : -1.0;
  for (int i = r0 + tid; i < r1; i += T) v[i] = (i == r0) ? xk + sg * nrm : M[i * ld + piv];
  const double beta = 1.0 / (nrm * (nrm + fabs(xk)));
  tsync();
  const int nc = c1 - c0, nr = r1 - r0;
  // thread -> (column c0 + jj, row segment sgm): rows r0 + sgm, r0 + sgm + S, ...
  // S * nc <= T when S > 1; with S == 1 threads step over columns
  const int S = max(1, min(nc > 0 ? T / nc : 1, nr));
  const int jj0 = (S > 1) ? tid % nc : tid, sgm = (S > 1) ? tid / nc : 0;
  const bool seg_ok = sgm < S;
  for (int jj = jj0; seg_ok && jj < nc; jj += (S > 1 ? nc : T)) {
    const int j = c0 + jj;
    double acc = 0.0;
    if (!((done && done[j]) || j == piv))
      for (int i = r0 + sgm; i < r1; i += S) acc = fma(v[i], M[i * ld + j], acc);
    if (S == 1) w[j] = beta * acc;
    else part[sgm * nc + jj] = acc;
  }
  tsync();
  if (S > 1) {
    for (int j2 = tid; j2 < nc; j2 += T) {
      double acc = part[j2];
      for (int k2 = 1; k2 < S; k2++) acc += part[k2 * nc + j2];
      w[c0 + j2] = beta * acc;
    }
    tsync();
  }
  for (int jj = jj0; seg_ok && jj < nc; jj += (S > 1 ? nc : T)) {
    const int j = c0 + jj;
    if ((done && done[j]) || j == piv) continue;
    const double wj = w[j];
    for (int i = r0 + sgm; i < r1; i += S) M[i * ld + j] = fma(-wj, v[i], M[i * ld + j]);
  }
  tsync();
  for (int i = r0 + tid; i < r1; i += T) M[i * ld + piv] = (i == r0) ? -sg * nrm : 0.0;
  tsync();
}

__device__ __forceinline__ double *hh_rowk() {
  __shared__ double rowk[kMaxCols];
  return rowk;
}

// One fused Householder step on rows [k, r) with pivot column piv in [a0, a1):
// one pass over the rows gives the raw products d_j = M_piv . M_j for the
// not-done columns of [a0, a1) together with d_piv = ||M_piv||^2.  If
// sqrt(d_piv) <= thr, M is left untouched and 0 is returned; otherwise the
// reflector (v = M_piv + sign(x_k) ||M_piv|| e_k) is applied to those columns,
// column piv becomes (-sign(x_k) ||M_piv||, 0, ..., 0), done[piv] is set when
// done is given, and the norm is returned.  Scratch: v (rows), d (columns).
// Each column's row segments sit on neighbouring lanes of one warp, so their
// partial products combine by shuffles.
static __device__ double hh_step(double *M, int ld, int k, int r, int piv, int a0, int a1, int *done, double *v,
                                 double *d, double thr) {
  const int tid = team_rank(), T = TEAM;
  double *mk = hh_rowk();
  const int nc = a1 - a0, nr = r - k;
  // S row segments per column, a power of two within a warp; thread -> (column a0 + jj, segment sgm)
  int S = 1;
  while (2 * S <= 32 && 2 * S * nc <= T && 2 * S <= nr) S *= 2;
  const int jj0 = (S > 1) ? tid / S : tid, sgm = (S > 1) ? (tid & (S - 1)) : 0;
  const int jstep = (S > 1) ? T : T;   // S > 1: one column per thread group (S * nc <= T)
  for (int i = k + tid; i < r; i += T) v[i] = M[i * ld + piv];
  for (int jj = tid; jj < nc; jj += T) mk[jj] = M[k * ld + a0 + jj];
  if (S > 1) {
    double acc = 0.0;
    const int j = a0 + jj0;
    if (jj0 < nc && (j == piv || !(done && done[j])))
      for (int i = k + sgm; i < r; i += S) acc = fma(M[i * ld + piv], M[i * ld + j], acc);
    for (int o = S >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o, S);
    if (jj0 < nc && sgm == 0) d[j] = acc;
  } else {
    for (int jj = jj0; jj < nc; jj += jstep) {
      const int j = a0 + jj;
      double acc = 0.0;
      if (j == piv || !(done && done[j]))
        for (int i = k; i < r; i++) acc = fma(M[i * ld + piv], M[i * ld + j], acc);
      d[j] = acc;
    }
  }
  tsync();
  const double nrm = sqrt(d[piv]);
  if (!(nrm > thr)) return 0.0;
  const double xk = v[k];
  const double sg = xk >= 0.0 ? 1.0 : -1.0;
  const double shift = sg * nrm;                 // v_k - x_k
  const double beta = 1.0 / (nrm * (nrm + fabs(xk)));
  for (int jj = jj0; jj < nc; jj += (S > 1 ? T : jstep)) {
    if (S > 1 && jj != jj0) break;
    const int j = a0 + jj;
    if (j == piv) {
      for (int i = k + sgm; i < r; i += S) M[i * ld + piv] = (i == k) ? -shift : 0.0;
      if (sgm == 0 && done) done[piv] = 1;
      continue;
    }
    if (done && done[j]) continue;
    const double wj = beta * fma(shift, mk[jj], d[j]);
    for (int i = k + sgm; i < r; i += S) {
      const double vi = (i == k) ? xk + shift : v[i];
      M[i * ld + j] = fma(-wj, vi, M[i * ld + j]);
    }
  }
  tsync();
  return nrm;
}

// Team arg-max with one barrier: partials alternate between two buffers by
// parity, so consecutive uses of one buffer must be separated by at least one
// other barrier.  Ties go to the smaller index.
__device__ __forceinline__ unsigned long long *argmax_keys() {
  __shared__ unsigned long long rk[2][32];
  return &rk[0][0];
}
__device__ __forceinline__ int *argmax_idx() {
  __shared__ int ri[2][32];
  return &ri[0][0];
}

// Warp stage of the arg-max: lane 0 leaves (key, index) of the warp's best in
// the parity buffer.  The key of a non-negative double orders like (high
// word, low word), so the reduction runs on the integer pipe.
__device__ __forceinline__ void warp_argmax_partial(double val, int idx, int parity) {
  const unsigned long long key = (unsigned long long)__double_as_longlong(val);
  const unsigned hi = (unsigned)(key >> 32), lo = (unsigned)key;
  const unsigned mhi = __reduce_max_sync(kFull, hi);
  const unsigned mlo = __reduce_max_sync(kFull, hi == mhi ? lo : 0u);
  const int widx = __reduce_min_sync(kFull, (hi == mhi && lo == mlo) ? idx : 0x7fffffff);
  if ((threadIdx.x & 31) == 0) {
    argmax_keys()[parity * 32 + (threadIdx.x >> 5)] = ((unsigned long long)mhi << 32) | mlo;
    argmax_idx()[parity * 32 + (threadIdx.x >> 5)] = widx;
  }
}

// Team stage: every thread reduces the warps' partials (after a barrier).
__device__ __forceinline__ void argmax_finish(int parity, double &bv, int &bi) {
  unsigned long long best = argmax_keys()[parity * 32];
  int besti = argmax_idx()[parity * 32];
  for (int w = 1; w < (int)(blockDim.x >> 5); w++) {
    const unsigned long long k2 = argmax_keys()[parity * 32 + w];
    const int i2 = argmax_idx()[parity * 32 + w];
    if (k2 > best || (k2 == best && i2 < besti)) { best = k2; besti = i2; }
  }
  bv = __longlong_as_double((long long)best);
  bi = besti;
}

__device__ __forceinline__ void team_argmax1(double val, int idx, int parity, double &bv, int &bi) {
  warp_argmax_partial(val, idx, parity);
  __syncthreads();
  argmax_finish(parity, bv, bi);
}

// The pivoted form of hh_step: the update pass also downdates the remaining
// norms of the candidate columns (re-evaluating a marked one from its rows,
// which sit on the same warp) and leaves each warp's best candidate in the
// arg-max buffer `parity`, so that the next pivot is known after the pass's
// own barrier.  Returns the norm, or 0 (M untouched) when it does not exceed thr.
static __device__ double hh_pivot_step(double *M, int ld, int k, int r, int piv, int a0, int a1, int *done,
                                       double *v, double *d, double thr, double *cn, double *cref, int cand0,
                                       int cand1, int parity) {
  const int tid = team_rank(), T = TEAM;
  double *mk = hh_rowk();
  const int nc = a1 - a0, nr = r - k;
  int S = 1;
  while (2 * S <= 32 && 2 * S * nc <= T && 2 * S <= nr) S *= 2;
  const int jj0 = (S > 1) ? tid / S : tid, sgm = (S > 1) ? (tid & (S - 1)) : 0;
  for (int i = k + tid; i < r; i += T) v[i] = M[i * ld + piv];
  for (int jj = tid; jj < nc; jj += T) mk[jj] = M[k * ld + a0 + jj];
  if (S > 1) {
    double acc = 0.0;
    const int j = a0 + jj0;
    if (jj0 < nc && (j == piv || !done[j]))
      for (int i = k + sgm; i < r; i += S) acc = fma(M[i * ld + piv], M[i * ld + j], acc);
    for (int o = S >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o, S);
    if (jj0 < nc && sgm == 0) d[j] = acc;
  } else {
    for (int jj = jj0; jj < nc; jj += T) {
      const int j = a0 + jj;
      double acc = 0.0;
      if (j == piv || !done[j])
        for (int i = k; i < r; i++) acc = fma(M[i * ld + piv], M[i * ld + j], acc);
      d[j] = acc;
    }
  }
  tsync();
  const double nrm = sqrt(d[piv]);
  if (!(nrm > thr)) return 0.0;
  const double xk = v[k];
  const double sg = xk >= 0.0 ? 1.0 : -1.0;
  const double shift = sg * nrm;
  const double beta = 1.0 / (nrm * (nrm + fabs(xk)));
  for (int jj = jj0; jj < nc && (S == 1 || jj == jj0); jj += T) {
    const int j = a0 + jj;
    if (j == piv) {
      for (int i = k + sgm; i < r; i += S) M[i * ld + piv] = (i == k) ? -shift : 0.0;
      if (sgm == 0) done[piv] = 1;
      continue;
    }
    if (done[j]) continue;
    const double wj = beta * fma(shift, mk[jj], d[j]);
    for (int i = k + sgm; i < r; i += S) {
      const double vi = (i == k) ? xk + shift : v[i];
      M[i * ld + j] = fma(-wj, vi, M[i * ld + j]);
    }
  }
  __syncwarp();  // a column's row segments are lanes of one warp
  double best = -1.0;
  int bidx = 0x7fffffff;
  for (int jj = jj0; jj < nc && (S == 1 || jj == jj0); jj += T) {
    const int j = a0 + jj;
    if (sgm != 0 || j == piv || j < cand0 || j >= cand1 || done[j]) continue;
    const double a = M[k * ld + j];
    double nw = cn[j] - a * a;
    if (nw <= 0x1p-26 * cref[j]) {
      nw = 0.0;
      for (int i = k + 1; i < r; i++) nw = fma(M[i * ld + j], M[i * ld + j], nw);
      cref[j] = nw;
    }
    cn[j] = nw;
    if (nw > best) { best = nw; bidx = j; }
  }
  warp_argmax_partial(best < 0.0 ? 0.0 : best, best < 0.0 ? 0x7fffffff : bidx, parity);
  tsync();
  return nrm;
}

// Column-pivoted Householder steps on rows [k, r).  Each step takes the
// candidate column (in [cand0, cand1), not done) of largest remaining norm;
// while its exact norm exceeds thr, its reflector is applied to the not-done
// columns of [app0, app1) (which must contain the candidates), it is marked
// done and recorded in pc (when given).  Remaining norms are downdated after
// every step and evaluated afresh once cancellation has consumed half their
// digits (the safeguard of LAPACK's xLAQP2, threshold sqrt(eps) = 2^-26).
// Returns the number of steps taken.
static __device__ int hh_pivoted(double *M, int ld, int k, int r, int cand0, int cand1, int app0, int app1,
                                 int *done, int *pc, double thr, double *v, double *w) {
  const int tid = team_rank(), T = TEAM;
  double *cn = hh_norms(), *cref = cn + kMaxCols;
  double mybest = -1.0;
  int mypiv = 0x7fffffff;
  for (int j = cand0 + tid; j < cand1; j += T) {
    double acc = 0.0;
    if (!done[j])
      for (int i = k; i < r; i++) acc = fma(M[i * ld + j], M[i * ld + j], acc);
    cn[j] = acc;
    cref[j] = acc;
    if (!done[j] && acc > mybest) { mybest = acc; mypiv = j; }
  }
  double b2;
  int piv;
  team_argmax1(mybest < 0.0 ? 0.0 : mybest, mybest < 0.0 ? 0x7fffffff : mypiv, 0, b2, piv);
  int steps = 0;
  while (k < r && piv != 0x7fffffff) {
    const double nrm = hh_pivot_step(M, ld, k, r, piv, app0, app1, done, v, w, thr, cn, cref, cand0, cand1,
                                     (steps + 1) & 1);
    if (nrm == 0.0) break;
    if (tid == 0 && pc) pc[steps] = piv;
    k++;
    steps++;
    if (k >= r) break;
    argmax_finish(steps & 1, b2, piv);
  }
  tsync();
  return steps;
}

// ---------------------------------------------------------------------------
// Lemma 1 by ordered column-pivoted Householder row reduction.
//
// M (r x nc, ld) holds, column-wise: ng groups of columns to eliminate (sizes
// gsz[]), then nkeep kept columns, then one offset column.  Tolerance policy
// (Sec. 8): every row is scaled to unit 2-norm over its coefficient columns;
// a pivot is accepted when its column norm over the remaining rows exceeds
// tau_rank * nu (nu = largest column norm of the scaled matrix); groups are
// pivoted in order, the eliminated variables first; a leftover row whose
// offset exceeds tau_inc * max(1, largest scaled offset) is inconsistent.
// On return rows [k0, k0 + krank) hold the kept relation in the kept columns
// (upper-trapezoidal in pivot order); they are also written, each renormalised
// to unit coefficient norm, to out (krank x (nkeep + 1), ldo) when out != 0.
// scr: >= 2 * nc + r + nc/2 + 1 doubles of scratch private to the task.
// ---------------------------------------------------------------------------
struct ProjResult {
  int grank[3];
  int krank;
  int k0;
  int inconsistent;
};

static __device__ ProjResult wproject(double *M, int ld, int r, int ng, const int *gsz, int nkeep,
                               double tau_rank, double tau_inc, double *out, int ldo,
                               double *scr) {
  const int tid = team_rank();
  int ncoef = nkeep;
  for (int g = 0; g < ng; g++) ncoef += gsz[g];
  const int nc = ncoef + 1, off = ncoef;
  double *v = scr;                 // r
  double *w = scr + r;             // nc
  int *done = (int *)(scr + r + nc);  // nc ints
  ProjResult res;
  res.grank[0] = res.grank[1] = res.grank[2] = 0;
  res.krank = 0;
  res.k0 = 0;
  res.inconsistent = 0;

  // row scaling
  for (int i = tid; i < r; i += TEAM) {
    double s0 = 0.0, s1 = 0.0;
    int j = 0;
    for (; j + 1 < ncoef; j += 2) {
      double a = M[i * ld + j], b = M[i * ld + j + 1];
      s0 = fma(a, a, s0);
      s1 = fma(b, b, s1);
    }
    if (j < ncoef) s0 = fma(M[i * ld + j], M[i * ld + j], s0);
    double s = s0 + s1;
    if (s > 0.0) {
      double inv = 1.0 / sqrt(s);
      for (j = 0; j < nc; j++) M[i * ld + j] *= inv;
    }
  }
  for (int j = tid; j < nc; j += TEAM) done[j] = 0;
  tsync();
  // nu and omega
  double nu = 0.0, om = 0.0;
  for (int j = tid; j < ncoef; j += TEAM) {
    double s0 = 0.0, s1 = 0.0;
    int i = 0;
    for (; i + 1 < r; i += 2) {
      s0 = fma(M[i * ld + j], M[i * ld + j], s0);
      s1 = fma(M[(i + 1) * ld + j], M[(i + 1) * ld + j], s1);
    }
    if (i < r) s0 = fma(M[i * ld + j], M[i * ld + j], s0);
    nu = fmax(nu, s0 + s1);
  }
  for (int i = tid; i < r; i += TEAM) om = fmax(om, fabs(M[i * ld + off]));
  nu = sqrt(team_max(nu));
  om = fmax(1.0, team_max(om));
  const double thr = tau_rank * nu;

  int k = 0, c0 = 0;
  for (int g = 0; g <= ng; g++) {
    const int c1 = c0 + (g < ng ? gsz[g] : nkeep);
    const int rk = hh_pivoted(M, ld, k, r, c0, c1, 0, nc, done, nullptr, thr, v, w);
    k += rk;
    if (g < ng) res.grank[g] = rk; else res.krank = rk;
    c0 = c1;
  }
  res.k0 = k - res.krank;
  int bad = 0;
  for (int i = k + tid; i < r; i += TEAM)
    if (fabs(M[i * ld + off]) > tau_inc * om) bad = 1;
  res.inconsistent = __syncthreads_or(bad);
  if (out) {
    const int kc0 = ncoef - nkeep;
    for (int a = tid; a < res.krank; a += TEAM) {
      const double *row = M + (res.k0 + a) * ld;
      double s = 0.0;
      for (int j = 0; j < nkeep; j++) s = fma(row[kc0 + j], row[kc0 + j], s);
      double inv = 1.0 / sqrt(s);
      for (int j = 0; j < nkeep; j++) out[a * ldo + j] = row[kc0 + j] * inv;
      out[a * ldo + nkeep] = row[off] * inv;
    }
  }
  tsync();
  return res;
}

// ---------------------------------------------------------------------------
// Null space and minimum-norm solutions of K X = -B through the column-
// pivoted Householder QR of K^T (pivoting over the rows of K):
//   K^T Pi = Q R,   rank = accepted pivots (tau_rank * largest row norm).
// W (nk x rk, ldw) receives K^T and is overwritten by R; Q (nk x nk, ldq) is
// formed explicitly: its first `rank` columns span range(K^T), the last
// nk - rank are an orthonormal basis of null(K).  perm: rk ints.
// ---------------------------------------------------------------------------
static __device__ int wtqr(const double *K, int ldk, int rk, int nk, double tau_rank, double *W, int ldw,
                    double *Q, int ldq, int *perm, double *scr /* >= nk + max(nk, rk) */) {
  const int tid = team_rank(), T = TEAM;
  double *v = scr, *w = scr + nk;
  double *part = hh_part();
  for (int idx = tid; idx < nk * rk; idx += T) {
    int i = idx / rk, j = idx - i * rk;
    W[i * ldw + j] = K[j * ldk + i];
  }
  for (int idx = tid; idx < nk * nk; idx += T) {
    int i = idx / nk, j = idx - i * nk;
    Q[i * ldq + j] = (i == j) ? 1.0 : 0.0;
  }
  for (int j = tid; j < rk; j += T) perm[j] = j;
  tsync();
  double nu = 0.0;
  for (int j = tid; j < rk; j += T) {
    double acc = 0.0;
    for (int i = 0; i < nk; i++) acc = fma(W[i * ldw + j], W[i * ldw + j], acc);
    nu = fmax(nu, acc);
  }
  nu = sqrt(team_max(nu));
  const double thr = tau_rank * nu;
  int rank = 0;
  for (int s = 0; s < rk && s < nk; s++) {
    double mybest = -1.0;
    int mypiv = 0x7fffffff;
    for (int j = s + tid; j < rk; j += T) {
      double t = 0.0;
      for (int i = s; i < nk; i++) t = fma(W[i * ldw + j], W[i * ldw + j], t);
      if (t > mybest) { mybest = t; mypiv = j; }
    }
    double b2;
    int piv;
    team_argmax(mybest < 0.0 ? 0.0 : mybest, mybest < 0.0 ? 0x7fffffff : mypiv, b2, piv);
    if (piv == 0x7fffffff) break;
    const double best = sqrt(b2);
    if (!(best > thr)) break;
    if (piv != s) {
      for (int i = tid; i < nk; i += T) {
        double t = W[i * ldw + s];
        W[i * ldw + s] = W[i * ldw + piv];
        W[i * ldw + piv] = t;
      }
      if (tid == 0) {
        int t = perm[s]; perm[s] = perm[piv]; perm[piv] = t;
      }
      tsync();
    }
    // W columns > s (the reflector stays in v)
    whouse_apply(W, ldw, s, nk, s, s + 1, rk, nullptr, v, w, best);
    const double beta = 1.0 / (best * fabs(v[s]));
    // Q <- Q H on columns [s, nk): row dots split by row of Q and segment of l
    const int nl = nk - s;
    const int S = max(1, min(T / nk, nl));
    for (int idx = tid; idx < S * nk; idx += T) {
      const int i = idx % nk, sgm = idx / nk;
      double acc = 0.0;
      for (int l = s + sgm; l < nk; l += S) acc = fma(Q[i * ldq + l], v[l], acc);
      if (S == 1) w[i] = beta * acc;
      else part[sgm * nk + i] = acc;
    }
    tsync();
    if (S > 1) {
      for (int i = tid; i < nk; i += T) {
        double acc = part[i];
        for (int sgm = 1; sgm < S; sgm++) acc += part[sgm * nk + i];
        w[i] = beta * acc;
      }
      tsync();
    }
    for (int idx = tid; idx < nk * nl; idx += T) {
      int i = idx / nl, l = s + idx % nl;
      Q[i * ldq + l] = fma(-w[i], v[l], Q[i * ldq + l]);
    }
    tsync();
    rank++;
  }
  return rank;
}

// After wtqr: X (nk x nb, ldx) = -Q1 R11^{-T} (Pi^T B)_1 for B (rk x nb, ldb),
// the min-norm solutions of K X = -B.  Returns the largest residual of the
// dependent rows relative to max(1, |B|_max) (a consistency check).
// Y: rank x nb scratch (ldy).  X must not alias B.
static __device__ double wtqr_solve(const double *W, int ldw, const double *Q, int ldq, const int *perm,
                             int rk, int nk, int rank, const double *B, int ldb, int nb, double *X,
                             int ldx, double *Y, int ldy) {
  const int tid = team_rank();
  double bmax = 0.0;
  for (int idx = tid; idx < rk * nb; idx += TEAM) {
    int i = idx / nb, j = idx - i * nb;
    bmax = fmax(bmax, fabs(B[i * ldb + j]));
  }
  bmax = fmax(1.0, team_max(bmax));
  double rmax = 0.0;
  for (int c = tid; c < nb; c += TEAM) {
    for (int i = 0; i < rank; i++) {
      double s = B[perm[i] * ldb + c];
      for (int l = 0; l < i; l++) s = fma(-W[l * ldw + i], Y[l * ldy + c], s);
      Y[i * ldy + c] = s / W[i * ldw + i];
    }
    for (int j = rank; j < rk; j++) {
      double s = B[perm[j] * ldb + c];
      for (int l = 0; l < rank; l++) s = fma(-W[l * ldw + j], Y[l * ldy + c], s);
      rmax = fmax(rmax, fabs(s));
    }
  }
  tsync();
  for (int idx = tid; idx < nk * nb; idx += TEAM) {
    int i = idx / nb, c = idx - i * nb;
    double s = 0.0;
    for (int l = 0; l < rank; l++) s = fma(Q[i * ldq + l], Y[l * ldy + c], s);
    X[i * ldx + c] = -s;
  }
  tsync();
  return team_max(rmax) / bmax;
}

// In-place Cholesky L L^T of an SPD n x n matrix (lower triangle, upper set
// to zero).  Returns 0 on success, 1 if a pivot is not positive.
static __device__ int wcholesky(double *Hm, int ld, int n) {
  const int tid = team_rank();
  int fail = 0;
  for (int j = 0; j < n; j++) {
    // diagonal
    double s = Hm[j * ld + j];
    for (int l = 0; l < j; l++) s = fma(-Hm[j * ld + l], Hm[j * ld + l], s);
    if (!(s > 0.0)) fail = 1;
    const double d = sqrt(fmax(s, 1e-300));
    const double inv = 1.0 / d;
    for (int i = j + 1 + tid; i < n; i += TEAM) {
      double t = Hm[i * ld + j];
      for (int l = 0; l < j; l++) t = fma(-Hm[i * ld + l], Hm[j * ld + l], t);
      Hm[i * ld + j] = t * inv;
    }
    tsync();
    if (tid == 0) {
      Hm[j * ld + j] = d;
      for (int i = 0; i < j; i++) Hm[i * ld + j] = 0.0;
    }
    tsync();
  }
  return fail;
}

// Solve (L L^T) X = B in place, B n x nb (ld ldb); lanes over right-hand sides.
static __device__ void wchol_solve(const double *L, int ldl, int n, double *B, int ldb, int nb) {
  for (int c = team_rank(); c < nb; c += TEAM) {
    for (int i = 0; i < n; i++) {
      double s = B[i * ldb + c];
      for (int l = 0; l < i; l++) s = fma(-L[i * ldl + l], B[l * ldb + c], s);
      B[i * ldb + c] = s / L[i * ldl + i];
    }
    for (int i = n - 1; i >= 0; i--) {
      double s = B[i * ldb + c];
      for (int l = i + 1; l < n; l++) s = fma(-L[l * ldl + i], B[l * ldb + c], s);
      B[i * ldb + c] = s / L[i * ldl + i];
    }
  }
  tsync();
}

// In-place LU with partial pivoting of an n x n matrix; piv: n ints.
static __device__ void wlu(double *A, int ld, int n, int *piv) {
  const int tid = team_rank();
  for (int j = 0; j < n; j++) {
    double mybest = -1.0;
    int myi = 0x7fffffff;
    for (int i = j + tid; i < n; i += TEAM) {
      double a = fabs(A[i * ld + j]);
      if (a > mybest) { mybest = a; myi = i; }
    }
    double b;
    int p;
    team_argmax(mybest < 0.0 ? 0.0 : mybest, myi, b, p);
    if (p == 0x7fffffff) p = j;
    if (p != j) {
      for (int c = tid; c < n; c += TEAM) {
        double t = A[j * ld + c]; A[j * ld + c] = A[p * ld + c]; A[p * ld + c] = t;
      }
    }
    if (tid == 0) piv[j] = p;
    tsync();
    const double inv = 1.0 / A[j * ld + j];
    for (int i = j + 1 + tid; i < n; i += TEAM) A[i * ld + j] *= inv;
    tsync();
    const int rows = n - j - 1, cols = n - j - 1;
    for (int idx = tid; idx < rows * cols; idx += TEAM) {
      int i = j + 1 + idx / cols, c = j + 1 + idx % cols;
      A[i * ld + c] = fma(-A[i * ld + j], A[j * ld + c], A[i * ld + c]);
    }
    tsync();
  }
}

// Solve A X = B (trans = 0) or A^T X = B (trans = 1) with the LU of wlu; B is
// n x nb, overwritten with X; lanes over right-hand sides.
static __device__ void wlu_solve(const double *LU, int ld, int n, const int *piv, double *B, int ldb, int nb,
                          int trans) {
  for (int c = team_rank(); c < nb; c += TEAM) {
    if (!trans) {
      for (int i = 0; i < n; i++)
        if (piv[i] != i) { double t = B[i * ldb + c]; B[i * ldb + c] = B[piv[i] * ldb + c]; B[piv[i] * ldb + c] = t; }
      for (int i = 0; i < n; i++) {
        double s = B[i * ldb + c];
        for (int l = 0; l < i; l++) s = fma(-LU[i * ld + l], B[l * ldb + c], s);
        B[i * ldb + c] = s;
      }
      for (int i = n - 1; i >= 0; i--) {
        double s = B[i * ldb + c];
        for (int l = i + 1; l < n; l++) s = fma(-LU[i * ld + l], B[l * ldb + c], s);
        B[i * ldb + c] = s / LU[i * ld + i];
      }
    } else {
      // A^T = U^T L^T P
      for (int i = 0; i < n; i++) {
        double s = B[i * ldb + c];
        for (int l = 0; l < i; l++) s = fma(-LU[l * ld + i], B[l * ldb + c], s);
        B[i * ldb + c] = s / LU[i * ld + i];
      }
      for (int i = n - 1; i >= 0; i--) {
        double s = B[i * ldb + c];
        for (int l = i + 1; l < n; l++) s = fma(-LU[l * ld + i], B[l * ldb + c], s);
        B[i * ldb + c] = s;
      }
      for (int i = n - 1; i >= 0; i--)
        if (piv[i] != i) { double t = B[i * ldb + c]; B[i * ldb + c] = B[piv[i] * ldb + c]; B[piv[i] * ldb + c] = t; }
    }
  }
  tsync();
}

}  // namespace eclqr

namespace eclqr {

// ---------------------------------------------------------------------------
// Elimination in a cost relation: rows [0, rc) are constraints (hold exactly),
// rows [rc, rc + rq) are least-squares cost rows (1/2 ||row . (vars, 1)||^2).
// Columns: ne eliminated | nk kept | 1 offset.  Minimises the cost over the
// eliminated variables subject to the constraints and returns the induced
// relation on the kept variables (equality-constrained least squares by
// direct elimination):
//   A. column-pivoted Householder on the (row-scaled) constraint rows over the
//      eliminated columns;
//   B. the constraint pivot rows remove their pivot variables from the cost
//      rows (adding multiples of an exact equation leaves the cost unchanged
//      on the constraint set);
//   C. column-pivoted Householder on the cost rows over the remaining
//      eliminated columns (their pivot rows vanish at the minimiser);
//   D. remaining constraint rows reduced to an independent basis over the kept
//      columns, leftover rows checked for 0 = gamma (tau_inc);
//   E. remaining cost rows compressed by Householder QR over the kept columns.
// Outputs: kc constraint rows (unit coefficient norm) to outC and kq cost rows
// to outQ, each (nk + 1) wide with leading dimension ldo.
// scr: >= 2 (rc + rq) + 2 (ne + nk + 1) + ne / 2 + 4 doubles.
// ---------------------------------------------------------------------------
struct LseResult {
  int k1, k2, kc, kq, inconsistent;
};

static __device__ LseResult wlse_elim(double *M, int ld, int rc, int rq, int ne, int nk, double tau_rank,
                                      double tau_inc, double *outC, double *outQ, int ldo, double *scr) {
  const int tid = team_rank();
  const int nc = ne + nk + 1, off = ne + nk, r = rc + rq;
  double *v = scr;
  double *w = v + r;
  int *done = (int *)(w + (nc > r ? nc : r));
  int *pc = done + nc;
  LseResult res;
  res.k1 = res.k2 = res.kc = res.kq = res.inconsistent = 0;
  // scale constraint rows to unit coefficient norm
  for (int i = tid; i < rc; i += TEAM) {
    double s = 0.0;
    for (int j = 0; j < off; j++) s = fma(M[i * ld + j], M[i * ld + j], s);
    if (s > 0.0) {
      double inv = 1.0 / sqrt(s);
      for (int j = 0; j < nc; j++) M[i * ld + j] *= inv;
    }
  }
  for (int j = tid; j < nc; j += TEAM) done[j] = 0;
  tsync();
  double nu = 0.0, om = 0.0;
  for (int j = tid; j < off; j += TEAM) {
    double s = 0.0;
    for (int i = 0; i < rc; i++) s = fma(M[i * ld + j], M[i * ld + j], s);
    nu = fmax(nu, s);
  }
  for (int i = tid; i < rc; i += TEAM) om = fmax(om, fabs(M[i * ld + off]));
  nu = sqrt(team_max(nu));
  om = fmax(1.0, team_max(om));
  const double thr = tau_rank * nu;
  // A
  res.k1 = hh_pivoted(M, ld, 0, rc, 0, ne, 0, nc, done, pc, thr, v, w);
  // B
  for (int p = 0; p < res.k1; p++) {
    const int col = pc[p];
    const double inv = 1.0 / M[p * ld + col];
    for (int q = tid; q < rq; q += TEAM) w[q] = M[(rc + q) * ld + col] * inv;
    tsync();
    for (int idx = tid; idx < rq * nc; idx += TEAM) {
      int q = idx / nc, j = idx - q * nc;
      double val = (j == col) ? 0.0 : fma(-w[q], M[p * ld + j], M[(rc + q) * ld + j]);
      M[(rc + q) * ld + j] = val;
    }
    tsync();
  }
  // C
  double nuq = 0.0;
  for (int j = tid; j < ne; j += TEAM) {
    if (done[j]) continue;
    double s = 0.0;
    for (int i = rc; i < r; i++) s = fma(M[i * ld + j], M[i * ld + j], s);
    nuq = fmax(nuq, s);
  }
  nuq = sqrt(team_max(nuq));
  res.k2 = hh_pivoted(M, ld, rc, r, 0, ne, 0, nc, done, nullptr, tau_rank * nuq, v, w);
  const int kk = rc + res.k2;
  // D
  res.kc = hh_pivoted(M, ld, res.k1, rc, ne, off, ne, nc, done, nullptr, thr, v, w);
  const int kd = res.k1 + res.kc;
  int bad = 0;
  for (int i = kd + tid; i < rc; i += TEAM)
    if (fabs(M[i * ld + off]) > tau_inc * om) bad = 1;
  res.inconsistent = __syncthreads_or(bad);
  for (int a = tid; a < res.kc; a += TEAM) {
    const double *row = M + (res.k1 + a) * ld;
    double s = 0.0;
    for (int j = 0; j < nk; j++) s = fma(row[ne + j], row[ne + j], s);
    double inv = (s > 0.0) ? 1.0 / sqrt(s) : 0.0;
    for (int j = 0; j < nk; j++) outC[a * ldo + j] = row[ne + j] * inv;
    outC[a * ldo + nk] = row[off] * inv;
  }
  tsync();
  // E: compress the remaining cost rows over the kept columns (no pivoting)
  int ke = kk;
  for (int col = ne; col < off && ke < r; col++)
    if (hh_step(M, ld, ke, r, col, col, nc, nullptr, v, w, 0.0) > 0.0) ke++;
  res.kq = ke - kk;
  for (int idx = tid; idx < res.kq * (nk + 1); idx += TEAM) {
    int a = idx / (nk + 1), j = idx - a * (nk + 1);
    outQ[a * ldo + j] = M[(kk + a) * ld + ne + j];
  }
  tsync();
  return res;
}

}  // namespace eclqr
