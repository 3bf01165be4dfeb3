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
// values at the last exact evaluation and two lists of active columns.  Sized
// for teams of up to kMaxTeam threads and matrices of up to kMaxCols columns
// (the header's dimension limits keep every factored matrix at or below
// 3 * 32 + 64 + 1 = 161 columns).  The static total stays below 10 KB, which
// the largest dynamic request (219 KB) leaves room for.
// ---------------------------------------------------------------------------
constexpr int kMaxTeam = 256;
constexpr int kMaxCols = 168;
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
// Active-column lists of the pivoted factorization (two, alternating by step).
__device__ __forceinline__ short *hh_lists() {
  __shared__ short lists[2 * kMaxCols];
  return lists;
}

// ---------------------------------------------------------------------------
// Work layout of a Householder pass.  The pass touches cnt columns (list
// positions 0 .. cnt-1) over nr rows.  Positions are dealt to the warps in
// equal contiguous blocks of cw, and each warp splits its columns into S row
// segments held by neighbouring lanes (rows k + sg, k + sg + S, ...), so the
// lanes of one column are always lanes of one warp.  An FP64 instruction costs
// its warp the same whatever its active mask, so the widest split that fits
// the warp, S = min(floor(32 / cw), nr), gives the fewest FP64 instructions
// per warp; S need not be a power of two.  With more than 16 columns per warp,
// S = 1 and each lane walks whole columns.  The integer work is kept free of
// hardware divisions, each of which costs about 80 cycles of latency.
// ---------------------------------------------------------------------------
struct HHLayout {
  int cw;  // list positions per warp
  int S;   // row segments per column
  int lc;  // this lane's column within its warp's block
  int sg;  // this lane's segment
};
// single-precision approximations (PTX rsqrt.approx / rcp.approx, relative
// error about 2^-22), used only as seeds and for small integer quotients
__device__ __forceinline__ float rsqrt_seed(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_seed(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// Branch-free, so that the compiler can schedule it inside the latency of
// the FP64 chains around it.  Teams have 1, 2, 4 or 8 warps.
__device__ __forceinline__ HHLayout hh_layout(int cnt, int nr) {
  HHLayout L;
  const int nw = (int)(blockDim.x >> 5), lane = (int)(threadIdx.x & 31);
  const int cw = (cnt + nw - 1) >> (__ffs(nw) - 1);
  // floor(32 / cw) for cw in [1, 16] (nibbles for cw >= 3), 1 beyond
  const int tab = (int)((0x2222223344568aull >> (4 * min(max(cw - 3, 0), 13))) & 0xf);
  const int s32 = cw <= 2 ? (32 >> min(max(cw - 1, 0), 1)) : (cw > 16 ? 1 : tab);
  L.cw = cw;
  L.S = min(s32, nr);
  // lane / S: (lane + 1/2) / S stays at least 1/64 away from an integer, far
  // beyond the error of the single-precision product
  L.lc = (int)(((float)lane + 0.5f) * rcp_seed((float)L.S));
  L.sg = lane - L.lc * L.S;
  return L;
}

// Sum over the S consecutive lanes of a segment group (S >= 2); the group's
// first lane (sg == 0) receives the total.  Called by the whole warp.
__device__ __forceinline__ double seg_sum(double acc, int sg, int S) {
  int o = 1;
  while (2 * o < S) o *= 2;
  for (; o > 0; o >>= 1) {
    const double t = __shfl_down_sync(kFull, acc, o);
    if (sg + o < S) acc += t;
  }
  return acc;
}

// Reflector of a column x with squared norm d = ||x||^2 and pivot entry x_k:
// nrm = sqrt(d), shift = sign(x_k) nrm (sign(0) = +1, also for -0),
// v_k = x_k + shift and beta = 2 / ||v||^2 with ||v||^2 = (d - x_k^2) + v_k^2
// evaluated from the v actually formed, so H = I - beta v v' is orthogonal to
// rounding whatever the last bits of nrm.  The FP64 square root and divide
// are long dependent chains (about 690 and 440 cycles), so both come from
// single-precision seeds (exponents handled on the integer pipe) refined by
// one third-order step: for d^(-1/2) the Householder iteration
// y = y0 (1 + e/2 + 3 e^2 / 8), e = 1 - d y0^2, and for 1/q the Newton-type
// step r = r0 (1 + e + e^2), e = 1 - q r0.  From a 2^-21 seed each leaves a
// truncation error below 2^-60 (5 e^3 / 16 and e^3).  The code is branch-
// free; it returns false, with the outputs unset, when d is zero, subnormal,
// above 2^1000 or not finite, where the seeds do not apply.
__device__ __forceinline__ bool hh_reflector(double d, double xk, double &nrm, double &shift, double &vk,
                                             double &beta) {
  const long long db = __double_as_longlong(d);
  const int dh = (int)(db >> 32);
  const int ex = ((dh >> 20) & 0x7ff) - 1023;
  // d = 2^(2 h) m, m in [1, 4): y0 = rsqrt(m) 2^-h
  const int odd = ex & 1, h = (ex - odd) >> 1;
  const unsigned m23 = ((unsigned)(dh & 0xfffff) << 3) | ((unsigned)db >> 29);
  const int yf = __float_as_int(rsqrt_seed(__int_as_float(((127 + odd) << 23) | (int)m23)));
  const double y0 =
      __hiloint2double(((((yf >> 23) & 0xff) + (1023 - 127) - h) << 20) | ((yf & 0x7fffff) >> 3), (yf & 7) << 29);
  const double dx = fma(-xk, xk, d);
  const double t = d * y0;
  const double e = fma(-t, y0, 1.0);
  const double p = fma(0.375, e, 0.5);
  nrm = fma(t * e, p, t);
  const bool neg = (__double_as_longlong(xk) < 0) && ((__double_as_longlong(xk) << 1) != 0);
  shift = neg ? -nrm : nrm;
  vk = xk + shift;
  const double q = fma(vk, vk, dx);
  // q = 2^g m, m in [1, 2): r0 = (1 / m) 2^-g ~ 1 / q, and beta = 2 / q from
  // the doubled seed (exponent + 1)
  const long long qb = __double_as_longlong(q);
  const int qh = (int)(qb >> 32);
  const int g = ((qh >> 20) & 0x7ff) - 1023;
  const unsigned n23 = ((unsigned)(qh & 0xfffff) << 3) | ((unsigned)qb >> 29);
  const int rf = __float_as_int(rcp_seed(__int_as_float((127 << 23) | (int)n23)));
  const int rhi = ((((rf >> 23) & 0xff) + (1023 - 127) - g) << 20) | ((rf & 0x7fffff) >> 3), rlo = (rf & 7) << 29;
  const double r0 = __hiloint2double(rhi, rlo), r2 = __hiloint2double(rhi + (1 << 20), rlo);
  const double f = fma(-q, r0, 1.0);
  beta = fma(r2, fma(f, f, f), r2);
  return ex >= -1000 && ex <= 1000;
}

// d^(-1/2) by the method of hh_reflector: a single-precision seed (exponent
// on the integer pipe) and one third-order step y = y0 (1 + e/2 + 3 e^2 / 8),
// e = 1 - d y0^2, truncation error below 2^-60.  ok is false, with the result
// unusable, unless d is positive, normal and within [2^-1000, 2^1001).
__device__ __forceinline__ double seeded_rsqrt(double d, bool &ok) {
  const long long db = __double_as_longlong(d);
  const int dh = (int)(db >> 32);
  const int ex = ((dh >> 20) & 0x7ff) - 1023;
  const int odd = ex & 1, h = (ex - odd) >> 1;
  const unsigned m23 = ((unsigned)(dh & 0xfffff) << 3) | ((unsigned)db >> 29);
  const int yf = __float_as_int(rsqrt_seed(__int_as_float(((127 + odd) << 23) | (int)m23)));
  const double y0 =
      __hiloint2double(((((yf >> 23) & 0xff) + (1023 - 127) - h) << 20) | ((yf & 0x7fffff) >> 3), (yf & 7) << 29);
  const double e = fma(-(d * y0), y0, 1.0);
  const double p = fma(0.375, e, 0.5);
  ok = (d > 0.0) && ex >= -1000 && ex <= 1000;
  return fma(y0 * e, p, y0);
}

// Team arg-max with one barrier: partials alternate between two buffers by
// parity, so consecutive uses of one buffer must be separated by at least one
// other barrier.  Keys are the bit patterns of non-negative doubles, which
// order like the values, so the reduction runs on the integer pipe; ties go to
// the smaller index.
__device__ __forceinline__ unsigned long long *argmax_keys() {
  __shared__ unsigned long long rk[2][32];
  return &rk[0][0];
}
__device__ __forceinline__ int *argmax_idx() {
  __shared__ int ri[2][32];
  return &ri[0][0];
}

// Warp stage: lane 0 leaves (key, index) of the warp's best in buffer parity.
__device__ __forceinline__ void warp_argmax_key(unsigned long long key, int idx, int parity) {
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

__device__ __forceinline__ unsigned long long dkey(double x) { return (unsigned long long)__double_as_longlong(x); }

// Whether a Householder step runs: d = ||x||^2 > 0 (a NaN d gives false) and
// nrm = sqrt(d) > thr, compared as bit patterns on the integer pipe: non-negative
// doubles order like their patterns, and a negative thr (sign bit set) is below
// every nrm of a positive d.
__device__ __forceinline__ bool hh_step_runs(double d, double nrm, double thr) {
  const long long db = __double_as_longlong(d), nb = __double_as_longlong(nrm), tb = __double_as_longlong(thr);
  return db > 0 && db <= 0x7ff0000000000000ll && (tb < 0 || nb > tb);
}

// One Householder step on rows [k, r) with pivot column piv among the cnt
// columns of the pass (column of position p: list ? list[p] : a0 + p; the
// pivot is one of them), laid out by L = hh_layout(cnt, r - k).  Dot pass:
// d_j = M_piv . M_j for every column j of the pass, d_piv = ||M_piv||^2, and
// the old row k kept in hh_rowk.  If sqrt(d_piv) <= thr (or d_piv = 0), M is
// left untouched and 0 is returned.  Otherwise the reflector
// H = I - beta v v' (v = M_piv + sign(x_k) ||M_piv|| e_k, beta =
// 1 / (||M_piv|| (||M_piv|| + |x_k|)), formed as 2 / ||v||^2 by hh_reflector)
// is applied to the other columns,
// column piv becomes (-sign(x_k) ||M_piv||, 0, ..., 0), and the norm is
// returned.  L is then replaced by the layout of the next step (cnt - 1
// columns on rows [k + 1, r)), computed in the shadow of the FP64 latency.
// Scratch: v (rows), d (columns).  With refl given, (v_k, beta) go to
// refl[0..1], so that v (with v[k] replaced by v_k) and beta describe H.
//
// Column pivoting (cn given): the update pass also downdates the remaining
// squared norms cn of the candidate columns in [cand0, cand1) (LAPACK
// xLAQP2's safeguard: a norm is evaluated afresh from its rows when it falls
// to 2^-26 = sqrt(eps) of its last exact value, crs holding that value times
// 2^-26), leaves each warp's best candidate in arg-max buffer parity, marks
// piv done and writes the list without piv to next (order kept).
static __device__ double hh_core(double *M, int ld, int k, int r, int piv, const short *list, int a0, int cnt,
                                 HHLayout &L, double *v, double *d, double thr, int *done = nullptr,
                                 short *next = nullptr, double *cn = nullptr, double *crs = nullptr,
                                 int cand0 = 0, int cand1 = 0, int parity = 0, double *refl = nullptr) {
  const int tid = team_rank(), T = TEAM, wid = tid >> 5;
  double *mk = hh_rowk();
  const int S = L.S, sg = L.sg;
  const int pw0 = wid * L.cw, pw1 = min(pw0 + L.cw, cnt);
  for (int i = k + tid; i < r; i += T) v[i] = M[i * ld + piv];
  for (int p = tid; p < cnt; p += T) {
    const int j = list ? list[p] : a0 + p;
    mk[j] = M[k * ld + j];
    if (next && j != piv) next[p - (j > piv ? 1 : 0)] = (short)j;
  }
  // dot pass
  const int p1 = pw0 + L.lc;
  const bool on1 = S > 1 && L.lc < L.cw && p1 < pw1;
  const int j1 = on1 ? (list ? list[p1] : a0 + p1) : piv;
  if (S > 1) {
    double acc = 0.0;
    if (on1)
      for (int i = k + sg; i < r; i += S) acc = fma(M[i * ld + piv], M[i * ld + j1], acc);
    acc = seg_sum(acc, sg, S);
    if (on1 && sg == 0) d[j1] = acc;
  } else {
    for (int p = pw0 + (tid & 31); p < pw1; p += 32) {
      const int j = list ? list[p] : a0 + p;
      double acc = 0.0;
      for (int i = k; i < r; i++) acc = fma(M[i * ld + piv], M[i * ld + j], acc);
      d[j] = acc;
    }
  }
  tsync();
  const double dp = d[piv];
  const double xk = v[k];
  double nrm, shift, vk, beta;
  const bool fast = hh_reflector(dp, xk, nrm, shift, vk, beta);
  const HHLayout Ln = hh_layout(cnt - 1, r - k - 1);
  if (!fast) {
    nrm = sqrt(dp);
    shift = ((__double_as_longlong(xk) < 0) && ((__double_as_longlong(xk) << 1) != 0)) ? -nrm : nrm;
    vk = xk + shift;
    beta = 1.0 / (nrm * (nrm + fabs(xk)));
  }
  if (!hh_step_runs(dp, nrm, thr)) return 0.0;
  L = Ln;
  if (refl && tid == 0) { refl[0] = vk; refl[1] = beta; }  // visible after the closing barrier
  // update pass (and, when pivoting, the norm downdate and the warp's arg-max)
  unsigned long long bkey = 0ull;
  int bidx = 0x7fffffff;
  if (S > 1) {
    if (on1) {
      if (j1 == piv) {
        for (int i = k + sg; i < r; i += S) M[i * ld + piv] = (i == k) ? -shift : 0.0;
        if (sg == 0 && done) done[piv] = 1;
      } else {
        const double wj = beta * fma(shift, mk[j1], d[j1]);
        for (int i = k + sg; i < r; i += S) M[i * ld + j1] = fma(-wj, (i == k) ? vk : v[i], M[i * ld + j1]);
      }
    }
    if (cn) {
      __syncwarp();  // a column's row segments are lanes of this warp
      const bool cand = on1 && j1 != piv && j1 >= cand0 && j1 < cand1;
      double nw = 0.0;
      bool fresh = false;
      if (cand) {
        const double a = M[k * ld + j1];
        nw = fma(-a, a, cn[j1]);
        fresh = !((long long)dkey(nw) > (long long)dkey(crs[j1]));
      }
      if (__any_sync(kFull, fresh)) {
        double acc = 0.0;
        if (fresh)
          for (int i = k + 1 + sg; i < r; i += S) acc = fma(M[i * ld + j1], M[i * ld + j1], acc);
        acc = seg_sum(acc, sg, S);
        if (fresh) nw = acc;
      }
      if (cand && sg == 0) {
        cn[j1] = nw;
        if (fresh) crs[j1] = 0x1p-26 * nw;
        bkey = dkey(nw);
        bidx = j1;
      }
    }
  } else {
    for (int p = pw0 + (tid & 31); p < pw1; p += 32) {
      const int j = list ? list[p] : a0 + p;
      if (j == piv) {
        for (int i = k; i < r; i++) M[i * ld + piv] = (i == k) ? -shift : 0.0;
        if (done) done[piv] = 1;
        continue;
      }
      const double wj = beta * fma(shift, mk[j], d[j]);
      M[k * ld + j] = fma(-wj, vk, M[k * ld + j]);
      for (int i = k + 1; i < r; i++) M[i * ld + j] = fma(-wj, v[i], M[i * ld + j]);
      if (cn && j >= cand0 && j < cand1) {
        const double a = M[k * ld + j];
        double nw = fma(-a, a, cn[j]);
        if (!((long long)dkey(nw) > (long long)dkey(crs[j]))) {
          nw = 0.0;
          for (int i = k + 1; i < r; i++) nw = fma(M[i * ld + j], M[i * ld + j], nw);
          crs[j] = 0x1p-26 * nw;
        }
        cn[j] = nw;
        if (bidx == 0x7fffffff || dkey(nw) > bkey) { bkey = dkey(nw); bidx = j; }
      }
    }
  }
  if (cn) warp_argmax_key(bkey, bidx, parity);
  tsync();
  return nrm;
}

// One Householder step applied to the columns [a0, a1) (piv among them).
static __device__ __forceinline__ double hh_step(double *M, int ld, int k, int r, int piv, int a0, int a1,
                                                 double *v, double *d, double thr, double *refl = nullptr) {
  HHLayout L = hh_layout(a1 - a0, r - k);
  return hh_core(M, ld, k, r, piv, nullptr, a0, a1 - a0, L, v, d, thr, nullptr, nullptr, nullptr, nullptr, 0, 0,
                 0, refl);
}

// Unpivoted steps down the diagonal: for col = c0, c0 + 1, ... < c1 while the
// row k < r, the reflector of column col on rows [k, r) applied to the
// columns [col, a1).  k advances when the column's norm exceeds thr, or after
// every column when keep_diag is set (row k then stays paired with column
// k).  Returns the final k.
static __device__ int hh_diag_steps(double *M, int ld, int k, int r, int c0, int c1, int a1, double *v, double *d,
                                    double thr, bool keep_diag) {
  HHLayout L = hh_layout(a1 - c0, r - k);
  for (int col = c0; col < c1 && k < r; col++) {
    const bool ok = hh_core(M, ld, k, r, col, nullptr, col, a1 - col, L, v, d, thr) > 0.0;
    if (ok || keep_diag) k++;
    if (!ok) L = hh_layout(a1 - col - 1, r - k);
  }
  return k;
}

// Column-pivoted Householder steps on rows [k, r).  Each step takes the
// candidate column (in [cand0, cand1), not done) of largest remaining norm;
// while its exact norm exceeds thr, its reflector is applied to the not-done
// columns of [app0, app1) (which must contain the candidates), it is marked
// done and recorded in pc (when given).  Remaining norms are downdated after
// every step and evaluated afresh once cancellation has consumed half their
// digits (the safeguard of LAPACK's xLAQP2, threshold sqrt(eps) = 2^-26).
// The passes run over a list of the not-done columns, shortened by one
// column per step.  Returns the number of steps taken.
static __device__ int hh_pivoted_list(double *M, int ld, int k, int r, int cand0, int cand1, int app0,
                                      int app1, int *done, int *pc, double thr, double *v, double *w) {
  const int tid = team_rank(), lane = tid & 31, wid = tid >> 5;
  double *cn = hh_norms(), *crs = cn + kMaxCols;
  short *lists = hh_lists();
  // the list: not-done columns of [app0, app1) in increasing order.  Every
  // warp builds it (identical values), so each warp can read its own writes
  // after __syncwarp and no team barrier is needed.
  int cnt = 0, pc0 = 0, pc1 = 0;
  for (int j0 = app0; j0 < app1; j0 += 32) {
    const int j = j0 + lane;
    const bool on = j < app1 && !done[j];
    const unsigned b = __ballot_sync(kFull, on);
    if (on) lists[cnt + __popc(b & ((1u << lane) - 1u))] = (short)j;
    pc0 += __popc(b & __ballot_sync(kFull, j < cand0));
    pc1 += __popc(b & __ballot_sync(kFull, j < cand1));
    cnt += __popc(b);
  }
  __syncwarp();
  const int ncand = pc1 - pc0;
  // exact squared norms of the candidates over rows [k, r)
  unsigned long long bkey = 0ull;
  int bidx = 0x7fffffff;
  {
    const HHLayout C = hh_layout(ncand, r - k);
    const int pw0 = wid * C.cw, pw1 = min(pw0 + C.cw, ncand);
    if (C.S > 1) {
      const int p = pw0 + C.lc;
      const bool on = C.lc < C.cw && p < pw1;
      const int j = on ? lists[pc0 + p] : 0;
      double acc = 0.0;
      if (on)
        for (int i = k + C.sg; i < r; i += C.S) acc = fma(M[i * ld + j], M[i * ld + j], acc);
      acc = seg_sum(acc, C.sg, C.S);
      if (on && C.sg == 0) {
        cn[j] = acc;
        crs[j] = 0x1p-26 * acc;
        bkey = dkey(acc);
        bidx = j;
      }
    } else {
      for (int p = pw0 + lane; p < pw1; p += 32) {
        const int j = lists[pc0 + p];
        double acc = 0.0;
        for (int i = k; i < r; i++) acc = fma(M[i * ld + j], M[i * ld + j], acc);
        cn[j] = acc;
        crs[j] = 0x1p-26 * acc;
        if (bidx == 0x7fffffff || dkey(acc) > bkey) { bkey = dkey(acc); bidx = j; }
      }
    }
  }
  warp_argmax_key(bkey, bidx, 0);
  HHLayout L = hh_layout(cnt, r - k);
  tsync();
  double b2;
  int piv;
  argmax_finish(0, b2, piv);
  // Between exact evaluations the downdated norms carry a relative error
  // below about 2^-22, so a largest estimate under thr^2 (1 - 2^-16) means
  // every candidate fails the exact test: stop without the step.
  const double stop2 = thr * thr * (1.0 - 0x1p-16);
  int steps = 0;
  while (k < r && piv != 0x7fffffff && !(b2 < stop2)) {
    const double nrm = hh_core(M, ld, k, r, piv, lists + (steps & 1) * kMaxCols, 0, cnt, L, v, w, thr, done,
                               lists + ((steps + 1) & 1) * kMaxCols, cn, crs, cand0, cand1, (steps + 1) & 1);
    if (nrm == 0.0) break;
    if (tid == 0 && pc) pc[steps] = piv;
    k++;
    steps++;
    cnt--;
    if (k >= r) break;
    argmax_finish(steps & 1, b2, piv);
  }
  tsync();
  return steps;
}

// Range form of a pivoted step: the passes cover every column of [a0, a1)
// (done ones idle) with power-of-two row segments, S (a1 - a0) <= team size,
// and the reflector scalars from hh_reflector (library functions only at
// extreme exponents).
// The update pass also downdates the remaining norms of the candidate
// columns (re-evaluating a marked one from its rows, which sit on the same
// warp) and leaves each warp's best candidate in the arg-max buffer `parity`,
// so that the next pivot is known after the pass's own barrier.  Returns the
// norm, or 0 (M untouched) when it does not exceed thr.
static __device__ double hh_range_step(double *M, int ld, int k, int r, int piv, int a0, int a1, int *done,
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
  const double dp = d[piv], xk = v[k];
  double nrm, shift, vk, beta;
  if (!hh_reflector(dp, xk, nrm, shift, vk, beta)) {
    nrm = sqrt(dp);
    shift = ((__double_as_longlong(xk) < 0) && ((__double_as_longlong(xk) << 1) != 0)) ? -nrm : nrm;
    vk = xk + shift;
    beta = 1.0 / (nrm * (nrm + fabs(xk)));
  }
  if (!hh_step_runs(dp, nrm, thr)) return 0.0;
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
      const double vi = (i == k) ? vk : v[i];
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
  warp_argmax_key(best < 0.0 ? 0ull : dkey(best), best < 0.0 ? 0x7fffffff : bidx, parity);
  tsync();
  return nrm;
}

// Range form of the column-pivoted steps (same contract as hh_pivoted_list):
// the passes cover every column of [app0, app1), done ones idle, with
// power-of-two row segments; the next pivot's candidates are downdated in
// the update pass.
static __device__ int hh_pivoted_range(double *M, int ld, int k, int r, int cand0, int cand1, int app0,
                                       int app1, int *done, int *pc, double thr, double *v, double *w) {
  const int tid = team_rank(), lane = tid & 31, wid = tid >> 5;
  double *cn = hh_norms(), *cref = cn + kMaxCols;
  // exact squared norms of the candidates over rows [k, r), on the balanced layout
  unsigned long long bkey = 0ull;
  int bidx = 0x7fffffff;
  {
    const int nc = cand1 - cand0;
    const HHLayout C = hh_layout(nc, max(r - k, 1));
    const int pw0 = wid * C.cw, pw1 = min(pw0 + C.cw, nc);
    if (C.S > 1) {
      const int j = cand0 + pw0 + C.lc;
      const bool on = C.lc < C.cw && pw0 + C.lc < pw1 && !done[j];
      double acc = 0.0;
      if (on)
        for (int i = k + C.sg; i < r; i += C.S) acc = fma(M[i * ld + j], M[i * ld + j], acc);
      acc = seg_sum(acc, C.sg, C.S);
      if (on && C.sg == 0) {
        cn[j] = acc;
        cref[j] = acc;
        bkey = dkey(acc);
        bidx = j;
      }
    } else {
      for (int p = pw0 + lane; p < pw1; p += 32) {
        const int j = cand0 + p;
        if (done[j]) continue;
        double acc = 0.0;
        for (int i = k; i < r; i++) acc = fma(M[i * ld + j], M[i * ld + j], acc);
        cn[j] = acc;
        cref[j] = acc;
        if (bidx == 0x7fffffff || dkey(acc) > bkey) { bkey = dkey(acc); bidx = j; }
      }
    }
  }
  double b2;
  int piv;
  warp_argmax_key(bkey, bidx, 0);
  tsync();
  argmax_finish(0, b2, piv);
  const double stop2 = thr * thr * (1.0 - 0x1p-16);  // see hh_pivoted_list
  int steps = 0;
  while (k < r && piv != 0x7fffffff && !(b2 < stop2)) {
    const double nrm = hh_range_step(M, ld, k, r, piv, app0, app1, done, v, w, thr, cn, cref, cand0, cand1,
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

// Column-pivoted Householder steps on rows [k, r) (contract of
// hh_pivoted_list).  Two forms: the list form packs the active columns
// evenly over the warps with any segment count, the range form keeps the
// fixed power-of-two layout over [app0, app1).  The list form has a larger
// fixed cost per factorization and per step (the list, its layout), so it is
// taken only where its first step saves at least kListGain row FMAs per lane
// and pass: tall, wide eliminations rather than short projections.
constexpr int kListGain = 4;
__device__ __forceinline__ bool hh_list_pays(int nc, int nr) {
  const int T = TEAM;
  int s_range = 1;
  while (2 * s_range <= 32 && 2 * s_range * nc <= T && 2 * s_range <= nr) s_range *= 2;
  const HHLayout L = hh_layout(nc, nr);
  return (nr + s_range - 1) / s_range - (nr + L.S - 1) / L.S >= kListGain;
}
static __device__ int hh_pivoted(double *M, int ld, int k, int r, int cand0, int cand1, int app0, int app1,
                                 int *done, int *pc, double thr, double *v, double *w) {
  if (hh_list_pays(app1 - app0, r - k))
    return hh_pivoted_list(M, ld, k, r, cand0, cand1, app0, app1, done, pc, thr, v, w);
  return hh_pivoted_range(M, ld, k, r, cand0, cand1, app0, app1, done, pc, thr, v, w);
}


// ---------------------------------------------------------------------------
// Row and column reductions of the factorizations, on the layout of the
// Householder passes (items dealt evenly over the warps, each split into
// segments on neighbouring lanes), so that no single lane walks a whole row
// or column while the other warps wait.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long *colmax_keys() {
  __shared__ unsigned long long k[2][32];
  return &k[0][0];
}

// Largest key (bit pattern of a non-negative double) over the warp, to lane 0.
__device__ __forceinline__ unsigned long long warp_max_key(unsigned long long key) {
  const unsigned hi = (unsigned)(key >> 32), lo = (unsigned)key;
  const unsigned mhi = __reduce_max_sync(kFull, hi);
  const unsigned mlo = __reduce_max_sync(kFull, hi == mhi ? lo : 0u);
  return ((unsigned long long)mhi << 32) | mlo;
}

// Scales each of the rows [0, r) of M to unit 2-norm over its columns
// [0, ncoef), applying the factor to the columns [0, nscale); rows of zero
// norm are left as they are.  Ends with a team barrier.
static __device__ void wscale_rows(double *M, int ld, int r, int ncoef, int nscale) {
  const int lane = team_rank() & 31, wid = team_rank() >> 5;
  const HHLayout L = hh_layout(r, max(ncoef, 1));
  const int pw0 = wid * L.cw, pw1 = min(pw0 + L.cw, r);
  if (L.S > 1) {
    const int i = pw0 + L.lc;
    const bool on = L.lc < L.cw && i < pw1;
    double acc = 0.0;
    if (on)
      for (int j = L.sg; j < ncoef; j += L.S) acc = fma(M[i * ld + j], M[i * ld + j], acc);
    acc = seg_sum(acc, L.sg, L.S);
    const double ss = __shfl_sync(kFull, acc, lane - L.sg);
    if (on && ss > 0.0) {
      const double inv = rsqrt(ss);
      for (int j = L.sg; j < nscale; j += L.S) M[i * ld + j] *= inv;
    }
  } else {
    for (int i = pw0 + lane; i < pw1; i += 32) {
      double ss = 0.0;
      for (int j = 0; j < ncoef; j++) ss = fma(M[i * ld + j], M[i * ld + j], ss);
      if (ss > 0.0) {
        const double inv = rsqrt(ss);
        for (int j = 0; j < nscale; j++) M[i * ld + j] *= inv;
      }
    }
  }
  tsync();
}

// Largest squared 2-norm over the rows [r0, r1) of the columns j in [0, nc)
// with skip[j] == 0 (skip may be null), and, for offc >= 0, the largest
// |M[i][offc]| over the same rows (0 otherwise).  One team barrier; the key
// buffers are reused by the next call, so calls must be separated by at
// least one other barrier.
static __device__ void wcol_max(const double *M, int ld, int r0, int r1, int nc, const int *skip, int offc,
                                double &nu2, double &om) {
  const int tid = team_rank(), lane = tid & 31, wid = tid >> 5;
  const HHLayout L = hh_layout(nc, max(r1 - r0, 1));
  const int pw0 = wid * L.cw, pw1 = min(pw0 + L.cw, nc);
  unsigned long long kn = 0ull, ko = 0ull;
  if (L.S > 1) {
    const int j = pw0 + L.lc;
    const bool on = L.lc < L.cw && j < pw1 && !(skip && skip[j]);
    double acc = 0.0;
    if (on)
      for (int i = r0 + L.sg; i < r1; i += L.S) acc = fma(M[i * ld + j], M[i * ld + j], acc);
    acc = seg_sum(acc, L.sg, L.S);
    if (on && L.sg == 0) kn = dkey(acc);
  } else {
    for (int j = pw0 + lane; j < pw1; j += 32) {
      if (skip && skip[j]) continue;
      double acc = 0.0;
      for (int i = r0; i < r1; i++) acc = fma(M[i * ld + j], M[i * ld + j], acc);
      if (dkey(acc) > kn) kn = dkey(acc);
    }
  }
  if (offc >= 0)
    for (int i = r0 + tid; i < r1; i += TEAM) {
      const unsigned long long k = dkey(fabs(M[i * ld + offc]));
      if (k > ko) ko = k;
    }
  kn = warp_max_key(kn);
  ko = warp_max_key(ko);
  unsigned long long *keys = colmax_keys();
  if (lane == 0) { keys[wid] = kn; keys[32 + wid] = ko; }
  tsync();
  kn = keys[0];
  ko = keys[32];
  for (int q = 1; q < (int)(blockDim.x >> 5); q++) {
    kn = max(kn, keys[q]);
    ko = max(ko, keys[32 + q]);
  }
  nu2 = __longlong_as_double((long long)kn);
  om = __longlong_as_double((long long)ko);
}

// out[a][0 : nk] = the row's columns [c0, c0 + nk) and out[a][nk] = its column
// offc, both divided by the 2-norm of the first part (0 for a zero row), for
// the rows r0 + a, a in [0, cnt).  Ends with a team barrier.
static __device__ void wnorm_rows_out(const double *M, int ld, int r0, int cnt, int c0, int nk, int offc,
                                      double *out, int ldo) {
  const int lane = team_rank() & 31, wid = team_rank() >> 5;
  const HHLayout L = hh_layout(cnt, max(nk, 1));
  const int pw0 = wid * L.cw, pw1 = min(pw0 + L.cw, cnt);
  if (L.S > 1) {
    const int a = pw0 + L.lc;
    const bool on = L.lc < L.cw && a < pw1;
    const double *row = M + (size_t)(r0 + (on ? a : 0)) * ld;
    double acc = 0.0;
    if (on)
      for (int j = L.sg; j < nk; j += L.S) acc = fma(row[c0 + j], row[c0 + j], acc);
    acc = seg_sum(acc, L.sg, L.S);
    const double ss = __shfl_sync(kFull, acc, lane - L.sg);
    if (on) {
      const double inv = (ss > 0.0) ? rsqrt(ss) : 0.0;
      for (int j = L.sg; j < nk; j += L.S) out[a * ldo + j] = row[c0 + j] * inv;
      if (L.sg == 0) out[a * ldo + nk] = row[offc] * inv;
    }
  } else {
    for (int a = pw0 + lane; a < pw1; a += 32) {
      const double *row = M + (size_t)(r0 + a) * ld;
      double ss = 0.0;
      for (int j = 0; j < nk; j++) ss = fma(row[c0 + j], row[c0 + j], ss);
      const double inv = (ss > 0.0) ? rsqrt(ss) : 0.0;
      for (int j = 0; j < nk; j++) out[a * ldo + j] = row[c0 + j] * inv;
      out[a * ldo + nk] = row[offc] * inv;
    }
  }
  tsync();
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

  // row scaling, then nu (largest column norm) and the offset scale omega
  wscale_rows(M, ld, r, ncoef, nc);
  for (int j = tid; j < nc; j += TEAM) done[j] = 0;
  double nu2, om;
  wcol_max(M, ld, 0, r, ncoef, nullptr, off, nu2, om);
  const double nu = sqrt(nu2);
  om = fmax(1.0, om);
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
  if (out) wnorm_rows_out(M, ld, res.k0, res.krank, ncoef - nkeep, nkeep, off, out, ldo);
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
static __device__ int wtqr_small(const double *K, int ldk, int rk, int nk, double tau_rank, double *W, int ldw,
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

static __device__ int wtqr_large(const double *K, int ldk, int rk, int nk, double tau_rank, double *W, int ldw,
                    double *Q, int ldq, int *perm, double *scr /* >= nk + max(nk, rk) + 2 */) {
  const int tid = team_rank(), T = TEAM, lane = tid & 31, wid = tid >> 5;
  double *v = scr, *w = scr + nk, *refl = w + (nk > rk ? nk : rk);
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
  double nu2, unused;
  wcol_max(W, ldw, 0, nk, rk, nullptr, -1, nu2, unused);
  const double thr = tau_rank * sqrt(nu2);
  int rank = 0;
  for (int s = 0; s < rk && s < nk; s++) {
    // exact remaining norms of the columns [s, rk) over rows [s, nk), balanced layout
    unsigned long long bkey = 0ull;
    int bidx = 0x7fffffff;
    {
      const HHLayout C = hh_layout(rk - s, nk - s);
      const int pw0 = wid * C.cw, pw1 = min(pw0 + C.cw, rk - s);
      if (C.S > 1) {
        const int p = pw0 + C.lc, j = s + p;
        const bool on = C.lc < C.cw && p < pw1;
        double acc = 0.0;
        if (on)
          for (int i = s + C.sg; i < nk; i += C.S) acc = fma(W[i * ldw + j], W[i * ldw + j], acc);
        acc = seg_sum(acc, C.sg, C.S);
        if (on && C.sg == 0) { bkey = dkey(acc); bidx = j; }
      } else {
        for (int p = pw0 + lane; p < pw1; p += 32) {
          const int j = s + p;
          double acc = 0.0;
          for (int i = s; i < nk; i++) acc = fma(W[i * ldw + j], W[i * ldw + j], acc);
          if (bidx == 0x7fffffff || dkey(acc) > bkey) { bkey = dkey(acc); bidx = j; }
        }
      }
    }
    warp_argmax_key(bkey, bidx, s & 1);
    tsync();
    double b2;
    int piv;
    argmax_finish(s & 1, b2, piv);
    if (piv == 0x7fffffff || !(sqrt(b2) > thr)) break;
    if (piv != s) {
      for (int i = tid; i < nk; i += T) {
        const double t = W[i * ldw + s];
        W[i * ldw + s] = W[i * ldw + piv];
        W[i * ldw + piv] = t;
      }
      if (tid == 0) {
        const int t = perm[s]; perm[s] = perm[piv]; perm[piv] = t;
      }
      tsync();
    }
    // W columns [s, rk): reflector of column s (v keeps it, refl = (v_s, beta))
    if (!(hh_step(W, ldw, s, nk, s, s, rk, v, w, 0.0, refl) > 0.0)) break;
    // Q <- Q H on columns [s, nk): each row of Q on one segment group of a warp
    {
      const double vs = refl[0], beta = refl[1];
      const HHLayout R = hh_layout(nk, nk - s);
      const int pw0 = wid * R.cw, pw1 = min(pw0 + R.cw, nk);
      if (R.S > 1) {
        const int i = pw0 + R.lc;
        const bool on = R.lc < R.cw && i < pw1;
        double acc = 0.0;
        if (on)
          for (int l = s + R.sg; l < nk; l += R.S) acc = fma(Q[i * ldq + l], (l == s) ? vs : v[l], acc);
        acc = seg_sum(acc, R.sg, R.S);
        const double ti = beta * __shfl_sync(kFull, acc, lane - R.sg);
        if (on)
          for (int l = s + R.sg; l < nk; l += R.S) Q[i * ldq + l] = fma(-ti, (l == s) ? vs : v[l], Q[i * ldq + l]);
      } else {
        for (int i = pw0 + lane; i < pw1; i += 32) {
          double acc = 0.0;
          for (int l = s; l < nk; l++) acc = fma(Q[i * ldq + l], (l == s) ? vs : v[l], acc);
          const double ti = beta * acc;
          for (int l = s; l < nk; l++) Q[i * ldq + l] = fma(-ti, (l == s) ? vs : v[l], Q[i * ldq + l]);
        }
      }
    }
    rank++;
  }
  tsync();
  return rank;
}

// Two forms with the same result contract.  wtqr_small (below 8 rows of
// W): one thread per column for the norms and the classic reflector
// application, little fixed cost per step, for the many small per-stage
// factorizations that run several CTAs to an SM.  wtqr_large: norms on the
// balanced layout, the one-barrier arg-max, the fused Householder step with
// seeded scalars, and a warp-local update of Q, for the factorizations on
// the critical path of the sweeps.
static __device__ int wtqr(const double *K, int ldk, int rk, int nk, double tau_rank, double *W, int ldw,
                    double *Q, int ldq, int *perm, double *scr /* >= nk + max(nk, rk) + 2 */) {
  if (nk < 8) return wtqr_small(K, ldk, rk, nk, tau_rank, W, ldw, Q, ldq, perm, scr);
  return wtqr_large(K, ldk, rk, nk, tau_rank, W, ldw, Q, ldq, perm, scr);
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
  // reciprocals of R's diagonal (into X's first column, rewritten below), so that the
  // substitution chains carry multiplies instead of divides
  double *rdiag = X;
  for (int i = tid; i < rank; i += TEAM) rdiag[i * ldx] = 1.0 / W[i * ldw + i];
  tsync();
  double rmax = 0.0;
  for (int c = tid; c < nb; c += TEAM) {
    for (int i = 0; i < rank; i++) {
      double s = B[perm[i] * ldb + c];
      for (int l = 0; l < i; l++) s = fma(-W[l * ldw + i], Y[l * ldy + c], s);
      Y[i * ldy + c] = s * rdiag[i * ldx];
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
// Cholesky factor of a bordered matrix, by ONE warp: on entry the lower
// triangle of the leading kh x kh block of Hm (row-major, ld) holds the
// symmetric H and row kh holds g (columns 0..kh-1); on exit the lower triangle
// holds L with L L' = H and row kh holds L^{-1} g (the factor of [H g; g' *]
// without its last diagonal).  Left-looking by columns: lane i owns rows i and
// i + 32 (kh + 1 <= 64), and column j is one dot product of length j per row,
// so each FP64 instruction carries every row still below the diagonal; the
// pivot's reciprocal square root comes from seeded_rsqrt.  The upper triangle
// is left as it was.  Returns nonzero when a pivot is not positive.
// Rows 32 .. kh (kh + 1 > 32) go to the lanes whose own row is already done:
// at column j lane l < j has finished row l, so it takes row l + 32, and one
// chain of length j per lane covers every open row; only for j < kh + 1 - 32
// does a lane hold two open rows and run a second chain.
static __device__ int wchol_bordered(double *Hm, int ld, int kh) {
  const int lane = threadIdx.x & 31;
  const int extra = kh + 1 - 32;  // rows beyond the warp's first 32 (<= 0: none)
  int fail = 0;
  for (int j = 0; j < kh; j++) {
    // this lane's open rows: ia (its chain), ib (a second chain, only while j < extra)
    int ia = (lane >= j && lane <= kh) ? lane : -1, ib = -1;
    if (lane + 32 <= kh && lane + 32 >= j) {
      if (ia < 0) ia = lane + 32;
      else ib = lane + 32;
    }
    const double *rj = Hm + j * ld;
    double s0 = 0.0, s1 = 0.0;
    if (ia >= 0) {
      const double *ri = Hm + ia * ld;
      s0 = ri[j];
      for (int l = 0; l < j; l++) s0 = fma(-ri[l], rj[l], s0);
    }
    if (j < extra && ib >= 0) {
      const double *ri = Hm + ib * ld;
      s1 = ri[j];
      for (int l = 0; l < j; l++) s1 = fma(-ri[l], rj[l], s1);
    }
    // row j is lane j's first row (j < 32) or lane j - 32's (then its only open row)
    const double sd = __shfl_sync(kFull, s0, j & 31);
    bool ok;
    double inv = seeded_rsqrt(sd, ok);
    if (!(sd > 0.0)) fail = 1;
    if (!ok) inv = 1.0 / sqrt(fmax(sd, 1e-300));
    const double dj = sd * inv;
    if (ia >= 0) Hm[ia * ld + j] = (ia == j) ? dj : s0 * inv;
    if (ib >= 0) Hm[ib * ld + j] = s1 * inv;
    __syncwarp();
  }
  return fail;
}

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

// Stable in-place reorder of the rows [r0, r0 + R) of M, columns [c0, c1), by key[i]
// ascending (ties keep their order): each thread moves whole columns along the cycles of
// the permutation.  key and rank are scratch of R ints each (key is overwritten).
static __device__ void rows_by_key(double *M, int ld, int r0, int R, int c0, int c1, int *key, int *rank) {
  const int tid = team_rank();
  for (int i = tid; i < R; i += TEAM) {
    int rk = 0;
    for (int j = 0; j < R; j++) rk += (key[j] < key[i] || (key[j] == key[i] && j < i)) ? 1 : 0;
    rank[i] = rk;  // row i moves to position rank[i]
  }
  tsync();
  for (int i = tid; i < R; i += TEAM) {  // key[i] <- i leads its cycle (its smallest index)
    int j = rank[i];
    bool first = true;
    while (j != i) {
      if (j < i) first = false;
      j = rank[j];
    }
    key[i] = first ? 1 : 0;
  }
  tsync();
  for (int c = c0 + tid; c < c1; c += TEAM) {
    double *col = M + (size_t)r0 * ld + c;
    for (int i = 0; i < R; i++) {
      if (!key[i]) continue;
      double carry = col[(size_t)i * ld];
      int j = rank[i];
      while (j != i) {
        const double t = col[(size_t)j * ld];
        col[(size_t)j * ld] = carry;
        carry = t;
        j = rank[j];
      }
      col[(size_t)i * ld] = carry;
    }
  }
  tsync();
}

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
  wscale_rows(M, ld, rc, off, nc);
  for (int j = tid; j < nc; j += TEAM) done[j] = 0;
  double nu2, om;
  wcol_max(M, ld, 0, rc, off, nullptr, off, nu2, om);
  const double nu = sqrt(nu2);
  om = fmax(1.0, om);
  const double thr = tau_rank * nu;
  // A
  res.k1 = hh_pivoted(M, ld, 0, rc, 0, ne, 0, nc, done, pc, thr, v, w);
  // B: the reciprocal pivots up front; the thread that updates a cost row's
  // next pivot entry also forms that row's next multiplier (two buffers), so
  // each pivot costs one barrier
  if (res.k1 > 0) {
    double *pinv = v, *wb[2] = {w, v + res.k1};  // k1 + rq <= r doubles of v
    for (int p = tid; p < res.k1; p += TEAM) pinv[p] = 1.0 / M[p * ld + pc[p]];
    tsync();
    for (int q = tid; q < rq; q += TEAM) wb[0][q] = M[(rc + q) * ld + pc[0]] * pinv[0];
    tsync();
    for (int p = 0; p < res.k1; p++) {
      const int col = pc[p], coln = (p + 1 < res.k1) ? pc[p + 1] : -1;
      const double *wc = wb[p & 1];
      double *wn = wb[(p + 1) & 1];
      for (int idx = tid; idx < rq * nc; idx += TEAM) {
        const int q = idx / nc, j = idx - q * nc;
        const double val = (j == col) ? 0.0 : fma(-wc[q], M[p * ld + j], M[(rc + q) * ld + j]);
        M[(rc + q) * ld + j] = val;
        if (j == coln) wn[q] = val * pinv[p + 1];
      }
      tsync();
    }
  }
  // C, on the cost rows with an entry in an eliminated column: the others (cost rows of
  // an operand that never involved these variables) are moved after them, unchanged by
  // the steps, which would leave them as they are
  int rce = r;
  if (rq > 1 && ne > 0) {
    int *has = (int *)v, *rank = has + rq;  // v holds r doubles
    for (int i = tid; i < rq; i += TEAM) {
      int h = 1;
      for (int j = 0; j < ne; j++)
        if ((__double_as_longlong(M[(rc + i) * ld + j]) << 1) != 0) { h = 0; break; }
      has[i] = h;  // 0: has an entry in an eliminated column (sorts first)
    }
    tsync();
    int cnt = 0;
    for (int i = 0; i < rq; i++) cnt += has[i] == 0 ? 1 : 0;
    rce = rc + cnt;
    tsync();
    if (cnt < rq) rows_by_key(M, ld, rc, rq, 0, nc, has, rank);
  }
  double nuq2, om_unused;
  wcol_max(M, ld, rc, rce, ne, done, -1, nuq2, om_unused);
  const double nuq = sqrt(nuq2);
  res.k2 = hh_pivoted(M, ld, rc, rce, 0, ne, 0, nc, done, nullptr, tau_rank * nuq, v, w);
  const int kk = rc + res.k2;
  // D
  res.kc = hh_pivoted(M, ld, res.k1, rc, ne, off, ne, nc, done, nullptr, thr, v, w);
  const int kd = res.k1 + res.kc;
  int bad = 0;
  for (int i = kd + tid; i < rc; i += TEAM)
    if (fabs(M[i * ld + off]) > tau_inc * om) bad = 1;
  res.inconsistent = __syncthreads_or(bad);
  wnorm_rows_out(M, ld, res.k1, res.kc, ne, nk, off, outC, ldo);
  // E: compress the remaining cost rows over the kept columns (no pivoting).  Rows with
  // no entry in the first kept columns (cost rows of an operand that the eliminated
  // variables never touched) are moved last, ordered by their first nonzero kept column
  // (exact zeros, compared as bit patterns), and each Householder step works only on
  // the rows with an entry in its column or before it: the others are zero there and a
  // reflector would leave them unchanged.  The rows' order does not change the factor
  // beyond rounding and row signs.  The rows move in place, one thread per column
  // following the permutation's cycles.
  int ke = kk;
  const int R = r - kk;
  if (R > 1 && nk > 0) {
    int *lead = (int *)v, *rank = lead + R;  // v holds r doubles: 2 r ints
    for (int i = tid; i < R; i += TEAM) {
      int c = nk;
      for (int j = 0; j < nk; j++)
        if ((__double_as_longlong(M[(kk + i) * ld + ne + j]) << 1) != 0) { c = j; break; }
      lead[i] = c;
    }
    tsync();
    for (int c = tid; c < nk; c += TEAM) {
      int cnt = 0;
      for (int i = 0; i < R; i++) cnt += lead[i] <= c ? 1 : 0;
      done[c] = kk + cnt;  // rows [kk, done[c]) may have an entry in kept column c
    }
    rows_by_key(M, ld, kk, R, ne, nc, lead, rank);
    for (int col = ne; col < off && ke < r; col++) {
      const int re = done[col - ne];
      if (re <= ke) continue;  // no row from ke on has an entry in this column
      HHLayout L = hh_layout(nc - col, re - ke);
      if (hh_core(M, ld, ke, re, col, nullptr, col, nc - col, L, v, w, 0.0) > 0.0) ke++;
    }
  } else {
    ke = hh_diag_steps(M, ld, ke, r, ne, off, nc, v, w, 0.0, false);
  }
  res.kq = ke - kk;
  for (int idx = tid; idx < res.kq * (nk + 1); idx += TEAM) {
    int a = idx / (nk + 1), j = idx - a * (nk + 1);
    outQ[a * ldo + j] = M[(kk + a) * ld + ne + j];
  }
  tsync();
  return res;
}

}  // namespace eclqr
