// Eigen_HH step 2 (Sec. 3: the paper calls LAPACK dstevx, i.e. bisection + inverse
// iteration): all eigenpairs of a real symmetric tridiagonal T = tridiag(e, d, e).
//
// * Splitting: an off-diagonal with e_i^2 <= eps^2 |d_i d_{i+1}| + tiny is set to zero;
//   each unreduced block is solved on its own and its eigenvectors vanish outside it.
//   Slot j of a problem holds eigenvalue (j - b0) of the block [b0, b1) containing row j.
// * Eigenvalues (kernel 1, several blocks per problem, one thread per slot):
//   Sturm counts are sign changes of the leading principal minors
//   p_i = (d_i - x) p_{i-1} - e_{i-1}^2 p_{i-2} (a zero minor takes the sign of its
//   predecessor), rescaled by powers of two: the division-free form of the LDL^T pivot
//   count, three operations per step.
//     1. bisection in FP32 (64x the FP64 rate on this GPU) to ~1e-7 |T|, counting negative
//        pivots of the LDL^T form with a fast reciprocal;
//     2. the FP32 bracket, widened by 8 eps_32 |T| (an FP32 count is exact for a matrix
//        within a few eps_32 |T| of T), is verified with two FP64 counts (the full
//        Gershgorin interval replaces it if a count disagrees);
//     3. an eigenvalue that the bracket isolates is finished by safeguarded Newton steps on
//        the characteristic polynomial and confirmed by FP64 counts; the others (and
//        any unconfirmed one) are queued and bisected in FP64 to eps |T| by a second kernel,
//        one thread per queue entry, so that its warps are full.
// * Eigenvectors (kernel 2, same block split): inverse iteration with a partially pivoted LU
//   of T - lambda I (tiny pivots perturbed to eps |T|), a scaled right-hand side, the growth
//   test |x|_inf >= sqrt(0.1/blocksize) within `maxits` solves plus two extra solves, and
//   modified Gram-Schmidt against the earlier members of a tight cluster (gap < 1e-11 |T|_1;
//   1e-9 |T|_1 when kernel 0 runs), whose leader walks the cluster in order.  Wider
//   near-degeneracies leave overlaps of order eps|T|/gap, which the caller removes with
//   Newton-Schulz steps Z <- Z (3I - Z^T Z)/2 (each squares them): one step for gaps
//   >= 1e-9 |T|_1 (overlaps <= ~1e-7), a second one for the problems flagged in ns2[] because
//   a gap lies in [1e-11, 1e-9) |T|_1 (overlaps <= ~1e-5).
//   A tight cluster of more than BIG members (the near-null spectrum of an ill-conditioned
//   overlap matrix can chain hundreds) is handed to kernel 3: one block per cluster, the
//   same iteration with the reorthogonalisation done by the whole block (classical
//   Gram-Schmidt applied twice) while one thread runs the tridiagonal solves.  A chain can
//   span far more than the tight band; a member is re-orthogonalised only against the
//   finished members within the band of its own eigenvalue (the others overlap it by at
//   most eps|T| over the band, which the Newton-Schulz steps remove).
// * Output: eigenvalues ascending (across blocks), eigenvectors in matching columns,
//   unit 2-norm, largest component positive.  All loops are bounded.
#include <cfloat>

#include "nao_internal.cuh"

namespace {

constexpr int ST_THREADS = 64;    // = slots per block (eigenvectors): the overlap phase (64 problems)
                                  // has ~36k of them, so 64-thread blocks spread over all SMs
constexpr int SZ_THREADS = 64;    // = slots per block (eigenvalues): ~8 blocks per SM for 128 problems
                                  // of n = 568, so the SMs' FP64 pipes finish within one block of each other
constexpr int EXTRA = 2;          // extra solves after the growth test passes (members of tight clusters)
constexpr int EXTRA_ISOLATED = 1; // the same for an eigenvalue outside any tight cluster: its gap is at
                                  // least 1e-11 |T|_1, so the other eigenvectors' components fall to
                                  // their rounding floor eps |T| / gap < 2.2e-5 within one solve past
                                  // the growth test; the Newton-Schulz steps remove that floor
constexpr double TIGHT = 1e-9;      // gaps below it need more than one Newton-Schulz step...
constexpr double TIGHT_GS = 1e-11;  // ...and below this, Gram-Schmidt (without MRRR vectors; with
                                    // them, Gram-Schmidt starts at TIGHT: the big clusters that the
                                    // wider band chains go to MRRR, which needs no serial walk)
constexpr int NARR = 6;           // scratch arrays per eigenvalue: L, U0inv, U1, U2, PIV, X
constexpr int BIG = 32;           // tight clusters with more members go to stein_cluster_kernel
constexpr int NEWTON_MAX = 6;     // Newton steps on an isolated eigenvalue before it is queued
constexpr int BQ_LANES = 4;       // lanes per queued eigenvalue in the FP64 bisection (multisection)

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Shared per-problem set-up: d, e (split), e^2 in shared memory; Gershgorin interval,
// max |T| and 1-norm; block boundaries.
struct TriInfo {
  double gl, gu, tnorm, onenrm;
};

__device__ TriInfo load_tridiag(int m, const double* __restrict__ din, const double* __restrict__ ein, double* d,
                                double* e, double* e2, int* bst, int* ben, double* red) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  const double eps = DBL_EPSILON * 0.5;
  for (int i = tid; i < m; i += nt) {
    const double di = din[i];
    d[i] = di;
    double ei = (i < m - 1) ? ein[i] : 0.0;
    if (i < m - 1) {
      const double dn = din[i + 1];
      if (ei * ei <= eps * eps * fabs(di * dn) + DBL_MIN) ei = 0.0;
    }
    e[i] = ei;
    e2[i] = ei * ei;
  }
  __syncthreads();
  double lmin = 1e300, lmax = -1e300, lnrm = 0.0;
  for (int i = tid; i < m; i += nt) {
    const double r = fabs(e[i]) + (i > 0 ? fabs(e[i - 1]) : 0.0);
    lmin = fmin(lmin, d[i] - r);
    lmax = fmax(lmax, d[i] + r);
    lnrm = fmax(lnrm, fabs(d[i]) + r);
  }
  lmin = warp_min(lmin);
  lmax = warp_max(lmax);
  lnrm = warp_max(lnrm);
  if (lane == 0) {
    red[wid] = lmin;
    red[32 + wid] = lmax;
    red[64 + wid] = lnrm;
  }
  if (tid == 0) {  // block boundaries (serial, O(m))
    int b0 = 0;
    for (int i = 0; i < m; ++i) {
      bst[i] = b0;
      if (i == m - 1 || e[i] == 0.0) {
        for (int k = b0; k <= i; ++k) ben[k] = i + 1;
        b0 = i + 1;
      }
    }
  }
  __syncthreads();
  TriInfo t;
  t.gl = 1e300;
  t.gu = -1e300;
  t.onenrm = 0.0;
  for (int k = 0; k < nw; ++k) {
    t.gl = fmin(t.gl, red[k]);
    t.gu = fmax(t.gu, red[32 + k]);
    t.onenrm = fmax(t.onenrm, red[64 + k]);
  }
  t.tnorm = fmax(fmax(fabs(t.gl), fabs(t.gu)), DBL_MIN);
  t.gl -= 4.0 * eps * t.tnorm * m + 2.0 * DBL_MIN;
  t.gu += 4.0 * eps * t.tnorm * m + 2.0 * DBL_MIN;
  if (t.onenrm == 0.0) t.onenrm = 1.0;
  return t;
}

// FP32 Sturm count of T[b0:b1) below x (matrix rounded to FP32), pivot form
// q_i = (d_i - x) - e_{i-1}^2 / q_{i-1} with a fast approximate reciprocal: this count only
// isolates eigenvalues; the bracket it gives is widened and re-verified in FP64.
__device__ int sturm_count32(const float* __restrict__ d, const float* __restrict__ e2, int b0, int b1, float x) {
  const float pivmin = 1e-30f;
  float q = d[b0] - x;
  if (fabsf(q) < pivmin) q = -pivmin;
  int cnt = q < 0.f;
  for (int i = b0 + 1; i < b1; ++i) {
    q = (d[i] - x) - __fdividef(e2[i - 1], q);
    if (fabsf(q) < pivmin) q = -pivmin;
    cnt += q < 0.f;
  }
  return cnt;
}

// FP64 Sturm count below x, and p_n(x), p_n'(x) up to a common positive power-of-two
// factor (for Newton's step p / p'), with the scale of p, p', and their predecessors checked
// once per four steps while |T| < 2^60 (see sturm64_count; p' grows by the same factor plus
// |p|), every step beyond.
__device__ int sturm64_deriv(const double* __restrict__ d, const double* __restrict__ e2, int b0, int b1, double x,
                             double tnorm, double* pn_out, double* dpn_out) {
  double pm1 = 1.0, p = d[b0] - x;
  double qm1 = 0.0, q = -1.0;  // derivatives
  long long bits = __double_as_longlong(p);
  int sn = (bits < 0) && ((bits << 1) != 0);
  int cnt = sn;
  auto step = [&](int i) {
    const double t = d[i] - x;
    const double pn = fma(t, p, -e2[i - 1] * pm1);
    const double qn = fma(t, q, fma(-e2[i - 1], qm1, -p));
    qm1 = q;
    q = qn;
    pm1 = p;
    p = pn;
    bits = __double_as_longlong(p);
    const int ns = ((bits << 1) == 0) ? sn : (int)(bits < 0);
    cnt += (ns != sn);
    sn = ns;
  };
  auto rescale = [&]() {
    const int ex = (int)((__double_as_longlong(p) >> 52) & 0x7ff), ex1 = (int)((__double_as_longlong(pm1) >> 52) & 0x7ff);
    const int eq = (int)((__double_as_longlong(q) >> 52) & 0x7ff), eq1 = (int)((__double_as_longlong(qm1) >> 52) & 0x7ff);
    const int emax = max(max(ex, ex1), max(eq, eq1));
    if (emax > 1023 + 400) {
      p *= 0x1p-400;
      pm1 *= 0x1p-400;
      q *= 0x1p-400;
      qm1 *= 0x1p-400;
    } else if (emax < 1023 - 400 && emax > 0) {
      p *= 0x1p400;
      pm1 *= 0x1p400;
      q *= 0x1p400;
      qm1 *= 0x1p400;
    }
  };
  int i = b0 + 1;
  const int b4 = tnorm < 0x1p60 ? b1 : b0 + 1;
  for (; i + 4 <= b4; i += 4) {
    step(i);
    step(i + 1);
    step(i + 2);
    step(i + 3);
    rescale();
  }
  for (; i < b1; ++i) {
    step(i);
    rescale();
  }
  *pn_out = p;
  *dpn_out = q;
  return cnt;
}

// FP64 Sturm count below x (the count of sturm64_deriv without the derivative): the same
// recurrence and rescaling, with the scale checked once per four steps while |T| < 2^60:
// four steps then grow |p| by at most (2|T| + |T|^2)^4 < 2^481, so the 2^400 threshold keeps
// every value finite (larger |T| checks every step, as sturm64 does).
__device__ int sturm64_count(const double* __restrict__ d, const double* __restrict__ e2, int b0, int b1, double x,
                             double tnorm) {
  double pm1 = 1.0, p = d[b0] - x;
  long long bits = __double_as_longlong(p);
  int sn = (bits < 0) && ((bits << 1) != 0);
  int cnt = sn;
  auto step = [&](int i) {
    const double t = d[i] - x;
    const double pn = fma(t, p, -e2[i - 1] * pm1);
    pm1 = p;
    p = pn;
    bits = __double_as_longlong(p);
    const int ns = ((bits << 1) == 0) ? sn : (int)(bits < 0);
    cnt += (ns != sn);
    sn = ns;
  };
  auto rescale = [&]() {
    const int ex = (int)((__double_as_longlong(p) >> 52) & 0x7ff), ex1 = (int)((__double_as_longlong(pm1) >> 52) & 0x7ff);
    const int emax = ex > ex1 ? ex : ex1;
    if (emax > 1023 + 400) {
      p *= 0x1p-400;
      pm1 *= 0x1p-400;
    } else if (emax < 1023 - 400 && emax > 0) {
      p *= 0x1p400;
      pm1 *= 0x1p400;
    }
  };
  int i = b0 + 1;
  const int b4 = tnorm < 0x1p60 ? b1 : b0 + 1;  // end of the four-step part
  for (; i + 4 <= b4; i += 4) {
    step(i);
    step(i + 1);
    step(i + 2);
    step(i + 3);
    rescale();
  }
  for (; i < b1; ++i) {
    step(i);
    rescale();
  }
  return cnt;
}

__device__ __forceinline__ double hash_uniform(unsigned long long key) {
  // splitmix64 finaliser -> uniform in (-1, 1)
  key += 0x9E3779B97F4A7C15ull;
  key = (key ^ (key >> 30)) * 0xBF58476D1CE4E5B9ull;
  key = (key ^ (key >> 27)) * 0x94D049BB133111EBull;
  key ^= key >> 31;
  return (double)(key >> 11) * 0x1p-52 - 1.0;
}

// Safeguarded Newton steps on p_n inside a bracket [lo, hi] that isolates eigenvalue idx of
// T[b0:b1) (count(lo) = idx, count(hi) = idx + 1); every evaluation's count narrows the
// bracket.  True when lam is confirmed within 2 tol, tol = max(2 eps |x|, eps |T|) (the
// bisection's final bracket width; the margin covers the counts' own backward error of a few
// eps |T|), by the last iterate's count on one side and one more FP64 count on the other.  A step within rounding of the root may leave the one-sided
// bracket, so convergence is tested before the step is kept inside it.
__device__ bool newton_finish(const double* __restrict__ d, const double* __restrict__ e2, int b0, int b1, int idx,
                              double tnorm, double& lo, double& hi, int& clo, int& chi, double& lam) {
  const double eps = DBL_EPSILON * 0.5;
  double x = 0.5 * (lo + hi);
  for (int it = 0; it < NEWTON_MAX; ++it) {
    double pn, dpn;
    const int c = sturm64_deriv(d, e2, b0, b1, x, tnorm, &pn, &dpn);
    if (c > idx) {
      hi = x;
      chi = c;
    } else {
      lo = x;
      clo = c;
    }
    const double tol = fmax(2.0 * eps * fabs(x), eps * tnorm);
    double xn = x - pn / dpn;
    if (fabs(xn - x) <= tol) {
      // x's count fixed one side of lambda (|xn - x| <= tol); one count 2 tol beyond xn on
      // the other side closes the bracket within [xn - 2 tol, xn + 2 tol]
      lam = xn;
      return c > idx ? sturm64_count(d, e2, b0, b1, xn - 2.0 * tol, tnorm) <= idx
                     : sturm64_count(d, e2, b0, b1, xn + 2.0 * tol, tnorm) > idx;
    }
    if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);  // outside, or not finite: bisect
    x = xn;
  }
  return false;
}

// ---------------------------------------------------------------- kernel 1: eigenvalues
__global__ void __launch_bounds__(SZ_THREADS)
stebz_kernel(int n, const int32_t* __restrict__ size, const double* __restrict__ dbase, const double* __restrict__ ebase,
             long long strideV, double* __restrict__ wslot, int32_t* __restrict__ status, int* __restrict__ qcount,
             int4* __restrict__ qent, double* __restrict__ qlo, double* __restrict__ qhi, double* __restrict__ e2g,
             double* __restrict__ tng) {
  extern __shared__ double smd[];
  double* d = smd;
  double* e = smd + n;
  double* e2 = smd + 2 * n;
  float* d32 = (float*)(smd + 3 * n);
  float* e232 = d32 + n;
  int* bst = (int*)(e232 + n);
  int* ben = bst + n;
  __shared__ double red[96];
  const int p = blockIdx.y;
  const int m = size ? size[p] : n;
  if (m <= 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && status) status[p] = 0;
    return;
  }
  const int j = blockIdx.x * blockDim.x + threadIdx.x;  // slot
  if ((int)(blockIdx.x * blockDim.x) >= m) return;     // uniform per block
  const TriInfo T = load_tridiag(m, dbase + (size_t)p * strideV, ebase + (size_t)p * strideV, d, e, e2, bst, ben, red);
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    d32[i] = (float)d[i];
    e232[i] = (float)e2[i];
    if (blockIdx.x == 0) e2g[(size_t)p * n + i] = e2[i];  // the split e^2, for the queue kernel
  }
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (status) status[p] = 0;
    tng[p] = T.tnorm;
  }
  if (j >= m) return;
  const int b0 = bst[j], b1 = ben[j];
  double lam;
  if (b1 - b0 == 1) {
    lam = d[b0];
  } else {
    const int idx = j - b0;
    // 1. FP32 bisection
    float lo32 = (float)T.gl, hi32 = (float)T.gu;
    const float tn32 = (float)T.tnorm;
    for (int it = 0; it < 64; ++it) {
      const float mid = 0.5f * (lo32 + hi32);
      if (hi32 - lo32 <= 4.0f * FLT_EPSILON * tn32 || mid <= lo32 || mid >= hi32) break;
      if (sturm_count32(d32, e232, b0, b1, mid) > idx) hi32 = mid;
      else lo32 = mid;
    }
    // 2. FP64 bracket from it, verified
    // the FP32 midpoint was measured within 1.9 eps_32 |T| of the eigenvalue (matrices of
    // the magnetite-shaped cell); 8 eps_32 |T| on each side, and the FP64 counts check it
    const double margin = 8.0 * (double)FLT_EPSILON * T.tnorm;
    double lo = fmax((double)lo32 - margin, T.gl), hi = fmin((double)hi32 + margin, T.gu);
    const int clo = sturm64_count(d, e2, b0, b1, lo, T.tnorm);
    const int chi = sturm64_count(d, e2, b0, b1, hi, T.tnorm);
    if (!(clo <= idx && idx < chi)) {
      lo = T.gl;
      hi = T.gu;
    }
    // 3. An eigenvalue that the bracket isolates is finished by newton_finish.  Every other
    //    one (a cluster the FP32 bracket does not split, or no confirmed convergence) goes
    //    to a queue that a second kernel bisects with full warps: bisecting it here would
    //    hold the whole warp for ~40 FP64 steps.
    int cl = clo, ch = chi;
    if (!(cl <= idx && idx < ch)) {
      cl = 0;
      ch = b1 - b0;
    }
    bool ok = false;
    if (cl == idx && ch == idx + 1) ok = newton_finish(d, e2, b0, b1, idx, T.tnorm, lo, hi, cl, ch, lam);
    if (!ok) {
      const int k = atomicAdd(qcount, 1);  // one queue over all problems
      qent[k] = make_int4(p, j, b0, b1);
      qlo[k] = lo;
      qhi[k] = hi;
      return;
    }
  }
  wslot[(size_t)p * n + j] = lam;
}

// Kernel 1b: FP64 bisection of the queued eigenvalues of all problems, one thread per queue
// entry, so that the warps are full however few entries each problem has.  An entry carries
// its problem, slot, split block and verified bracket; d and the split e^2 are read from
// global memory (each lane streams its own problem's arrays).  (Switching a lane to Newton
// once its bracket isolates the eigenvalue was measured slower: the lanes of a warp reach
// isolation at different steps, so the two paths serialise.)
__global__ void __launch_bounds__(SZ_THREADS)
stebz_bisect_kernel(int n, const double* __restrict__ dbase, long long strideV, const double* __restrict__ e2g,
                    const double* __restrict__ tng, double* __restrict__ wslot, const int* __restrict__ qcount,
                    const int4* __restrict__ qent, const double* __restrict__ qlo, const double* __restrict__ qhi) {
  // BQ_LANES lanes per entry: each step counts at BQ_LANES interior points of the bracket,
  // one per lane, and keeps the sub-interval that holds the eigenvalue (log2(BQ_LANES + 1)
  // bits per step instead of one): the dependent chain of steps, which sets this kernel's
  // time, is ~2.3x shorter
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int q = gt / BQ_LANES, sub = gt % BQ_LANES;
  if (q >= *qcount) return;  // uniform over the entry's lanes
  const unsigned gmask = ((1u << BQ_LANES) - 1u) << ((threadIdx.x & 31) & ~(BQ_LANES - 1));
  const int4 en = qent[q];
  const int p = en.x, j = en.y, b0 = en.z, b1 = en.w, idx = j - b0;
  const double* d = dbase + (size_t)p * strideV;
  const double* e2 = e2g + (size_t)p * n;
  const double tn = tng[p];
  const double eps = DBL_EPSILON * 0.5;
  double lo = qlo[q], hi = qhi[q];
  for (int it = 0; it < 128; ++it) {
    const double mid = 0.5 * (lo + hi);
    const double tol = fmax(2.0 * eps * fmax(fabs(lo), fabs(hi)), eps * tn);
    if (hi - lo <= tol || mid <= lo || mid >= hi) break;
    const double h = (hi - lo) / (BQ_LANES + 1);
    const double x = lo + h * (sub + 1);
    const bool above = (x > lo && x < hi) ? sturm64_count(d, e2, b0, b1, x, tn) > idx : x >= hi;
    // the lowest point with more than idx eigenvalues below it bounds the eigenvalue from
    // above, the point before it from below (every lane forms the same bracket)
    const unsigned ab = __ballot_sync(gmask, above) & gmask;
    const int k = ab ? __ffs(ab) - 1 - ((threadIdx.x & 31) & ~(BQ_LANES - 1)) : BQ_LANES;
    const double xk = lo + h * (k + 1), xk1 = lo + h * k;
    if (k < BQ_LANES) hi = xk;
    if (k > 0) lo = xk1;
  }
  if (sub == 0) wslot[(size_t)p * n + j] = 0.5 * (lo + hi);
}

// ---------------------------------------------------------------- kernel 2: eigenvectors
__global__ void __launch_bounds__(ST_THREADS, 8)  // up to 8 blocks per SM (shared memory allows ~9)
stein_vec_kernel(int n, const int32_t* __restrict__ size, const double* __restrict__ dbase, const double* __restrict__ ebase,
                 long long strideV, const double* __restrict__ wslot, double* __restrict__ wbase,
                 double* __restrict__ Zbase, int ldz, long long strideZ, double* __restrict__ scratch,
                 int32_t* __restrict__ status, int* __restrict__ biglist, int bigcap,
                 const int32_t* __restrict__ nvec, int nvec_max, int maxits, const int* __restrict__ mdone,
                 int* __restrict__ ns2, double tgs) {
  extern __shared__ double smd[];
  double* d = smd;
  double* e = smd + n;
  double* e2 = smd + 2 * n;
  double* w = smd + 3 * n;
  int* bst = (int*)(smd + 4 * n);
  int* ben = bst + n;
  __shared__ double red[96];
  __shared__ int s_fail;
  const int p = blockIdx.y;
  const int m = size ? size[p] : n;
  if (m <= 0 || (int)(blockIdx.x * blockDim.x) >= m) return;  // uniform per block
  const TriInfo T = load_tridiag(m, dbase + (size_t)p * strideV, ebase + (size_t)p * strideV, d, e, e2, bst, ben, red);
  const double* ws = wslot + (size_t)p * n;
  for (int i = threadIdx.x; i < m; i += blockDim.x) w[i] = ws[i];
  if (threadIdx.x == 0) s_fail = 0;
  __syncthreads();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int nv = min(nvec ? nvec[p] : m, nvec_max);  // vectors of the lowest nv eigenvalues only
  double* wout = wbase + (size_t)p * strideV;
  double* Z = Zbase + (size_t)p * strideZ;
  double* scr = scratch + (size_t)p * NARR * n * n;
  const double eps = DBL_EPSILON * 0.5;
  const double tight = tgs * T.onenrm, tight1 = TIGHT * T.onenrm;
  const double pivtol = eps * T.tnorm;
  const size_t nn = (size_t)n * n;
  if (j < m && ns2 && j > bst[j]) {  // a gap that one Newton-Schulz step does not cover
    const double gap = w[j] - w[j - 1];
    if (gap < tight1 && !(gap < tight)) ns2[p] = 1;
  }
  if (j < m) {
    // global ascending order (ties broken by slot)
    const double wj = w[j];
    int rk = 0;
    for (int t = 0; t < m; ++t) {
      const double wt = w[t];
      rk += (wt < wj) || (wt == wj && t < j);
    }
    wout[rk] = wj;
  }
  __syncthreads();
  if (j < m) {
    const int b0 = bst[j], b1 = ben[j];
    const bool leader = !(j > b0 && w[j] - w[j - 1] < tight);
    int jend = j + 1;
    if (leader)
      while (jend < b1 && w[jend] - w[jend - 1] < tight) ++jend;
    if (leader && jend - j > BIG) {  // hand the cluster to kernel 3
      const int slot = atomicAdd(&biglist[0], 1);
      if (slot < bigcap) {
        biglist[1 + 3 * slot] = p;
        biglist[2 + 3 * slot] = j;
        biglist[3 + 3 * slot] = jend;
      } else {
        s_fail = 1;
      }
    } else if (leader) {
      const int bs = b1 - b0;
      double* __restrict__ Lr = scr + 0 * nn;
      double* __restrict__ U0i = scr + 1 * nn;
      double* __restrict__ U1 = scr + 2 * nn;
      double* __restrict__ U2 = scr + 3 * nn;
      double* __restrict__ PV = scr + 4 * nn;
      double* __restrict__ X = scr + 5 * nn;
      const int sl = j;  // scratch column of this leader
#define AT(arr, i) arr[(size_t)(i) * n + sl]
      double lamprev = 0.0;
      for (int q = j; q < jend; ++q) {
        // rank of slot q (recomputed: members of a cluster may belong to other threads' slots)
        const double wq = w[q];
        int rq = 0;
        for (int t = 0; t < m; ++t) {
          const double wt = w[t];
          rq += (wt < wq) || (wt == wq && t < q);
        }
        if (rq >= nv) break;  // members ascend: the rest of the cluster is not wanted either
        const int* dn = mdone ? mdone + (size_t)p * n : nullptr;
        if (dn && dn[q]) {  // an MRRR vector (kernel 0) is already in Z
          lamprev = wq;
          continue;
        }
        double* zc = Z + (size_t)rq * ldz;
        if (bs == 1) {
          for (int i = 0; i < m; ++i) zc[i] = (i == b0) ? 1.0 : 0.0;
          lamprev = wq;
          continue;
        }
        double lam = wq;
        if (q > j) {
          const double pertol = 10.0 * fabs(eps * lam);
          if (lam - lamprev < pertol) lam = lamprev + pertol;
        }
        lamprev = lam;
        // LU with partial pivoting of T[b0:b1) - lam I
        double al = d[b0] - lam, be = e[b0];
        for (int k = b0; k < b1 - 1; ++k) {
          const double c = e[k];
          const double an = d[k + 1] - lam;
          const double bn = (k + 1 < b1 - 1) ? e[k + 1] : 0.0;
          // the pivot (perturbed when tiny) serves both the multiplier l = num / u0 and
          // the stored 1/u0: one FP64 reciprocal instead of two divisions
          double u0, u1, u2, num, piv;
          if (fabs(al) >= fabs(c)) {
            piv = 0.0;
            u0 = al;
            u1 = be;
            u2 = 0.0;
            num = c;
          } else {
            piv = 1.0;
            u0 = c;
            u1 = an;
            u2 = bn;
            num = al;
          }
          if (fabs(u0) < pivtol) u0 = copysign(pivtol, u0);
          const double rinv = 1.0 / u0;
          const double l = num * rinv;
          const double al2 = piv == 0.0 ? an - l * be : be - l * an;
          const double be2 = piv == 0.0 ? bn : -l * bn;
          AT(U0i, k) = rinv;
          AT(U1, k) = u1;
          AT(U2, k) = u2;
          AT(Lr, k) = l;
          AT(PV, k) = piv;
          al = al2;
          be = be2;
        }
        if (fabs(al) < pivtol) al = copysign(pivtol, al);
        const double ulast = al;
        AT(U0i, b1 - 1) = 1.0 / al;
        // x1 = |X|_1 of the next right-hand side, summed in row order as it is written (the
        // start vector) or read by the previous iteration's norm pass
        double x1 = 0.0;
        for (int i = b0; i < b1; ++i) {
          const double xi =
              hash_uniform(((unsigned long long)p << 40) ^ ((unsigned long long)q << 20) ^ (unsigned long long)i);
          AT(X, i) = xi;
          x1 += fabs(xi);
        }
        int its = 0, nrmchk = 0;
        bool ok = false;
        while (its < maxits + EXTRA) {
          ++its;
          const double scl = (double)bs * T.onenrm * fmax(eps, fabs(ulast)) / fmax(x1, DBL_MIN);
          double r = AT(X, b0) * scl;
#pragma unroll 4
          for (int k = b0; k < b1 - 1; ++k) {
            const double xn = AT(X, k + 1) * scl;
            const double l = AT(Lr, k);
            if (AT(PV, k) == 0.0) {
              AT(X, k) = r;
              r = xn - l * r;
            } else {
              AT(X, k) = xn;
              r = r - l * xn;
            }
          }
          AT(X, b1 - 1) = r;
          double x2 = 0.0, x1v = AT(X, b1 - 1) * AT(U0i, b1 - 1);
          AT(X, b1 - 1) = x1v;
#pragma unroll 4
          for (int k = b1 - 2; k >= b0; --k) {
            const double xv = (AT(X, k) - AT(U1, k) * x1v - AT(U2, k) * x2) * AT(U0i, k);
            AT(X, k) = xv;
            x2 = x1v;
            x1v = xv;
          }
          for (int t = j; t < jend; ++t) {  // reorthogonalise against the cluster's finished members
            if (t == q || (t > q && !(dn && dn[t]))) continue;
            const double wt = w[t];
            int rt = 0;
            for (int u = 0; u < m; ++u) rt += (w[u] < wt) || (w[u] == wt && u < t);
            const double* zt = Z + (size_t)rt * ldz;
            double dot = 0.0;
            for (int i = b0; i < b1; ++i) dot = fma(AT(X, i), zt[i], dot);
            for (int i = b0; i < b1; ++i) AT(X, i) = fma(-dot, zt[i], AT(X, i));
          }
          double xinf = 0.0;
          bool finite = true;
          x1 = 0.0;
          for (int i = b0; i < b1; ++i) {
            const double a = fabs(AT(X, i));
            finite = finite && (a <= DBL_MAX);
            xinf = fmax(xinf, a);
            x1 += a;
          }
          if (!finite) break;
          if (its > maxits && nrmchk == 0) break;
          if (xinf < sqrt(0.1 / bs)) continue;
          ++nrmchk;
          if (nrmchk < (jend - j > 1 ? EXTRA : EXTRA_ISOLATED) + 1) continue;
          ok = true;
          break;
        }
        if (!ok) s_fail = 1;
        double nrm2 = 0.0, big = 0.0;
        int jmax = b0;
        for (int i = b0; i < b1; ++i) {
          const double a = AT(X, i);
          nrm2 = fma(a, a, nrm2);
          if (fabs(a) > big) {
            big = fabs(a);
            jmax = i;
          }
        }
        double sc = (nrm2 > 0.0 && nrm2 <= DBL_MAX) ? 1.0 / sqrt(nrm2) : 0.0;
        if (AT(X, jmax) < 0.0) sc = -sc;
        for (int i = 0; i < m; ++i) zc[i] = (i >= b0 && i < b1) ? AT(X, i) * sc : 0.0;
        if (sc == 0.0) zc[b0 + (q - b0) % bs] = 1.0;  // keep a unit vector even on failure
      }
#undef AT
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && s_fail && status) atomicExch(&status[p], NAO_E_NOCONV);
}

// ---------------------------------------------------------------- kernel 3: big tight clusters
// One block per cluster listed by kernel 2: members in ascending order; thread 0 factors
// T - lambda I and runs the solves (as kernel 2), the block re-orthogonalises each iterate
// against the earlier members (classical Gram-Schmidt, twice) and takes the norms.
__device__ __forceinline__ double block_sum1(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double r = 0.0;
  for (int k = 0; k < nw; ++k) r += red[k];
  return r;
}

__device__ __forceinline__ double block_max1(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double r = 0.0;
  for (int k = 0; k < nw; ++k) r = fmax(r, red[k]);
  return r;
}

constexpr int SC_THREADS = 256;

__global__ void __launch_bounds__(SC_THREADS, 1)
stein_cluster_kernel(int n, const int32_t* __restrict__ size, const double* __restrict__ dbase,
                     const double* __restrict__ ebase, long long strideV, const double* __restrict__ wslot,
                     double* __restrict__ Zbase, int ldz, long long strideZ, double* __restrict__ scratch,
                     int32_t* __restrict__ status, const int* __restrict__ biglist, int bigcap,
                     const int32_t* __restrict__ nvec, int nvec_max, int maxits, const int* __restrict__ mdone,
                     double tgs) {
  extern __shared__ double smc[];
  double* d = smc;
  double* e = smc + n;
  double* e2 = smc + 2 * n;
  double* w = smc + 3 * n;
  double* sx = smc + 4 * n;
  double* dots = e2;  // e^2 is not needed after the load: it holds the Gram-Schmidt coefficients
  int* bst = (int*)(smc + 5 * n);
  int* ben = bst + n;
  int* rnk = ben + n;
  int* fin = rnk + n;  // the finished members a member is re-orthogonalised against
  __shared__ double red[96];
  __shared__ int s_go, s_ok, s_nf;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  const int count = min(biglist[0], bigcap);
  for (int ent = blockIdx.x; ent < count; ent += gridDim.x) {
    const int p = biglist[1 + 3 * ent], j = biglist[2 + 3 * ent], jend = biglist[3 + 3 * ent];
    const int m = size ? size[p] : n;
    __syncthreads();
    const TriInfo T = load_tridiag(m, dbase + (size_t)p * strideV, ebase + (size_t)p * strideV, d, e, e2, bst, ben, red);
    const double* ws = wslot + (size_t)p * n;
    for (int i = tid; i < m; i += nt) w[i] = ws[i];
    __syncthreads();
    for (int q = j + tid; q < jend; q += nt) {  // ranks of the members (global ascending order)
      const double wq = w[q];
      int r = 0;
      for (int t = 0; t < m; ++t) r += (w[t] < wq) || (w[t] == wq && t < q);
      rnk[q - j] = r;
    }
    __syncthreads();
    double* Z = Zbase + (size_t)p * strideZ;
    double* scr = scratch + (size_t)p * NARR * n * n;
    const double eps = DBL_EPSILON * 0.5;
    const double pivtol = eps * T.tnorm;
    const size_t nn = (size_t)n * n;
    const int b0 = bst[j], b1 = ben[j], bs = b1 - b0;
    // the solves below run in one thread: their factor loads are independent of the
    // recurrence, so the loops are unrolled for the loads of several rows to be in flight
    double* __restrict__ Lr = scr + 0 * nn;
    double* __restrict__ U0i = scr + 1 * nn;
    double* __restrict__ U1 = scr + 2 * nn;
    double* __restrict__ U2 = scr + 3 * nn;
    double* __restrict__ PV = scr + 4 * nn;
    double lamprev = 0.0, ulast = 0.0;
    bool fail = false;
    const int nv = min(nvec ? nvec[p] : m, nvec_max);
    const int* dn = mdone ? mdone + (size_t)p * n : nullptr;
    for (int q = j; q < jend; ++q) {
      if (rnk[q - j] >= nv) break;  // uniform: ranks ascend with q
      if (dn && dn[q]) {  // an MRRR vector (kernel 0) is already in Z
        lamprev = w[q];
        continue;
      }
      if (tid == 0) {  // finished members within the tight band of w[q]: the earlier ones and
                       // the later MRRR vectors
        const double tband = tgs * T.onenrm, wq = w[q];
        int c = 0;
        for (int t = 0; t < jend - j; ++t)
          if ((t < q - j || (t > q - j && dn && dn[j + t])) && fabs(w[j + t] - wq) < tband) fin[c++] = t;
        s_nf = c;
      }
      const int sl = q;
#define AT(arr, i) arr[(size_t)(i) * n + sl]
      if (tid == 0) {  // LU with partial pivoting of T[b0:b1) - lam I (as kernel 2)
        double lam = w[q];
        if (q > j) {
          const double pertol = 10.0 * fabs(eps * lam);
          if (lam - lamprev < pertol) lam = lamprev + pertol;
        }
        lamprev = lam;
        double al = d[b0] - lam, be = e[b0];
        for (int k = b0; k < b1 - 1; ++k) {
          const double c = e[k];
          const double an = d[k + 1] - lam;
          const double bn = (k + 1 < b1 - 1) ? e[k + 1] : 0.0;
          // the pivot (perturbed when tiny) serves both the multiplier l = num / u0 and
          // the stored 1/u0: one FP64 reciprocal instead of two divisions
          double u0, u1, u2, num, piv;
          if (fabs(al) >= fabs(c)) {
            piv = 0.0;
            u0 = al;
            u1 = be;
            u2 = 0.0;
            num = c;
          } else {
            piv = 1.0;
            u0 = c;
            u1 = an;
            u2 = bn;
            num = al;
          }
          if (fabs(u0) < pivtol) u0 = copysign(pivtol, u0);
          const double rinv = 1.0 / u0;
          const double l = num * rinv;
          const double al2 = piv == 0.0 ? an - l * be : be - l * an;
          const double be2 = piv == 0.0 ? bn : -l * bn;
          AT(U0i, k) = rinv;
          AT(U1, k) = u1;
          AT(U2, k) = u2;
          AT(Lr, k) = l;
          AT(PV, k) = piv;
          al = al2;
          be = be2;
        }
        if (fabs(al) < pivtol) al = copysign(pivtol, al);
        ulast = al;
        AT(U0i, b1 - 1) = 1.0 / al;
      }
      for (int i = b0 + tid; i < b1; i += nt)
        sx[i] = hash_uniform(((unsigned long long)p << 40) ^ ((unsigned long long)q << 20) ^ (unsigned long long)i);
      __syncthreads();
      int its = 0, nrmchk = 0;
      bool ok = false;
      while (its < maxits + EXTRA) {
        ++its;
        double a1 = 0.0;
        for (int i = b0 + tid; i < b1; i += nt) a1 += fabs(sx[i]);
        const double x1 = block_sum1(a1, red);
        if (tid == 0) {  // scaled right-hand side, forward and back substitution
          const double scl = (double)bs * T.onenrm * fmax(eps, fabs(ulast)) / fmax(x1, DBL_MIN);
          double r = sx[b0] * scl;
          #pragma unroll 8
          for (int k = b0; k < b1 - 1; ++k) {
            const double xn = sx[k + 1] * scl;
            const double l = AT(Lr, k);
            if (AT(PV, k) == 0.0) {
              sx[k] = r;
              r = xn - l * r;
            } else {
              sx[k] = xn;
              r = r - l * xn;
            }
          }
          double x2 = 0.0, x1v = r * AT(U0i, b1 - 1);
          sx[b1 - 1] = x1v;
          #pragma unroll 8
          for (int k = b1 - 2; k >= b0; --k) {
            const double xv = (sx[k] - AT(U1, k) * x1v - AT(U2, k) * x2) * AT(U0i, k);
            sx[k] = xv;
            x2 = x1v;
            x1v = xv;
          }
        }
        __syncthreads();
        const int nf = s_nf;  // (published by the barriers above)
        for (int pass = 0; pass < 2 && nf > 0; ++pass) {
          for (int u = wid; u < nf; u += nw) {
            const double* zt = Z + (size_t)rnk[fin[u]] * ldz;
            double dt = 0.0;
            for (int i = b0 + lane; i < b1; i += 32) dt = fma(sx[i], zt[i], dt);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) dt += __shfl_xor_sync(0xffffffffu, dt, o);
            if (lane == 0) dots[u] = dt;
          }
          __syncthreads();
          for (int i = b0 + tid; i < b1; i += nt) {
            double v = sx[i];
            for (int u = 0; u < nf; ++u) v = fma(-dots[u], Z[(size_t)rnk[fin[u]] * ldz + i], v);
            sx[i] = v;
          }
          __syncthreads();
        }
        double am = 0.0;
        bool fin = true;
        for (int i = b0 + tid; i < b1; i += nt) {
          const double a = fabs(sx[i]);
          fin = fin && (a <= DBL_MAX);
          am = fmax(am, a);
        }
        const double xinf = block_max1(fin ? am : INFINITY, red);
        if (!(xinf <= DBL_MAX)) break;
        if (its > maxits && nrmchk == 0) break;
        if (xinf < sqrt(0.1 / bs)) continue;
        ++nrmchk;
        if (nrmchk < EXTRA + 1) continue;
        ok = true;
        break;
      }
      if (!ok) fail = true;
      // normalise, sign: largest component positive (first of equal magnitude)
      double a2 = 0.0, big = 0.0;
      int jm = b1;
      for (int i = b0 + tid; i < b1; i += nt) {
        const double a = sx[i];
        a2 = fma(a, a, a2);
        if (fabs(a) > big) {
          big = fabs(a);
          jm = i;
        }
      }
      const double nrm2 = block_sum1(a2, red);
      const double bigmax = block_max1(big, red);
      if (tid == 0) s_go = b1;
      __syncthreads();
      if (big == bigmax && bigmax > 0.0) atomicMin(&s_go, jm);
      __syncthreads();
      double sc = (nrm2 > 0.0 && nrm2 <= DBL_MAX) ? 1.0 / sqrt(nrm2) : 0.0;
      if (s_go < b1 && sx[s_go] < 0.0) sc = -sc;
      double* zc = Z + (size_t)rnk[q - j] * ldz;
      for (int i = tid; i < m; i += nt) zc[i] = (i >= b0 && i < b1) ? sx[i] * sc : 0.0;
      if (sc == 0.0 && tid == 0) zc[b0 + (q - b0) % bs] = 1.0;
      __syncthreads();
#undef AT
    }
    if (tid == 0) s_ok = fail ? 0 : 1;
    __syncthreads();
    if (tid == 0 && !s_ok && status) atomicExch(&status[p], NAO_E_NOCONV);
  }
}


// ---------------------------------------------------------------- kernel 0: MRRR vectors
// Eigenvectors from a relatively robust representation (the method of LAPACK's dstegr /
// dstemr, which the paper names beside dstevx; one root representation, not the whole
// representation tree): for every unreduced block of a positive semidefinite tridiagonal (the
// overlap's), shift to just below its smallest eigenvalue, T - sigma I = L D L^T with D > 0.
// A definite L D L^T determines its eigenvalues to high relative accuracy, so the near-null
// spectrum of an ill-conditioned overlap, hundreds of eigenvalues within 1e-9 |T| of each
// other but relatively far apart, becomes well separated.
//   A member of a big tight cluster (gaps < 1e-9 |T|_1, more than BIG members: the ones
// inverse iteration would re-orthogonalise at O(k^2 n)) whose shifted eigenvalue
// mu = lambda - sigma has a relative gap of at least MR_MINRGP to both neighbours is refined
// by bisection on negative-pivot counts of L D L^T - x I (the stationary qd transform) to
// relative accuracy, and its eigenvector comes from one twisted factorization of
// L D L^T - mu I: the forward (stationary) and backward (progressive) transforms give
// gamma_k = s_k + p_k + mu, and with r = argmin |gamma_k|, z_r = 1, z_k = -L+_k z_{k+1} above
// r, z_{k+1} = -U-_k z_k below it.
//   Vectors of one representation are orthogonal to O(n eps / relgap) without any
// Gram-Schmidt (LAPACK asks relgap >= 1e-3 for 1e-13 orthogonality; here the Newton-Schulz
// step that follows removes overlaps up to ~1e-6, so relgap >= 1e-5 suffices: overlaps
// <= n eps / 1e-5 ~ 3e-8 at n = 3000).  Slots with smaller relative gaps are left
// (mdone = 0) to inverse iteration, which re-orthogonalises them against the finished members.
constexpr double MR_MINRGP = 1e-5;
constexpr int MR_THREADS = 64;

// negative pivots of L D L^T - x I over [b0, b1) (stationary qd; tiny pivots set to -pivmin)
__device__ int mr_negcount(const double* __restrict__ D, const double* __restrict__ L, int b0, int b1, double x,
                           double pivmin) {
  double s = -x;
  int cnt = 0;
  for (int k = b0; k < b1 - 1; ++k) {
    double dp = D[k] + s;
    if (fabs(dp) < pivmin) dp = -pivmin;
    cnt += dp < 0.0;
    s = (L[k] * L[k] * D[k]) * s / dp - x;
  }
  double dp = D[b1 - 1] + s;
  if (fabs(dp) < pivmin) dp = -pivmin;
  return cnt + (dp < 0.0);
}

__global__ void __launch_bounds__(MR_THREADS)
mrrr_vec_kernel(int n, const int32_t* __restrict__ size, const double* __restrict__ dbase,
                const double* __restrict__ ebase, long long strideV, const double* __restrict__ wslot,
                double* __restrict__ Zbase, int ldz, long long strideZ, double* __restrict__ scratch,
                int* __restrict__ mdone, const int32_t* __restrict__ nvec, int nvec_max, int all, double tgs) {
  extern __shared__ double smr[];
  double* w = smr;           // [n] eigenvalues (slot order)
  double* D = smr + n;       // [n] root representation of each unreduced block
  double* L = smr + 2 * n;   // [n]
  double* sig = smr + 3 * n; // [n] the block's shift, per row
  int* bst = (int*)(smr + 4 * n);
  int* ben = bst + n;
  __shared__ double s_tn;
  const int p = blockIdx.y;
  const int m = size ? size[p] : n;
  if (m <= 0 || (int)(blockIdx.x * blockDim.x) >= m) return;  // uniform per block
  const double* din = dbase + (size_t)p * strideV;
  const double* ein = ebase + (size_t)p * strideV;
  const double* ws = wslot + (size_t)p * n;
  const double eps = DBL_EPSILON * 0.5;
  {
    // nothing to do for a block of slots none of which lies in a tight cluster (a
    // conservative test on the neighbouring slots, the tridiagonal's 1-norm bounded by
    // 3 max(|d|, |e|) from a block-wide maximum)
    const int jj = blockIdx.x * blockDim.x + threadIdx.x;
    if (jj < m) mdone[(size_t)p * n + jj] = 0;  // kernel 2 reads every slot's flag
    double am = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) am = fmax(am, fmax(fabs(din[i]), i < m - 1 ? fabs(ein[i]) : 0.0));
    __shared__ double s_am;
    if (threadIdx.x == 0) s_am = 0.0;
    __syncthreads();
    atomicMax((unsigned long long*)&s_am, (unsigned long long)__double_as_longlong(am));  // am >= 0
    __syncthreads();
    const double tb = tgs * 3.0 * s_am;
    for (int i = threadIdx.x; i < m; i += blockDim.x) w[i] = ws[i];
    __syncthreads();
    // only the members of big tight clusters (more than BIG members, the ones kernel 3 would
    // re-orthogonalise at O(k^2 n)); smaller clusters are cheap by inverse iteration
    bool big = all != 0;  // all: every slot whose relative gap allows, not only big clusters
    if (jj < m && !big) {
      int c = 1;
      for (int t = jj; t > 0 && c <= BIG && fabs(w[t] - w[t - 1]) < tb; --t) ++c;
      for (int t = jj; t < m - 1 && c <= BIG && fabs(w[t + 1] - w[t]) < tb; ++t) ++c;
      big = c > BIG;
    }
    if (!__syncthreads_or(big)) return;
  }
  if (threadIdx.x == 0) {
    // split (as kernel 1), max |T| for the shift margins
    double tn = 0.0;
    for (int i = 0; i < m; ++i) {
      const double r = (i > 0 ? fabs(ein[i - 1]) : 0.0) + (i < m - 1 ? fabs(ein[i]) : 0.0);
      tn = fmax(tn, fabs(din[i]) + r);
    }
    tn = fmax(tn, DBL_MIN);
    s_tn = tn;
    int b0 = 0;
    for (int i = 0; i < m; ++i) {
      bst[i] = b0;
      bool cut = i == m - 1;
      if (!cut) {
        const double ei = ein[i];
        cut = ei * ei <= eps * eps * fabs(din[i] * din[i + 1]) + DBL_MIN;
      }
      if (cut) {
        for (int k = b0; k <= i; ++k) ben[k] = i + 1;
        b0 = i + 1;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // root representation per block: sigma just below the block's smallest eigenvalue (slot
    // b0 holds it), D > 0 checked, the margin doubled until it holds
    const double tn = s_tn;
    for (int b0 = 0; b0 < m; b0 = ben[b0]) {
      const int b1 = ben[b0];
      double off = 32.0 * eps * tn;
      bool ok = false;
      double sg = 0.0;
      for (int tr = 0; tr < 40 && !ok; ++tr, off *= 2.0) {
        sg = w[b0] - off;
        ok = true;
        double dk = din[b0] - sg;
        for (int k = b0; k < b1 - 1 && ok; ++k) {
          if (!(dk > 0.0)) ok = false;
          const double ek = ein[k];
          const double lk = ek / dk;
          D[k] = dk;
          L[k] = lk;
          dk = (din[k + 1] - sg) - lk * ek;
        }
        if (!(dk > 0.0)) ok = false;
        D[b1 - 1] = dk;
        L[b1 - 1] = 0.0;
      }
      for (int k = b0; k < b1; ++k) sig[k] = ok ? sg : NAN;  // NaN: no representation, inverse iteration
    }
  }
  __syncthreads();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  const int nv = min(nvec ? nvec[p] : m, nvec_max);
  const double wj = w[j];
  int rk = 0;  // rank of slot j in the global ascending order (ties by slot), as kernel 2
  for (int t = 0; t < m; ++t) {
    const double wt = w[t];
    rk += (wt < wj) || (wt == wj && t < j);
  }
  int* done = mdone + (size_t)p * n;
  done[j] = 0;
  if (rk >= nv) return;
  const int b0 = bst[j], b1 = ben[j], bs = b1 - b0;
  const double sg = sig[j];
  if (bs == 1 || !(sg == sg)) return;  // singletons and blocks without a representation: kernel 2
  const double mu0 = wj - sg;
  const double gl = j > b0 ? wj - w[j - 1] : INFINITY, gr = j < b1 - 1 ? w[j + 1] - wj : INFINITY;
  const double tn = s_tn;
  // only members of big tight clusters (as above, now within the split block), unless all
  if (!all) {
    int c = 1;
    for (int t = j; t > b0 && c <= BIG && w[t] - w[t - 1] < tgs * tn; --t) ++c;
    for (int t = j; t < b1 - 1 && c <= BIG && w[t + 1] - w[t] < tgs * tn; ++t) ++c;
    if (c <= BIG) return;
  }
  if (!(fmin(gl, gr) >= MR_MINRGP * mu0)) return;  // a relative cluster: kernel 2
  const double pivmin = DBL_MIN * fmax(1.0, tn * tn);
  // relative bisection of eigenvalue idx of the block, from the absolute bracket of kernel 1
  const int idx = j - b0;
  double lo = fmax(mu0 - 8.0 * eps * tn, 0.0), hi = mu0 + 8.0 * eps * tn;
  if (!(mr_negcount(D, L, b0, b1, lo, pivmin) <= idx && mr_negcount(D, L, b0, b1, hi, pivmin) > idx)) {
    lo = 0.0;
    hi = 2.0 * tn + fabs(sg) + 4.0 * eps * tn;
  }
  for (int it = 0; it < 160; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (hi - lo <= 4.0 * eps * hi || mid <= lo || mid >= hi) break;
    if (mr_negcount(D, L, b0, b1, mid, pivmin) > idx) hi = mid;
    else lo = mid;
  }
  const double mu = 0.5 * (lo + hi);
  // twisted factorization at mu: forward (stationary) multipliers Lp and s, backward
  // (progressive) multipliers Um with gamma_k = s_k + p_k + mu on the way
  double* scr = scratch + (size_t)p * NARR * n * n;
  const size_t nn = (size_t)n * n;
  double* Lp = scr + 0 * nn;
  double* Sa = scr + 1 * nn;
  double* Um = scr + 2 * nn;
  double* Xz = scr + 3 * nn;
#define AT(arr, i) arr[(size_t)(i) * n + j]
  double sv = -mu;
  for (int k = b0; k < b1 - 1; ++k) {
    AT(Sa, k) = sv;
    double dp = D[k] + sv;
    if (fabs(dp) < pivmin) dp = -pivmin;
    const double lp = L[k] * D[k] / dp;
    AT(Lp, k) = lp;
    sv = lp * L[k] * sv - mu;
  }
  AT(Sa, b1 - 1) = sv;
  double pv = D[b1 - 1] - mu;
  double gbest = sv + pv + mu;
  int r = b1 - 1;
  for (int k = b1 - 2; k >= b0; --k) {
    double dm = L[k] * L[k] * D[k] + pv;
    if (fabs(dm) < pivmin) dm = -pivmin;
    const double t = D[k] / dm;
    AT(Um, k) = L[k] * t;
    pv = pv * t - mu;
    const double g = AT(Sa, k) + pv + mu;
    if (fabs(g) < fabs(gbest)) {
      gbest = g;
      r = k;
    }
  }
  // z from the twist index outwards; the running magnitude is kept finite by rescaling
  AT(Xz, r) = 1.0;
  double zk = 1.0;
  for (int k = r - 1; k >= b0; --k) {
    zk = -AT(Lp, k) * zk;
    if (fabs(zk) > 0x1p500) {
      for (int q = k + 1; q <= r; ++q) AT(Xz, q) *= 0x1p-500;
      zk *= 0x1p-500;
    }
    AT(Xz, k) = zk;
  }
  double scale_up = 1.0;  // factor applied to [b0, r] by rescales of the lower part
  zk = 1.0;
  for (int k = r; k < b1 - 1; ++k) {
    zk = -AT(Um, k) * zk;
    if (fabs(zk) > 0x1p500) {
      for (int q = r + 1; q <= k; ++q) AT(Xz, q) *= 0x1p-500;
      scale_up *= 0x1p-500;
      zk *= 0x1p-500;
    }
    AT(Xz, k + 1) = zk;
  }
  if (scale_up != 1.0)
    for (int q = b0; q <= r; ++q) AT(Xz, q) *= scale_up;
  double nrm2 = 0.0, big = 0.0;
  int jmax = b0;
  for (int i = b0; i < b1; ++i) {
    const double a = AT(Xz, i);
    nrm2 = fma(a, a, nrm2);
    if (fabs(a) > big) {
      big = fabs(a);
      jmax = i;
    }
  }
  if (!(nrm2 > 0.0 && nrm2 <= DBL_MAX)) return;  // no usable vector: kernel 2
  double sc = 1.0 / sqrt(nrm2);
  if (AT(Xz, jmax) < 0.0) sc = -sc;
  double* zc = Zbase + (size_t)p * strideZ + (size_t)rk * ldz;
  for (int i = 0; i < m; ++i) zc[i] = (i >= b0 && i < b1) ? AT(Xz, i) * sc : 0.0;
#undef AT
  done[j] = 1;
}
}  // namespace

// scratch: NARR n^2 doubles per problem, the eigenvalue slots (n per problem), and the
// big-cluster list (count + 3 ints per cluster, at most n / (BIG + 1) clusters per problem)
static int big_capacity(int n, int nprob) { return nprob * (n / (BIG + 1) + 1); }

size_t stein_scratch_doubles(int n, int nprob) {
  // the bisection queue (5 n + 1 doubles per problem, + 1) fits in the first NARR n^2 per
  // problem for n >= 2; the pad covers n = 1
  return (size_t)NARR * n * n * nprob + (size_t)n * nprob + (3 * (size_t)big_capacity(n, nprob) + 2) / 2 + 1 +
         ((size_t)n * nprob + 1) / 2 + 1 + nprob + 2;
}

cudaError_t launch_stein(int n, int nprob, const int32_t* size, const double* d, const double* e, long long strideV,
                         double* w, double* Z, int ld, long long strideZ, double* scratch, int32_t* status,
                         const int32_t* nvec, int nvec_max, int maxits, int mrrr, cudaStream_t st, int* ns2) {
  double* wslot = scratch + (size_t)NARR * n * n * nprob;
  const size_t smem1 = sizeof(double) * 3 * (size_t)n + sizeof(float) * 2 * (size_t)n + sizeof(int) * 2 * (size_t)n;
  cudaError_t err = cudaFuncSetAttribute(stebz_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1);
  if (err != cudaSuccess) return err;
  // the bisection queue (all problems) and the split e^2 live in the inverse-iteration
  // scratch, unused until kernel 2
  const size_t cap = (size_t)n * nprob;
  double* qlo = scratch;
  double* qhi = qlo + cap;
  int4* qent = (int4*)(qhi + cap);
  double* e2g = (double*)(qent + cap);
  double* tng = e2g + cap;                                            // 5 cap + nprob <= NARR n^2 nprob
  int* qcount = (int*)(scratch + stein_scratch_doubles(n, nprob) - 2);  // the pad at the end
  err = cudaMemsetAsync(qcount, 0, sizeof(int), st);
  if (err != cudaSuccess) return err;
  dim3 grid1((n + SZ_THREADS - 1) / SZ_THREADS, nprob);
  stebz_kernel<<<grid1, SZ_THREADS, smem1, st>>>(n, size, d, e, strideV, wslot, status, qcount, qent, qlo, qhi, e2g,
                                                 tng);
  err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  stebz_bisect_kernel<<<(unsigned)((cap * BQ_LANES + SZ_THREADS - 1) / SZ_THREADS), SZ_THREADS, 0, st>>>(n, d, strideV, e2g, tng,
                                                                                             wslot, qcount, qent, qlo,
                                                                                             qhi);
  dim3 grid((n + ST_THREADS - 1) / ST_THREADS, nprob);
  err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  int* biglist = (int*)(wslot + (size_t)n * nprob);
  const int bigcap = big_capacity(n, nprob);
  err = cudaMemsetAsync(biglist, 0, sizeof(int), st);
  if (err != cudaSuccess) return err;
  // kernel 0 (MRRR vectors where the representation separates the eigenvalues), when asked
  int* mdone = nullptr;
  // Gram-Schmidt band: TIGHT where MRRR takes the members of big clusters (a wide band costs
  // nothing there; a narrow one splits the near-null spectrum of an ill-conditioned overlap
  // into small clusters that one thread walks serially), TIGHT_GS and a second Newton-Schulz
  // step for the band in between where inverse iteration works alone
  const double tgs = mrrr ? TIGHT : TIGHT_GS;
  if (mrrr) {
    mdone = biglist + 1 + 3 * (size_t)bigcap + 1;  // n ints per problem after the cluster list
    const size_t smem0 = sizeof(double) * 4 * (size_t)n + sizeof(int) * 2 * (size_t)n;
    err = cudaFuncSetAttribute(mrrr_vec_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem0);
    if (err != cudaSuccess) return err;
    dim3 grid0((n + MR_THREADS - 1) / MR_THREADS, nprob);
    mrrr_vec_kernel<<<grid0, MR_THREADS, smem0, st>>>(n, size, d, e, strideV, wslot, Z, ld, strideZ, scratch, mdone,
                                                       nvec, nvec_max, mrrr == 2, tgs);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
  }
  const size_t smem2 = sizeof(double) * 4 * (size_t)n + sizeof(int) * 2 * (size_t)n;
  err = cudaFuncSetAttribute(stein_vec_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
  if (err != cudaSuccess) return err;
  if (ns2) {
    err = cudaMemsetAsync(ns2, 0, sizeof(int) * (size_t)nprob, st);
    if (err != cudaSuccess) return err;
  }
  stein_vec_kernel<<<grid, ST_THREADS, smem2, st>>>(n, size, d, e, strideV, wslot, w, Z, ld, strideZ, scratch, status,
                                                    biglist, bigcap, nvec, nvec_max, maxits, mdone, ns2, tgs);
  err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  // kernel 3: a grid that stays resident; blocks without a listed cluster exit at once
  const size_t smem3 = sizeof(double) * 5 * (size_t)n + sizeof(int) * 4 * (size_t)n;
  err = cudaFuncSetAttribute(stein_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem3);
  if (err != cudaSuccess) return err;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  stein_cluster_kernel<<<sms, SC_THREADS, smem3, st>>>(n, size, d, e, strideV, wslot, Z, ld, strideZ, scratch, status,
                                                       biglist, bigcap, nvec, nvec_max, maxits, mdone, tgs);
  return cudaGetLastError();
}
