// Eigen_HH step 2 (Sec. 3: the paper calls LAPACK dstevx, i.e. bisection + inverse
// iteration): all eigenpairs of a real symmetric tridiagonal T = tridiag(e, d, e), one
// thread block per problem, one thread per eigenvalue.
//
// * Splitting: an off-diagonal with e_i^2 <= eps^2 |d_i d_{i+1}| + tiny is set to zero;
//   each unreduced block is solved on its own and its eigenvectors vanish outside it.
// * Eigenvalues: bisection on Sturm counts.  The count is the number of sign changes of
//   the leading principal minors p_i = (d_i - x) p_{i-1} - e_{i-1}^2 p_{i-2} (a zero minor
//   takes the sign of its predecessor), rescaled by powers of two to stay in range.  This
//   is the division-free form of the LDL^T pivot count (pivot q_i = p_i / p_{i-1}): three
//   FP64 operations per step instead of a division, which costs ~10 FMAs on this GPU.
// * Eigenvectors: inverse iteration with a partially pivoted LU of T - lambda I (tiny
//   pivots perturbed to eps*|T|), a scaled right-hand side, the growth test
//   |x|_inf >= sqrt(0.1/blocksize) plus two extra solves, and modified Gram-Schmidt against
//   the previous members of a TIGHT cluster (gap < 1e-7 |T|_1).  Wider near-degeneracies
//   leave overlaps of order eps|T|/gap <= ~1e-9, which the caller removes with one
//   Newton-Schulz step Z <- Z (3I - Z^T Z)/2.
// * Output: eigenvalues ascending (across blocks), eigenvectors in matching columns,
//   unit 2-norm, largest component positive.
#include <cfloat>

#include "nao_internal.cuh"

namespace {

constexpr int ST_THREADS = 1024;
constexpr int MAXITS = 5;    // inverse-iteration solves before giving up
constexpr int EXTRA = 2;     // extra solves after the growth test passes
constexpr double TIGHT = 1e-7;
constexpr int NARR = 6;      // scratch arrays per eigenvalue: L, U0inv, U1, U2, PIV, X

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

// Number of eigenvalues of T[b0:b1) strictly below x.
__device__ int sturm_count(const double* __restrict__ d, const double* __restrict__ e2, int b0, int b1, double x) {
  double pm1 = 1.0;
  double p = d[b0] - x;
  long long bits = __double_as_longlong(p);
  int sn = (bits < 0) && ((bits << 1) != 0);
  int cnt = sn;
  for (int i = b0 + 1; i < b1; ++i) {
    const double pn = fma(d[i] - x, p, -e2[i - 1] * pm1);
    pm1 = p;
    p = pn;
    bits = __double_as_longlong(p);
    const int zero = (bits << 1) == 0;
    const int ns = zero ? sn : (int)(bits < 0);
    cnt += (ns != sn);
    sn = ns;
    // keep |p|, |pm1| away from overflow / underflow (exact power-of-two scaling)
    const int ex = (int)((bits >> 52) & 0x7ff);
    const int ex1 = (int)((__double_as_longlong(pm1) >> 52) & 0x7ff);
    const int emax = ex > ex1 ? ex : ex1;
    if (emax > 1023 + 400) {
      p *= 0x1p-400;
      pm1 *= 0x1p-400;
    } else if (emax < 1023 - 400) {
      p *= 0x1p400;
      pm1 *= 0x1p400;
    }
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

__global__ void __launch_bounds__(ST_THREADS)
stein_kernel(int n, const int32_t* __restrict__ size, const double* __restrict__ dbase, const double* __restrict__ ebase,
             long long strideV, double* __restrict__ wbase, double* __restrict__ Zbase, int ldz, long long strideZ,
             double* __restrict__ scratch, int32_t* __restrict__ status) {
  extern __shared__ double smd[];
  double* d = smd;             // [n]
  double* e = smd + n;         // [n]   (e[i] couples rows i and i+1; split entries zeroed)
  double* e2 = smd + 2 * n;    // [n]
  double* w = smd + 3 * n;     // [n]   eigenvalue of slot j
  int* rank = (int*)(smd + 4 * n);  // [n]
  int* bst = rank + n;              // [n] first row of the block containing row j
  int* ben = bst + n;               // [n] one past its last row
  __shared__ double red[64];
  __shared__ int s_fail;

  const int p = blockIdx.x;
  const int m = size ? size[p] : n;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5;
  if (m <= 0) {
    if (tid == 0 && status) status[p] = 0;
    return;
  }
  const double* din = dbase + (size_t)p * strideV;
  const double* ein = ebase + (size_t)p * strideV;
  double* wout = wbase + (size_t)p * strideV;
  double* Z = Zbase + (size_t)p * strideZ;
  double* scr = scratch + (size_t)p * NARR * n * n;
  const double eps = DBL_EPSILON * 0.5;

  if (tid == 0) s_fail = 0;
  // load + split test + Gershgorin interval + 1-norm
  double lmin = 1e300, lmax = -1e300, lnrm = 0.0;
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
  }
  __syncthreads();
  double gl = 1e300, gu = -1e300;
  for (int k = 0; k < (nt >> 5); ++k) {
    gl = fmin(gl, red[k]);
    gu = fmax(gu, red[32 + k]);
  }
  __syncthreads();
  if (lane == 0) red[wid] = lnrm;
  __syncthreads();
  double onenrm = 0.0;
  for (int k = 0; k < (nt >> 5); ++k) onenrm = fmax(onenrm, red[k]);
  const double tnorm = fmax(fmax(fabs(gl), fabs(gu)), DBL_MIN);
  gl -= 4.0 * eps * tnorm * m + 2.0 * DBL_MIN;
  gu += 4.0 * eps * tnorm * m + 2.0 * DBL_MIN;
  if (onenrm == 0.0) onenrm = 1.0;

  // block boundaries (a serial scan is O(m) and negligible)
  if (tid == 0) {
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

  // ---- bisection: slot j holds eigenvalue (j - b0) of its block
  for (int j = tid; j < m; j += nt) {
    const int b0 = bst[j], b1 = ben[j];
    double lam;
    if (b1 - b0 == 1) {
      lam = d[b0];
    } else {
      const int idx = j - b0;
      double lo = gl, hi = gu;
      for (int it = 0; it < 128; ++it) {
        const double mid = 0.5 * (lo + hi);
        const double tol = fmax(2.0 * eps * fmax(fabs(lo), fabs(hi)), eps * tnorm);
        if (hi - lo <= tol || mid <= lo || mid >= hi) break;
        if (sturm_count(d, e2, b0, b1, mid) > idx) hi = mid;
        else lo = mid;
      }
      lam = 0.5 * (lo + hi);
    }
    w[j] = lam;
  }
  __syncthreads();
  // ---- global ascending order (ties broken by slot)
  for (int j = tid; j < m; j += nt) {
    const double wj = w[j];
    int r = 0;
    for (int t = 0; t < m; ++t) {
      const double wt = w[t];
      r += (wt < wj) || (wt == wj && t < j);
    }
    rank[j] = r;
    wout[r] = wj;
  }
  __syncthreads();

  // ---- inverse iteration (cluster leaders walk their tight cluster in order)
  const double tight = TIGHT * onenrm;
  const double pivtol = eps * tnorm;
  const size_t nn = (size_t)n * n;
  for (int j = tid; j < m; j += nt) {
    const int b0 = bst[j], b1 = ben[j];
    if (j > b0 && w[j] - w[j - 1] < tight) continue;  // not a leader
    int jend = j + 1;
    while (jend < b1 && w[jend] - w[jend - 1] < tight) ++jend;
    const int bs = b1 - b0;
    double* Lr = scr + 0 * nn;
    double* U0i = scr + 1 * nn;
    double* U1 = scr + 2 * nn;
    double* U2 = scr + 3 * nn;
    double* PV = scr + 4 * nn;
    double* X = scr + 5 * nn;
    const int sl = j;  // scratch column of this leader
#define AT(arr, i) arr[(size_t)(i) * n + sl]
    double lamprev = 0.0;
    for (int q = j; q < jend; ++q) {
      double* zc = Z + (size_t)rank[q] * ldz;
      if (bs == 1) {
        for (int i = 0; i < m; ++i) zc[i] = (i == b0) ? 1.0 : 0.0;
        lamprev = w[q];
        continue;
      }
      double lam = w[q];
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
        double u0, u1, u2, l, piv, al2, be2;
        if (fabs(al) >= fabs(c)) {
          piv = 0.0;
          u0 = al;
          u1 = be;
          u2 = 0.0;
          l = (al != 0.0) ? c / al : 0.0;
          al2 = an - l * be;
          be2 = bn;
        } else {
          piv = 1.0;
          u0 = c;
          u1 = an;
          u2 = bn;
          l = al / c;
          al2 = be - l * an;
          be2 = -l * bn;
        }
        if (fabs(u0) < pivtol) u0 = copysign(pivtol, u0);
        AT(U0i, k) = 1.0 / u0;
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
      // random start
      for (int i = b0; i < b1; ++i)
        AT(X, i) = hash_uniform(((unsigned long long)p << 40) ^ ((unsigned long long)q << 20) ^ (unsigned long long)i);
      int its = 0, nrmchk = 0;
      bool ok = false;
      while (its < MAXITS + EXTRA) {
        ++its;
        double x1 = 0.0;
        for (int i = b0; i < b1; ++i) x1 += fabs(AT(X, i));
        const double scl = (double)bs * onenrm * fmax(eps, fabs(ulast)) / fmax(x1, DBL_MIN);
        // forward: apply the row interchanges and L
        double r = AT(X, b0) * scl;
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
        // back substitution with U (diagonal, two superdiagonals)
        double x2 = 0.0, x1v = AT(X, b1 - 1) * AT(U0i, b1 - 1);
        AT(X, b1 - 1) = x1v;
        for (int k = b1 - 2; k >= b0; --k) {
          const double xv = (AT(X, k) - AT(U1, k) * x1v - AT(U2, k) * x2) * AT(U0i, k);
          AT(X, k) = xv;
          x2 = x1v;
          x1v = xv;
        }
        // reorthogonalise against the earlier members of the tight cluster
        for (int t = j; t < q; ++t) {
          const double* zt = Z + (size_t)rank[t] * ldz;
          double dot = 0.0;
          for (int i = b0; i < b1; ++i) dot = fma(AT(X, i), zt[i], dot);
          for (int i = b0; i < b1; ++i) AT(X, i) = fma(-dot, zt[i], AT(X, i));
        }
        double xinf = 0.0;
        bool finite = true;
        for (int i = b0; i < b1; ++i) {
          const double a = fabs(AT(X, i));
          finite = finite && (a <= DBL_MAX);
          xinf = fmax(xinf, a);
        }
        if (!finite) break;
        if (its > MAXITS && nrmchk == 0) break;
        if (xinf < sqrt(0.1 / bs)) continue;
        ++nrmchk;
        if (nrmchk < EXTRA + 1) continue;
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
  __syncthreads();
  if (tid == 0 && status) status[p] = s_fail ? NAO_E_NOCONV : 0;
}

}  // namespace

size_t stein_scratch_doubles(int n, int nprob) { return (size_t)NARR * n * n * nprob; }

cudaError_t launch_stein(int n, int nprob, const int32_t* size, const double* d, const double* e, long long strideV,
                         double* w, double* Z, int ld, long long strideZ, double* scratch, int32_t* status,
                         cudaStream_t st) {
  size_t smem = sizeof(double) * 4 * (size_t)n + sizeof(int) * 3 * (size_t)n;
  cudaError_t err = cudaFuncSetAttribute(stein_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  stein_kernel<<<nprob, ST_THREADS, smem, st>>>(n, size, d, e, strideV, w, Z, ld, strideZ, scratch, status);
  return cudaGetLastError();
}
