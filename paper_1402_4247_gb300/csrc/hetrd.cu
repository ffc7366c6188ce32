// Eigen_HH step 1 (Sec. 3, Procedures 1-6): Householder reduction of a Hermitian matrix to
// real symmetric tridiagonal form, one thread block per problem.
//
// Column i: x = A(i+1:m, i) (Procedure 1); a reflector H_i = I - tau v v^H with v(0) = 1 and
// a REAL beta, H_i^H x = beta e_1, is formed from |x| (Procedure 2) and kept in place for the
// back-transformation (Procedure 3); p = tau A22 v (Procedure 4); w = p - (tau/2)(p^H v) v
// (Procedure 5); A22 <- A22 - v w^H - w v^H (Procedure 6).  Choosing beta real removes the
// separate phase pass: Q^H A Q = T with Q = H_0 H_1 ... H_{m-2}.
//
// Storage: full Hermitian matrix, column-major (element (r, c) at A[r + c*ld]); both
// triangles are kept current so that the Hermitian matrix-vector product streams whole
// columns.  Output: d[0..m), e[0..m-1) (e[m-1] = 0), tau[0..m) (tau[m-1] = 0), and v_i in
// A(i+2:m, i).
#include "nao_internal.cuh"

namespace {

constexpr int HT_THREADS = 1024;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of (a, b) over the block, returned to every thread.  red: >= 64 doubles of shared memory.
__device__ __forceinline__ double2 block_sum2(double a, double b, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  a = warp_sum(a);
  b = warp_sum(b);
  __syncthreads();  // red may still be read from the previous call
  if (lane == 0) {
    red[wid] = a;
    red[32 + wid] = b;
  }
  __syncthreads();
  a = (lane < nw) ? red[lane] : 0.0;
  b = (lane < nw) ? red[32 + lane] : 0.0;
  a = warp_sum(a);
  b = warp_sum(b);
  return make_double2(a, b);
}

__global__ void __launch_bounds__(HT_THREADS)
hetrd_kernel(int n, const int32_t* __restrict__ size, z64* __restrict__ Abase, int ld, long long strideA,
             double* __restrict__ dbase, double* __restrict__ ebase, z64* __restrict__ taubase, long long strideV) {
  extern __shared__ z64 sm[];
  z64* v = sm;          // [n]
  z64* w = sm + n;      // [n]
  z64* part = sm + 2 * n;  // [HT_THREADS]
  __shared__ double red[64];
  __shared__ z64 s_tau, s_scale;

  const int p = blockIdx.x;
  const int m = size ? size[p] : n;
  z64* A = Abase + (size_t)p * strideA;
  double* d = dbase + (size_t)p * strideV;
  double* e = ebase + (size_t)p * strideV;
  z64* tau = taubase + (size_t)p * strideV;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (m <= 0) return;

  for (int i = 0; i < m - 1; ++i) {
    const int mt = m - i - 1;          // order of the trailing block A22 = A(i+1:m, i+1:m)
    z64* col = A + (size_t)i * ld;     // column i
    // Procedure 1-2: |x(1:)|^2 of x = A(i+1:m, i)
    double s = 0.0;
    for (int r = i + 2 + tid; r < m; r += nt) s += zabs2(col[r]);
    s = block_sum2(s, 0.0, red).x;
    if (tid == 0) {
      const z64 alpha = col[i + 1];
      const double xnorm = sqrt(s);
      z64 t, scale;
      double beta;
      if (xnorm == 0.0 && alpha.y == 0.0) {
        t = zmk(0.0, 0.0);
        scale = zmk(0.0, 0.0);
        beta = alpha.x;
      } else {
        beta = -copysign(sqrt(alpha.x * alpha.x + alpha.y * alpha.y + s), alpha.x);
        t = zmk((beta - alpha.x) / beta, -alpha.y / beta);
        const z64 den = zmk(alpha.x - beta, alpha.y);  // scale = 1 / (alpha - beta)
        const double dd = zabs2(den);
        scale = zmk(den.x / dd, -den.y / dd);
      }
      s_tau = t;
      s_scale = scale;
      d[i] = A[(size_t)i * ld + i].x;
      e[i] = beta;
      tau[i] = t;
      col[i + 1] = zmk(beta, 0.0);
    }
    __syncthreads();
    const z64 t = s_tau;
    const z64 scale = s_scale;
    // Procedure 3: v (implicit leading 1) kept in A(i+2:m, i) and in shared memory
    for (int r = i + 1 + tid; r < m; r += nt) {
      z64 val;
      if (r == i + 1) {
        val = zmk(1.0, 0.0);
      } else {
        val = zmul(col[r], scale);
        col[r] = val;
      }
      v[r - i - 1] = val;
    }
    __syncthreads();
    if (t.x == 0.0 && t.y == 0.0) continue;  // H_i = I (uniform branch: s_tau is shared)

    // Procedure 4: p = tau * A22 v.  Threads own rows (coalesced column reads); when the
    // block is narrower than the thread count, CS column groups split the columns.
    z64* A22 = A + (size_t)(i + 1) * ld + (i + 1);
    const int rows = mt < nt ? mt : nt;
    const int CS = mt < nt ? nt / mt : 1;
    const int g = tid / rows, r0 = tid - g * rows;
    if (g < CS) {
      for (int r = r0; r < mt; r += rows) {
        z64 acc = zmk(0.0, 0.0);
        const z64* Ar = A22 + r;
        for (int c = g; c < mt; c += CS) acc = zfma(Ar[(size_t)c * ld], v[c], acc);
        if (CS == 1) w[r] = acc;
        else part[g * mt + r] = acc;
      }
    }
    __syncthreads();
    if (CS > 1) {
      for (int r = tid; r < mt; r += nt) {
        z64 acc = zmk(0.0, 0.0);
        for (int gg = 0; gg < CS; ++gg) acc = zadd(acc, part[gg * mt + r]);
        w[r] = acc;
      }
      __syncthreads();
    }
    // p = tau * (A22 v); dot = p^H v
    double dre = 0.0, dim = 0.0;
    for (int r = tid; r < mt; r += nt) {
      const z64 pr = zmul(t, w[r]);
      w[r] = pr;
      const z64 c = zcfma(pr, v[r], zmk(0.0, 0.0));
      dre += c.x;
      dim += c.y;
    }
    const double2 dot = block_sum2(dre, dim, red);
    // Procedure 5: w = p - (tau/2) (p^H v) v
    const z64 alpha2 = zscale(zmul(t, zmk(dot.x, dot.y)), -0.5);
    for (int r = tid; r < mt; r += nt) w[r] = zfma(alpha2, v[r], w[r]);
    __syncthreads();
    // Procedure 6: A22 -= v w^H + w v^H (both triangles)
    const long long tot = (long long)mt * mt;
    for (long long idx = tid; idx < tot; idx += nt) {
      const int c = (int)(idx / mt), r = (int)(idx - (long long)c * mt);
      z64 a = A22[(size_t)c * ld + r];
      const z64 vr = v[r], wr = w[r], vc = v[c], wc = w[c];
      // a -= vr * conj(wc) + wr * conj(vc)
      a.x -= vr.x * wc.x + vr.y * wc.y + wr.x * vc.x + wr.y * vc.y;
      a.y -= vr.y * wc.x - vr.x * wc.y + wr.y * vc.x - wr.x * vc.y;
      A22[(size_t)c * ld + r] = a;
    }
    __syncthreads();
  }
  if (tid == 0) {
    d[m - 1] = A[(size_t)(m - 1) * ld + (m - 1)].x;
    e[m - 1] = 0.0;
    tau[m - 1] = zmk(0.0, 0.0);
  }
}

}  // namespace

cudaError_t launch_hetrd(int n, int nprob, const int32_t* size, z64* A, int ld, long long strideA, double* d,
                         double* e, z64* tau, long long strideV, cudaStream_t st) {
  size_t smem = sizeof(z64) * (2 * (size_t)n + HT_THREADS);
  cudaError_t err = cudaFuncSetAttribute(hetrd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  hetrd_kernel<<<nprob, HT_THREADS, smem, st>>>(n, size, A, ld, strideA, d, e, tau, strideV);
  return cudaGetLastError();
}
