// Ritz refinement of approximate generalized eigenpairs (not in the paper: it wins back the
// accuracy of the mixed-precision products).  One sweep of the Ogita-Aishima iteration
// (T. Ogita, K. Aishima, "Iterative refinement for symmetric eigenvalue decomposition",
// Japan J. Indust. Appl. Math. 35, 2018) carried to the S inner product:
//
//   given C^ (n x m, columns approximately S-orthonormal eigenvectors of H c = eps S c),
//   R' = C^^H S C^,  G = C^^H H C^            (FP64-accurate products, by the caller)
//   lambda_i = G_ii / R'_ii                   (Rayleigh quotients of the old vectors)
//   F_ii = (1 - R'_ii) / 2
//   F_ij = (G_ij - lambda_j R'_ij) / (lambda_j - lambda_i)   when |F_ij| <= OA_FMAX,
//        = -R'_ij / 2                                       otherwise (near-degenerate pair)
//   C = C^ (I + F)                            (caller)
// The off-diagonal formula is the first-order solution of (I+F)^H R' (I+F) = I and
// (I+F)^H G (I+F) = diag: with R = I - R', F + F^H = R and G + F^H D + D F = D give
// F_ij (lambda_j - lambda_i) = G_ij + lambda_j R_ij.  After the update the eigenvalues are
// the Rayleigh quotients of the new columns, c^H H c / c^H S c, and each column is scaled to
// c^H S c = 1; the last step sorts them ascending.
//
// Matrices are column-major with leading dimension ld and per-problem stride; m = size[p].
#include <cfloat>

#include "nao_internal.cuh"

namespace {

constexpr double OA_FMAX = 0.25;  // largest first-order rotation taken; beyond it the pair is a cluster

__global__ void oa_lambda_kernel(int n, int nprob, const int32_t* __restrict__ size, const z64* __restrict__ Rp,
                                 const z64* __restrict__ G, int ld, long long stride, double* __restrict__ lam,
                                 long long lstride) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)nprob * n) return;
  const int p = (int)(idx / n), i = (int)(idx % n);
  if (i >= size[p]) return;
  const size_t o = (size_t)p * stride + (size_t)i * ld + i;
  lam[(size_t)p * lstride + i] = G[o].x / Rp[o].x;
}

// In place over G: G <- I + F (reads R' and G element-wise, lambda per row / column)
__global__ void oa_f_kernel(int n, const int32_t* __restrict__ size, const z64* __restrict__ Rp, z64* __restrict__ G,
                            int ld, long long stride, const double* __restrict__ lam, long long lstride) {
  const int p = blockIdx.z;
  const int m = size[p];
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= m || j >= m) return;
  const size_t o = (size_t)p * stride + (size_t)j * ld + i;
  const z64 r = Rp[o];
  z64 f;
  if (i == j) {
    f = zmk(1.0 + 0.5 * (1.0 - r.x), 0.0);
  } else {
    const double li = lam[(size_t)p * lstride + i], lj = lam[(size_t)p * lstride + j];
    const z64 g = G[o];
    const z64 num = zmk(g.x - lj * r.x, g.y - lj * r.y);
    const double den = lj - li;
    if (sqrt(zabs2(num)) <= OA_FMAX * fabs(den)) f = zmk(num.x / den, num.y / den);
    else f = zmk(-0.5 * r.x, -0.5 * r.y);
  }
  G[o] = f;
}

// One warp per column j < m: lambda_j = Re(c^H W2) / Re(c^H W1), c <- c / sqrt(Re(c^H W1)),
// with W1 = S c, W2 = H c.
__global__ void oa_rq_kernel(int n, int nprob, const int32_t* __restrict__ size, z64* __restrict__ Cn, int ldc,
                             long long cstride, const z64* __restrict__ W1, const z64* __restrict__ W2, int ldw,
                             long long wstride, double* __restrict__ lam, long long lstride) {
  const int lane = threadIdx.x & 31;
  const size_t wg = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (wg >= (size_t)nprob * n) return;
  const int p = (int)(wg / n), j = (int)(wg % n);
  if (j >= size[p]) return;
  z64* c = Cn + (size_t)p * cstride + (size_t)j * ldc;
  const z64* w1 = W1 + (size_t)p * wstride + (size_t)j * ldw;
  const z64* w2 = W2 + (size_t)p * wstride + (size_t)j * ldw;
  double s = 0.0, h = 0.0;
  for (int r = lane; r < n; r += 32) {
    const z64 cr = c[r];
    s += cr.x * w1[r].x + cr.y * w1[r].y;  // Re(conj(c) w)
    h += cr.x * w2[r].x + cr.y * w2[r].y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    h += __shfl_xor_sync(0xffffffffu, h, o);
  }
  if (lane == 0) lam[(size_t)p * lstride + j] = h / s;
  const double sc = 1.0 / sqrt(s);
  for (int r = lane; r < n; r += 32) c[r] = zscale(c[r], sc);
}

// One block per problem: sort lambda[0, m) ascending (bitonic, padded with +inf), write eps
// (+inf beyond m) and the permutation.
__global__ void oa_sort_kernel(int n, const int32_t* __restrict__ size, const double* __restrict__ lam,
                               long long lstride, int P2, double* __restrict__ eps, int32_t* __restrict__ perm) {
  extern __shared__ unsigned char sm_raw[];
  double* key = (double*)sm_raw;
  int* idx = (int*)(key + P2);
  const int p = blockIdx.x;
  const int m = size[p];
  for (int i = threadIdx.x; i < P2; i += blockDim.x) {
    key[i] = i < m ? lam[(size_t)p * lstride + i] : INFINITY;
    idx[i] = i;
  }
  __syncthreads();
  for (int k = 2; k <= P2; k <<= 1) {
    for (int jj = k >> 1; jj > 0; jj >>= 1) {
      for (int i = threadIdx.x; i < P2; i += blockDim.x) {
        const int l = i ^ jj;
        if (l > i) {
          const bool up = (i & k) == 0;
          const double a = key[i], b = key[l];
          const bool swap = up ? (a > b || (a == b && idx[i] > idx[l])) : (a < b || (a == b && idx[i] < idx[l]));
          if (swap) {
            key[i] = b;
            key[l] = a;
            const int t = idx[i];
            idx[i] = idx[l];
            idx[l] = t;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    eps[(size_t)p * n + i] = i < m ? key[i] : INFINITY;
    perm[(size_t)p * n + i] = i < m ? idx[i] : -1;
  }
}

// C[p][r][j] (row-major, nb columns) = Cn(r, perm[j]) for j < m, 0 beyond.
__global__ void oa_gather_kernel(int n, int nprob, int nb, const int32_t* __restrict__ perm, const z64* __restrict__ Cn,
                                 int ldc, long long cstride, z64* __restrict__ C) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)nprob * n * nb) return;
  const int j = (int)(idx % nb);
  const size_t pr = idx / nb;
  const int r = (int)(pr % n), p = (int)(pr / n);
  const int src = perm[(size_t)p * n + j];
  C[idx] = src >= 0 ? Cn[(size_t)p * cstride + (size_t)src * ldc + r] : zmk(0.0, 0.0);
}

}  // namespace

cudaError_t launch_oa_lambda(int n, int nprob, const int32_t* size, const z64* Rp, const z64* G, int ld,
                             long long stride, double* lam, long long lstride, cudaStream_t st) {
  const size_t tot = (size_t)nprob * n;
  oa_lambda_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, nprob, size, Rp, G, ld, stride, lam, lstride);
  return cudaGetLastError();
}

cudaError_t launch_oa_f(int n, int nprob, const int32_t* size, const z64* Rp, z64* G, int ld, long long stride,
                        const double* lam, long long lstride, cudaStream_t st) {
  dim3 grid((n + 127) / 128, n, nprob);
  oa_f_kernel<<<grid, 128, 0, st>>>(n, size, Rp, G, ld, stride, lam, lstride);
  return cudaGetLastError();
}

cudaError_t launch_oa_rq(int n, int nprob, const int32_t* size, z64* Cn, int ldc, long long cstride, const z64* W1,
                         const z64* W2, int ldw, long long wstride, double* lam, long long lstride, cudaStream_t st) {
  const size_t warps = (size_t)nprob * n;
  oa_rq_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(n, nprob, size, Cn, ldc, cstride, W1, W2, ldw,
                                                                      wstride, lam, lstride);
  return cudaGetLastError();
}

cudaError_t launch_oa_sort(int n, int nprob, const int32_t* size, const double* lam, long long lstride, double* eps,
                           int32_t* perm, cudaStream_t st) {
  int P2 = 1;
  while (P2 < n) P2 <<= 1;
  const size_t smem = (size_t)P2 * (sizeof(double) + sizeof(int));
  cudaError_t e = cudaFuncSetAttribute(oa_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  oa_sort_kernel<<<nprob, 1024, smem, st>>>(n, size, lam, lstride, P2, eps, perm);
  return cudaGetLastError();
}

cudaError_t launch_oa_gather(int n, int nprob, int nb, const int32_t* perm, const z64* Cn, int ldc, long long cstride,
                             z64* C, cudaStream_t st) {
  const size_t tot = (size_t)nprob * n * nb;
  oa_gather_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, nprob, nb, perm, Cn, ldc, cstride, C);
  return cudaGetLastError();
}
