// Part 1 (Sec. 3): giving k dependence to H and S, and its inverse for the density matrix
// (Part 6).  Both are phase-weighted sums over the lattice images R.
#include "nao_internal.cuh"

namespace {

constexpr int KB = 8;          // k-points per pass (accumulators per thread: 2*KB)
constexpr int BLOCH_THREADS = 256;

// (cos, sin)(2 pi frac(k.R)); the integer part of k.R is removed first so that the
// argument of sincospi stays in [-1, 1].
__device__ __forceinline__ double2 phase_of(const double* k, const int32_t* R) {
  double t = k[0] * (double)R[0] + k[1] * (double)R[1] + k[2] * (double)R[2];
  t -= rint(t);
  double s, c;
  sincospi(2.0 * t, &s, &c);
  return make_double2(c, s);
}

// Lower-triangle element t -> (i, j), i >= j, t = i(i+1)/2 + j.
__device__ __forceinline__ void tri_index(long long t, int& i, int& j) {
  int r = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while ((long long)(r + 1) * (r + 2) / 2 <= t) ++r;
  while ((long long)r * (r + 1) / 2 > t) --r;
  i = r;
  j = (int)(t - (long long)r * (r + 1) / 2);
}

// grid: x over lower-triangle elements, y over (matrix a, k-block)
__global__ void __launch_bounds__(BLOCH_THREADS)
bloch_sum_kernel(int n, int nR, const int32_t* __restrict__ R, const double* __restrict__ MR, int nk,
                 const double* __restrict__ kpts, z64* __restrict__ Mk, int nkb) {
  extern __shared__ double2 ph[];  // [KB][nR]
  const int a = blockIdx.y / nkb;
  const int q0 = (blockIdx.y % nkb) * KB;
  const int nq = min(KB, nk - q0);
  for (int idx = threadIdx.x; idx < KB * nR; idx += blockDim.x) {
    int q = idx / nR, r = idx % nR;
    ph[idx] = (q < nq) ? phase_of(kpts + 3 * (q0 + q), R + 3 * r) : make_double2(0.0, 0.0);
  }
  __syncthreads();
  const long long ntri = (long long)n * (n + 1) / 2;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntri) return;
  int i, j;
  tri_index(t, i, j);
  const size_t nn = (size_t)n * n;
  const double* src = MR + (size_t)a * nR * nn + (size_t)i * n + j;
  double re[KB], im[KB];
#pragma unroll
  for (int q = 0; q < KB; ++q) re[q] = im[q] = 0.0;
  for (int r = 0; r < nR; ++r) {
    const double m = src[(size_t)r * nn];
#pragma unroll
    for (int q = 0; q < KB; ++q) {
      const double2 p = ph[q * nR + r];
      re[q] = fma(p.x, m, re[q]);
      im[q] = fma(p.y, m, im[q]);
    }
  }
  for (int q = 0; q < nq; ++q) {
    z64* out = Mk + ((size_t)a * nk + q0 + q) * nn;
    out[(size_t)i * n + j] = zmk(re[q], im[q]);
    if (i != j) out[(size_t)j * n + i] = zmk(re[q], -im[q]);
    else out[(size_t)i * n + j] = zmk(re[q], 0.0);
  }
}

// rho[s][r][i][j] = g sum_q w_q Re(P[s][q][i][j] e^{-2 pi i k_q.R_r})
//                 = g sum_q w_q (Re P cos + Im P sin)
constexpr int RB = 8;  // images per pass
__global__ void __launch_bounds__(BLOCH_THREADS)
rho_phase_kernel(int n, int nk, int nR, const int32_t* __restrict__ R, const double* __restrict__ kpts,
                 const double* __restrict__ wk, double g, const z64* __restrict__ P, double* __restrict__ rho,
                 int nrb) {
  extern __shared__ double2 ph[];  // [nk][RB], pre-multiplied by g w_q
  const int s = blockIdx.y / nrb;
  const int r0 = (blockIdx.y % nrb) * RB;
  const int nr = min(RB, nR - r0);
  for (int idx = threadIdx.x; idx < nk * RB; idx += blockDim.x) {
    int q = idx / RB, r = idx % RB;
    double2 v = make_double2(0.0, 0.0);
    if (r < nr) {
      v = phase_of(kpts + 3 * q, R + 3 * (r0 + r));
      const double gw = g * wk[q];
      v.x *= gw;
      v.y *= gw;
    }
    ph[idx] = v;
  }
  __syncthreads();
  const size_t nn = (size_t)n * n;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nn) return;
  double acc[RB];
#pragma unroll
  for (int r = 0; r < RB; ++r) acc[r] = 0.0;
  const z64* src = P + (size_t)s * nk * nn + e;
  for (int q = 0; q < nk; ++q) {
    const z64 pv = src[(size_t)q * nn];
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const double2 c = ph[q * RB + r];
      acc[r] = fma(pv.x, c.x, fma(pv.y, c.y, acc[r]));
    }
  }
  for (int r = 0; r < nr; ++r) rho[((size_t)s * nR + r0 + r) * nn + e] = acc[r];
}

// Full Hermitian, column-major dst from a row-major lower-triangle src (32x32 tiles so that
// both the read and the write are coalesced).
__global__ void herm_fill_kernel(int n, const z64* __restrict__ src, long long sstride, const int32_t* __restrict__ map,
                                 z64* __restrict__ dst, int ld, long long dstride) {
  __shared__ z64 tile[32][33];
  const int p = blockIdx.z;
  const z64* S = src + (size_t)(map ? map[p] : p) * sstride;
  z64* D = dst + (size_t)p * dstride;
  const int bi = blockIdx.y * 32, bj = blockIdx.x * 32;  // dst tile rows bi.., cols bj..
  const int tx = threadIdx.x, ty = threadIdx.y;            // 32 x 8
  if (bi >= bj) {
    // dst(i, j) = src[i][j] for i >= j: read rows of src (coalesced in j), write columns of dst.
    for (int r = ty; r < 32; r += 8) {
      int i = bi + r, j = bj + tx;
      tile[r][tx] = (i < n && j < n) ? S[(size_t)i * n + j] : zmk(0, 0);
    }
    __syncthreads();
    for (int c = ty; c < 32; c += 8) {
      int j = bj + c, i = bi + tx;
      if (i < n && j < n) {
        z64 v = tile[tx][c];
        if (i < j) v = zconj(S[(size_t)j * n + i]);  // only on the diagonal tile
        if (i == j) v.y = 0.0;
        D[(size_t)j * ld + i] = v;
      }
    }
  } else {
    // upper tile: dst(i, j) = conj(src[j][i]) with j > i: src row j is contiguous in i.
    for (int c = ty; c < 32; c += 8) {
      int j = bj + c, i = bi + tx;
      if (i < n && j < n) D[(size_t)j * ld + i] = zconj(S[(size_t)j * n + i]);
    }
  }
}

}  // namespace

cudaError_t launch_bloch_sum(int n, int nR, const int32_t* R, int nmat, const double* MR, int nk,
                             const double* kpts, z64* Mk, cudaStream_t st) {
  const long long ntri = (long long)n * (n + 1) / 2;
  const int nkb = (nk + KB - 1) / KB;
  dim3 grid((unsigned)((ntri + BLOCH_THREADS - 1) / BLOCH_THREADS), (unsigned)(nmat * nkb));
  size_t smem = sizeof(double2) * KB * nR;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(bloch_sum_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  bloch_sum_kernel<<<grid, BLOCH_THREADS, smem, st>>>(n, nR, R, MR, nk, kpts, Mk, nkb);
  return cudaGetLastError();
}

cudaError_t launch_rho_phase_sum(int n, int nspin, int nk, int nR, const int32_t* R, const double* kpts,
                                 const double* wk, double g, const z64* P, double* rho, cudaStream_t st) {
  const size_t nn = (size_t)n * n;
  const int nrb = (nR + RB - 1) / RB;
  dim3 grid((unsigned)((nn + BLOCH_THREADS - 1) / BLOCH_THREADS), (unsigned)(nspin * nrb));
  size_t smem = sizeof(double2) * nk * RB;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(rho_phase_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  rho_phase_kernel<<<grid, BLOCH_THREADS, smem, st>>>(n, nk, nR, R, kpts, wk, g, P, rho, nrb);
  return cudaGetLastError();
}

cudaError_t launch_herm_fill(int n, int nprob, const z64* src, long long src_stride, const int32_t* map,
                             z64* dst, int ld, long long dst_stride, cudaStream_t st) {
  dim3 grid((n + 31) / 32, (n + 31) / 32, nprob), block(32, 8);
  herm_fill_kernel<<<grid, block, 0, st>>>(n, src, src_stride, map, dst, ld, dst_stride);
  return cudaGetLastError();
}
