// Batched FP64 GEMM for the GEMM-shaped steps (Sec. 3: Parts 3-4 use ZGEMM; the
// back-transform re-orthogonalisation and Part 6 reuse it): C = alpha op(A) op(B) + beta C
// with arbitrary element strides, optional conjugation, per-problem dimensions and an
// optional batch-index map per operand.
//
// FP64 CUDA-core kernel: 64x64 output tile per 256-thread block, 4x4 outputs per thread,
// K staged through shared memory in slices of 8.  On this GPU the FP64 pipe (not memory)
// bounds it: 16 complex multiply-adds per 8 shared-memory loads per thread.
#include "nao_internal.cuh"

namespace {

constexpr int BM = 64, BN = 64, BK = 8, TM = 4, TN = 4, GT = 256;

template <typename T> struct Num;
template <> struct Num<double> {
  __device__ static double zero() { return 0.0; }
  __device__ static double conj(double a) { return a; }
  __device__ static double fma_(double a, double b, double c) { return fma(a, b, c); }
  __device__ static double mul(double a, double b) { return a * b; }
  __device__ static double add(double a, double b) { return a + b; }
  __device__ static bool is_zero(double a) { return a == 0.0; }
};
template <> struct Num<z64> {
  __device__ static z64 zero() { return zmk(0.0, 0.0); }
  __device__ static z64 conj(z64 a) { return zconj(a); }
  __device__ static z64 fma_(z64 a, z64 b, z64 c) { return zfma(a, b, c); }
  __device__ static z64 mul(z64 a, z64 b) { return zmul(a, b); }
  __device__ static z64 add(z64 a, z64 b) { return zadd(a, b); }
  __device__ static bool is_zero(z64 a) { return a.x == 0.0 && a.y == 0.0; }
};

template <typename T>
__global__ void __launch_bounds__(GT)
gemm_kernel(GemmDims dims, T alpha, GemmOperand A, GemmOperand B, T beta, T* __restrict__ C, long long Cbs,
            long long Crs, long long Ccs) {
  typedef Num<T> N_;
  __shared__ T As[BK][BM];
  __shared__ T Bs[BK][BN];
  const int p = blockIdx.z;
  const int M = dims.Mp ? dims.Mp[p] : dims.M;
  const int Nn = dims.Np ? dims.Np[p] : dims.N;
  const int K = gemm_k(dims, p);
  const int i0 = blockIdx.y * BM, j0 = blockIdx.x * BN;
  if (i0 >= M || j0 >= Nn) return;
  if (dims.lower && j0 > i0 + BM - 1) return;  // tile entirely above the diagonal
  const T* Ap = (const T*)A.ptr + (size_t)(A.map ? A.map[p] : p) * A.bs;
  const T* Bp = (const T*)B.ptr + (size_t)(B.map ? B.map[p] : p) * B.bs;
  T* Cp = C + (size_t)p * Cbs;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const bool a_rowfast = llabs(A.rs) <= llabs(A.cs);
  const bool b_rowfast = llabs(B.rs) <= llabs(B.cs);
  T acc[TM][TN];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TN; ++b) acc[a][b] = N_::zero();

  for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
    for (int s = 0; s < (BM * BK) / GT; ++s) {
      const int e = tid + GT * s;
      int row, kk;
      if (a_rowfast) { row = e % BM; kk = e / BM; }
      else { kk = e % BK; row = e / BK; }
      const int gi = i0 + row, gk = k0 + kk;
      T v = N_::zero();
      if (gi < M && gk < K) {
        v = Ap[(long long)gi * A.rs + (long long)gk * A.cs];
        if (A.conj) v = N_::conj(v);
      }
      As[kk][row] = v;
    }
#pragma unroll
    for (int s = 0; s < (BN * BK) / GT; ++s) {
      const int e = tid + GT * s;
      int col, kk;
      if (b_rowfast) { kk = e % BK; col = e / BK; }
      else { col = e % BN; kk = e / BN; }
      const int gj = j0 + col, gk = k0 + kk;
      T v = N_::zero();
      if (gj < Nn && gk < K) {
        v = Bp[(long long)gk * B.rs + (long long)gj * B.cs];
        if (B.conj) v = N_::conj(v);
      }
      Bs[kk][col] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T av[TM], bv[TN];
#pragma unroll
      for (int a = 0; a < TM; ++a) av[a] = As[kk][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < TN; ++b) bv[b] = Bs[kk][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TN; ++b) acc[a][b] = N_::fma_(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
  const bool use_beta = !N_::is_zero(beta);
#pragma unroll
  for (int a = 0; a < TM; ++a) {
    const int gi = i0 + ty + 16 * a;
    if (gi >= M) continue;
#pragma unroll
    for (int b = 0; b < TN; ++b) {
      const int gj = j0 + tx + 16 * b;
      if (gj >= Nn) continue;
      T* cp = Cp + (long long)gi * Crs + (long long)gj * Ccs;
      T r = N_::mul(alpha, acc[a][b]);
      if (use_beta) r = N_::fma_(beta, *cp, r);
      *cp = r;
    }
  }
}

template <typename T>
cudaError_t launch_gemm_t(int nprob, GemmDims dims, T alpha, GemmOperand A, GemmOperand B, T beta, T* C,
                          long long Cbs, long long Crs, long long Ccs, cudaStream_t st) {
  if (nprob <= 0 || dims.M <= 0 || dims.N <= 0) return cudaSuccess;
  dim3 grid((dims.N + BN - 1) / BN, (dims.M + BM - 1) / BM, nprob);
  gemm_kernel<T><<<grid, GT, 0, st>>>(dims, alpha, A, B, beta, C, Cbs, Crs, Ccs);
  return cudaGetLastError();
}

// Z2 = Z - 0.5 Z (G - I), G symmetric from its lower triangle; FP32 product.
constexpr int NB = 64, NK = 16;
__global__ void __launch_bounds__(256)
ns_correct_kernel(int n, const int32_t* __restrict__ size, const int32_t* __restrict__ ncols,
                  const double* __restrict__ Zb, const double* __restrict__ Gb, int ld, long long stride,
                  double* __restrict__ Z2b) {
  __shared__ float Zs[NK][NB + 1];
  __shared__ float Es[NK][NB + 1];
  const int p = blockIdx.z;
  const int m = size ? size[p] : n;
  const int nc = ncols ? ncols[p] : m;  // columns of Z (and order of G)
  const int i0 = blockIdx.y * NB, j0 = blockIdx.x * NB;
  if (i0 >= m || j0 >= nc) return;
  const double* Z = Zb + (size_t)p * stride;
  const double* G = Gb + (size_t)p * stride;
  double* Z2 = Z2b + (size_t)p * stride;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
  for (int k0 = 0; k0 < nc; k0 += NK) {
#pragma unroll
    for (int s = 0; s < (NB * NK) / 256; ++s) {
      const int e = tid + 256 * s;
      const int row = e % NB, kk = e / NB;  // Z(i0+row, k0+kk): column-major, rows fast
      const int gi = i0 + row, gk = k0 + kk;
      Zs[kk][row] = (gi < m && gk < nc) ? (float)Z[(size_t)gk * ld + gi] : 0.f;
      const int col = e % NB, kk2 = e / NB;  // E(k0+kk2, j0+col)
      const int gj = j0 + col, gk2 = k0 + kk2;
      float ev = 0.f;
      if (gj < nc && gk2 < nc) {
        double g = (gk2 >= gj) ? G[(size_t)gj * ld + gk2] : G[(size_t)gk2 * ld + gj];
        if (gk2 == gj) g -= 1.0;
        ev = (float)g;
      }
      Es[kk2][col] = ev;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < NK; ++kk) {
      float av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = Zs[kk][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Es[kk][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int gi = i0 + ty + 16 * a;
    if (gi >= m) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int gj = j0 + tx + 16 * b;
      if (gj >= nc) continue;
      const size_t o = (size_t)gj * ld + gi;
      Z2[o] = Z[o] - 0.5 * (double)acc[a][b];
    }
  }
}

// E = G - I made full in place from G = Z^T Z given by its lower triangle (column-major, ld):
// the upper triangle mirrored from the lower, 1 subtracted on the diagonal; order ncols[p]
// (n when ncols is null).  A block owns one 32 x 32 tile on or above the diagonal and reads
// its mirror through shared memory, so that both the read and the write are coalesced.
__global__ void sym_minus_identity_kernel(int n, const int32_t* __restrict__ ncols, double* __restrict__ Gb, int ld,
                                          long long stride) {
  __shared__ double tile[32][33];
  const int p = blockIdx.z;
  const int nc = ncols ? ncols[p] : n;
  const int bi = blockIdx.y * 32, bj = blockIdx.x * 32;  // target rows bi.., columns bj..
  if (bi > bj || bj >= nc) return;                        // uniform per block
  double* G = Gb + (size_t)p * stride;
  const int tx = threadIdx.x, ty = threadIdx.y;           // 32 x 8
  for (int c = ty; c < 32; c += 8) {  // source G(j, i), j = bj + tx, i = bi + c: contiguous in j
    const int i = bi + c, j = bj + tx;
    tile[c][tx] = (i < nc && j < nc && j >= i) ? G[(size_t)i * ld + j] : 0.0;
  }
  __syncthreads();
  for (int c = ty; c < 32; c += 8) {  // target E(i, j), i = bi + tx, j = bj + c: contiguous in i
    const int i = bi + tx, j = bj + c;
    if (i < nc && j < nc && i <= j) G[(size_t)j * ld + i] = (i == j) ? tile[tx][c] - 1.0 : tile[tx][c];
  }
}

}  // namespace

cudaError_t launch_sym_minus_identity(int n, int nprob, const int32_t* ncols, double* G, int ld, long long stride,
                                      cudaStream_t st) {
  dim3 grid((n + 31) / 32, (n + 31) / 32, nprob), block(32, 8);
  sym_minus_identity_kernel<<<grid, block, 0, st>>>(n, ncols, G, ld, stride);
  return cudaGetLastError();
}

cudaError_t launch_ns_correct(int n, int nprob, const int32_t* size, const int32_t* ncols, const double* Z,
                              const double* G, int ld, long long stride, double* Z2, cudaStream_t st) {
  dim3 grid((n + NB - 1) / NB, (n + NB - 1) / NB, nprob);
  ns_correct_kernel<<<grid, 256, 0, st>>>(n, size, ncols, Z, G, ld, stride, Z2);
  return cudaGetLastError();
}

cudaError_t launch_zgemm(int nprob, GemmDims dims, z64 alpha, GemmOperand A, GemmOperand B, z64 beta, z64* C,
                         long long Cbs, long long Crs, long long Ccs, cudaStream_t st) {
  return launch_gemm_t<z64>(nprob, dims, alpha, A, B, beta, C, Cbs, Crs, Ccs, st);
}

cudaError_t launch_dgemm(int nprob, GemmDims dims, double alpha, GemmOperand A, GemmOperand B, double beta, double* C,
                         long long Cbs, long long Crs, long long Ccs, cudaStream_t st) {
  return launch_gemm_t<double>(nprob, dims, alpha, A, B, beta, C, Cbs, Crs, Ccs, st);
}
