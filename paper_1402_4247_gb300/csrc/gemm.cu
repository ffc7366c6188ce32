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
  const int K = dims.Kp ? dims.Kp[p] : dims.K;
  const int i0 = blockIdx.y * BM, j0 = blockIdx.x * BN;
  if (i0 >= M || j0 >= Nn) return;
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

}  // namespace

cudaError_t launch_zgemm(int nprob, GemmDims dims, z64 alpha, GemmOperand A, GemmOperand B, z64 beta, z64* C,
                         long long Cbs, long long Crs, long long Ccs, cudaStream_t st) {
  return launch_gemm_t<z64>(nprob, dims, alpha, A, B, beta, C, Cbs, Crs, Ccs, st);
}

cudaError_t launch_dgemm(int nprob, GemmDims dims, double alpha, GemmOperand A, GemmOperand B, double beta, double* C,
                         long long Cbs, long long Crs, long long Ccs, cudaStream_t st) {
  return launch_gemm_t<double>(nprob, dims, alpha, A, B, beta, C, Cbs, Crs, Ccs, st);
}
