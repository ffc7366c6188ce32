// Eigen_HH steps 3-4 (Sec. 3: "rearrangement of eigenvectors" and "normalization") and the
// small element-wise steps around them.  The eigenvectors of A are U = Q Z with
// Q = H_0 H_1 ... H_{m-2} from the tridiagonalization; Q is applied in compact WY blocks
// (Q_j = I - V_j T_j V_j^H: W = V_j^H U, then U -= (V_j T_j) W, products issued by the caller), then
// the columns are scaled to unit 2-norm.  For the overlap matrix the normalization also
// applies Part 2's canonical orthogonalization X = U_m diag(s_m^{-1/2}).
#include "nao_internal.cuh"

namespace {

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void count_kept_kernel(int n, int nprob, const int32_t* __restrict__ size, const double* __restrict__ w,
                                  long long strideV, double s_cut, int32_t* __restrict__ m,
                                  int32_t* __restrict__ status) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nprob) return;
  const double* wp = w + (size_t)p * strideV;
  const int np = size ? size[p] : n;  // the problem's order: eigenvalues 0 .. np-1
  int k = 0;
  for (int j = 0; j < np; ++j) k += (wp[j] >= s_cut);
  m[p] = k;
  if (k == 0 && status[p] == 0) status[p] = NAO_E_ALLCUT;
}

__global__ void hermitize_kernel(int n, const int32_t* __restrict__ size, z64* __restrict__ Abase, int ld,
                                 long long strideA) {
  const int p = blockIdx.z;
  const int m = size ? size[p] : n;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;  // row
  const int c = blockIdx.y;                             // column
  if (r >= m || c >= m || r > c) return;
  z64* A = Abase + (size_t)p * strideA;
  if (r == c) {
    A[(size_t)c * ld + r].y = 0.0;
  } else {
    A[(size_t)c * ld + r] = zconj(A[(size_t)r * ld + c]);  // upper (r < c) from lower (c, r)
  }
}

__global__ void write_eps_kernel(int n, int nprob, const int32_t* __restrict__ m, const double* __restrict__ w,
                                 long long strideV, double* __restrict__ eps) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * nprob) return;
  const int p = (int)(idx / n), j = (int)(idx % n);
  eps[idx] = (j < m[p]) ? w[(size_t)p * strideV + j] : __longlong_as_double(0x7ff0000000000000ll);
}

__global__ void zero_cols_kernel(int n, int nprob, int nb, const int32_t* __restrict__ m, z64* __restrict__ C) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * nb * nprob) return;
  const int p = (int)(idx / ((size_t)n * nb));
  const int j = (int)(idx % nb);
  if (j >= m[p]) C[idx] = zmk(0.0, 0.0);
}

__global__ void scale_cols_sqrt_kernel(int n, int nprob, int nb, const z64* __restrict__ C, const double* __restrict__ f,
                                       z64* __restrict__ Cs) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * nb * nprob) return;
  const int p = (int)(idx / ((size_t)n * nb));
  const int j = (int)(idx % nb);
  const double fj = f[(size_t)p * n + j];
  Cs[idx] = zscale(C[idx], fj > 0.0 ? sqrt(fj) : 0.0);
}

// Ce = Cs diag(eps) over the occupied columns (eps is +inf where f = 0: those stay zero)
__global__ void scale_cols_eps_kernel(int n, int nprob, int nb, const z64* __restrict__ Cs, const double* __restrict__ f,
                                      const double* __restrict__ eps, z64* __restrict__ Ce) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * nb * nprob) return;
  const int p = (int)(idx / ((size_t)n * nb));
  const int j = (int)(idx % nb);
  const double fj = f[(size_t)p * n + j];
  Ce[idx] = fj > 0.0 ? zscale(Cs[idx], eps[(size_t)p * n + j]) : zmk(0.0, 0.0);
}

}  // namespace

cudaError_t launch_count_kept(int n, int nprob, const int32_t* size, const double* w, long long strideV, double s_cut,
                              int32_t* m, int32_t* status, cudaStream_t st) {
  count_kept_kernel<<<(nprob + 127) / 128, 128, 0, st>>>(n, nprob, size, w, strideV, s_cut, m, status);
  return cudaGetLastError();
}

cudaError_t launch_hermitize(int n, int nprob, const int32_t* size, z64* A, int ld, long long strideA, cudaStream_t st) {
  dim3 grid((n + 127) / 128, n, nprob);
  hermitize_kernel<<<grid, 128, 0, st>>>(n, size, A, ld, strideA);
  return cudaGetLastError();
}

cudaError_t launch_write_eps(int n, int nprob, const int32_t* m, const double* w, long long strideV, double* eps,
                             cudaStream_t st) {
  const size_t tot = (size_t)n * nprob;
  write_eps_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, nprob, m, w, strideV, eps);
  return cudaGetLastError();
}

cudaError_t launch_zero_cols(int n, int nprob, int nb, const int32_t* m, z64* C, cudaStream_t st) {
  const size_t tot = (size_t)n * nb * nprob;
  zero_cols_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, nprob, nb, m, C);
  return cudaGetLastError();
}

cudaError_t launch_scale_cols_eps(int n, int nprob, int nb, const z64* Cs, const double* f, const double* eps, z64* Ce,
                                  cudaStream_t st) {
  const size_t tot = (size_t)n * nb * nprob;
  scale_cols_eps_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, nprob, nb, Cs, f, eps, Ce);
  return cudaGetLastError();
}

cudaError_t launch_scale_cols_sqrt(int n, int nprob, int nb, const z64* C, const double* f, z64* Cs, cudaStream_t st) {
  const size_t tot = (size_t)n * nb * nprob;
  scale_cols_sqrt_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, nprob, nb, C, f, Cs);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Blocked form of steps 3-4 (compact WY): Q = Q_0 Q_1 ... with Q_j = H_{j nb} ... H_{j nb+nb-1}
// = I - V_j T_j V_j^H, applied as two matrix products per block with V_j T_j formed once (run
// on the tensor cores by the caller).  The kernels below prepare the operands.
// ---------------------------------------------------------------------------------------
namespace {

// Vfull(:, i) = explicit reflector i (1 at row i + off, A(r, i) below, 0 elsewhere) for
// i < m - off, zero columns otherwise (ncolv >= n columns); tauc[i] = tau[i] or 0.
__global__ void extract_v_kernel(int n, const int32_t* __restrict__ size, const z64* __restrict__ Abase, int lda,
                                 long long strideA, const z64* __restrict__ taubase, long long strideV, int ncolv,
                                 z64* __restrict__ Vbase, int ldv, long long strideVf, z64* __restrict__ taucbase,
                                 int off) {
  const int p = blockIdx.z;
  const int m = size ? size[p] : n;
  const int i = blockIdx.y;  // column
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n || i >= ncolv) return;
  const z64* A = Abase + (size_t)p * strideA;
  z64 val = zmk(0.0, 0.0);
  if (i < m - off) {
    if (r == i + off) val = zmk(1.0, 0.0);
    else if (r > i + off && r < m) val = A[(size_t)i * lda + r];
  }
  Vbase[(size_t)p * strideVf + (size_t)i * ldv + r] = val;
  if (r == 0) taucbase[(size_t)p * ncolv + i] = (i < m - off) ? taubase[(size_t)p * strideV + i] : zmk(0.0, 0.0);
}

// U(:, c) = Z(:, m - nc + c) (or Z(:, c) when lowest) as complex for c < nc, rows < m; zero
// elsewhere (n x n).
__global__ void init_u_kernel(int n, const int32_t* __restrict__ size, const int32_t* __restrict__ ncols,
                              const double* __restrict__ Zbase, int ldz, long long strideZ, z64* __restrict__ Ubase,
                              int ldu, long long strideU, int lowest) {
  const int p = blockIdx.z;
  const int m = size ? size[p] : n;
  const int nc = ncols ? ncols[p] : m;
  const int c = blockIdx.y;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  double v = 0.0;
  if (c < nc && r < m) v = Zbase[(size_t)p * strideZ + (size_t)(lowest ? c : m - nc + c) * ldz + r];
  Ubase[(size_t)p * strideU + (size_t)c * ldu + r] = zmk(v, 0.0);
}

// T (nb x nb, row-major, upper triangular) of block j from G = V^H V (row-major, Hermitian):
// T_ii = tau_i, T(0:i, i) = -tau_i T(0:i, 0:i) G(0:i, i).  One block of nb threads per
// (block j, problem p); thread r owns row r of T, which it writes and reads back itself (in
// global memory, cached).  Columns are formed BT_B at a time: the part of each dot product
// over the finished columns is accumulated for all BT_B new columns from one read of the row
// (the reads of T fall BT_B-fold), then the new columns follow one by one from registers;
// the terms are added in the same order as one column at a time.  G's columns of the batch
// sit in shared memory (row stride BT_B + 1: no bank conflicts).  G and T of block j of
// problem p at (j nprob + p) nb^2.
constexpr int BT_B = 8;
__global__ void build_t_kernel(int nb, int nprob, const z64* __restrict__ Gbase, const z64* __restrict__ taucbase,
                               int ncolv, z64* __restrict__ Tbase) {
  extern __shared__ z64 gs[];  // G(c, i0 + k) at gs[c (BT_B + 1) + k]
  const int p = blockIdx.x % nprob, j = blockIdx.x / nprob;
  const int r = threadIdx.x;
  const z64* G = Gbase + (size_t)blockIdx.x * nb * nb;
  const z64* tau = taucbase + (size_t)p * ncolv + (size_t)j * nb;
  z64* Tr = Tbase + (size_t)blockIdx.x * nb * nb + (size_t)r * nb;  // row r
  for (int c = 0; c < r; ++c) Tr[c] = zmk(0.0, 0.0);
  for (int i0 = 0; i0 < nb; i0 += BT_B) {
    const int nbat = nb - i0 < BT_B ? nb - i0 : BT_B, L = i0 + nbat;
    __syncthreads();  // the previous batch's reads of gs are done
    // G(c, i) = conj(G(i, c)) (G is Hermitian): coalesced loads of rows i0 .. i0 + nbat - 1
    for (int idx = r; idx < L * nbat; idx += nb) {
      const int k = idx / L, c = idx - k * L;
      gs[c * (BT_B + 1) + k] = zconj(G[(size_t)(i0 + k) * nb + c]);
    }
    __syncthreads();
    z64 acc[BT_B], tb[BT_B];
#pragma unroll
    for (int k = 0; k < BT_B; ++k) acc[k] = zmk(0.0, 0.0);
    for (int c = r; c < i0; ++c) {  // finished columns
      const z64 t = Tr[c];
#pragma unroll
      for (int k = 0; k < BT_B; ++k) acc[k] = zfma(t, gs[c * (BT_B + 1) + k], acc[k]);
    }
#pragma unroll
    for (int k = 0; k < BT_B; ++k) {
      if (k < nbat) {
        const int i = i0 + k;
        z64 a = acc[k];
#pragma unroll
        for (int c2 = 0; c2 < k; ++c2)  // the batch's earlier columns c = i0 + c2 >= r
          if (i0 + c2 >= r) a = zfma(tb[c2], gs[(i0 + c2) * (BT_B + 1) + k], a);
        const z64 ti = tau[i];
        z64 tv = zmk(0.0, 0.0);
        if (r < i) tv = zmul(zmk(-ti.x, -ti.y), a);
        else if (r == i) tv = ti;
        tb[k] = tv;
        if (r <= i) Tr[i] = tv;
      }
    }
  }
}

// column c < nc: U(:, c) /= ||U(:, c)||, times 1/sqrt(w[m - nc + c]) when use_rsqrt
__global__ void normalize_cols_kernel(int n, const int32_t* __restrict__ size, const int32_t* __restrict__ ncols,
                                      const double* __restrict__ wbase, long long strideV, int use_rsqrt,
                                      z64* __restrict__ Ubase, int ldu, long long strideU) {
  const int p = blockIdx.y;
  const int m = size ? size[p] : n;
  const int nc = ncols ? ncols[p] : m;
  const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= nc) return;
  z64* u = Ubase + (size_t)p * strideU + (size_t)c * ldu;
  double s = 0.0;
  for (int r = lane; r < m; r += 32) s += zabs2(u[r]);
  s = wsum(s);
  double sc = 1.0 / sqrt(s);
  if (use_rsqrt) sc /= sqrt(wbase[(size_t)p * strideV + (m - nc + c)]);
  for (int r = lane; r < m; r += 32) u[r] = zscale(u[r], sc);
}

}  // namespace

cudaError_t launch_extract_v(int n, int nprob, const int32_t* size, const z64* A, int lda, long long strideA,
                             const z64* tau, long long strideV, int ncolv, z64* V, int ldv, long long strideVf,
                             z64* tauc, int off, cudaStream_t st) {
  dim3 grid((n + 127) / 128, ncolv, nprob);
  extract_v_kernel<<<grid, 128, 0, st>>>(n, size, A, lda, strideA, tau, strideV, ncolv, V, ldv, strideVf, tauc, off);
  return cudaGetLastError();
}

cudaError_t launch_init_u(int n, int nprob, const int32_t* size, const int32_t* ncols, const double* Z, int ldz,
                          long long strideZ, z64* U, int ldu, long long strideU, int lowest, cudaStream_t st) {
  dim3 grid((n + 127) / 128, n, nprob);
  init_u_kernel<<<grid, 128, 0, st>>>(n, size, ncols, Z, ldz, strideZ, U, ldu, strideU, lowest);
  return cudaGetLastError();
}

cudaError_t launch_build_t(int nb, int nprob, int nblk, const z64* G, const z64* tauc, int ncolv, z64* T,
                           cudaStream_t st) {
  const size_t smem = (size_t)nb * (BT_B + 1) * sizeof(z64);
  build_t_kernel<<<nprob * nblk, nb, smem, st>>>(nb, nprob, G, tauc, ncolv, T);
  return cudaGetLastError();
}

cudaError_t launch_normalize_cols(int n, int nprob, const int32_t* size, const int32_t* ncols, const double* w,
                                  long long strideV, int use_rsqrt, z64* U, int ldu, long long strideU,
                                  cudaStream_t st) {
  dim3 grid((n + 7) / 8, nprob);
  normalize_cols_kernel<<<grid, 256, 0, st>>>(n, size, ncols, w, strideV, use_rsqrt, U, ldu, strideU);
  return cudaGetLastError();
}
