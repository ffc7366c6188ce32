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

// ---------------------------------------------------------------- tensor-core form
// Both phase sums are one contraction each over a short index (images R or k-points) with
// n^2 independent columns (matrix elements), so they run as FP64-accurate digit-plane GEMMs
// (csrc/ozgemm.cu) instead of FP64 FMAs:
//   Part 1:  [Re Mk; Im Mk](q, e) = sum_r [cos; sin](2 pi k_q.R_r) M(r, e), one GEMM with
//            the cos and sin rows stacked (M = 2 nk rows), then a pack that interleaves the
//            two halves and mirrors the lower triangle;
//   Part 6:  rho(r, e) = sum_q g w_q cos(.) Re P(q, e) + sum_q g w_q sin(.) Im P(q, e), two
//            real GEMMs, the second accumulating (beta = 1).
// The element columns go in chunks so that the digit planes stay within a bounded workspace.

// A[h nk + q][r] = (cos, sin)(2 pi k_q.R_r)[h]
__global__ void bloch_phase_kernel(int nk, int nR, const int32_t* __restrict__ R, const double* __restrict__ kpts,
                                   double* __restrict__ A) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nk * nR) return;
  const int q = t / nR, r = t % nR;
  const double2 ph = phase_of(kpts + 3 * q, R + 3 * r);
  A[(size_t)q * nR + r] = ph.x;
  A[(size_t)(nk + q) * nR + r] = ph.y;
}

// Ac[r][q] = g w_q cos(2 pi k_q.R_r), As[r][q] = g w_q sin(2 pi k_q.R_r)
__global__ void rho_phase_matrix_kernel(int nk, int nR, const int32_t* __restrict__ R, const double* __restrict__ kpts,
                                        const double* __restrict__ wk, double g, double* __restrict__ Ac,
                                        double* __restrict__ As) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nk * nR) return;
  const int r = t / nk, q = t % nk;
  const double2 ph = phase_of(kpts + 3 * q, R + 3 * r);
  const double gw = g * wk[q];
  Ac[t] = gw * ph.x;
  As[t] = gw * ph.y;
}

// Mk[a][q] rows i0 .. i0+rows-1 from the GEMM result Ct[a][h nk + q][(i - i0) n + j]:
// Mk(i, j) = Re + i Im for j <= i (real diagonal), Mk(j, i) = conj(Mk(i, j)) for j < i.
// 32 x 32 tiles through shared memory, so that the mirrored writes are coalesced too.
__global__ void bloch_pack_kernel(int n, int nk, int i0, int rows, const double* __restrict__ Ct, long long Cbs,
                                  long long Crs, z64* __restrict__ Mk) {
  __shared__ z64 tile[32][33];
  const int a = blockIdx.z / nk, q = blockIdx.z % nk;
  const int bi = i0 + blockIdx.y * 32, bj = blockIdx.x * 32;
  if (bj > bi + 31) return;  // tile above the diagonal (uniform per block)
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  const double* Cre = Ct + (size_t)a * Cbs + (size_t)q * Crs;
  const double* Cim = Cre + (size_t)nk * Crs;
  z64* M = Mk + ((size_t)a * nk + q) * n * n;
  const int iend = i0 + rows;
  for (int r = ty; r < 32; r += 8) {
    const int i = bi + r, j = bj + tx;
    z64 v = zmk(0.0, 0.0);
    if (i < iend && j <= i) {
      const size_t c = (size_t)(i - i0) * n + j;
      v = zmk(Cre[c], i == j ? 0.0 : Cim[c]);
      M[(size_t)i * n + j] = v;
    }
    tile[r][tx] = v;
  }
  __syncthreads();
  for (int c = ty; c < 32; c += 8) {
    const int j = bj + c, i = bi + tx;
    if (i < iend && j < i) M[(size_t)j * n + i] = zconj(tile[tx][c]);
  }
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

// ---------------------------------------------------------------- tensor-core launchers
namespace {
constexpr size_t PHASE_TC_CAP = (size_t)1 << 28;  // workspace bound of one chunk (bytes)

size_t wsalign(size_t b) { return (b + 255) & ~(size_t)255; }

// rows of the element matrix per chunk: a multiple of 32 (the pack tiles), all n when they fit
int bloch_chunk_rows(int n, int nR, int nmat, int nk) {
  const size_t per_row = (size_t)nmat * n * (2 * (size_t)nk * 8 + (size_t)NAO_OZ_DIGITS_FP64 * ((nR + 15) / 16 * 16) * 2 + 8);
  int rc = (int)(PHASE_TC_CAP / (per_row ? per_row : 1)) / 32 * 32;
  const int nr = (n + 31) / 32 * 32;
  if (rc < 32) rc = 32;
  return rc < nr ? rc : nr;
}

long long rho_chunk_cols(int n, int nspin, int nk) {
  const size_t per_col = (size_t)nspin * ((size_t)NAO_OZ_DIGITS_FP64 * ((nk + 15) / 16 * 16) * 2 + 8);
  long long nc = (long long)(PHASE_TC_CAP / per_col) / 64 * 64;
  if (nc < 64) nc = 64;
  const long long nn = (long long)n * n;
  return nc < nn ? nc : nn;
}
}  // namespace

size_t bloch_tc_ws_bytes(int n, int nR, int nmat, int nk) {
  const int rc = bloch_chunk_rows(n, nR, nmat, nk);
  const int Nc = rc * n;
  return wsalign(sizeof(double) * 2 * (size_t)nk * nR) + wsalign(sizeof(double) * (size_t)nmat * 2 * nk * Nc) +
         wsalign(dgemm_oz_workspace(nmat, GemmDims{2 * nk, Nc, nR, nullptr, nullptr, nullptr}));
}

cudaError_t launch_bloch_sum_tc(int n, int nR, const int32_t* R, int nmat, const double* MR, int nk,
                                const double* kpts, z64* Mk, void* ws, int* err, cudaStream_t st, int* nlaunch) {
  const int rc = bloch_chunk_rows(n, nR, nmat, nk);
  const int Ncmax = rc * n;
  char* w = (char*)ws;
  double* A = (double*)w;
  w += wsalign(sizeof(double) * 2 * (size_t)nk * nR);
  double* Ct = (double*)w;
  w += wsalign(sizeof(double) * (size_t)nmat * 2 * nk * Ncmax);
  void* ozws = w;
  *nlaunch = 1;
  bloch_phase_kernel<<<(nk * nR + 255) / 256, 256, 0, st>>>(nk, nR, R, kpts, A);
  cudaError_t e = cudaGetLastError();
  const long long nn = (long long)n * n;
  for (int i0 = 0; i0 < n && e == cudaSuccess; i0 += rc) {
    const int rows = n - i0 < rc ? n - i0 : rc;
    const int Nc = rows * n;
    const long long Cbs = 2LL * nk * Nc;
    GemmDims d{2 * nk, Nc, nR, nullptr, nullptr, nullptr};
    e = launch_dgemm_oz(nmat, d, 1.0, GemmOperand{A, 0, nR, 1, 0, nullptr},
                        GemmOperand{MR + (size_t)i0 * n, (long long)nR * nn, nn, 1, 0, nullptr}, 0.0, Ct, Cbs, Nc, 1,
                        ozws, err, st, NAO_OZ_DIGITS_FP64);
    if (e != cudaSuccess) break;
    dim3 grid((n + 31) / 32, (rows + 31) / 32, nmat * nk), block(32, 8);
    bloch_pack_kernel<<<grid, block, 0, st>>>(n, nk, i0, rows, Ct, Cbs, Nc, Mk);
    e = cudaGetLastError();
    *nlaunch += 4;
  }
  return e;
}

size_t rho_phase_tc_ws_bytes(int n, int nspin, int nk, int nR) {
  const long long Nc = rho_chunk_cols(n, nspin, nk);
  return 2 * wsalign(sizeof(double) * (size_t)nk * nR) +
         wsalign(dgemm_oz_workspace(nspin, GemmDims{nR, (int)Nc, nk, nullptr, nullptr, nullptr}));
}

cudaError_t launch_rho_phase_tc(int n, int nspin, int nk, int nR, const int32_t* R, const double* kpts,
                                const double* wk, double g, const z64* P, double* rho, void* ws, int* err,
                                cudaStream_t st, int* nlaunch) {
  const long long nn = (long long)n * n;
  const long long Ncmax = rho_chunk_cols(n, nspin, nk);
  char* w = (char*)ws;
  double* Ac = (double*)w;
  w += wsalign(sizeof(double) * (size_t)nk * nR);
  double* As = (double*)w;
  w += wsalign(sizeof(double) * (size_t)nk * nR);
  void* ozws = w;
  *nlaunch = 1;
  rho_phase_matrix_kernel<<<(nk * nR + 255) / 256, 256, 0, st>>>(nk, nR, R, kpts, wk, g, Ac, As);
  cudaError_t e = cudaGetLastError();
  const double* Pd = (const double*)P;  // [s][q][e] complex as (re, im) doubles
  for (long long c0 = 0; c0 < nn && e == cudaSuccess; c0 += Ncmax) {
    const int Nc = (int)(nn - c0 < Ncmax ? nn - c0 : Ncmax);
    GemmDims d{nR, Nc, nk, nullptr, nullptr, nullptr};
    for (int h = 0; h < 2 && e == cudaSuccess; ++h) {  // cos Re P, then + sin Im P
      e = launch_dgemm_oz(nspin, d, 1.0, GemmOperand{h ? As : Ac, 0, nk, 1, 0, nullptr},
                          GemmOperand{Pd + 2 * c0 + h, 2LL * nk * nn, 2 * nn, 2, 0, nullptr}, h ? 1.0 : 0.0,
                          rho + c0, (long long)nR * nn, nn, 1, ozws, err, st, NAO_OZ_DIGITS_FP64);
      *nlaunch += 3;
    }
  }
  return e;
}
