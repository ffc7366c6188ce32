// Two-stage form of Eigen_HH step 1 (Sec. 3; the paper's conclusion asks for an algorithm
// change in its Householder part): A Hermitian -> band (lower bandwidth B) -> real symmetric
// tridiagonal, and the matching second back-transformation.
//
// * Stage 1, dense -> band, one panel of B columns at a time (host loop in api.cu):
//   QR of the panel below its diagonal block (he2hb_qr_kernel, FP64), Q = I - V T V^H, then
//   the two-sided update A22 <- Q^H A22 Q = A22 - V W^H - W V^H with X = A22 V T and
//   W = X - V (T^H V^H X) / 2.  Every product there (V^H V, V T, A22 (V T), V^H X, T^H M,
//   the W correction and the rank-2B update) runs on the tensor cores (digit planes).
// * Stage 2, band -> tridiagonal (hb2st_kernel, one block per matrix, FP64): sweep j
//   annihilates column j below its subdiagonal with a reflector of length <= B, applies it
//   from both sides to the diagonal block it spans and from the right to the block below,
//   which fills that block; the next step of the sweep annihilates the first column of the
//   fill, and so on down the band.  The rest of the fill is removed by later sweeps, so the
//   band never holds more than 2B - 1 subdiagonals.  Every reflector leaves a real
//   subdiagonal entry, so the result is real.
// * Back-transformation of stage 2 (q2_apply_kernel, FP64): U = Q2 Z with Q2 the product of
//   the stage-2 reflectors in the order they were made; the reflectors of one sweep act on
//   disjoint rows and are applied in parallel (one warp each), sweeps from the last to the
//   first, on a block of columns held in shared memory.  Stage 1's reflectors follow as
//   compact WY blocks on the tensor cores (backtransform_blocked with head offset B).
//
// Band storage: element (r, c) of the lower band, 0 <= r - c < 2B, at AB[c 2B + (r - c)].
// Stage-2 reflector (sweep j, step k) at index q2_index(n, B, j) + k: B complex entries
// (v_0 = 1, zero past its length) and tau.
#include "nao_internal.cuh"

namespace {

constexpr int SBR_THREADS = 256;

__device__ __forceinline__ double wsum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Reflector H = I - tau v v^H (v_0 = 1) with H^H (alpha, x)^T = (beta, 0)^T, beta real,
// v_i = x_i scale; xnorm2 = |x|^2.  tau = 0 (H = I) when x = 0 and alpha is real.
struct Refl {
  z64 tau;
  double beta;
  z64 scale;
};
__device__ __forceinline__ Refl make_refl(z64 alpha, double xnorm2) {
  Refl h;
  if (xnorm2 == 0.0 && alpha.y == 0.0) {
    h.tau = zmk(0.0, 0.0);
    h.beta = alpha.x;
    h.scale = zmk(0.0, 0.0);
    return h;
  }
  const double nrm = sqrt(alpha.x * alpha.x + alpha.y * alpha.y + xnorm2);
  const double beta = alpha.x >= 0.0 ? -nrm : nrm;
  h.beta = beta;
  h.tau = zmk((beta - alpha.x) / beta, -alpha.y / beta);
  const z64 dd = zmk(alpha.x - beta, alpha.y);  // 1 / (alpha - beta)
  const double den = dd.x * dd.x + dd.y * dd.y;
  h.scale = zmk(dd.x / den, -dd.y / den);
  return h;
}

// ---------------------------------------------------------------- stage 1: panel QR
// Panel columns c0 .. c0+B-1, rows r0 = c0 + B .. m-1 of the column-major A (ld n).  Each
// warp owns the columns q with (q - c0) % 8 == warp: it forms that column's reflector when
// its turn comes and applies the earlier reflectors to it (lanes over rows, coalesced).
// Leaves R (upper part) and the reflector tails in A, tau in tauc[p][B], and the explicit
// reflectors (1 at the head, zero above it and at rows >= m) in columns 0..B-1 and
// 2B..3B-1 of VW ([n][3B] row-major, rows r0 .. n-1).
template <int B>
__global__ void __launch_bounds__(SBR_THREADS) he2hb_qr_kernel(int n, const int32_t* __restrict__ size,
                                                               z64* __restrict__ Abase, long long sA, int c0,
                                                               z64* __restrict__ taucbase, z64* __restrict__ taubase,
                                                               long long stau, z64* __restrict__ VWbase, long long sVW) {
  const int p = blockIdx.x;
  const int m = size ? size[p] : n;
  z64* A = Abase + (size_t)p * sA;
  z64* VW = VWbase + (size_t)p * sVW;
  const int r0 = c0 + B;
  const int L = m - r0;
  const int nrefl = L <= 0 ? 0 : (L < B ? L : B);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ z64 s_tau[B];
  for (int i = 0; i < nrefl; ++i) {
    const int col = c0 + i, head = r0 + i;
    z64* a = A + (size_t)col * n;
    if (warp == (i & 7)) {
      double s = 0.0;
      for (int r = head + 1 + lane; r < m; r += 32) s += zabs2(a[r]);
      s = wsum_d(s);
      const z64 alpha = a[head];
      Refl h;
      if (head + 1 >= m) {  // length 1: nothing to annihilate
        h.tau = zmk(0.0, 0.0);
        h.beta = 0.0;
        h.scale = zmk(0.0, 0.0);
      } else {
        h = make_refl(alpha, s);
      }
      if (h.tau.x != 0.0 || h.tau.y != 0.0) {
        for (int r = head + 1 + lane; r < m; r += 32) a[r] = zmul(a[r], h.scale);
        if (lane == 0) a[head] = zmk(h.beta, 0.0);
      }
      if (lane == 0) s_tau[i] = h.tau;
    }
    __syncthreads();
    const z64 tau = s_tau[i];
    if (tau.x != 0.0 || tau.y != 0.0) {
      const z64 ctau = zconj(tau);
      for (int q = c0 + i + 1 + ((warp - (i + 1)) & 7); q < c0 + B; q += 8) {
        z64* aq = A + (size_t)q * n;
        z64 acc = zmk(0.0, 0.0);
        for (int r = head + 1 + lane; r < m; r += 32) acc = zcfma(a[r], aq[r], acc);
        acc.x = wsum_d(acc.x);
        acc.y = wsum_d(acc.y);
        acc = zadd(acc, aq[head]);   // v_head = 1
        const z64 t = zmul(ctau, acc);  // conj(tau) v^H a_q
        for (int r = head + 1 + lane; r < m; r += 32) aq[r] = zfms(a[r], t, aq[r]);
        __syncwarp();
        if (lane == 0) aq[head] = zsub(aq[head], t);
      }
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < B; i += blockDim.x) {
    const z64 t = i < nrefl ? s_tau[i] : zmk(0.0, 0.0);
    taucbase[(size_t)p * B + i] = t;
    if (c0 + i < n) taubase[(size_t)p * stau + c0 + i] = t;
  }
  // explicit reflectors, rows r0 .. n-1
  const int nrow = n - r0;
  for (int idx = threadIdx.x; idx < nrow * B; idx += blockDim.x) {
    const int r = r0 + idx / B, i = idx % B;
    z64 v = zmk(0.0, 0.0);
    if (i < nrefl && r < m) {
      const int head = r0 + i;
      if (r == head) v = zmk(1.0, 0.0);
      else if (r > head) v = A[(size_t)(c0 + i) * n + r];
    }
    VW[(size_t)r * 3 * B + i] = v;
    VW[(size_t)r * 3 * B + 2 * B + i] = v;
  }
}

// Lower band (offsets 0..B, and zero for B+1..2B-1) of the reduced matrix into AB.
template <int B>
__global__ void band_extract_kernel(int n, const int32_t* __restrict__ size, const z64* __restrict__ Abase,
                                    long long sA, z64* __restrict__ ABbase, long long sAB) {
  const int p = blockIdx.y;
  const int m = size ? size[p] : n;
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * 2 * B) return;
  const int c = (int)(idx / (2 * B)), o = (int)(idx % (2 * B));
  z64 v = zmk(0.0, 0.0);
  if (o <= B && c + o < m) {
    v = Abase[(size_t)p * sA + (size_t)c * n + c + o];
    if (o == 0) v.y = 0.0;
  }
  ABbase[(size_t)p * sAB + idx] = v;
}

// Rows and columns >= size[p] of A set to zero (the product steps of stage 1 read all n).
__global__ void zero_outside_kernel(int n, const int32_t* __restrict__ size, z64* __restrict__ Abase, long long sA) {
  const int p = blockIdx.y;
  const int m = size[p];
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * n) return;
  const int c = (int)(idx / n), r = (int)(idx % n);
  if (r >= m || c >= m) Abase[(size_t)p * sA + idx] = zmk(0.0, 0.0);
}

// ---------------------------------------------------------------- stage 2: bulge chasing
__host__ __device__ inline long long floor_sum(long long T, int B) {  // sum_{t=0}^{T} floor(t / B)
  if (T < 0) return 0;
  const long long q = (T + 1) / B, r = (T + 1) % B;
  return (long long)B * q * (q - 1) / 2 + q * r;
}

// Block of one step: P = rows [s1, s2] x columns [c, c + wP) (the column being annihilated
// and, after the first step, the rest of the previous fill block), D = the Hermitian
// diagonal block [s1, s2]^2, C = rows [s2 + 1, s2 + Lb] x columns [s1, s2] (filled by this
// step, the next step's P).  Shared-memory blocks are column-major with leading dimension
// B + 1 (no bank conflicts on either index).
template <int B>
__global__ void __launch_bounds__(SBR_THREADS) hb2st_kernel(int n, const int32_t* __restrict__ size,
                                                            z64* __restrict__ ABbase, long long sAB,
                                                            double* __restrict__ dbase, double* __restrict__ ebase,
                                                            long long sv, z64* __restrict__ V2base,
                                                            z64* __restrict__ tau2base, long long sq) {
  constexpr int LD = B + 1;
  constexpr int W2 = 2 * B;
  const int p = blockIdx.x;
  const int m = size ? size[p] : n;
  z64* AB = ABbase + (size_t)p * sAB;
  z64* V2 = V2base + (size_t)p * sq * B;
  z64* tau2 = tau2base + (size_t)p * sq;
  extern __shared__ z64 hb_smem[];  // P and C (ping-pong), D, then v, w, p, y and tau
  z64* sPC[2] = {hb_smem, hb_smem + B * LD};
  z64* sD = hb_smem + 2 * B * LD;
  z64* s_v = sD + B * LD;
  z64* s_w = s_v + B;
  z64* s_p = s_w + B;
  z64* s_y = s_p + B;
  z64& s_tau = s_y[B];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long fs_n = floor_sum(n - 2, B);
  for (int j = 0; j < m - 1; ++j) {
    const long long qbase = j + fs_n - floor_sum(n - 2 - j, B);  // q2_index(n, B, j)
    int c = j, s1 = j + 1, wP = 1, k = 0, cur = 0;
    while (true) {
      const int s2 = min(s1 + B - 1, m - 1), L = s2 - s1 + 1;
      const int t0 = s2 + 1;
      const int Lb = max(0, min(B, m - t0));
      z64* P = sPC[cur];
      z64* C = sPC[cur ^ 1];
      if (k == 0)
        for (int r = tid; r < L; r += SBR_THREADS) P[r] = AB[(size_t)c * W2 + (s1 + r - c)];
      for (int idx = tid; idx < L * L; idx += SBR_THREADS) {
        const int q = idx / L, r = idx % L;
        sD[q * LD + r] = r >= q ? AB[(size_t)(s1 + q) * W2 + (r - q)] : zconj(AB[(size_t)(s1 + r) * W2 + (q - r)]);
      }
      for (int idx = tid; idx < Lb * L; idx += SBR_THREADS) {
        const int q = idx / Lb, r = idx % Lb;
        C[q * LD + r] = AB[(size_t)(s1 + q) * W2 + (t0 + r - s1 - q)];
      }
      __syncthreads();
      if (warp == 0) {  // reflector from P's first column
        const z64 x = lane < L ? P[lane] : zmk(0.0, 0.0);
        const double s = wsum_d(lane >= 1 ? zabs2(x) : 0.0);
        const z64 alpha = zmk(__shfl_sync(0xffffffffu, x.x, 0), __shfl_sync(0xffffffffu, x.y, 0));
        Refl h;
        if (k > 0 && L == 1) {
          h.tau = zmk(0.0, 0.0);
          h.beta = 0.0;
          h.scale = zmk(0.0, 0.0);
        } else {
          h = make_refl(alpha, s);
        }
        const bool act = h.tau.x != 0.0 || h.tau.y != 0.0;
        if (lane < B) s_v[lane] = lane == 0 ? zmk(1.0, 0.0) : (act && lane < L ? zmul(x, h.scale) : zmk(0.0, 0.0));
        if (act && lane < L) P[lane] = lane == 0 ? zmk(h.beta, 0.0) : zmk(0.0, 0.0);
        if (lane == 0) s_tau = h.tau;
      }
      __syncthreads();
      const z64 tau = s_tau;
      const long long qi = qbase + k;
      if (tid < B) V2[(size_t)qi * B + tid] = s_v[tid];
      if (tid == 0) tau2[qi] = tau;
      if (tau.x != 0.0 || tau.y != 0.0) {
        // dot products: left w_q = v^H P(:, q) (q >= 1), p_r = (D v)_r, y_r = (C v)_r;
        // two threads per dot, halves combined by one shuffle
        const int nl = wP - 1;
        const int nitems = nl + L + Lb;
        {
          const int item = tid >> 1, half = tid & 1;
          z64 acc = zmk(0.0, 0.0);
          if (item < nitems) {
            if (item < nl) {
              const z64* col = P + (item + 1) * LD;
              for (int r = half; r < L; r += 2) acc = zcfma(s_v[r], col[r], acc);
            } else if (item < nl + L) {
              const int r = item - nl;
              for (int q = half; q < L; q += 2) acc = zfma(sD[q * LD + r], s_v[q], acc);
            } else {
              const int r = item - nl - L;
              for (int q = half; q < L; q += 2) acc = zfma(C[q * LD + r], s_v[q], acc);
            }
          }
          acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
          acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
          if (item < nitems && half == 0) {
            if (item < nl) s_w[item + 1] = zmul(zconj(tau), acc);         // conj(tau) v^H P(:, q)
            else if (item < nl + L) s_p[item - nl] = zmul(tau, acc);       // tau D v
            else s_y[item - nl - L] = zmul(tau, acc);                      // tau C v
          }
        }
        __syncthreads();
        if (warp == 0) {  // q = p - K v with K = conj(tau) (v^H p) / 2
          const z64 pv = lane < L ? s_p[lane] : zmk(0.0, 0.0);
          const z64 vv = lane < L ? s_v[lane] : zmk(0.0, 0.0);
          z64 t = zmk(0.0, 0.0);
          t = zcfma(vv, pv, t);
          t.x = wsum_d(t.x);
          t.y = wsum_d(t.y);
          const z64 K = zscale(zmul(zconj(tau), t), 0.5);
          if (lane < L) s_p[lane] = zfms(K, vv, pv);
        }
        __syncthreads();
        const int n1 = nl * L, n2 = n1 + L * L, n3 = n2 + Lb * L;
        for (int idx = tid; idx < n3; idx += SBR_THREADS) {
          if (idx < n1) {  // P(:, q) -= v (conj(tau) v^H P(:, q))
            const int q = 1 + idx / L, r = idx % L;
            P[q * LD + r] = zfms(s_v[r], s_w[q], P[q * LD + r]);
          } else if (idx < n2) {  // D -= q v^H + v q^H (lower triangle)
            const int i2 = idx - n1, q = i2 / L, r = i2 % L;
            if (r >= q) {
              z64 dv = sD[q * LD + r];
              dv = zfmsc(s_p[r], s_v[q], dv);
              dv = zfmsc(s_v[r], s_p[q], dv);
              sD[q * LD + r] = dv;
            }
          } else {  // C -= (tau C v) v^H
            const int i3 = idx - n2, q = i3 / Lb, r = i3 % Lb;
            C[q * LD + r] = zfmsc(s_y[r], s_v[q], C[q * LD + r]);
          }
        }
        __syncthreads();
      }
      // write back P and D's lower triangle; C stays as the next step's P
      for (int idx = tid; idx < wP * L; idx += SBR_THREADS) {
        const int q = idx / L, r = idx % L;
        AB[(size_t)(c + q) * W2 + (s1 + r - c - q)] = P[q * LD + r];
      }
      for (int idx = tid; idx < L * L; idx += SBR_THREADS) {
        const int q = idx / L, r = idx % L;
        if (r >= q) {
          z64 v = sD[q * LD + r];
          if (r == q) v.y = 0.0;
          AB[(size_t)(s1 + q) * W2 + (r - q)] = v;
        }
      }
      __syncthreads();
      if (Lb <= 0) break;
      c = s1;
      s1 = t0;
      wP = L;
      cur ^= 1;
      ++k;
    }
  }
  double* d = dbase + (size_t)p * sv;
  double* e = ebase + (size_t)p * sv;
  for (int i = tid; i < n; i += SBR_THREADS) {
    d[i] = i < m ? AB[(size_t)i * W2].x : 0.0;
    e[i] = i < m - 1 ? AB[(size_t)i * W2 + 1].x : 0.0;
  }
}

// ---------------------------------------------------------------- stage 2 back-transformation
// U(:, c) <- Q2 U(:, c) for c < ncols[p], rows < m.  One block per W columns of one problem,
// the columns held in shared memory as [m][W]; lane (cc, h) of a warp owns column cc and the
// reflector rows r = h (mod 32 / W).
template <int B, int W>
__global__ void __launch_bounds__(SBR_THREADS) q2_apply_kernel(int n, const int32_t* __restrict__ size,
                                                               const int32_t* __restrict__ ncols,
                                                               const z64* __restrict__ V2base,
                                                               const z64* __restrict__ tau2base, long long sq,
                                                               z64* __restrict__ Ubase, int ldu, long long sU) {
  constexpr int G = 32 / W;   // row groups per warp
  constexpr int RPL = B / G;  // reflector rows per lane (B >= G)
  constexpr int NW = SBR_THREADS / 32;
  extern __shared__ z64 Us[];
  const int p = blockIdx.y;
  const int m = size ? size[p] : n;
  const int nc = ncols ? ncols[p] : m;
  const int c0 = blockIdx.x * W;
  if (c0 >= nc) return;
  const z64* V2 = V2base + (size_t)p * sq * B;
  const z64* tau2 = tau2base + (size_t)p * sq;
  z64* U = Ubase + (size_t)p * sU;
  for (int idx = threadIdx.x; idx < m * W; idx += SBR_THREADS) {
    const int r = idx % m, cc = idx / m;
    Us[r * W + cc] = c0 + cc < nc ? U[(size_t)(c0 + cc) * ldu + r] : zmk(0.0, 0.0);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int cc = lane % W, h = lane / W;
  const long long fs_n = floor_sum(n - 2, B);
  for (int j = m - 2; j >= 0; --j) {
    const long long qbase = j + fs_n - floor_sum(n - 2 - j, B);
    const int nst = (m - 2 - j) / B + 1;
    for (int k = warp; k < nst; k += NW) {
      const long long qi = qbase + k;
      const z64 tau = tau2[qi];
      if (tau.x == 0.0 && tau.y == 0.0) continue;
      const int s1 = j + 1 + k * B;
      const int L = min(B, m - s1);
      const z64* v = V2 + (size_t)qi * B;
      z64 vr[RPL];
      z64 acc = zmk(0.0, 0.0);
#pragma unroll
      for (int i = 0; i < RPL; ++i) {
        const int r = h + G * i;
        vr[i] = r < L ? v[r] : zmk(0.0, 0.0);
        if (r < L) acc = zcfma(vr[i], Us[(s1 + r) * W + cc], acc);
      }
#pragma unroll
      for (int o = W; o < 32; o <<= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
      }
      const z64 t = zmul(tau, acc);
#pragma unroll
      for (int i = 0; i < RPL; ++i) {
        const int r = h + G * i;
        if (r < L) Us[(s1 + r) * W + cc] = zfms(vr[i], t, Us[(s1 + r) * W + cc]);
      }
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < m * W; idx += SBR_THREADS) {
    const int r = idx % m, cc2 = idx / m;
    if (c0 + cc2 < nc) U[(size_t)(c0 + cc2) * ldu + r] = Us[r * W + cc2];
  }
}

template <int B, int W>
cudaError_t q2_launch(int n, int nprob, const int32_t* size, const int32_t* ncols, const z64* V2, const z64* tau2,
                      long long sq, z64* U, int ldu, long long sU, cudaStream_t st) {
  const size_t smem = (size_t)n * W * sizeof(z64);
  cudaError_t e = cudaFuncSetAttribute(q2_apply_kernel<B, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((n + W - 1) / W, nprob);
  q2_apply_kernel<B, W><<<grid, SBR_THREADS, smem, st>>>(n, size, ncols, V2, tau2, sq, U, ldu, sU);
  return cudaGetLastError();
}

template <int B>
cudaError_t q2_dispatch(int n, int nprob, const int32_t* size, const int32_t* ncols, const z64* V2, const z64* tau2,
                        long long sq, z64* U, int ldu, long long sU, cudaStream_t st) {
  const size_t col = (size_t)n * sizeof(z64);  // shared-memory bytes per column
  constexpr size_t cap = 200 * 1024;
  if (16 * col <= cap) return q2_launch<B, 16>(n, nprob, size, ncols, V2, tau2, sq, U, ldu, sU, st);
  if (8 * col <= cap) return q2_launch<B, 8>(n, nprob, size, ncols, V2, tau2, sq, U, ldu, sU, st);
  if (4 * col <= cap) return q2_launch<B, 4>(n, nprob, size, ncols, V2, tau2, sq, U, ldu, sU, st);
  return q2_launch<B, 2>(n, nprob, size, ncols, V2, tau2, sq, U, ldu, sU, st);
}

}  // namespace

long long sbr_q2_count(int n, int B) {
  // sum over sweeps j = 0 .. n-2 of floor((n - 2 - j) / B) + 1
  return n < 2 ? 1 : (long long)(n - 1) + floor_sum(n - 2, B);
}

cudaError_t launch_sbr_qr(int B, int n, int nprob, const int32_t* size, z64* A, long long sA, int c0, z64* tauc,
                          z64* tau, long long stau, z64* VW, long long sVW, cudaStream_t st) {
  if (B == 32) he2hb_qr_kernel<32><<<nprob, SBR_THREADS, 0, st>>>(n, size, A, sA, c0, tauc, tau, stau, VW, sVW);
  else if (B == 16) he2hb_qr_kernel<16><<<nprob, SBR_THREADS, 0, st>>>(n, size, A, sA, c0, tauc, tau, stau, VW, sVW);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_sbr_band(int B, int n, int nprob, const int32_t* size, const z64* A, long long sA, z64* AB,
                            long long sAB, cudaStream_t st) {
  const size_t tot = (size_t)n * 2 * B;
  dim3 grid((unsigned)((tot + 255) / 256), nprob);
  if (B == 32) band_extract_kernel<32><<<grid, 256, 0, st>>>(n, size, A, sA, AB, sAB);
  else if (B == 16) band_extract_kernel<16><<<grid, 256, 0, st>>>(n, size, A, sA, AB, sAB);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_zero_outside(int n, int nprob, const int32_t* size, z64* A, long long sA, cudaStream_t st) {
  const size_t tot = (size_t)n * n;
  dim3 grid((unsigned)((tot + 255) / 256), nprob);
  zero_outside_kernel<<<grid, 256, 0, st>>>(n, size, A, sA);
  return cudaGetLastError();
}

template <int B>
cudaError_t chase_launch(int n, int nprob, const int32_t* size, z64* AB, long long sAB, double* d, double* e,
                         long long sv, z64* V2, z64* tau2, long long sq, cudaStream_t st) {
  const size_t smem = (size_t)(3 * B * (B + 1) + 4 * B + 1) * sizeof(z64);
  cudaError_t err = cudaFuncSetAttribute(hb2st_kernel<B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  hb2st_kernel<B><<<nprob, SBR_THREADS, smem, st>>>(n, size, AB, sAB, d, e, sv, V2, tau2, sq);
  return cudaGetLastError();
}

cudaError_t launch_sbr_chase(int B, int n, int nprob, const int32_t* size, z64* AB, long long sAB, double* d, double* e,
                             long long sv, z64* V2, z64* tau2, long long sq, cudaStream_t st) {
  if (B == 32) return chase_launch<32>(n, nprob, size, AB, sAB, d, e, sv, V2, tau2, sq, st);
  if (B == 16) return chase_launch<16>(n, nprob, size, AB, sAB, d, e, sv, V2, tau2, sq, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_sbr_q2(int B, int n, int nprob, const int32_t* size, const int32_t* ncols, const z64* V2,
                          const z64* tau2, long long sq, z64* U, int ldu, long long sU, cudaStream_t st) {
  if (B == 32) return q2_dispatch<32>(n, nprob, size, ncols, V2, tau2, sq, U, ldu, sU, st);
  if (B == 16) return q2_dispatch<16>(n, nprob, size, ncols, V2, tau2, sq, U, ldu, sU, st);
  return cudaErrorInvalidValue;
}
