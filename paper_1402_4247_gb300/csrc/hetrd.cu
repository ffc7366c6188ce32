// Eigen_HH step 1 (Sec. 3, Procedures 1-6): Householder reduction of a Hermitian matrix to
// real symmetric tridiagonal form, blocked by panels of NAO_HT_NB columns (the rank-2
// update of Procedure 6 is deferred within a panel and applied once per panel as a
// rank-2 NB product on the tensor cores by the caller).
//
// Column i: x = A(i+1:m, i) (Procedure 1); a reflector H_i = I - tau v v^H with v(0) = 1 and
// a REAL beta, H_i^H x = beta e_1, is formed from |x| (Procedure 2) and kept in place for the
// back-transformation (Procedure 3); p = tau A22 v (Procedure 4); w = p - (tau/2)(p^H v) v
// (Procedure 5); A22 <- A22 - v w^H - w v^H (Procedure 6).  Choosing beta real removes the
// separate phase pass: Q^H A Q = T with Q = H_0 H_1 ... H_{m-2}.
//
// GB300 layout of the work.  On this chip the FP64 pipe (1/64 of FP32) bounds the kernel,
// so the design minimises FP64 operations and spreads one matrix over several SMs:
//  * only the lower triangle is stored and updated (column-major, element (r, c) at
//    A[r + c*ld], r >= c): the Hermitian product reads row r's part left of the diagonal
//    and column r's part below it, so the rank-2 update costs 8 (m-i)^2 flops, not 16;
//  * a thread-block cluster of C blocks (C = 1..8) shares one matrix: rows are dealt out in
//    pairs (r, mt-1-r) so every pair costs the same in both the product and the update;
//  * each block computes p for its rows, the pieces meet through distributed shared memory,
//    and every block then forms the full w itself (identical, fixed-order arithmetic);
//  * each pair's work (its full Hermitian row: row part + column part, and its share of the
//    rank-2 update) is split over K threads so that ~1000 threads per block keep the FP64
//    pipe fed; the K partial sums meet in shared memory in a fixed order;
//  * four barriers per column: cluster barriers (release/acquire at cluster scope, so rows
//    written by another block in the previous column are visible to ordinary loads
//    afterwards) when C > 1, block barriers when one block holds the matrix.
// Output: d[0..m), e[0..m-1) (e[m-1] = 0), tau[0..m) (tau[m-1] = 0), v_i in A(i+2:m, i).
#include <cooperative_groups.h>

#include "nao_internal.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int HT_THREADS = 1024;
constexpr int HT_MAXK = 8;  // threads per row pair
constexpr int HT_FP64_WARPS = 8;  // digit path: warps doing the FP64 work beside the digit products

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of (a, b) over the first HT_RED_WARPS warps (the threads that hold data; the others pass
// nothing), returned to every thread of the block.  On this GPU an FP64 warp instruction
// holds the FP64 pipe for 16 cycles of the SM, so a reduction tree in all 32 warps of a block
// costs ~10 us per column; in four warps it costs a tenth of that.  red: >= 8 doubles.
constexpr int HT_RED_WARPS = 4;
__device__ __forceinline__ double2 red_sum2(double a, double b, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (wid < HT_RED_WARPS) {
    a = warp_sum(a);
    b = warp_sum(b);
    if (lane == 0) {
      red[wid] = a;
      red[HT_RED_WARPS + wid] = b;
    }
  }
  __syncthreads();
  double2 r = make_double2(0.0, 0.0);
#pragma unroll
  for (int k = 0; k < HT_RED_WARPS; ++k) {
    r.x += red[k];
    r.y += red[HT_RED_WARPS + k];
  }
  __syncthreads();  // red may be reused at once
  return r;
}



// ---------------------------------------------------------------------------------------
// Exact integer form of the panel's Hermitian matrix-vector product (used with the
// tensor-core product method).  On this GPU FP64 runs at 2 FMA/clk/SM while the integer
// 4-way dot product (DP4A) runs at 60/clk/SM (240 8-bit MACs), so the product
// p = A22 v, which dominates the reduction, is formed from 8-bit digits:
//  * once per panel, every row r of the Hermitian trailing matrix (both triangles) is scaled
//    by its own power of two 2^{e_r} (|a| < 2^{e_r}) and q = round(a 2^{62 - e_r}) written in
//    eight balanced base-256 digits d_0..d_7 in [-128, 127] (62 bits: FP64 accuracy with
//    margin for entries below their row maximum), real and imaginary parts separately;
//  * per column, v is split the same way with one scale 2^f;
//  * DP4A sums digit products of one order G = s + t exactly in int32 (|d d'| <= 2^14, two
//    products per pair, at most 8 pairs per order, K <= 4096: below 2^30): RR_G collects
//    Re a Re v + Im a (-Im v) (-Im v is split as its own
//    value, so no digit is negated), RI_G the cross terms, for G <= 7 (the orders beyond are
//    below 2^-68 of the row scale);
//  * p_r = 2^{e_r + f - 12} sum_G (RR_G + i RI_G) 2^{-8 G}, combined in integer arithmetic.
// Digit layout: dig[p][rr][w][16 words], rr = r - (i0 + 1), word w holds columns
// i0 + 1 + 4w .. +3 (4 int8 lanes) of plane s, part t at word index 2 s + t.
// The digit count S is a template parameter: S = 8 (62 bits, FP64 accuracy; the orders
// G <= 7 are kept) for every reduction of the FP64 mode and for the overlap, S = 6 (46 bits,
// orders G <= 5, truncation below 2^-43 of |row| |v|) for the H' reduction of the mixed mode,
// whose results the Ritz refinement corrects.  A digit row holds 2 S words per four columns.
constexpr int HD_S = 8;      // digits per value of the FP64 form
// words (4 columns) per digit row: rows and columns i0 + 1 .. n - 1
__host__ __device__ inline int hd_words(int n) { return n > 1 ? (n - 1 + 3) / 4 : 1; }

__device__ __forceinline__ int hd_exp(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7ff); }

// q = round(x 2^{8S - 2 - e}) for |x| < 2^e (integer arithmetic on the bits of x)
template <int S>
__device__ __forceinline__ long long hd_fixed(double x, int e) {
  const long long bits = __double_as_longlong(x);
  const int b = (int)((bits >> 52) & 0x7ff);
  if (b == 0) return 0;
  long long m = (bits & 0xFFFFFFFFFFFFFll) | 0x10000000000000ll;
  const int sh = b - 1075 + 8 * S - 2 - e;
  long long q;
  if (sh >= 0) q = m << sh;
  else if (sh <= -62) q = 0;
  else q = (m + (1ll << (-sh - 1))) >> (-sh);
  return bits < 0 ? -q : q;
}

// S balanced base-256 digits of q (|q| < 2^{8S-2}), most significant first, as unsigned bytes
template <int S>
__device__ __forceinline__ void hd_digits(long long q, unsigned int* d) {
#pragma unroll
  for (int s = S - 1; s >= 1; --s) {
    const int ds = (int)((q + 128) & 255) - 128;
    d[s] = (unsigned int)(ds & 255);
    q = (q - ds) >> 8;
  }
  d[0] = (unsigned int)((int)q & 255);
}

// digit words of 4 complex values x[0..3]: out[2 s + t] = plane s of part t (t = 0 re, 1 im);
// S / 2 uint4 per four columns
template <int S>
__device__ __forceinline__ void hd_pack4(const z64* x, int e, uint4* out4) {
  unsigned int w[2 * S];
#pragma unroll
  for (int k = 0; k < 2 * S; ++k) w[k] = 0u;
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    unsigned int dr[S], di[S];
    hd_digits<S>(hd_fixed<S>(x[l].x, e), dr);
    hd_digits<S>(hd_fixed<S>(x[l].y, e), di);
#pragma unroll
    for (int s = 0; s < S; ++s) {
      w[2 * s] |= dr[s] << (8 * l);
      w[2 * s + 1] |= di[s] << (8 * l);
    }
  }
#pragma unroll
  for (int k = 0; k < S / 2; ++k) out4[k] = make_uint4(w[4 * k], w[4 * k + 1], w[4 * k + 2], w[4 * k + 3]);
}

// digit words of 4 real values x[0..3]: out[t] = plane t
template <int S>
__device__ __forceinline__ void hd_pack4p(const double* x, int e, unsigned int* out) {
#pragma unroll
  for (int t = 0; t < S; ++t) out[t] = 0u;
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    unsigned int dg[S];
    hd_digits<S>(hd_fixed<S>(x[l], e), dg);
#pragma unroll
    for (int t = 0; t < S; ++t) out[t] |= dg[t] << (8 * l);
  }
}

// digit words of v's 4 values: out[3 t + k], k = 0: Re v, 1: Im v, 2: -Im v (plane t)
template <int S>
__device__ __forceinline__ void hd_pack4v(const z64* x, int e, unsigned int* out) {
#pragma unroll
  for (int k = 0; k < 3 * S; ++k) out[k] = 0u;
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    unsigned int dr[S], di[S], dn[S];
    hd_digits<S>(hd_fixed<S>(x[l].x, e), dr);
    hd_digits<S>(hd_fixed<S>(x[l].y, e), di);
    hd_digits<S>(hd_fixed<S>(-x[l].y, e), dn);
#pragma unroll
    for (int t = 0; t < S; ++t) {
      out[3 * t] |= dr[t] << (8 * l);
      out[3 * t + 1] |= di[t] << (8 * l);
      out[3 * t + 2] |= dn[t] << (8 * l);
    }
  }
}

// sum_{G < NG} R[G] 2^{-8 G} 2^ex as a double (NG <= 8), in integer arithmetic: the orders
// G < 4 and G >= 4 are combined exactly in two int64 words (|R[G]| < 2^31 gives |.| < 2^56
// each), which are then joined in one 63-bit integer, with a rounding of the low word far
// below the result's last bit, and converted with one rounding
template <int NG>
__device__ __forceinline__ double hd_combine(const int* R, int ex) {
  long long hi = 0, lo = 0;
#pragma unroll
  for (int G = 0; G < 4 && G < NG; ++G) hi += (long long)R[G] * (1ll << (8 * (3 - G)));
#pragma unroll
  for (int G = 4; G < NG; ++G) lo += (long long)R[G] * (1ll << (8 * (7 - G)));
  // value = (hi 2^32 + lo) 2^{ex - 56}; shift hi up by s <= 32 so that |hi 2^s| < 2^61
  const unsigned long long ah = hi < 0 ? 0ull - (unsigned long long)hi : (unsigned long long)hi;
  const int s = min(max(__clzll((long long)ah) - 3, 0), 32);
  long long t = (long long)((unsigned long long)hi << s);
  if (s == 32) t += lo;
  else t += (lo + (1ll << (31 - s))) >> (32 - s);
  return fix_to_double(t, ex - 56 - s + 32, false);
}

// element (r, c) of the Hermitian matrix stored as its lower triangle (column-major)
__device__ __forceinline__ z64 herm_at(const z64* A, int ld, int r, int c) {
  return c <= r ? A[(size_t)c * ld + r] : zconj(A[(size_t)r * ld + c]);
}

// Digits of the trailing matrix rows/columns i0+1 .. m-1 at the start of a panel.  One warp
// per row; lanes over words.  Lmax rows x W words per problem.
template <int S>
__global__ void __launch_bounds__(256)
hetrd_digits_kernel(int n, const int32_t* __restrict__ size, const z64* __restrict__ Abase, int ld,
                    long long strideA, int i0, int Lmax, int W, uint4* __restrict__ dig, int* __restrict__ erow) {
  const int p = blockIdx.y;
  const int lane = threadIdx.x & 31;
  const int rr = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int m = size ? size[p] : n;
  const int L = m - i0 - 1;
  if (rr >= Lmax || rr >= L || L <= 0) return;
  const z64* A = Abase + (size_t)p * strideA;
  const int r = i0 + 1 + rr;
  int bmax = 0;
  for (int c = lane; c < L; c += 32) {
    const z64 a = herm_at(A, ld, r, i0 + 1 + c);
    bmax = max(bmax, max(hd_exp(a.x), hd_exp(a.y)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) bmax = max(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
  const int e = bmax == 0 ? -1100 : bmax - 1022;
  if (lane == 0) erow[(size_t)p * Lmax + rr] = e;
  uint4* row = dig + ((size_t)p * Lmax + rr) * W * (S / 2);
  const int Wp = (L + 3) >> 2;
  for (int w = lane; w < Wp; w += 32) {
    z64 x[4];
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int c = 4 * w + l;
      x[l] = c < L ? herm_at(A, ld, r, i0 + 1 + c) : zmk(0.0, 0.0);
    }
    hd_pack4<S>(x, e, row + (size_t)w * (S / 2));
  }
}

// first pair index of block k when npairs pairs are dealt to C blocks
__device__ __forceinline__ int pair_start(int k, int npairs, int C) { return (int)(((long long)k * npairs) / C); }

// One panel of NAO_HT_NB columns i0.. of the blocked reduction.  The rank-2 updates of the
// panel's columns are deferred: column i first receives the updates of the earlier panel
// columns (a), its reflector is formed (b), and the Hermitian product with the trailing
// matrix as it stood at the panel start is corrected by the panel's V and W columns:
//   p = A22 v - V (W^H v) - W (V^H v)   (c, d),   w = tau p - (tau/2)(p^H tau p ...) v (e).
// The caller applies A22 -= V W^H + W V^H to the rest of the matrix after the panel
// (a rank-2 NB product on the tensor cores).  VW holds the panel's columns [V | W | V]
// column-major: VW(r, c) at VW[c n + r] (c < 3 NB), so that the FP64 warps, which walk
// rows, read them coalesced.
//
// Digit path: the 24 digit-product warps take groups of four rows dynamically (a counter in
// shared memory), eight lanes per row.  (Streaming the digit rows through per-warp rings of
// shared memory with asynchronous copies was measured slower: 96 vs 90 ms per step on the
// magnetite-shaped cell; the rows then pass the shared-memory pipe twice.)  With one block
// per matrix (C = 1) the barriers are block barriers; clusters use cluster barriers
// (release/acquire at cluster scope).
template <int S>
__global__ void __launch_bounds__(HT_THREADS)
hetrd_panel_kernel(int n, const int32_t* __restrict__ size, z64* __restrict__ Abase, int ld, long long strideA,
                   double* __restrict__ dbase, double* __restrict__ ebase, z64* __restrict__ taubase, long long strideV,
                   z64* __restrict__ VWbase, long long strideVW, int i0, const uint4* __restrict__ dig,
                   const int* __restrict__ erow, int Lmax, int W, z64* __restrict__ VWrbase) {
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  constexpr int NB = NAO_HT_NB;
  constexpr int QW = S / 2;  // uint4 per four columns of a digit row
  extern __shared__ z64 sm[];
  z64* v = sm;               // [n] reflector (trailing coordinates); first x itself
  z64* w = sm + n;           // [n] w; in the digit path first the corrections of p (one-block clusters)
  z64* pown = sm + 2 * n;    // [n] p for this block's rows (read by the others)
  z64* part = sm + 3 * n;    // FP64 path: [2 * HT_THREADS] partial sums of the K threads of each pair
  unsigned int* vd = (unsigned int*)(sm + 3 * n);  // digit path, same region: [3 S][W] digit words of v
  __shared__ int ired[32];
  __shared__ z64 ypart[2 * NB], yfull[2 * NB];
  __shared__ double red[64];
  __shared__ z64 s_tau, s_scale;
  __shared__ double s_beta;
  __shared__ int s_next;

  const int p = blockIdx.x / C;
  const int m = size ? size[p] : n;
  z64* A = Abase + (size_t)p * strideA;
  double* d = dbase + (size_t)p * strideV;
  double* e = ebase + (size_t)p * strideV;
  z64* tau = taubase + (size_t)p * strideV;
  z64* VW = VWbase + (size_t)p * strideVW;
#define VWAT(r, c) VW[(size_t)(c) * n + (r)]
  z64* VWr = VWrbase + (size_t)p * strideVW;  // row-major copy: VWr[r * 3 NB + c]
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  const int iend = min(i0 + NB, m);  // uniform over the cluster (one problem per cluster)
  // Digit path: warps [0, NWD) form the digit products while the last HT_FP64_WARPS warps
  // do the FP64 work that does not depend on them (W^H v and V^H v, the corrections when the
  // cluster is one block, and the next column's updates from panel columns 0..j-1), so the
  // integer and FP64 pipes work at the same time.
  const bool dp = dig != nullptr;
  const int NWD = dp ? nw - HT_FP64_WARPS : nw;
  auto csync = [&]() {
    if (C == 1) __syncthreads();
    else cluster.sync();
  };

  for (int i = i0; i < iend; ++i) {
    const int j = i - i0;
    // (a) column i (rows i..m-1) receives the updates of panel columns 0..j-1 (in the digit
    // path those of columns 0..j-2 were applied while column i-1 was reduced)
    if (j > 0) {
      const int jj0 = dp ? j - 1 : 0;
      for (int r = i + rank * nt + tid; r < m; r += C * nt) {
        z64 acc = A[(size_t)i * ld + r];
        for (int jj = jj0; jj < j; ++jj) {
          acc = zfmsc(VWAT(r, jj), VWAT(i, NB + jj), acc);  // - V(r,jj) conj(W(i,jj))
          acc = zfmsc(VWAT(r, NB + jj), VWAT(i, jj), acc);  // - W(r,jj) conj(V(i,jj))
        }
        if (r == i) acc.y = 0.0;
        A[(size_t)i * ld + r] = acc;
      }
    }
    csync();  // S1: column i is final everywhere
    if (i == m - 1) {  // last diagonal element, no reflector
      if (rank == 0 && tid == 0) {
        d[m - 1] = A[(size_t)(m - 1) * ld + (m - 1)].x;
        e[m - 1] = 0.0;
        tau[m - 1] = zmk(0.0, 0.0);
      }
      break;
    }
    const int mt = m - i - 1;
    const z64* col = A + (size_t)i * ld;
    // (b) Procedures 1-2 (every block, redundantly): x = A(i+1:m, i) read once into v, the
    // norm of x(1:) summed on the way; then the reflector, and v = x / (alpha - beta)
    double s = 0.0;
    if (tid < 32 * HT_RED_WARPS)
      for (int r = tid; r < mt; r += 32 * HT_RED_WARPS) {
        const z64 x = col[i + 1 + r];
        v[r] = x;
        if (r > 0) s += zabs2(x);
      }
    s = red_sum2(s, 0.0, red).x;  // (its barriers also publish v)
    if (tid == 0) {
      const z64 alpha = v[0];
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
      s_beta = beta;
      if (rank == 0) {
        d[i] = A[(size_t)i * ld + i].x;
        e[i] = beta;
        tau[i] = t;
      }
    }
    __syncthreads();
    const z64 t = s_tau;
    const z64 scale = s_scale;
    for (int r = tid; r < mt; r += nt) v[r] = (r == 0) ? zmk(1.0, 0.0) : zmul(v[r], scale);
    __syncthreads();
    const bool active = !(t.x == 0.0 && t.y == 0.0);  // H_i = I otherwise (uniform)

    // (c) Procedure 4 on the panel-start trailing matrix: p_raw = A22 v for this block's
    // row pairs, and the partial corrections y1 = W^H v, y2 = V^H v over the same rows
    const z64* A22 = A + (size_t)(i + 1) * ld + (i + 1);
    const int npairs = (mt + 1) >> 1;
    const int g0 = pair_start(rank, npairs, C), g1 = pair_start(rank + 1, npairs, C);
    const int P = g1 - g0;
    int K = P > 0 ? nt / P : 1;
    K = K < 1 ? 1 : (K > HT_MAXK ? HT_MAXK : K);
    if (active && dig) {
      // (c) with 8-bit digits and DP4A (see the note above hetrd_digits_kernel)
      int bm = 0;
      for (int c = tid; c < mt; c += nt) bm = max(bm, max(hd_exp(v[c].x), hd_exp(v[c].y)));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) bm = max(bm, __shfl_xor_sync(0xffffffffu, bm, o));
      if (lane == 0) ired[wid] = bm;
      __syncthreads();
      bm = 0;
      for (int k = 0; k < nw; ++k) bm = max(bm, ired[k]);
      const int f = bm == 0 ? -1100 : bm - 1022;
      const int kk0 = i - i0;  // column i + 1 relative to i0 + 1
      const int w0 = kk0 >> 2, Wp = (m - i0 - 1 + 3) >> 2;
      for (int idx = tid; idx < 3 * (Wp - w0); idx += nt) {  // one (word, part) per thread
        const int w = w0 + idx / 3, part = idx % 3;
        double x[4];
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          const int c = 4 * w + l - kk0;
          const z64 vc = (c >= 0 && c < mt) ? v[c] : zmk(0.0, 0.0);
          x[l] = part == 0 ? vc.x : (part == 1 ? vc.y : -vc.y);
        }
        unsigned int t[S];
        hd_pack4p<S>(x, f, t);
#pragma unroll
        for (int k = 0; k < S; ++k) vd[(3 * k + part) * W + w] = t[k];
      }
      if (tid == 0) s_next = 0;
      __syncthreads();
      // rows of this block's pairs, in groups of two taken dynamically: sixteen lanes per row
      const int nrows = 2 * P, rslot = lane >> 4, wl = lane & 15;
      const int ngroups = (nrows + 1) >> 1;
      while (wid < NWD) {
        int grp = 0;
        if (lane == 0) grp = atomicAdd(&s_next, 1);
        grp = __shfl_sync(0xffffffffu, grp, 0);
        if (grp >= ngroups) break;
        const int qq = grp * 2 + rslot;
        int r = -1;
        if (qq < nrows) {
          const int g = g0 + (qq >> 1);
          r = (qq & 1) ? mt - 1 - g : g;
          if ((qq & 1) && r == g) r = -1;
        }
        int RR[S], RI[S];
#pragma unroll
        for (int G = 0; G < S; ++G) RR[G] = RI[G] = 0;
        const int rr = r + kk0;  // digit row
        if (r >= 0) {
          const uint4* row = dig + ((size_t)p * Lmax + rr) * W * QW;
          for (int ww = w0 + wl; ww < Wp; ww += 16) {
            unsigned int a[2 * S];
            const uint4* aw = row + (size_t)ww * QW;
            // the lane's word two iterations on, into L2 (the row stream comes from DRAM)
            if (ww + 32 < Wp) asm volatile("prefetch.global.L2 [%0];" :: "l"(row + (size_t)(ww + 32) * QW));
#pragma unroll
            for (int q = 0; q < QW; ++q) {
              const uint4 q4 = __ldcs(aw + q);
              a[4 * q] = q4.x;
              a[4 * q + 1] = q4.y;
              a[4 * q + 2] = q4.z;
              a[4 * q + 3] = q4.w;
            }
#pragma unroll
            for (int t2 = 0; t2 < S; ++t2) {
              const int bre = (int)vd[(3 * t2) * W + ww], bim = (int)vd[(3 * t2 + 1) * W + ww],
                        bni = (int)vd[(3 * t2 + 2) * W + ww];
#pragma unroll
              for (int s2 = 0; s2 + t2 < S; ++s2) {
                const int G = s2 + t2;
                RR[G] = __dp4a((int)a[2 * s2], bre, RR[G]);      // Re a Re v
                RR[G] = __dp4a((int)a[2 * s2 + 1], bni, RR[G]);  // Im a (-Im v)
                RI[G] = __dp4a((int)a[2 * s2], bim, RI[G]);      // Re a Im v
                RI[G] = __dp4a((int)a[2 * s2 + 1], bre, RI[G]);  // Im a Re v
              }
            }
          }
        }
#pragma unroll
        for (int o = 1; o < 16; o <<= 1)
#pragma unroll
          for (int G = 0; G < S; ++G) {
            RR[G] += __shfl_xor_sync(0xffffffffu, RR[G], o);
            RI[G] += __shfl_xor_sync(0xffffffffu, RI[G], o);
          }
        if (r >= 0 && wl < 2) {  // lane 0 the real part, lane 1 the imaginary part
          // a = 2^{e_r - (8S-2)} q_a, v = 2^{f - (8S-2)} q_v, q_a q_v = sum_G R_G 2^{8(2S-2-G)}:
          // the product is 2^{e_r + f - 12} sum_G R_G 2^{-8G} for every S
          double* dst = (double*)&pown[r] + wl;
          *dst = hd_combine<S>(wl ? RI : RR, erow[(size_t)p * Lmax + rr] + f - 12);
        }
      }
    }
    if (active && !dig) {
      for (int tt = tid; tt < K * P; tt += nt) {
        const int k = tt / P, gl = tt - k * P, g = g0 + gl;
        const int c0 = (int)(((long long)k * mt) / K), c1 = (int)(((long long)(k + 1) * mt) / K);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int r = h ? mt - 1 - g : g;
          z64 acc = zmk(0.0, 0.0);
          if (!(h && r == g)) {
            const int ce = min(c1, r + 1);
            for (int c = c0; c < ce; ++c) acc = zfma(A22[(size_t)c * ld + r], v[c], acc);
            const z64* colr = A22 + (size_t)r * ld;
            for (int c = max(c0, r + 1); c < c1; ++c) acc = zcfma(colr[c], v[c], acc);
          }
          part[(size_t)k * 2 * P + 2 * gl + h] = acc;
        }
      }
    }
    if (active && !dp) {
      // partial y over this block's rows: warp-strided over the 2j entries
      for (int jj = wid; jj < 2 * j; jj += nw) {
        const int cidx = jj < j ? NB + jj : jj - j;  // W column jj, or V column jj - j
        z64 acc = zmk(0.0, 0.0);
        for (int g = g0 + lane; g < g1; g += 32) {
          const int ra = g, rb = mt - 1 - g;
          acc = zcfma(VWAT(i + 1 + ra, cidx), v[ra], acc);
          if (rb != ra) acc = zcfma(VWAT(i + 1 + rb, cidx), v[rb], acc);
        }
        const double sre = warp_sum(acc.x), sim = warp_sum(acc.y);
        if (lane == 0) ypart[jj] = zmk(sre, sim);
      }
      __syncthreads();
      for (int tt = tid; tt < 2 * P; tt += nt) {
        const int gl = tt >> 1, h = tt & 1, g = g0 + gl;
        const int r = h ? mt - 1 - g : g;
        if (h && r == g) continue;
        z64 acc = zmk(0.0, 0.0);
        for (int k = 0; k < K; ++k) acc = zadd(acc, part[(size_t)k * 2 * P + tt]);
        pown[r] = acc;
      }
    }
    if (dp && wid >= NWD) {
      // the FP64 warps, while the others form the digit products
      const int fw = wid - NWD, nfw = nw - NWD, ft = tid - NWD * 32, nft = nfw * 32;
      if (active) {
        // partial y over this block's rows: y1 = W^H v (entries 0..j-1), y2 = V^H v (j..2j-1)
        for (int jj = fw; jj < 2 * j; jj += nfw) {
          const int cidx = jj < j ? NB + jj : jj - j;
          z64 acc = zmk(0.0, 0.0);
          for (int g = g0 + lane; g < g1; g += 32) {
            const int ra = g, rb = mt - 1 - g;
            acc = zcfma(VWAT(i + 1 + ra, cidx), v[ra], acc);
            if (rb != ra) acc = zcfma(VWAT(i + 1 + rb, cidx), v[rb], acc);
          }
          const double sre = warp_sum(acc.x), sim = warp_sum(acc.y);
          if (lane == 0) ypart[jj] = zmk(sre, sim);
        }
        if (C == 1 && j > 0) {
          // one-block cluster: y is complete, so the corrections V y1 + W y2 of every row
          // are formed here too, into w (subtracted from p in (e))
          asm volatile("bar.sync 1, %0;" :: "r"(nft) : "memory");
          for (int r = ft; r < mt; r += nft) {
            z64 acc = zmk(0.0, 0.0);
            for (int jj = 0; jj < j; ++jj) {
              acc = zfma(VWAT(i + 1 + r, jj), ypart[jj], acc);           // V(r,jj) (W^H v)_jj
              acc = zfma(VWAT(i + 1 + r, NB + jj), ypart[j + jj], acc);  // W(r,jj) (V^H v)_jj
            }
            w[r] = acc;
          }
        }
      }
      // column i+1 (same panel) receives the updates of panel columns 0..j-1 now; the one of
      // column j follows in its (a)
      if (j > 0 && j + 1 < NB && i + 1 < iend) {
        const int i1 = i + 1;
        for (int r = i1 + rank * nft + ft; r < m; r += C * nft) {
          z64 acc = A[(size_t)i1 * ld + r];
          for (int jj = 0; jj < j; ++jj) {
            acc = zfmsc(VWAT(r, jj), VWAT(i1, NB + jj), acc);
            acc = zfmsc(VWAT(r, NB + jj), VWAT(i1, jj), acc);
          }
          A[(size_t)i1 * ld + r] = acc;
        }
      }
    }
    csync();  // S2: partial results ready; every block is done reading column i
    if (rank == 0) {  // Procedure 3: keep v below the subdiagonal of column i, and in V
      z64* colw = A + (size_t)i * ld;
      for (int r = tid; r < mt; r += nt) {
        colw[i + 1 + r] = (r == 0) ? zmk(s_beta, 0.0) : v[r];
        const z64 vr = active ? v[r] : zmk(0.0, 0.0);
        VWAT(i + 1 + r, j) = vr;
        VWAT(i + 1 + r, 2 * NB + j) = vr;
        VWr[(size_t)(i + 1 + r) * 3 * NB + j] = vr;
        VWr[(size_t)(i + 1 + r) * 3 * NB + 2 * NB + j] = vr;
      }
    }
    if (active && (!dp || C > 1)) {
      // (d) y = sum over the cluster's blocks (fixed order), then the corrections of this
      // block's rows: p_raw -= V y2 + W y1  (y1 = W^H v multiplies V, y2 = V^H v multiplies W)
      for (int jj = tid; jj < 2 * j; jj += nt) {
        z64 acc = zmk(0.0, 0.0);
        for (int k = 0; k < C; ++k) acc = zadd(acc, cluster.map_shared_rank(ypart, k)[jj]);
        yfull[jj] = acc;
      }
      __syncthreads();
      if (j > 0)
        for (int tt = tid; tt < 2 * P; tt += nt) {
          const int gl = tt >> 1, h = tt & 1, g = g0 + gl;
          const int r = h ? mt - 1 - g : g;
          if (h && r == g) continue;
          z64 acc = pown[r];
          for (int jj = 0; jj < j; ++jj) {
            acc = zfms(VWAT(i + 1 + r, jj), yfull[jj], acc);           // - V(r,jj) (W^H v)_jj
            acc = zfms(VWAT(i + 1 + r, NB + jj), yfull[j + jj], acc);  // - W(r,jj) (V^H v)_jj
          }
          pown[r] = acc;
        }
    }
    csync();  // S3: corrected pieces of p ready
    if (active) {
      // (e) Procedure 5: w = tau p - (tau/2) ((tau p)^H v) v on the full vector (in the digit
      // path with a one-block cluster, p = pown - w: the corrections formed beside (c))
      const bool dpc = dp && C == 1 && j > 0;
      z64 dacc = zmk(0.0, 0.0);
      for (int g = tid; tid < 32 * HT_RED_WARPS && g < npairs; g += 32 * HT_RED_WARPS) {
        int k = 0;
        while (k + 1 < C && pair_start(k + 1, npairs, C) <= g) ++k;
        const z64* src = C == 1 ? pown : cluster.map_shared_rank(pown, k);
        const int ra = g, rb = mt - 1 - g;
        const z64 pa = zmul(t, dpc ? zsub(src[ra], w[ra]) : src[ra]);
        w[ra] = pa;
        dacc = zcfma(pa, v[ra], dacc);
        if (rb != ra) {
          const z64 pb = zmul(t, dpc ? zsub(src[rb], w[rb]) : src[rb]);
          w[rb] = pb;
          dacc = zcfma(pb, v[rb], dacc);
        }
      }
      const double2 dot = red_sum2(dacc.x, dacc.y, red);  // (its barriers also publish w)
      const z64 alpha2 = zscale(zmul(t, zmk(dot.x, dot.y)), -0.5);
      for (int r = tid; r < mt; r += nt) {
        const z64 wr = zfma(alpha2, v[r], w[r]);
        w[r] = wr;
        if (rank == 0) {
          VWAT(i + 1 + r, NB + j) = wr;
          VWr[(size_t)(i + 1 + r) * 3 * NB + NB + j] = wr;
        }
      }
    } else if (rank == 0) {
      for (int r = tid; r < mt; r += nt) {
        VWAT(i + 1 + r, NB + j) = zmk(0.0, 0.0);
        VWr[(size_t)(i + 1 + r) * 3 * NB + NB + j] = zmk(0.0, 0.0);
      }
    }
    csync();  // S4: V and W column j visible to the whole cluster
  }
#undef VWAT
}
}  // namespace

// v, w, pown, then one region shared by the FP64 path's partial sums and the digit path's
// digit words of v (digits: 0 for the FP64 path, else the digit count S)
static size_t panel_smem(int n, int digits) {
  const size_t region = digits ? sizeof(unsigned int) * 3 * digits * hd_words(n) : sizeof(z64) * 2 * HT_THREADS;
  return sizeof(z64) * 3 * (size_t)n + region;
}

static int smem_optin() {
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return optin;
}

static const void* panel_fn(int digits) {
  return digits == 6 ? (const void*)hetrd_panel_kernel<6> : (const void*)hetrd_panel_kernel<HD_S>;
}

bool hetrd_digits_fit(int n, int digits) { return panel_smem(n, digits) <= (size_t)smem_optin(); }

// Largest cluster size C (1..8, at most one block per 128 rows) for which the nprob clusters
// of C blocks are all resident at once, as the occupancy calculator reports for this kernel.
int hetrd_cluster_size(int n, int nprob, int num_sms, int digits) {
  const size_t smem = panel_smem(n, digits);
  const void* fn = panel_fn(digits);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 0) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  const int cmax = max(1, min(8, n / 128));
  for (int c = cmax; c > 1; --c) {
    if ((long long)nprob * c > num_sms) continue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nprob * c));
    cfg.blockDim = dim3(HT_THREADS);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = c;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, fn, &cfg) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (clusters >= nprob) return c;
  }
  return 1;
}

cudaError_t launch_hetrd_panel(int n, int nprob, const int32_t* size, z64* A, int ld, long long strideA, double* d,
                               double* e, z64* tau, long long strideV, z64* VW, long long strideVW, int i0, int cluster,
                               const void* dig, const int* erow, int digits, z64* VWr, cudaStream_t st) {
  if (!dig) digits = 0;
  if (digits != 0 && digits != 6 && digits != HD_S) return cudaErrorInvalidValue;
  size_t smem = panel_smem(n, digits);
  cudaError_t err = cudaFuncSetAttribute(panel_fn(digits), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(nprob * cluster));
  cfg.blockDim = dim3(HT_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (digits == 6)
    return cudaLaunchKernelEx(&cfg, hetrd_panel_kernel<6>, n, size, A, ld, strideA, d, e, tau, strideV, VW, strideVW,
                              i0, (const uint4*)dig, erow, n > 1 ? n - 1 : 1, hd_words(n), VWr);
  return cudaLaunchKernelEx(&cfg, hetrd_panel_kernel<HD_S>, n, size, A, ld, strideA, d, e, tau, strideV, VW, strideVW,
                            i0, (const uint4*)dig, erow, n > 1 ? n - 1 : 1, hd_words(n), VWr);
}

size_t hetrd_digits_bytes(int n, int nprob, int digits) {
  const size_t L = n > 1 ? n - 1 : 1;
  return L * hd_words(n) * 8 * (size_t)digits * (size_t)nprob;
}

cudaError_t launch_hetrd_digits(int n, int nprob, const int32_t* size, const z64* A, int ld, long long strideA, int i0,
                                void* dig, int* erow, int digits, cudaStream_t st) {
  const int Lmax = n > 1 ? n - 1 : 1, L = n - i0 - 1;
  if (L <= 0) return cudaSuccess;
  dim3 grid((L + 7) / 8, nprob);
  if (digits == 6)
    hetrd_digits_kernel<6><<<grid, 256, 0, st>>>(n, size, A, ld, strideA, i0, Lmax, hd_words(n), (uint4*)dig, erow);
  else if (digits == HD_S)
    hetrd_digits_kernel<HD_S><<<grid, 256, 0, st>>>(n, size, A, ld, strideA, i0, Lmax, hd_words(n), (uint4*)dig, erow);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}
