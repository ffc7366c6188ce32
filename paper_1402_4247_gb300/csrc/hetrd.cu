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
//  * two cluster barriers per column (release/acquire at cluster scope, so rows written by
//    another block in the previous column are visible to ordinary loads afterwards).
// Output: d[0..m), e[0..m-1) (e[m-1] = 0), tau[0..m) (tau[m-1] = 0), v_i in A(i+2:m, i).
#include <cooperative_groups.h>

#include "nao_internal.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int HT_THREADS = 1024;
constexpr int HT_MAXK = 8;  // threads per row pair

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


// first pair index of block k when npairs pairs are dealt to C blocks
__device__ __forceinline__ int pair_start(int k, int npairs, int C) { return (int)(((long long)k * npairs) / C); }

// One panel of NAO_HT_NB columns i0.. of the blocked reduction.  The rank-2 updates of the
// panel's columns are deferred: column i first receives the updates of the earlier panel
// columns (a), its reflector is formed (b), and the Hermitian product with the trailing
// matrix as it stood at the panel start is corrected by the panel's V and W columns:
//   p = A22 v - V (W^H v) - W (V^H v)   (c, d),   w = tau p - (tau/2)(p^H tau p ...) v (e).
// The caller applies A22 -= V W^H + W V^H to the rest of the matrix after the panel
// (a rank-2 NB update, run as one tensor-core product).  VW holds, per row, [V | W | V].
__global__ void __launch_bounds__(HT_THREADS)
hetrd_panel_kernel(int n, const int32_t* __restrict__ size, z64* __restrict__ Abase, int ld, long long strideA,
                   double* __restrict__ dbase, double* __restrict__ ebase, z64* __restrict__ taubase, long long strideV,
                   z64* __restrict__ VWbase, long long strideVW, int i0) {
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  constexpr int NB = NAO_HT_NB;
  constexpr int LDVW = 3 * NB;
  extern __shared__ z64 sm[];
  z64* v = sm;               // [n] reflector (trailing coordinates)
  z64* w = sm + n;           // [n] p, then w
  z64* pown = sm + 2 * n;    // [n] corrected p for this block's rows (read by the others)
  z64* part = sm + 3 * n;    // [2 * HT_THREADS] partial sums of the K threads of each pair
  __shared__ z64 ypart[2 * NB], yfull[2 * NB];
  __shared__ double red[64];
  __shared__ z64 s_tau, s_scale;
  __shared__ double s_beta;

  const int p = blockIdx.x / C;
  const int m = size ? size[p] : n;
  z64* A = Abase + (size_t)p * strideA;
  double* d = dbase + (size_t)p * strideV;
  double* e = ebase + (size_t)p * strideV;
  z64* tau = taubase + (size_t)p * strideV;
  z64* VW = VWbase + (size_t)p * strideVW;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  const int iend = min(i0 + NB, m);  // uniform over the cluster (one problem per cluster)

  for (int i = i0; i < iend; ++i) {
    const int j = i - i0;
    // (a) column i (rows i..m-1) receives the updates of panel columns 0..j-1
    if (j > 0) {
      for (int r = i + rank * nt + tid; r < m; r += C * nt) {
        z64 acc = A[(size_t)i * ld + r];
        const z64* Vr = VW + (size_t)r * LDVW;
        const z64* Vi = VW + (size_t)i * LDVW;
        for (int jj = 0; jj < j; ++jj) {
          acc = zsub(acc, zmul(Vr[jj], zconj(Vi[NB + jj])));  // V(r,jj) conj(W(i,jj))
          acc = zsub(acc, zmul(Vr[NB + jj], zconj(Vi[jj])));  // W(r,jj) conj(V(i,jj))
        }
        if (r == i) acc.y = 0.0;
        A[(size_t)i * ld + r] = acc;
      }
    }
    cluster.sync();  // S1: column i is final everywhere
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
    // (b) Procedures 1-2 (every block, redundantly): the reflector of x = A(i+1:m, i)
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
    for (int r = tid; r < mt; r += nt) v[r] = (r == 0) ? zmk(1.0, 0.0) : zmul(col[i + 1 + r], scale);
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
    if (active) {
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
      // partial y over this block's rows: warp-strided over the 2j entries
      for (int jj = wid; jj < 2 * j; jj += nw) {
        const int cidx = jj < j ? NB + jj : jj - j;  // W column jj, or V column jj - j
        double sre = 0.0, sim = 0.0;
        for (int g = g0 + lane; g < g1; g += 32) {
          const int ra = g, rb = mt - 1 - g;
          const z64 a = VW[(size_t)(i + 1 + ra) * LDVW + cidx];
          const z64 ca = zcfma(a, v[ra], zmk(0.0, 0.0));
          sre += ca.x;
          sim += ca.y;
          if (rb != ra) {
            const z64 b = VW[(size_t)(i + 1 + rb) * LDVW + cidx];
            const z64 cb = zcfma(b, v[rb], zmk(0.0, 0.0));
            sre += cb.x;
            sim += cb.y;
          }
        }
        sre = warp_sum(sre);
        sim = warp_sum(sim);
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
    cluster.sync();  // S2: partial results ready; every block is done reading column i
    if (rank == 0) {  // Procedure 3: keep v below the subdiagonal of column i, and in V
      z64* colw = A + (size_t)i * ld;
      for (int r = tid; r < mt; r += nt) {
        colw[i + 1 + r] = (r == 0) ? zmk(s_beta, 0.0) : v[r];
        z64* row = VW + (size_t)(i + 1 + r) * LDVW;
        row[j] = active ? v[r] : zmk(0.0, 0.0);
        row[2 * NB + j] = row[j];
      }
    }
    if (active) {
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
          const z64* row = VW + (size_t)(i + 1 + r) * LDVW;
          z64 acc = pown[r];
          for (int jj = 0; jj < j; ++jj) {
            acc = zsub(acc, zmul(row[jj], yfull[jj]));           // V(r,jj) (W^H v)_jj
            acc = zsub(acc, zmul(row[NB + jj], yfull[j + jj]));  // W(r,jj) (V^H v)_jj
          }
          pown[r] = acc;
        }
    }
    cluster.sync();  // S3: corrected pieces of p ready
    if (active) {
      // (e) Procedure 5: w = tau p - (tau/2) ((tau p)^H v) v on the full vector
      double dre = 0.0, dim = 0.0;
      for (int g = tid; g < npairs; g += nt) {
        int k = 0;
        while (k + 1 < C && pair_start(k + 1, npairs, C) <= g) ++k;
        const z64* src = cluster.map_shared_rank(pown, k);
        const int ra = g, rb = mt - 1 - g;
        const z64 pa = zmul(t, src[ra]);
        w[ra] = pa;
        const z64 c1 = zcfma(pa, v[ra], zmk(0.0, 0.0));
        dre += c1.x;
        dim += c1.y;
        if (rb != ra) {
          const z64 pb = zmul(t, src[rb]);
          w[rb] = pb;
          const z64 c2 = zcfma(pb, v[rb], zmk(0.0, 0.0));
          dre += c2.x;
          dim += c2.y;
        }
      }
      const double2 dot = block_sum2(dre, dim, red);
      const z64 alpha2 = zscale(zmul(t, zmk(dot.x, dot.y)), -0.5);
      for (int r = tid; r < mt; r += nt) w[r] = zfma(alpha2, v[r], w[r]);
      __syncthreads();
    }
    if (rank == 0)
      for (int r = tid; r < mt; r += nt) VW[(size_t)(i + 1 + r) * LDVW + NB + j] = active ? w[r] : zmk(0.0, 0.0);
    cluster.sync();  // S4: V and W column j visible to the whole cluster
  }
}

}  // namespace

// Largest cluster size C (1..8, at most one block per 128 rows) for which the nprob clusters
// of C blocks are all resident at once, as the occupancy calculator reports for this kernel.
int hetrd_cluster_size(int n, int nprob, int num_sms) {
  const size_t smem = sizeof(z64) * (3 * (size_t)n + 2 * HT_THREADS);
  if (cudaFuncSetAttribute(hetrd_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaFuncSetAttribute(hetrd_panel_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 0) != cudaSuccess) {
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
    if (cudaOccupancyMaxActiveClusters(&clusters, hetrd_panel_kernel, &cfg) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (clusters >= nprob) return c;
  }
  return 1;
}

cudaError_t launch_hetrd_panel(int n, int nprob, const int32_t* size, z64* A, int ld, long long strideA, double* d,
                               double* e, z64* tau, long long strideV, z64* VW, long long strideVW, int i0, int cluster,
                               cudaStream_t st) {
  size_t smem = sizeof(z64) * (3 * (size_t)n + 2 * HT_THREADS);
  cudaError_t err = cudaFuncSetAttribute(hetrd_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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
  return cudaLaunchKernelEx(&cfg, hetrd_panel_kernel, n, size, A, ld, strideA, d, e, tau, strideV, VW, strideVW, i0);
}
