// Part 5 (Sec. 3): chemical potential and band energy.  mu solves
//   N(mu) = g sum_p w_p sum_{j < m_p} f((eps_pj - mu)/kT) = N_e,  f(x) = 1/(1 + e^x),
// by bisection on [min eps - 40 kT, max eps + 40 kT] (N is strictly increasing for kT > 0),
// then f_pj and E_band = g sum w f eps.  All eigenvalues of all (k, spin) problems enter
// one sum, so the kernel runs on the whole GPU: each round every block sums its share of
// the Fermi factors, the partial sums meet after a grid-wide barrier, and every block
// applies the same (deterministic, fixed-order) total to its copy of the bracket.
#include <cooperative_groups.h>

#include <cfloat>

#include "nao_internal.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int FT = 256;

__device__ __forceinline__ double fermi_fn(double x) {
  if (x <= 0.0) return 1.0 / (1.0 + exp(x));
  const double ex = exp(-x);
  return ex / (1.0 + ex);
}

__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = 0.0;
  for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
  return t;
}

__device__ double block_minmax(double v, double* red, bool is_max) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double u = __shfl_xor_sync(0xffffffffu, v, o);
    v = is_max ? fmax(v, u) : fmin(v, u);
  }
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = red[0];
  for (int k = 1; k < (int)(blockDim.x >> 5); ++k) t = is_max ? fmax(t, red[k]) : fmin(t, red[k]);
  return t;
}

// Grid-wide sum in a fixed order; buf alternates so that a fast block never overwrites
// partials that a slow block is still reading.
__device__ double grid_sum(cg::grid_group& grid, double v, double* red, double* scratch, int& buf) {
  v = block_sum(v, red);
  double* part = scratch + (size_t)buf * gridDim.x;
  if (threadIdx.x == 0) part[blockIdx.x] = v;
  buf ^= 1;
  grid.sync();
  double t = 0.0;
  for (unsigned b = 0; b < gridDim.x; ++b) t += part[b];
  return t;
}

__global__ void __launch_bounds__(FT)
fermi_kernel(int n, int nprob, int nk, double g, const double* __restrict__ wk, const double* __restrict__ eps,
             const int32_t* __restrict__ m, int nb, double n_electrons, double kT, double f_min,
             double* __restrict__ f, int32_t* __restrict__ nocc, double* __restrict__ mu_out, double* __restrict__ eband_out,
             int32_t* __restrict__ status, double* __restrict__ scratch) {
  cg::grid_group grid = cg::this_grid();
  __shared__ double red[32];
  int buf = 0;
  const size_t total = (size_t)nprob * n;
  const size_t gtid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t gstride = (size_t)gridDim.x * blockDim.x;

  double lmin = DBL_MAX, lmax = -DBL_MAX, cap = 0.0;
  for (size_t idx = gtid; idx < total; idx += gstride) {
    const int p = (int)(idx / n), j = (int)(idx % n);
    if (j < m[p]) {
      const double e = eps[idx];
      lmin = fmin(lmin, e);
      lmax = fmax(lmax, e);
      cap += g * wk[p % nk];
    }
    if (j == 0) nocc[p] = 0;
  }
  // min and max through the sum machinery: two grid sums of +-large sentinels would lose
  // precision, so reduce them with dedicated partial slots
  lmin = block_minmax(lmin, red, false);
  lmax = block_minmax(lmax, red, true);
  double* mm = scratch + 2 * (size_t)gridDim.x;
  if (threadIdx.x == 0) {
    mm[2 * blockIdx.x] = lmin;
    mm[2 * blockIdx.x + 1] = lmax;
  }
  cap = grid_sum(grid, cap, red, scratch, buf);  // (contains a grid.sync)
  double emin = DBL_MAX, emax = -DBL_MAX;
  for (unsigned b = 0; b < gridDim.x; ++b) {
    emin = fmin(emin, mm[2 * b]);
    emax = fmax(emax, mm[2 * b + 1]);
  }
  int32_t st = 0;
  if (!(n_electrons >= 0.0 && n_electrons <= cap * (1.0 + 1e-14)) || !(emin <= emax)) st = NAO_E_RANGE;
  double lo = emin - 40.0 * kT, hi = emax + 40.0 * kT;
  if (st == 0) {
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (mid <= lo || mid >= hi || hi - lo <= 1e-15 * fmax(1.0, fabs(mid))) break;
      double s = 0.0;
      for (size_t idx = gtid; idx < total; idx += gstride) {
        const int p = (int)(idx / n), j = (int)(idx % n);
        if (j < m[p]) s += wk[p % nk] * fermi_fn((eps[idx] - mid) / kT);
      }
      s = g * grid_sum(grid, s, red, scratch, buf);
      if (s < n_electrons) lo = mid;
      else hi = mid;
    }
  }
  const double mu = 0.5 * (lo + hi);
  // occupations, band energy, occupied-band counts
  double eb = 0.0;
  for (size_t idx = gtid; idx < total; idx += gstride) {
    const int p = (int)(idx / n), j = (int)(idx % n);
    double fj = 0.0;
    if (st == 0 && j < m[p]) {
      fj = fermi_fn((eps[idx] - mu) / kT);
      eb += g * wk[p % nk] * fj * eps[idx];
      if (fj > f_min) atomicMax(&nocc[p], j + 1);
    }
    f[idx] = fj;
  }
  eb = grid_sum(grid, eb, red, scratch, buf);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *mu_out = (st == 0) ? mu : __longlong_as_double(0x7ff8000000000000ll);
    *eband_out = (st == 0) ? eb : __longlong_as_double(0x7ff8000000000000ll);
  }
  grid.sync();
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    // bands beyond the nb returned eigenvectors must be empty; the count is clamped so
    // that the density-matrix product never reads past column nb
    int32_t s2 = st;
    for (int p = 0; p < nprob; ++p)
      if (nocc[p] > nb) {
        if (s2 == 0) s2 = NAO_E_INVALID;
        nocc[p] = nb;
      }
    if (status) *status = s2;
  }
}

}  // namespace

size_t fermi_scratch_doubles(int num_sms) { return (size_t)4 * num_sms + 64; }

cudaError_t launch_fermi(int num_sms, int n, int nprob, int nk, double g, const double* wk, const double* eps,
                         const int32_t* m, int nb, double n_electrons, double kT, double f_min, double* f,
                         int32_t* nocc, double* mu, double* eband, int32_t* status, double* scratch, cudaStream_t st) {
  int per_sm = 0;
  cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fermi_kernel, FT, 0);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  int grid = num_sms;  // one block per SM is enough: ~nprob*n/(num_sms*FT) values per thread
  void* args[] = {&n,  &nprob, &nk,   &g,  &wk,    &eps,   &m,       &nb,     &n_electrons,
                  &kT, &f_min, &f,    &nocc, &mu,  &eband, &status, &scratch};
  return cudaLaunchCooperativeKernel((const void*)fermi_kernel, dim3(grid), dim3(FT), args, 0, st);
}

// ---------------------------------------------------------------------------------------
// Allocation-free variant of Part 5 (no counterpart in the paper).
//
// The entry point above takes its scratch (grid partial sums, per-problem occupied-band
// counts) from the context's workspace, which the library grows with cudaMalloc.  Some
// callers cannot allow that: host codes that hand the library a fixed device-memory pool
// and forbid allocations behind their back (DFT drivers in Fortran/MPI with their own
// allocators), and serving loops that must never synchronise the device in the middle
// of a step (cudaMalloc/cudaFree can synchronise).  For them nao_fermi_level_noalloc
// runs the same kernel on a scratch array that is part of the library image itself.
// ---------------------------------------------------------------------------------------

#include <mutex>

namespace {
constexpr int NOALLOC_MAX_BLOCKS = 1024;           // grid blocks whose partial sums fit
constexpr int NOALLOC_MAX_PROBLEMS = 65536;        // (spin, k) problems whose band counts fit
constexpr size_t NOALLOC_PART_DOUBLES = 4 * (size_t)NOALLOC_MAX_BLOCKS + 64;
constexpr size_t NOALLOC_DOUBLES = NOALLOC_PART_DOUBLES + NOALLOC_MAX_PROBLEMS / 2;  // + int32 counts
}  // namespace

// 288.5 KiB (295,424 bytes) of device memory, held by every GPU that loads the library until
// the process exits.
static __device__ __align__(256) double nao_fermi_scratch[NOALLOC_DOUBLES];

namespace {
std::mutex g_noalloc_mu;
constexpr int NOALLOC_MAX_DEVICES = 64;
void* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

// Device address of nao_fermi_scratch on the current device, looked up once per device and
// kept for the life of the process (a cudaDeviceReset of the device in between would leave
// it stale; the entry point's documentation excludes that).  In host code the symbol names
// a host-side shadow, not device memory.
cudaError_t noalloc_scratch(int dev, double** out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, nao_fermi_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = p;
  }
  *out = (double*)g_noalloc_ptr[dev];
  return cudaSuccess;
}
}  // namespace

extern "C" int nao_fermi_level_noalloc(int n, int nspin, int nk, const double* wk, const double* eps,
                                       const int32_t* m_kept, int nb, double n_electrons, double kT, double* f_out,
                                       double* mu_out, double* eband_out, int32_t* status, void* stream) {
  if (n < 1 || nk < 1 || (nspin != 1 && nspin != 2) || nb < 1 || nb > n)
    return nao_fail(nullptr, NAO_E_INVALID, "nao_fermi_level_noalloc: bad sizes");
  if ((long long)nspin * nk > NOALLOC_MAX_PROBLEMS)
    return nao_fail(nullptr, NAO_E_INVALID,
                    "nao_fermi_level_noalloc: %d problems exceed the fixed scratch limit of %d",
                    nspin * nk, NOALLOC_MAX_PROBLEMS);
  if (!wk || !eps || !m_kept || !f_out || !mu_out || !eband_out || !status)
    return nao_fail(nullptr, NAO_E_INVALID, "nao_fermi_level_noalloc: NULL array");
  if (!(kT > 0.0)) return nao_fail(nullptr, NAO_E_INVALID, "nao_fermi_level_noalloc: kT must be > 0");
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  double* scratch = nullptr;
  if (e == cudaSuccess) e = noalloc_scratch(dev, &scratch);
  if (e != cudaSuccess)
    return nao_fail(nullptr, NAO_E_CUDA, "nao_fermi_level_noalloc: %s", cudaGetErrorString(e));
  const int grid = sms < NOALLOC_MAX_BLOCKS ? sms : NOALLOC_MAX_BLOCKS;
  int32_t* nocc = (int32_t*)(scratch + NOALLOC_PART_DOUBLES);
  e = launch_fermi(grid, n, nspin * nk, nk, nspin == 1 ? 2.0 : 1.0, wk, eps, m_kept, nb, n_electrons, kT,
                   NAO_F_MIN_DEFAULT, f_out, nocc, mu_out, eband_out, status, scratch, (cudaStream_t)stream);
  if (e != cudaSuccess)
    return nao_fail(nullptr, NAO_E_CUDA, "nao_fermi_level_noalloc: launch failed: %s", cudaGetErrorString(e));
  return NAO_OK;
}
