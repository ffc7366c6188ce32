// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/nao.h"

typedef double2 z64;  // complex128 as (x = re, y = im)

// ---------------------------------------------------------------- complex helpers
__host__ __device__ __forceinline__ z64 zmk(double r, double i) { return make_double2(r, i); }
__host__ __device__ __forceinline__ z64 zadd(z64 a, z64 b) { return zmk(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ z64 zsub(z64 a, z64 b) { return zmk(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ z64 zmul(z64 a, z64 b) {
  return zmk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ z64 zconj(z64 a) { return zmk(a.x, -a.y); }
__host__ __device__ __forceinline__ z64 zscale(z64 a, double s) { return zmk(a.x * s, a.y * s); }
// acc + a*b
__host__ __device__ __forceinline__ z64 zfma(z64 a, z64 b, z64 acc) {
  return zmk(fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y)));
}
// acc + conj(a)*b
__host__ __device__ __forceinline__ z64 zcfma(z64 a, z64 b, z64 acc) {
  return zmk(fma(a.x, b.x, fma(a.y, b.y, acc.x)), fma(a.x, b.y, fma(-a.y, b.x, acc.y)));
}
// acc - a*b
__host__ __device__ __forceinline__ z64 zfms(z64 a, z64 b, z64 acc) {
  return zmk(fma(-a.x, b.x, fma(a.y, b.y, acc.x)), fma(-a.x, b.y, fma(-a.y, b.x, acc.y)));
}
// acc - a*conj(b)
__host__ __device__ __forceinline__ z64 zfmsc(z64 a, z64 b, z64 acc) {
  return zmk(fma(-a.x, b.x, fma(-a.y, b.y, acc.x)), fma(-a.y, b.x, fma(a.x, b.y, acc.y)));
}
__host__ __device__ __forceinline__ double zabs2(z64 a) { return a.x * a.x + a.y * a.y; }

// The double nearest to t 2^ex (ties to even), negated if neg, by integer operations (on
// this GPU the FP64 pipe, which the int64 -> double conversion and a scaling multiply
// would use, runs at 1/64 of the integer rate).  Results outside the normal range (not met by the
// operands of this method) take an FP64 ldexp (a subnormal result may then round twice).
__device__ __forceinline__ double fix_to_double(long long t, int ex, bool neg) {
  if (t == 0) return 0.0;
  const unsigned long long sgn = ((unsigned long long)t >> 63 ^ (neg ? 1ull : 0ull)) << 63;
  unsigned long long u = t < 0 ? 0ull - (unsigned long long)t : (unsigned long long)t;
  const int nlz = __clzll((long long)u);
  u <<= nlz;                                          // leading one at bit 63
  unsigned long long mant = u >> 11;                  // 53 bits
  const unsigned int rest = (unsigned int)u & 0x7ffu;  // the 11 bits below them
  if (rest > 0x400u || (rest == 0x400u && (mant & 1ull))) ++mant;
  const int e = 63 - nlz + ex;  // exponent of the leading one; a carry out of the rounding
  if (e >= -1022 && e <= 1022)  // moves it up by one, through the add into the exponent field
    return __longlong_as_double((long long)((((unsigned long long)(e + 1022) << 52) + mant) | sgn));
  const double r = ldexp((double)mant, e - 52);
  return sgn ? -r : r;
}

// ---------------------------------------------------------------- context
struct NaoStageStat {
  const char* name;
  double ms;
  long long calls, launches;
};
struct NaoPending {
  int stage;
  cudaEvent_t a, b;
};
struct nao_ctx {
  int device = 0;
  int num_sms = 0;
  void* ws = nullptr;       // device workspace arena
  size_t ws_bytes = 0;
  std::string last_error;
  long long launches = 0;   // kernels launched by this context
  bool profiling = false;
  std::vector<NaoStageStat> stages;
  std::vector<NaoPending> pending;
  std::vector<cudaEvent_t> event_pool;
  int gemm_method = NAO_GEMM_TC;
  int refine_sweeps = 0;     // mixed mode: -1 none, 0 Rayleigh quotients, 1-2 Ritz sweeps + quotients
  int* dev_flags = nullptr;  // NAO_FLAG_*: device words shared by the context's kernels
  size_t hbm_budget = 0;     // bound on the workspace arena (0: none)
  nao_config cfg{};          // run-time settings (nao_init / nao_set_config)
  struct NaoServer* server = nullptr;  // request scheduler (csrc/serve.cu), made on first use
  cudaStream_t aux_stream = nullptr;   // second stream of split Parts 3-4 (made on first use)
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
};

// Layout of nao_ctx::dev_flags (64 ints of device memory):
//   [NAO_FLAG_TIMEOUT]   set to 1 by a tensor-core product whose bounded wait expired;
//                        reported (and cleared) by the next nao_gen_eig / nao_density_matrix
//   [NAO_FLAG_WAIT .. +1] long long: the wait bound in SM cycles (nao_config.tc_wait_cycles),
//                        read by the tensor-core kernels at their start
constexpr int NAO_FLAG_TIMEOUT = 0;
constexpr int NAO_FLAG_WAIT = 2;
// Defaults of nao_config.
constexpr double NAO_F_MIN_DEFAULT = 1e-16;
constexpr int NAO_INV_ITER_DEFAULT = 5;
constexpr long long NAO_TC_WAIT_DEFAULT = 4000000000LL;  // ~2 s at 2 GHz
constexpr int NAO_MIXED_PLANES_DEFAULT = 6;
constexpr int NAO_OVERLAP_MRRR_DEFAULT = 1;
constexpr int NAO_BAND_WIDTH_DEFAULT = 0;  // one-stage tridiagonalization
constexpr int NAO_MRRR_ALL_DEFAULT = 0;    // MRRR vectors only for the overlap's big clusters
constexpr int NAO_SPLIT_HPRIME_DEFAULT = 0;  // one pass of Parts 3-4 (2: split from NAO_SPLIT_MIN_PROBLEMS on)
constexpr int NAO_SPLIT_MIN_PROBLEMS = 32;

// Workspace bytes nao_gen_eig / nao_density_matrix reserve on this context (before the
// arena's 1/8 headroom); the scheduler's admission test uses them.
size_t gen_eig_ws_bytes(const nao_ctx* ctx, int n, int nprob, int nSe);
size_t density_ws_bytes(const nao_ctx* ctx, int n, int nspin, int nk, int nR, int nb);
size_t bloch_ws_bytes(const nao_ctx* ctx, int n, int nR, int nmat, int nk);  // 0: no workspace
// Stops the scheduler thread of ctx (if any), waits for its batches, frees its memory.
void serve_shutdown(nao_ctx* ctx);

// Stage bracketing for tracing (no-ops unless profiling is on).
struct NaoStage {
  nao_ctx* ctx;
  cudaStream_t st;
  int idx = -1;
  cudaEvent_t a = nullptr;
  NaoStage(nao_ctx* c, const char* name, cudaStream_t s, int nlaunch);
  ~NaoStage();
  void add_launches(int k);  // kernels counted after the stage began
};

// Bump allocator over the context's workspace (256-byte aligned slices).
struct WsPlan {
  size_t off = 0;
  template <class T>
  size_t take(size_t count) {
    size_t o = (off + 255) & ~size_t(255);
    off = o + count * sizeof(T);
    return o;
  }
};

int nao_ws_reserve(nao_ctx* ctx, size_t bytes);  // grow workspace (synchronises the device)
int nao_fail(nao_ctx* ctx, int code, const char* fmt, ...);

#define NAO_CUDA_TRY(ctx, call)                                                             \
  do {                                                                                      \
    cudaError_t _e = (call);                                                                \
    if (_e != cudaSuccess)                                                                  \
      return nao_fail((ctx), NAO_E_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(_e), \
                      __FILE__, __LINE__);                                                  \
  } while (0)

// ---------------------------------------------------------------- launchers (host side)
// Each returns cudaSuccess or the launch error; all are stream-ordered.

// Part 1: Mk[a][q] = sum_r e^{2 pi i k_q.R_r} MR[a][r], lower triangle + mirror.
cudaError_t launch_bloch_sum(int n, int nR, const int32_t* R, int nmat, const double* MR, int nk,
                             const double* kpts, z64* Mk, cudaStream_t st);

// Build the full Hermitian matrix (column-major, ld) from a row-major lower triangle.
// src(p) = src + p*src_stride (row-major n x n), dst(p) = dst + p*dst_stride.
// If map != null, the source of problem p is map[p].
cudaError_t launch_herm_fill(int n, int nprob, const z64* src, long long src_stride, const int32_t* map,
                             z64* dst, int ld, long long dst_stride, cudaStream_t st);

// Eigen_HH step 1: Householder tridiagonalization, one block per problem, in place on the
// full Hermitian column-major matrix A (ld).  size[p] (or n when size == null) is the order.
// Only the lower triangle of A is read and updated.  `cluster` blocks (1..8, a thread-block
// cluster) share each matrix; hetrd_cluster_size picks it from the problem count.
// One launch reduces the panel of columns i0 .. i0+NAO_HT_NB-1; VW ([nprob][3 NB][n], the
// columns [V | W | V]) receives the panel's reflectors and update vectors, and the caller
// applies A(i0+NB:, i0+NB:) -= V W^H + W V^H before the next panel.
constexpr int NAO_HT_NB = 32;
// Digit counts of the panel's integer matrix-vector products: 8 (62 bits, FP64 accuracy) or
// 6 (46 bits: the H' reduction of the mixed mode); 0 selects the FP64 FMA path.
constexpr int NAO_HT_DIGITS_FP64 = 8;
constexpr int NAO_HT_DIGITS_MIXED = 6;
int hetrd_cluster_size(int n, int nprob, int num_sms, int digits);
bool hetrd_digits_fit(int n, int digits);  // the digit path's shared memory fits a block at order n
// dig / erow (nullable): 8-bit digit planes of the trailing matrix made by launch_hetrd_digits
// for this panel (with the same digit count); with them the panel forms its Hermitian
// matrix-vector products exactly with integer dot products (DP4A) instead of FP64 FMAs.
cudaError_t launch_hetrd_panel(int n, int nprob, const int32_t* size, z64* A, int ld, long long strideA, double* d,
                               double* e, z64* tau, long long strideV, z64* VW, long long strideVW, int i0, int cluster,
                               const void* dig, const int* erow, int digits, z64* VWr, cudaStream_t st);
// digit planes (row exponents: (n - 1) nprob ints)
size_t hetrd_digits_bytes(int n, int nprob, int digits);
cudaError_t launch_hetrd_digits(int n, int nprob, const int32_t* size, const z64* A, int ld, long long strideA, int i0,
                                void* dig, int* erow, int digits, cudaStream_t st);

// Two-stage form of Eigen_HH step 1 (csrc/sbr.cu), lower bandwidth B (16 or 32).
// Stage 1 panel QR of columns c0 .. c0+B-1 below row c0 + B (in place in the column-major A,
// ld n): tau of the panel into tauc[p][B] and tau[p stau + c0 + i], explicit reflectors into
// columns 0..B-1 and 2B..3B-1 of VW ([n][3B] row-major, rows c0+B .. n-1).
cudaError_t launch_sbr_qr(int B, int n, int nprob, const int32_t* size, z64* A, long long sA, int c0, z64* tauc,
                          z64* tau, long long stau, z64* VW, long long sVW, cudaStream_t st);
// Rows and columns >= size[p] of A set to zero.
cudaError_t launch_zero_outside(int n, int nprob, const int32_t* size, z64* A, long long sA, cudaStream_t st);
// The band of the reduced A into AB ([n][2B] per problem: element (r, c) at c 2B + r - c).
cudaError_t launch_sbr_band(int B, int n, int nprob, const int32_t* size, const z64* A, long long sA, z64* AB,
                            long long sAB, cudaStream_t st);
// Stage 2: band -> real tridiagonal (d, e) by bulge chasing; reflectors into V2 ([sq][B] per
// problem) and tau2 ([sq]), sq = sbr_q2_count(n, B).
long long sbr_q2_count(int n, int B);
cudaError_t launch_sbr_chase(int B, int n, int nprob, const int32_t* size, z64* AB, long long sAB, double* d, double* e,
                             long long sv, z64* V2, z64* tau2, long long sq, cudaStream_t st);
// U(:, c) <- Q2 U(:, c) for c < ncols[p] (column-major U, ld ldu).
cudaError_t launch_sbr_q2(int B, int n, int nprob, const int32_t* size, const int32_t* ncols, const z64* V2,
                          const z64* tau2, long long sq, z64* U, int ldu, long long sU, cudaStream_t st);

// Eigen_HH step 2: eigenvalues w (ascending) and orthonormal eigenvectors Z (column-major,
// ld) of tridiag(e, d, e) by bisection + inverse iteration.  scratch: see stein_scratch_doubles.
size_t stein_scratch_doubles(int n, int nprob);
// nvec (nullable: all) and nvec_max bound the eigenvectors computed per problem to the lowest
// min(nvec[p], nvec_max); the eigenvalues are always all computed.
// maxits: inverse-iteration solves per vector before NAO_E_NOCONV (nao_config).  mrrr: first
// compute vectors from a relatively robust representation L D L^T of T - sigma I (sigma just
// below each unreduced block's smallest eigenvalue) for the members of big tight clusters
// whose relative gap allows (1), or for every eigenvalue whose relative gap allows (2);
// inverse iteration takes the rest (and everything at 0).
cudaError_t launch_stein(int n, int nprob, const int32_t* size, const double* d, const double* e,
                         long long strideV, double* w, double* Z, int ld, long long strideZ,
                         double* scratch, int32_t* status, const int32_t* nvec, int nvec_max, int maxits,
                         int mrrr, cudaStream_t st, int* ns2 = nullptr);
// ns2 (nullable, [nprob]): set to 1 for a problem whose vectors need a second Newton-Schulz
// step (a gap in [1e-11, 1e-9) |T|_1, where inverse iteration leaves overlaps up to ~1e-5)

// Blocked (compact WY) back-transformation helpers, see backtr.cu.
constexpr int NAO_WY_NB = 128;
// off: row of reflector i's head is i + off (1: one-stage; B: stage 1 of the two-stage form)
cudaError_t launch_extract_v(int n, int nprob, const int32_t* size, const z64* A, int lda, long long strideA,
                             const z64* tau, long long strideV, int ncolv, z64* V, int ldv, long long strideVf,
                             z64* tauc, int off, cudaStream_t st);
// init_u: column c of U takes Z's column m - nc + c (the top nc) or, when lowest, column c.
cudaError_t launch_init_u(int n, int nprob, const int32_t* size, const int32_t* ncols, const double* Z, int ldz,
                          long long strideZ, z64* U, int ldu, long long strideU, int lowest, cudaStream_t st);
// T_j of every WY block j < nblk and problem p at once: G_j, T_j at (j nprob + p) nb^2.
cudaError_t launch_build_t(int nb, int nprob, int nblk, const z64* G, const z64* tauc, int ncolv, z64* T,
                           cudaStream_t st);
cudaError_t launch_normalize_cols(int n, int nprob, const int32_t* size, const int32_t* ncols, const double* w,
                                  long long strideV, int use_rsqrt, z64* U, int ldu, long long strideU,
                                  cudaStream_t st);

// Generic batched GEMM:  C(p) = alpha * opA(A(p)) * opB(B(p)) + beta * C(p)
// Element (i, j) of an operand X at X.ptr + p*X.bs + i*X.rs + j*X.cs; conj flags per operand.
// Dimensions: M, N, K fixed, or per problem from dim arrays when non-null.
struct GemmOperand {
  const void* ptr;
  long long bs, rs, cs;
  int conj;
  const int32_t* map;  // nullable: problem p reads batch entry map[p]
};
struct GemmDims {
  int M, N, K;                          // maxima (grid sizing) / fixed values
  const int32_t *Mp, *Np, *Kp;          // per-problem overrides (nullable)
  int lower = 0;                        // 1: only output tiles that meet the lower triangle
  int k0 = 0;                           // contraction chunk start: with Kp, problem p's length
                                        // is min(max(Kp[p] - k0, 0), K)
};
// per-problem contraction length of a (possibly chunked) product
__host__ __device__ inline int gemm_k(const GemmDims& d, int p) {
  if (!d.Kp) return d.K;
  const int k = d.Kp[p] - d.k0;
  return k < 0 ? 0 : (k > d.K ? d.K : k);
}
cudaError_t launch_zgemm(int nprob, GemmDims dims, z64 alpha, GemmOperand A, GemmOperand B, z64 beta,
                         z64* C, long long Cbs, long long Crs, long long Ccs, cudaStream_t st);
cudaError_t launch_dgemm(int nprob, GemmDims dims, double alpha, GemmOperand A, GemmOperand B, double beta,
                         double* C, long long Cbs, long long Crs, long long Ccs, cudaStream_t st);

// Newton-Schulz re-orthogonalisation, second half: Z2 = Z - Z E / 2 with E = G - I and G
// = Z^T Z given by its lower triangle (column-major, ld).  E is ~1e-9, so the product runs
// in FP32 on the FP32 pipe; its rounding (~1e-7 relative of a 1e-9 term) stays below FP64
// rounding of Z.
// E = G - I made full in place (upper triangle mirrored from the lower), order ncols[p] or n.
cudaError_t launch_sym_minus_identity(int n, int nprob, const int32_t* ncols, double* G, int ld, long long stride,
                                      cudaStream_t st);
cudaError_t launch_ns_correct(int n, int nprob, const int32_t* size, const int32_t* ncols, const double* Z,
                              const double* G, int ld, long long stride, double* Z2, cudaStream_t st);

// FP64-accurate complex GEMM on the BF16 tensor cores (digit-plane splitting): C = alpha
// op(A) op(B) + beta C with real alpha, beta.  Contractions longer than 896 (1792 real) run
// as chunks whose FP32 group sums stay exact, accumulated in FP64.  ws: zgemm_oz_workspace
// bytes; err: the context's dev_flags (err[NAO_FLAG_TIMEOUT] set to 1 if a bounded wait
// expired; the bound is the long long at err + NAO_FLAG_WAIT).  digits: base-64 planes per
// operand: NAO_OZ_DIGITS_FP64 (ten planes, 60 bits: FP64 accuracy, 55 tensor-core products),
// or 5, 6, 7 (30, 36, 42 bits: 15, 21, 28 products) for terms that tolerate less, or
// NAO_OZ_DIGITS_B128: nine base-128 planes (63 bits, 45 products in 17 MMAs per K step
// instead of 27-31), FP64 accuracy for short contractions (chunks of 256, 512 real).
constexpr int NAO_OZ_DIGITS_FP64 = 10;
constexpr int NAO_OZ_DIGITS_B128 = 9;
constexpr int NAO_OZ_DIGITS_NS = 5;   // the Newton-Schulz correction term (~1e-9 of Z)
// the mixed mode's products take nao_config.mixed_planes (5, 6 or 7) planes
bool zgemm_oz_supported(GemmDims dims);
size_t zgemm_oz_workspace(int nprob, GemmDims dims);
cudaError_t launch_zgemm_oz(int nprob, GemmDims dims, double alpha, GemmOperand A, GemmOperand B, double beta, z64* C,
                            long long Cbs, long long Crs, long long Ccs, void* ws, int* err, cudaStream_t st,
                            int digits = NAO_OZ_DIGITS_FP64);

// The same method for real float64 operands (C = alpha op(A) op(B) + beta C, K <= 1792);
// fits in the workspace of a complex product of the same M, N, K.
bool dgemm_oz_supported(GemmDims dims);
size_t dgemm_oz_workspace(int nprob, GemmDims dims);  // bytes of ws for launch_dgemm_oz
cudaError_t launch_dgemm_oz(int nprob, GemmDims dims, double alpha, GemmOperand A, GemmOperand B, double beta, double* C,
                            long long Cbs, long long Crs, long long Ccs, void* ws, int* err, cudaStream_t st,
                            int digits = NAO_OZ_DIGITS_FP64);

// Ritz refinement (csrc/refine.cu): Rayleigh quotients G_ii / R'_ii; I + F in place over G;
// Rayleigh quotients of the refined columns (W1 = S C, W2 = H C) with S-normalisation;
// ascending sort with permutation; gather of the first nb sorted columns into C [n][nb].
cudaError_t launch_oa_lambda(int n, int nprob, const int32_t* size, const z64* Rp, const z64* G, int ld,
                             long long stride, double* lam, long long lstride, cudaStream_t st);
cudaError_t launch_oa_f(int n, int nprob, const int32_t* size, const z64* Rp, z64* G, int ld, long long stride,
                        const double* lam, long long lstride, cudaStream_t st);
cudaError_t launch_oa_rq(int n, int nprob, const int32_t* size, z64* Cn, int ldc, long long cstride, const z64* W1,
                         const z64* W2, int ldw, long long wstride, double* lam, long long lstride, cudaStream_t st);
cudaError_t launch_oa_sort(int n, int nprob, const int32_t* size, const double* lam, long long lstride, double* eps,
                           int32_t* perm, cudaStream_t st);
cudaError_t launch_oa_gather(int n, int nprob, int nb, const int32_t* perm, const z64* Cn, int ldc, long long cstride,
                             z64* C, cudaStream_t st);

// Small helpers of the gen-eig chain.
// size (nullable): each problem's order (eigenvalues 0 .. size[p]-1 are counted)
cudaError_t launch_count_kept(int n, int nprob, const int32_t* size, const double* w, long long strideV, double s_cut,
                              int32_t* m, int32_t* status, cudaStream_t st);
cudaError_t launch_hermitize(int n, int nprob, const int32_t* size, z64* A, int ld, long long strideA,
                             cudaStream_t st);
cudaError_t launch_write_eps(int n, int nprob, const int32_t* m, const double* w, long long strideV,
                             double* eps, cudaStream_t st);
cudaError_t launch_zero_cols(int n, int nprob, int nb, const int32_t* m, z64* C, cudaStream_t st);

// Part 5: mu by bisection on the electron count, f, E_band, and per problem the number of
// occupied bands (f > f_min), in one cooperative grid-wide kernel.
cudaError_t launch_fermi(int num_sms, int n, int nprob, int nk, double g, const double* wk, const double* eps,
                         const int32_t* m, int nb, double n_electrons, double kT, double f_min, double* f,
                         int32_t* nocc, double* mu, double* eband, int32_t* status, double* scratch, cudaStream_t st);
// status[0] <- NAO_E_TIMEOUT if the context's timeout flag is set and status[0] is 0; the
// flag is cleared (it is reported once).  status may be NULL (then the flag is only cleared).
cudaError_t launch_report_timeout(int* flags, int32_t* status, int nstatus, cudaStream_t st);
size_t fermi_scratch_doubles(int num_sms);

// Part 6 helpers: Cs = C diag(sqrt f), Ce = Cs diag(eps) (occupied columns), and the inverse
// phase sum to rho(R).
cudaError_t launch_scale_cols_sqrt(int n, int nprob, int nb, const z64* C, const double* f, z64* Cs,
                                   cudaStream_t st);
cudaError_t launch_scale_cols_eps(int n, int nprob, int nb, const z64* Cs, const double* f, const double* eps, z64* Ce,
                                  cudaStream_t st);
cudaError_t launch_rho_phase_sum(int n, int nspin, int nk, int nR, const int32_t* R, const double* kpts,
                                 const double* wk, double g, const z64* P, double* rho, cudaStream_t st);
// The same two phase sums as FP64-accurate tensor-core GEMMs (digit planes), for k grids
// of at least NAO_PHASE_TC_MIN_NK points; ws holds *_ws_bytes; *nlaunch counts the kernels.
constexpr int NAO_PHASE_TC_MIN_NK = 8;
size_t bloch_tc_ws_bytes(int n, int nR, int nmat, int nk);
cudaError_t launch_bloch_sum_tc(int n, int nR, const int32_t* R, int nmat, const double* MR, int nk,
                                const double* kpts, z64* Mk, void* ws, int* err, cudaStream_t st, int* nlaunch);
size_t rho_phase_tc_ws_bytes(int n, int nspin, int nk, int nR);
cudaError_t launch_rho_phase_tc(int n, int nspin, int nk, int nR, const int32_t* R, const double* kpts,
                                const double* wk, double g, const z64* P, double* rho, void* ws, int* err,
                                cudaStream_t st, int* nlaunch);
