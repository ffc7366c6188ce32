/*
 * nao.h -- C ABI of the GB300 band-step library (numerical-atomic-orbital band DFT,
 * the Band_DFT_Col step of Parq, Sevre & Lee, arXiv:1402.4247, Sec. 3).
 *
 * One process, one GPU.  Every compute entry point is stream-ordered: it validates its
 * arguments on the host (returning NAO_E_INVALID before any launch), enqueues kernels on
 * `stream` (a cudaStream_t passed as void*; NULL = the legacy default stream) and returns
 * without synchronising.  Results are valid once the stream has reached that point.
 *
 * Memory: unless stated otherwise, every array argument is DEVICE memory owned by the
 * caller; the library never frees it.  The library owns an internal workspace (device
 * memory held by the context and grown on demand).  Complex numbers are interleaved
 * (re, im) float64 pairs.  Matrices are row-major, C-contiguous.  Only the lower triangle
 * (i >= j) of a Hermitian input is read.
 *
 * Errors: a negative NAO_E_* code is returned for host-detectable failures (invalid
 * arguments, allocation failure, CUDA launch errors) and nao_last_error() describes it.
 * Numerical failures found on the device are reported per problem in `status` arrays
 * (0 = ok) and never trap or hang the GPU: every device-side iteration is bounded.
 */
#ifndef NAO_H
#define NAO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nao_ctx nao_ctx;
typedef struct { double re, im; } nao_c128;

enum {
  NAO_OK = 0,
  NAO_E_INVALID = -1,  /* bad argument (host-side check)                                   */
  NAO_E_NOMEM = -2,    /* device workspace could not be allocated                            */
  NAO_E_NOCONV = -3,   /* an iterative step hit its iteration bound (per-problem status)     */
  NAO_E_TIMEOUT = -4,  /* a bounded wait expired                                             */
  NAO_E_CUDA = -5,     /* a CUDA runtime call failed                                         */
  NAO_E_ALLCUT = -6,   /* every overlap eigenvalue fell below s_cut (per-problem status)     */
  NAO_E_BUSY = -7,     /* resource temporarily unavailable                                   */
  NAO_E_RANGE = -8     /* electron count outside [0, number of states] (density matrix)      */
};

enum { NAO_FP64 = 0, NAO_MIXED_TF32 = 1, NAO_MIXED_BF16X3 = 2 };

/* How the FP64 matrix products of the band step are computed (both FP64-accurate). */
enum {
  NAO_GEMM_FP64 = 0,  /* FP64 FMA on the CUDA cores                                        */
  NAO_GEMM_TC = 1     /* BF16 tensor cores on exact 6-bit digit planes of the FP64 operands
                         (60-bit splitting, FP32-exact partial sums; FP64-level accuracy);
                         used where the contraction length allows (2K <= 1792), else FP64 */
};

/* Library / context ------------------------------------------------------------------ */

/* Create a context bound to CUDA device `device`.  *out receives the handle.             */
int nao_init(nao_ctx** out, int device);
/* Release the context and its workspace (after all its work has completed).             */
void nao_destroy(nao_ctx* ctx);
/* Text of the last host-side error on this context ("" if none).  Valid until the next
 * call on the context.  ctx may be NULL (then: the last error of nao_init).              */
const char* nao_last_error(const nao_ctx* ctx);
/* Bytes of device workspace currently held by the context.                              */
size_t nao_workspace_bytes(const nao_ctx* ctx);

/* Select the product method of this context's band-step calls (default NAO_GEMM_TC).    */
int nao_set_gemm_method(nao_ctx* ctx, int method);

/* Ritz refinement sweeps after a mixed-precision nao_gen_eig: 1 (default; eigenvalues to
 * the mixed-mode bound), 2 (eigenvectors to FP64 accuracy too) or 0 (none: raw mixed
 * results).  Returns NAO_E_INVALID for other values.  No effect on NAO_FP64 calls.        */
int nao_set_refinement(nao_ctx* ctx, int sweeps);

/* Batched complex GEMM (the products of Parts 3, 4 and 6):
 *   C[p] = alpha op(A[p]) op(B[p]) + beta C[p],  p = 0..nprob-1, real alpha and beta.
 * Row-major storage: A[p] at A + p*strideA with leading dimension lda (elements); op(X) is
 * X (trans = 0), X^T (1) or X^H (2).  op(A) is M x K, op(B) is K x N, C[p] is M x N with
 * leading dimension ldc.  method: NAO_GEMM_FP64 or NAO_GEMM_TC (NAO_E_INVALID if 2K > 1792
 * for NAO_GEMM_TC).  Device arrays; stream-ordered.                                       */
int nao_zgemm(nao_ctx* ctx, int method, int nprob, int M, int N, int K, double alpha,
              const nao_c128* A, int lda, long long strideA, int transA,
              const nao_c128* B, int ldb, long long strideB, int transB, double beta,
              nao_c128* C, int ldc, long long strideC, void* stream);

/* Part 1: k dependence (Sec. 3, Part 1) ---------------------------------------------- *
 * Mk[a][q][i][j] = sum_r exp(+2 pi i kpts[q].R[r]) MR[a][r][i][j]   for i >= j, and
 * Mk[a][q][j][i] = conj(Mk[a][q][i][j]), so every output matrix is exactly Hermitian
 * when MR[a][r][i][j] = MR[a][r'][j][i] for the image r' = -R[r] (caller's contract).
 *   n     basis size (>= 1);  nR images (>= 1);  nmat matrices (e.g. spin channels, >= 1)
 *   R     int32 [nR][3] integer cell vectors (device)
 *   MR    float64 [nmat][nR][n][n] real-space blocks (device); only i >= j is read
 *   kpts  float64 [nk][3] fractional k-points (device)
 *   Mk    complex128 [nmat][nk][n][n] output (device)                                    */
int nao_bloch_sum(nao_ctx* ctx, int n, int nR, const int32_t* R, int nmat, const double* MR,
                  int nk, const double* kpts, nao_c128* Mk, void* stream);

/* Parts 2-4: generalized Hermitian eigenproblem H C = S C eps (Sec. 3, Parts 2-4) ----- *
 * Solved the paper's way: Eigen_HH(S) -> s, U (Householder tridiagonalization, a
 * bisection + inverse-iteration tridiagonal solve, back-transformation and normalization);
 * X = U_m diag(s_m^{-1/2}) over the m eigenvalues s_j >= s_cut; H' = X^H H X;
 * Eigen_HH(H') -> eps, V; C = X V.
 *   n         basis size (>= 1); nprob problems (>= 1)
 *   H         complex128 [nprob][n][n] Hermitian (lower triangle read)
 *   S         complex128 [nS][n][n] Hermitian positive semi-definite (lower triangle read)
 *   s_of_prob int32 [nprob]: index of the S matrix of each problem, or NULL for the
 *             identity map (then nS = nprob).  Each distinct S is reduced once.
 *   nS        number of S matrices (ignored when s_of_prob is NULL)
 *   s_cut     absolute cutoff on the eigenvalues of S (e.g. 1e-10)
 *   precision NAO_FP64: every product FP64-accurate (ten-digit tensor-core products, or
 *             FP64 CUDA cores with NAO_GEMM_FP64).
 *             NAO_MIXED_BF16X3: the back-transformations, X^H H X, the rank-2k updates of H'
 *             and X V use 30-bit tensor-core products (five BF16 digit planes); the reduction
 *             of S, the tridiagonal solves and s^{-1/2} stay FP64.  Then one Ritz refinement
 *             sweep (Ogita-Aishima in the S inner product, FP64-accurate products of the
 *             input H and S; not in the paper) restores the accuracy: eps are the Rayleigh
 *             quotients of the refined vectors, sorted.  nao_set_refinement chooses 0-2
 *             sweeps (default 1).
 *             NAO_MIXED_TF32: rejected (NAO_E_INVALID): 12-bit products leave errors that
 *             one sweep does not remove.
 *   nb        eigenvector columns wanted, 1 <= nb <= n
 *   eps       float64 [nprob][n] out: ascending eigenvalues; entries j >= m are +inf
 *   C         complex128 [nprob][n][nb] out (may be NULL): column j is the eigenvector of
 *             eps[j], S-orthonormal (C^H S C = I); columns j >= m are zero
 *   m_kept    int32 [nprob] out: m, the number of kept overlap directions
 *   status    int32 [nprob] out: 0, NAO_E_NOCONV (a vector did not converge within the
 *             iteration bound; results still written) or NAO_E_ALLCUT (m = 0)          */
int nao_gen_eig(nao_ctx* ctx, int n, int nprob, const nao_c128* H, const nao_c128* S,
                const int32_t* s_of_prob, int nS, double s_cut, int precision, int nb,
                double* eps, nao_c128* C, int32_t* m_kept, int32_t* status, void* stream);

/* Parts 5-6: chemical potential, occupations, band energy, density matrix ------------ *
 * Problem p = sigma * nk + q (spin-major), as produced by nao_gen_eig on H(k) from
 * nao_bloch_sum.  g = 2 when nspin = 1, else 1.  Fermi-Dirac occupations
 * f = 1 / (1 + exp((eps - mu)/kT)); mu solves g sum_p wk[q] sum_{j<m_p} f = n_electrons
 * (Sec. 3 Part 5); E_band = g sum_p wk[q] sum_j f eps.  Density matrix (Part 6):
 *   rhoR[sigma][r][i][j] = Re[ g sum_q wk[q] sum_{j'} f c_{i j'} conj(c_{j j'})
 *                              exp(-2 pi i kpts[q].R[r]) ].
 *   eps, C, m_kept as written by nao_gen_eig (C [nprob][n][nb]); bands j >= nb must be
 *     unoccupied (f <= 1e-16), else status NAO_E_INVALID is written.
 *   mu_out, eband_out  float64 [1] out (device);  f_out float64 [nprob][n] out or NULL
 *   rhoR   float64 [nspin][nR][n][n] out (device)
 *   status int32 [1] out (device): 0, NAO_E_RANGE or NAO_E_INVALID                    */
int nao_density_matrix(nao_ctx* ctx, int n, int nspin, int nk, const double* wk,
                       const double* kpts, const double* eps, const nao_c128* C, int nb,
                       const int32_t* m_kept, double n_electrons, double kT, int nR,
                       const int32_t* R, double* mu_out, double* eband_out, double* f_out,
                       double* rhoR, int32_t* status, void* stream);

/* Tracing ------------------------------------------------------------------------------ *
 * With profiling on, every stage of the calls above is bracketed by CUDA events recorded
 * on the call's stream (no extra synchronisation while work is queued).  Stages: e.g.
 * "bloch_sum", "hetrd", "stein", "ortho_ns", "backtransform", "zgemm_HX", ... .
 * nao_profile_enable(ctx, 1) clears the counters and starts recording; (ctx, 0) stops.   */
int nao_profile_enable(nao_ctx* ctx, int on);
/* Waits for the recorded events, then fills up to `max` entries: names[i] (static
 * strings), total milliseconds, number of stage executions and of kernel launches.
 * Returns the number of stages recorded (may exceed max), or a negative error.          */
int nao_profile_read(nao_ctx* ctx, int max, const char** names, double* ms, int64_t* calls,
                     int64_t* launches);
/* Kernels this context has launched since nao_init (always counted).                    */
int64_t nao_launch_count(const nao_ctx* ctx);

/* Part 5 without allocation (no counterpart in the paper) ----------------------------- *
 * Same result as the mu / f / E_band part of nao_density_matrix, for callers that must not
 * let the library allocate device memory: codes that give the library a fixed memory pool
 * and forbid allocations behind their back, and loops that cannot afford the device
 * synchronisation a cudaMalloc/cudaFree may cause.  It takes no context and never calls
 * cudaMalloc, cudaFree or an allocating library routine: its scratch (grid partial sums
 * and per-problem occupied-band counts, 296 KiB) is a static array in the library image,
 * resident on every GPU that loads the library until the process exits.
 *   Limits: nspin * nk <= 65536 problems (else NAO_E_INVALID); runs on the current
 *   device, on `stream`; f_out float64 [nspin*nk][n] is required.
 *   Set-up: the first call on a device looks up the scratch array's device address
 *   (cudaGetSymbolAddress, once per device, with that device current); make that first
 *   call before any stream capture.
 *   Sharing: every call uses the same scratch and leaves its contents behind (the kernel
 *   resets what must start at zero).  Calls that overlap on the GPU (other streams, other
 *   host threads) race on it and must be serialised by the caller.
 *   Arguments and outputs as in nao_density_matrix; errors: NAO_E_INVALID, NAO_E_CUDA
 *   (text via nao_last_error(NULL)).                                                      */
int nao_fermi_level_noalloc(int n, int nspin, int nk, const double* wk, const double* eps,
                            const int32_t* m_kept, int nb, double n_electrons, double kT,
                            double* f_out, double* mu_out, double* eband_out, int32_t* status,
                            void* stream);

#ifdef __cplusplus
}
#endif

#endif /* NAO_H */
