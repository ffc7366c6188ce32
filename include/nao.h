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
                         contractions longer than 896 run as chunks summed in FP64.  With
                         this method the Householder matrix-vector products also run on
                         exact 8-bit digits (62 bits, int32 dot products on the integer
                         pipe) up to the order whose digits fit a block (n ~ 3200)        */
};

/* Library / context ------------------------------------------------------------------ */

/* Run-time settings of a context (nao_config_defaults fills the defaults).              */
typedef struct {
  double f_min;               /* occupation at or below which a band is left out of the
                                 density matrices and treated as empty (Part 6); default
                                 1e-16, range [0, 1e-3]                                      */
  int inverse_iteration_max;  /* inverse-iteration solves per eigenvector of the
                                 tridiagonal solve (Eigen_HH step 2) before it is declared
                                 not converged (status NAO_E_NOCONV, vector still written);
                                 default 5, range [0, 64]; 0 makes every vector fail         */
  long long tc_wait_cycles;   /* bound, in SM clock cycles, on each wait of a tensor-core
                                 product's copy/MMA pipeline; when it expires the product's
                                 block lets its copies land, skips its output, frees its
                                 tensor memory and raises the context's timeout flag
                                 (reported as NAO_E_TIMEOUT by the next status, below);
                                 default 4e9 (~2 s), range [1, 1e12]; below 1024 each wait
                                 is a single non-blocking test (to exercise that path)       */
  int mixed_planes;           /* BF16 digit planes per operand of the products that the
                                 mixed mode (NAO_MIXED_BF16X3) computes to reduced precision:
                                 5, 6 or 7 (30, 36 or 42 bits); default 6                    */
  int overlap_mrrr;           /* eigenvectors of the overlap's tridiagonal (Eigen_HH step 2
                                 of Part 2): 1 (default) from a relatively robust
                                 representation L D L^T of T - sigma I (dstegr's method, which
                                 the paper names) wherever an eigenvalue's relative gap is at
                                 least 1e-3, inverse iteration for the rest; 0: inverse
                                 iteration (dstevx's method) for all                         */
  int band_width;             /* Householder reduction of Eigen_HH step 1 (Sec. 3; the
                                 paper's conclusion calls for a change of this algorithm):
                                 0 (default) one stage, blocked Householder straight to
                                 tridiagonal form; 16 or 32: two stages, dense -> band of that
                                 lower bandwidth (panel QR and tensor-core updates), then
                                 band -> tridiagonal by bulge chasing, with a second
                                 back-transformation of the eigenvectors                      */
  int mrrr_all;               /* 1: eigenvectors of both tridiagonals (Eigen_HH step 2 of
                                 Parts 2 and 4) from the relatively robust representation of
                                 each unreduced block shifted below its smallest eigenvalue
                                 (dstegr's method) for every eigenvalue whose relative gap is
                                 at least 1e-5, inverse iteration for the rest; 0 (default):
                                 as overlap_mrrr says                                        */
  int split_hprime;           /* Parts 3-4 of an FP64 one-stage nao_gen_eig call as two halves
                                 of the problems on two streams of the context, the second
                                 starting once the first half's Part 3 products are done, so
                                 that its products run beside the first half's Householder
                                 panels; the results are ordered on the caller's stream as
                                 before.  0 (default): one pass; 1: split whenever there are
                                 at least 2 problems; 2: split from 32 problems on           */
} nao_config;

void nao_config_defaults(nao_config* cfg);

/* Create a context bound to CUDA device `device`.  *out receives the handle.
 *   hbm_budget_bytes  upper bound on the device memory the context itself holds (its
 *                     workspace arena); a call whose workspace would exceed it fails with
 *                     NAO_E_NOMEM before any launch.  0: no bound.  The serving scheduler
 *                     (below) admits requests within this budget unless nao_serve_config
 *                     sets another.
 *   cfg               settings, or NULL for the defaults.                                  */
int nao_init(nao_ctx** out, int device, size_t hbm_budget_bytes, const nao_config* cfg);
/* Read / replace the settings of a context (between calls; the new ones apply to work
 * enqueued afterwards).  NAO_E_INVALID for values outside the ranges above.                */
int nao_get_config(const nao_ctx* ctx, nao_config* cfg);
int nao_set_config(nao_ctx* ctx, const nao_config* cfg);
/* Release the context and its workspace (after all its work has completed).             */
void nao_destroy(nao_ctx* ctx);
/* Text of the last host-side error on this context ("" if none).  Valid until the next
 * call on the context.  ctx may be NULL (then: the last error of nao_init).              */
const char* nao_last_error(const nao_ctx* ctx);
/* Bytes of device workspace currently held by the context.                              */
size_t nao_workspace_bytes(const nao_ctx* ctx);

/* Select the product method of this context's band-step calls (default NAO_GEMM_TC).    */
int nao_set_gemm_method(nao_ctx* ctx, int method);

/* Refinement after a mixed-precision nao_gen_eig (no effect on NAO_FP64 calls):
 *   0 (default): eigenvalues = Rayleigh quotients c^H H c / c^H S c of the mixed-precision
 *      vectors, with FP64-accurate products of the input H and S: the eigenvalue error is
 *      second order in the vectors' (~1e-7 with 6 planes), so eigenvalues meet the mixed-mode
 *      bound; the vectors keep their mixed-precision accuracy;
 *   1 or 2: that many Ritz (Ogita-Aishima) sweeps first, each squaring the vector error
 *      (2: eigenvectors to FP64 accuracy), then the Rayleigh quotients;
 *   -1: none (raw mixed results, for measurements).
 * Returns NAO_E_INVALID for other values.                                                  */
int nao_set_refinement(nao_ctx* ctx, int sweeps);

/* Batched complex GEMM (the products of Parts 3, 4 and 6):
 *   C[p] = alpha op(A[p]) op(B[p]) + beta C[p],  p = 0..nprob-1, real alpha and beta.
 * Row-major storage: A[p] at A + p*strideA with leading dimension lda (elements); op(X) is
 * X (trans = 0), X^T (1) or X^H (2).  op(A) is M x K, op(B) is K x N, C[p] is M x N with
 * leading dimension ldc.  method: NAO_GEMM_FP64 or NAO_GEMM_TC.  Device arrays;
 * stream-ordered.                                                                         */
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
 *   MR    float64 [nmat][nR][n][n] real-space blocks (device); only i >= j enters the
 *         result (the tensor-core form reads all n^2 entries and discards the upper ones)
 *   kpts  float64 [nk][3] fractional k-points (device)
 *   Mk    complex128 [nmat][nk][n][n] output (device)
 * With NAO_GEMM_TC (the default) and nk >= 8 the sum is one FP64-accurate tensor-core
 * product per chunk of rows (phase matrix [cos; sin] times the element columns; the
 * context's workspace grows by up to 256 MB); otherwise FP64 FMAs.  A tensor-core wait that
 * expired (see nao_config.tc_wait_cycles) shows as NAO_E_TIMEOUT in the status of the
 * context's next nao_gen_eig or nao_density_matrix, which reports it once.                 */
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
 *             identity map (then nS = nprob).  Each distinct S is reduced once.  The
 *             entries must lie in [0, nS): they live on the device and are not checked
 *             (that would cost a device-to-host read per call); an entry outside the range
 *             makes the kernels read outside S and the workspace.
 *   nS        number of S matrices (ignored when s_of_prob is NULL)
 *   s_cut     absolute cutoff on the eigenvalues of S (e.g. 1e-10)
 *   precision NAO_FP64: every product FP64-accurate (ten-digit tensor-core products, or
 *             FP64 CUDA cores with NAO_GEMM_FP64); the one exception is the Newton-Schulz
 *             correction of the tridiagonal eigenvectors, a term ~1e-9 of them, formed with
 *             five digits (30 bits), far below the FP64 rounding of the vectors it corrects.
 *             NAO_MIXED_BF16X3: the back-transformations, X^H H X, the rank-2k updates of H'
 *             and X V use reduced-precision tensor-core products (nao_config.mixed_planes
 *             BF16 digit planes, 36 bits by default), and the Householder matrix-vector
 *             products of H' 46-bit integer digits; the reduction of S, the tridiagonal
 *             solves and s^{-1/2} stay FP64.  Then the refinement (not in the paper) restores
 *             the accuracy with FP64-accurate products of the input H and S: by default eps
 *             are the Rayleigh quotients of the mixed-precision vectors, sorted; with
 *             nao_set_refinement(1 or 2) Ritz (Ogita-Aishima) sweeps refine the vectors
 *             first.
 *             NAO_MIXED_TF32: rejected (NAO_E_INVALID): 12-bit products leave errors that
 *             one sweep does not remove.
 *   nb        eigenvector columns wanted, 1 <= nb <= n
 *   eps       float64 [nprob][n] out: ascending eigenvalues; entries j >= m are +inf
 *   C         complex128 [nprob][n][nb] out (may be NULL): column j is the eigenvector of
 *             eps[j], S-orthonormal (C^H S C = I); columns j >= m are zero
 *   m_kept    int32 [nprob] out: m, the number of kept overlap directions
 *   status    int32 [nprob] out: 0, NAO_E_NOCONV (a vector did not converge within the
 *             iteration bound nao_config.inverse_iteration_max; results still written),
 *             NAO_E_ALLCUT (m = 0) or NAO_E_TIMEOUT (a tensor-core wait of this call, or of
 *             an earlier call on the context not yet reported, expired: results invalid).
 * Workspace: grows on demand (NAO_E_NOMEM past the context's hbm_budget_bytes).             */
int nao_gen_eig(nao_ctx* ctx, int n, int nprob, const nao_c128* H, const nao_c128* S,
                const int32_t* s_of_prob, int nS, double s_cut, int precision, int nb,
                double* eps, nao_c128* C, int32_t* m_kept, int32_t* status, void* stream);

/* Parts 2-4 for problems of different basis sizes in one call (the same method as
 * nao_gen_eig): s_size int32 [nS] (device) gives the order n_s <= n of each overlap matrix,
 * and every problem takes the order of its S.  Each matrix of H and S is stored n x n with
 * its own n_s x n_s matrix in the leading block and zeros in the rest (the caller pads);
 * the results follow the same layout: eps[p][j] for j < m_p (m_p <= n_s) and +inf beyond,
 * rows n_s .. n-1 of C[p] zero.  s_size NULL is nao_gen_eig.  Orders outside [1, n] are the
 * caller's error (not checked: the array is device memory).                                */
int nao_gen_eig_sized(nao_ctx* ctx, int n, int nprob, const nao_c128* H, const nao_c128* S,
                      const int32_t* s_of_prob, int nS, const int32_t* s_size, double s_cut,
                      int precision, int nb, double* eps, nao_c128* C, int32_t* m_kept,
                      int32_t* status, void* stream);

/* Parts 5-6: chemical potential, occupations, band energy, density matrix ------------ *
 * Problem p = sigma * nk + q (spin-major), as produced by nao_gen_eig on H(k) from
 * nao_bloch_sum.  g = 2 when nspin = 1, else 1.  Fermi-Dirac occupations
 * f = 1 / (1 + exp((eps - mu)/kT)); mu solves g sum_p wk[q] sum_{j<m_p} f = n_electrons
 * (Sec. 3 Part 5); E_band = g sum_p wk[q] sum_j f eps.  Charge and energy density
 * matrices (Part 6):
 *   rhoR[sigma][r][i][j] = Re[ g sum_q wk[q] sum_{j'} f c_{i j'} conj(c_{j j'})
 *                              exp(-2 pi i kpts[q].R[r]) ],
 *   edmR: the same with weights f eps instead of f.
 * The k sum runs, like Part 1's, as FP64-accurate tensor-core products (cos Re P + sin Im P)
 * with NAO_GEMM_TC and nk >= 8, else with FP64 FMAs.
 *   eps, C, m_kept as written by nao_gen_eig (C [nprob][n][nb]); bands j >= nb must be
 *     unoccupied (f <= f_min), else status NAO_E_INVALID is written.
 *   mu_out, eband_out  float64 [1] out (device);  f_out float64 [nprob][n] out or NULL
 *   rhoR   float64 [nspin][nR][n][n] out (device)
 *   edmR   float64 [nspin][nR][n][n] out (device), or NULL to skip it
 *   status int32 [1] out (device): 0, NAO_E_RANGE, NAO_E_INVALID or NAO_E_TIMEOUT (a
 *          tensor-core wait expired, as in nao_gen_eig)
 * Bands with f <= nao_config.f_min are left out of rhoR and edmR.                          */
int nao_density_matrix(nao_ctx* ctx, int n, int nspin, int nk, const double* wk,
                       const double* kpts, const double* eps, const nao_c128* C, int nb,
                       const int32_t* m_kept, double n_electrons, double kT, int nR,
                       const int32_t* R, double* mu_out, double* eband_out, double* f_out,
                       double* rhoR, double* edmR, int32_t* status, void* stream);

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
 * and per-problem occupied-band counts, 288.5 KiB = 295,424 bytes) is a static array in the
 * library image, resident on every GPU that loads the library until the process exits.
 *   Limits: nspin * nk <= 65536 problems (else NAO_E_INVALID); runs on the current
 *   device, on `stream`; f_out float64 [nspin*nk][n] is required.
 *   Set-up: the first call on a device looks up the scratch array's device address
 *   (cudaGetSymbolAddress, once per device, with that device current); make that first
 *   call before any stream capture.  The address is kept for the life of the process: do
 *   not cudaDeviceReset a device between calls (the kept address would be stale).
 *   The band cut f_min is the default of nao_config (1e-16).
 *   Sharing: every call uses the same scratch and leaves its contents behind (the kernel
 *   resets what must start at zero).  Calls that overlap on the GPU (other streams, other
 *   host threads) race on it and must be serialised by the caller.
 *   Arguments and outputs as in nao_density_matrix; errors: NAO_E_INVALID, NAO_E_CUDA
 *   (text via nao_last_error(NULL)).                                                      */
int nao_fermi_level_noalloc(int n, int nspin, int nk, const double* wk, const double* eps,
                            const int32_t* m_kept, int nb, double n_electrons, double kT,
                            double* f_out, double* mu_out, double* eband_out, int32_t* status,
                            void* stream);

/* Workspace bytes that nao_gen_eig (precision as given) allocates in this context for n,
 * nprob problems and nS overlap matrices (nS = nprob without a map).  *bytes out.       */
int nao_gen_eig_workspace(nao_ctx* ctx, int n, int nprob, int nS, int precision, size_t* bytes);

/* ---- Serving: continuous batching of band steps (not in the paper) ------------------- *
 * A request is one band step (Parts 1-6) of its own cell: real-space H(R), S(R), images R,
 * its k-points and weights.  nao_serve_submit copies the inputs (host or device memory) and
 * returns at once with a ticket.  A scheduler thread inside the context:
 *   - groups queued requests of equal (n, precision, nb, s_cut), in arrival order, into one
 *     batch of at most max_batch_problems (spin, k) problems, solved by one nao_gen_eig;
 *   - runs each batch on a free slot (a stream with its own workspace), so batches of
 *     different sizes overlap on the GPU, and admits a batch only when its device bytes
 *     (inputs, outputs, workspace growth) fit in hbm_budget_bytes next to what running
 *     batches and unreleased results hold;
 *   - keeps each result on the device until nao_serve_release.
 * A request that alone exceeds the budget fails with NAO_E_NOMEM.                         */
typedef struct {
  int n, nspin, nk, nR;
  const double* HR;    /* float64 [nspin][nR][n][n] (host or device) */
  const double* SR;    /* float64 [nR][n][n] */
  const int32_t* R;    /* int32 [nR][3] integer image vectors */
  const double* kpts;  /* float64 [nk][3] fractional */
  const double* wk;    /* float64 [nk] weights */
  double n_electrons, kT, s_cut;
  int precision;       /* NAO_FP64 or NAO_MIXED_BF16X3 */
  int nb;              /* eigenvector columns per problem, 1..n; 0 means n */
  int want_rho;        /* 1: Parts 5-6 (mu, f, E_band, rho) as well */
} nao_request;

typedef struct {
  int status;          /* NAO_OK; NAO_E_BUSY: not finished within the poll's timeout;
                          otherwise the code the request failed with */
  int n, nprob, nb, nspin, nR;
  const double* eps;             /* device [nprob][n], as from nao_gen_eig */
  const nao_c128* C;             /* device [nprob][n][nb] */
  const int32_t* m_kept;         /* device [nprob] */
  const int32_t* prob_status;    /* device [nprob] */
  const double* mu;              /* device [1]; NULL unless want_rho (also eband, f, rho) */
  const double* eband;           /* device [1] */
  const double* f;               /* device [nprob][n] */
  const double* rho;             /* device [nspin][nR][n][n] */
  const int32_t* rho_status;     /* device [1] */
  double queue_ms;     /* submit -> its batch was launched (host clock) */
  double latency_ms;   /* submit -> its batch finished on the GPU */
  int batch_requests;  /* requests that shared its nao_gen_eig launch */
} nao_result;

/* Scheduler settings; call before the first submit (or when nothing is queued or running).
 * Defaults: the context's hbm_budget_bytes, or (when that is 0) 80 % of the free device
 * memory at the first submit; 256 problems; 2 slots.                                        */
int nao_serve_config(nao_ctx* ctx, size_t hbm_budget_bytes, int max_batch_problems, int slots);
/* Hold (on = 1) or resume (on = 0) admission: while held, requests queue but none starts;
 * running batches finish.  For draining a device or assembling a batch deliberately.     */
int nao_serve_pause(nao_ctx* ctx, int on);
/* Queue a request; *ticket receives its id.  NAO_E_INVALID for bad sizes or pointers.     */
int nao_serve_submit(nao_ctx* ctx, const nao_request* req, uint64_t* ticket);
/* Wait up to timeout_us (0: do not wait; < 0: no limit) for the request, then fill *out.
 * Returns out->status.  Device pointers stay valid until nao_serve_release.               */
int nao_serve_poll(nao_ctx* ctx, uint64_t ticket, int timeout_us, nao_result* out);
/* Free a finished request's device memory (NAO_E_BUSY while it is queued or running).    */
int nao_serve_release(nao_ctx* ctx, uint64_t ticket);
/* Device bytes held by the scheduler now and at most so far, requests queued / running.   */
int nao_serve_stats(nao_ctx* ctx, size_t* used_bytes, size_t* peak_bytes, int* queued, int* running);

#ifdef __cplusplus
}
#endif

#endif /* NAO_H */
