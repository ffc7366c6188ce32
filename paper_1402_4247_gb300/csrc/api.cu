// C ABI of the band-step library: argument checks, workspace layout and the stream-ordered
// launch sequence of Band_DFT_Col (Sec. 3, Parts 1-6).
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "nao_internal.cuh"

static std::string g_init_error;

int nao_fail(nao_ctx* ctx, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (ctx) ctx->last_error = buf;
  else g_init_error = buf;
  return code;
}

int nao_ws_reserve(nao_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->ws_bytes) return NAO_OK;
  if (ctx->hbm_budget && bytes > ctx->hbm_budget)
    return nao_fail(ctx, NAO_E_NOMEM, "workspace of %zu bytes exceeds the context's HBM budget of %zu bytes", bytes,
                    ctx->hbm_budget);
  // Growing the arena frees the old one: wait for work that may still use it.
  NAO_CUDA_TRY(ctx, cudaDeviceSynchronize());
  if (ctx->ws) {
    cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
  }
  size_t want = bytes + bytes / 8;
  if (ctx->hbm_budget && want > ctx->hbm_budget) want = ctx->hbm_budget;
  cudaError_t e = cudaMalloc(&ctx->ws, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ctx->ws = nullptr;
    return nao_fail(ctx, NAO_E_NOMEM, "workspace allocation of %zu bytes failed: %s", want, cudaGetErrorString(e));
  }
  ctx->ws_bytes = want;
  return NAO_OK;
}

static cudaEvent_t take_event(nao_ctx* c) {
  if (!c->event_pool.empty()) {
    cudaEvent_t e = c->event_pool.back();
    c->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

static void drain_pending(nao_ctx* c) {
  for (auto& p : c->pending) {
    float ms = 0.f;
    cudaEventSynchronize(p.b);
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) c->stages[p.stage].ms += ms;
    c->event_pool.push_back(p.a);
    c->event_pool.push_back(p.b);
  }
  c->pending.clear();
}

NaoStage::NaoStage(nao_ctx* c, const char* name, cudaStream_t s, int nlaunch) : ctx(c), st(s) {
  c->launches += nlaunch;
  if (!c->profiling) return;
  for (size_t i = 0; i < c->stages.size(); ++i)
    if (strcmp(c->stages[i].name, name) == 0) idx = (int)i;
  if (idx < 0) {
    c->stages.push_back(NaoStageStat{name, 0.0, 0, 0});
    idx = (int)c->stages.size() - 1;
  }
  c->stages[idx].calls += 1;
  c->stages[idx].launches += nlaunch;
  if (c->pending.size() > 8192) drain_pending(c);
  a = take_event(c);
  cudaEventRecord(a, s);
}

void NaoStage::add_launches(int k) {
  ctx->launches += k;
  if (idx >= 0) ctx->stages[idx].launches += k;
}

NaoStage::~NaoStage() {
  if (idx < 0 || !a) return;
  cudaEvent_t b = take_event(ctx);
  cudaEventRecord(b, st);
  ctx->pending.push_back(NaoPending{idx, a, b});
}

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

inline cudaStream_t as_stream(void* s) { return (cudaStream_t)s; }

// Run one launcher inside a traced stage.
#define NAO_STAGE(name, nl, call)              \
  do {                                         \
    NaoStage stage_(ctx, name, st, nl);        \
    NAO_CUDA_TRY(ctx, call);                   \
  } while (0)

// tiny gather: m of each problem from its S, the number of C columns, and the status
__global__ void gather_m_kernel(int nprob, const int32_t* map, const int32_t* mS, const int32_t* statS, int nb,
                                int32_t* mP, int32_t* nbP, int32_t* statP) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nprob) return;
  const int s = map ? map[p] : p;
  const int m = mS[s];
  mP[p] = m;
  nbP[p] = m < nb ? m : nb;
  statP[p] = statS[s];
}

__global__ void finish_status_kernel(int nprob, const int32_t* mP, const int32_t* statP, const int32_t* statH,
                                     const int* flags, int32_t* m_kept, int32_t* status) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nprob) return;
  m_kept[p] = mP[p];
  int32_t s = statP[p];
  if (s == 0) s = statH[p];
  if (s == 0 && flags[NAO_FLAG_TIMEOUT]) s = NAO_E_TIMEOUT;
  status[p] = s;
}

// after the statuses that report it: status[0..nstatus) of a one-word status array takes
// NAO_E_TIMEOUT if the flag is set and it is 0; the flag is cleared (reported once)
__global__ void report_timeout_kernel(int* flags, int32_t* status, int nstatus) {
  if (threadIdx.x != 0) return;
  if (status && flags[NAO_FLAG_TIMEOUT])
    for (int i = 0; i < nstatus; ++i)
      if (status[i] == 0) status[i] = NAO_E_TIMEOUT;
  flags[NAO_FLAG_TIMEOUT] = 0;
}

// One batched complex product of the band step, on the tensor cores (digit planes) when the
// context asks for it and the contraction length allows, else on the FP64 CUDA cores.
// digits: NAO_OZ_DIGITS_FP64, or nao_config.mixed_planes for the products the mixed mode
// computes to 30 bits (the FP64 CUDA-core route ignores it).
cudaError_t run_zgemm(nao_ctx* ctx, const char* stage, int nprob, GemmDims d, double alpha, GemmOperand A,
                      GemmOperand B, double beta, z64* C, long long Cbs, long long Crs, long long Ccs, void* ozws,
                      cudaStream_t st, int digits = NAO_OZ_DIGITS_FP64) {
  if (ctx->gemm_method == NAO_GEMM_TC && ozws && zgemm_oz_supported(d)) {
    NaoStage stage_(ctx, stage, st, 3);
    return launch_zgemm_oz(nprob, d, alpha, A, B, beta, C, Cbs, Crs, Ccs, ozws, ctx->dev_flags, st, digits);
  }
  NaoStage stage_(ctx, stage, st, 1);
  return launch_zgemm(nprob, d, zmk(alpha, 0.0), A, B, zmk(beta, 0.0), C, Cbs, Crs, Ccs, st);
}

// Real counterpart of run_zgemm (the Newton-Schulz Gram matrix).
cudaError_t run_dgemm(nao_ctx* ctx, const char* stage, int nprob, GemmDims d, double alpha, GemmOperand A,
                      GemmOperand B, double beta, double* C, long long Cbs, long long Crs, long long Ccs, void* ozws,
                      cudaStream_t st) {
  if (ctx->gemm_method == NAO_GEMM_TC && ozws && dgemm_oz_supported(d)) {
    NaoStage stage_(ctx, stage, st, 3);
    return launch_dgemm_oz(nprob, d, alpha, A, B, beta, C, Cbs, Crs, Ccs, ozws, ctx->dev_flags, st);
  }
  NaoStage stage_(ctx, stage, st, 1);
  return launch_dgemm(nprob, d, alpha, A, B, beta, C, Cbs, Crs, Ccs, st);
}

// Workspace layout of nao_gen_eig (byte offsets into the context's arena) and its size.
struct GenEigPlan {
  size_t oAS, oTauS, odS, oeS, owS, oZ, oZ2, oG, oScr, omS, ostS, oX, oHf, oY, oHp, oV, oTauH, odH, oeH, owH, omP, onbP, ostP, ostH, oOz, oVf, oTc, oG2, oT2, oW, oW2, oVW, oDig, oErow;
  // two-stage reduction (band width B2 > 0): V T, the panel's small matrices, band, stage-2 reflectors
  size_t oSVT, oSG, oST, oSM, oSN, oSTc, oSAB, oSV2, oSTau2;
  // split Parts 3-4: the second half's inverse-iteration scratch and product workspace
  size_t oScr2, oOz2;
  // per problem: the second Newton-Schulz step's flag and column count
  size_t oNs2, oNc2;
  size_t bytes;
};

GenEigPlan plan_gen_eig(int n, int nprob, int nSe, bool use_tc, int B2, bool split = false) {
  GenEigPlan W;
  WsPlan P;
  const size_t nn = (size_t)n * n;
  const int nmax = nSe > nprob ? nSe : nprob;
  // overlap chain
  W.oAS = P.take<z64>(nn * nSe);
  W.oTauS = P.take<z64>((size_t)n * nSe);
  W.odS = P.take<double>((size_t)n * nSe);
  W.oeS = P.take<double>((size_t)n * nSe);
  W.owS = P.take<double>((size_t)n * nSe);
  W.omS = P.take<int32_t>(nSe);
  W.ostS = P.take<int32_t>(nSe);
  W.oX = P.take<z64>(nn * nSe);
  // tridiagonal eigenvectors, Newton-Schulz, inverse-iteration scratch (both chains)
  W.oZ = P.take<double>(nn * nmax);
  W.oZ2 = P.take<double>(use_tc ? 1 : nn * nmax);  // the tensor-core Newton-Schulz step works in place
  W.oG = P.take<double>(nn * nmax);
  W.oScr = P.take<double>(stein_scratch_doubles(n, nmax));
  // Hamiltonian chain
  W.oHf = P.take<z64>(nn * nprob);
  W.oY = P.take<z64>(nn * nprob);
  W.oHp = P.take<z64>(nn * nprob);
  W.oV = P.take<z64>(nn * nprob);
  W.oTauH = P.take<z64>((size_t)n * nprob);
  W.odH = P.take<double>((size_t)n * nprob);
  W.oeH = P.take<double>((size_t)n * nprob);
  W.owH = P.take<double>((size_t)n * nprob);
  W.omP = P.take<int32_t>(nprob);
  W.onbP = P.take<int32_t>(nprob);
  W.ostP = P.take<int32_t>(nprob);
  W.ostH = P.take<int32_t>(nprob);
  // digit planes of the largest product: n x n x n, or the back-transform's nb-wide ones
  const int nd = n > NAO_WY_NB ? n : NAO_WY_NB;
  const GemmDims dmax{nd, nd, nd, nullptr, nullptr, nullptr, 0};
  W.oOz = P.take<char>(use_tc ? zgemm_oz_workspace(nmax, dmax) : 1);
  // compact WY operands and the Householder panel's [V | W | V]
  const int ncolv = (n + NAO_WY_NB - 1) / NAO_WY_NB * NAO_WY_NB;
  W.oVf = P.take<z64>((size_t)n * ncolv * nmax);
  W.oTc = P.take<z64>((size_t)ncolv * nmax);
  const int nblk = n > 1 ? (n - 1 + NAO_WY_NB - 1) / NAO_WY_NB : 1;  // WY blocks: G_j and T_j of all
  W.oG2 = P.take<z64>((size_t)NAO_WY_NB * NAO_WY_NB * nmax * nblk);
  W.oT2 = P.take<z64>((size_t)NAO_WY_NB * NAO_WY_NB * nmax * nblk);
  W.oW = P.take<z64>((size_t)NAO_WY_NB * n * nmax);
  W.oW2 = P.take<z64>((size_t)n * ncolv * nmax);  // V_j T_j of all blocks
  W.oVW = P.take<z64>((size_t)2 * 3 * NAO_HT_NB * n * nmax);  // column-major + row-major copies
  // 8-bit digit planes of the Householder trailing matrix (tensor-core product method)
  W.oDig = P.take<char>(use_tc ? hetrd_digits_bytes(n, nmax, NAO_HT_DIGITS_FP64) : 16);
  W.oErow = P.take<int>((size_t)(n > 1 ? n - 1 : 1) * nmax);
  const size_t b2 = B2 > 0 ? (size_t)B2 : 0;
  const size_t sq = B2 > 0 ? (size_t)sbr_q2_count(n, B2) : 0;
  W.oSVT = P.take<z64>(b2 * n * nmax + 1);
  W.oSG = P.take<z64>(b2 * b2 * nmax + 1);
  W.oST = P.take<z64>(b2 * b2 * nmax + 1);
  W.oSM = P.take<z64>(b2 * b2 * nmax + 1);
  W.oSN = P.take<z64>(b2 * b2 * nmax + 1);
  W.oSTc = P.take<z64>(b2 * nmax + 1);
  W.oSAB = P.take<z64>(2 * b2 * n * nmax + 1);
  W.oSV2 = P.take<z64>(sq * b2 * nmax + 1);
  W.oSTau2 = P.take<z64>(sq * nmax + 1);
  const int np2 = nprob - nprob / 2;
  W.oScr2 = P.take<double>(split ? stein_scratch_doubles(n, np2) : 1);
  W.oOz2 = P.take<char>(split && use_tc ? zgemm_oz_workspace(np2, dmax) : 1);
  W.oNs2 = P.take<int>(nmax);
  W.oNc2 = P.take<int32_t>(nmax);
  W.bytes = P.off;
  return W;
}

// Workspace layout of nao_density_matrix.
struct DensityPlan {
  size_t of, onocc, oscr, ost, oCs, oCe, oP, oOz;
  size_t bytes;
};

// The phase sum of Part 6 (rho_tc: on the tensor cores) reuses the product workspace oOz:
// it runs after the P(k) product, in stream order.
DensityPlan plan_density(int n, int nspin, int nk, int nR, int nb, int num_sms, bool use_tc, bool rho_tc, bool edm) {
  const int nprob = nspin * nk;
  DensityPlan W;
  WsPlan P;
  W.of = P.take<double>((size_t)nprob * n);
  W.onocc = P.take<int32_t>(nprob);
  W.oscr = P.take<double>(fermi_scratch_doubles(num_sms));
  W.ost = P.take<int32_t>(1);
  W.oCs = P.take<z64>((size_t)nprob * n * nb);
  W.oCe = P.take<z64>(edm ? (size_t)nprob * n * nb : 1);
  W.oP = P.take<z64>((size_t)n * n * nprob);
  size_t oz = use_tc ? zgemm_oz_workspace(nprob, GemmDims{n, n, nb, nullptr, nullptr, nullptr, 0}) : 1;
  if (rho_tc) {
    const size_t r = rho_phase_tc_ws_bytes(n, nspin, nk, nR);
    if (r > oz) oz = r;
  }
  W.oOz = P.take<char>(oz);
  W.bytes = P.off;
  return W;
}

// Eigen_HH steps 3-4 in blocked form: U(:, c) = Q Z(:, m - nc + c) for c < nc (nc = ncols[p];
// Z(:, c) when lowest),
// normalised (times 1/sqrt(w) when use_rsqrt), with Q = prod_j (I - V_j T_j V_j^H) applied from
// the last block of NAO_WY_NB reflectors to the first.  Nothing about V_j and T_j depends on
// U, so the Gram matrices V_j^H V_j of all blocks come first, then all T_j in one launch,
// then the products VT_j = V_j T_j; each block then costs two products on the chain through
// U: W = V_j^H U and U -= VT_j W.  VT: [nprob][ncolv][n] (column-major like Vf, block j in
// columns j nb ..).
// The second reduction stage of the two-stage form: its reflectors (csrc/sbr.cu).
struct Q2Ref {
  int B;
  const z64* V2;
  const z64* tau2;
  long long sq;
};

cudaError_t backtransform_blocked(nao_ctx* ctx, int n, int nprob, const int32_t* size, const int32_t* ncols, const z64* A,
                                  const z64* tau, const double* Z, const double* w, int use_rsqrt, z64* U, z64* Vf,
                                  z64* tauc, z64* G, z64* T, z64* W, z64* VT, void* ozws, cudaStream_t st,
                                  int digits, int lowest, int off = 1, const Q2Ref* q2 = nullptr) {
  const int nb = NAO_WY_NB;
  const int ncolv = (n + nb - 1) / nb * nb;
  const long long snn = (long long)n * n, svf = (long long)n * ncolv, snb2 = (long long)nb * nb,
                  snbn = (long long)nb * n;
  cudaError_t e;
  {
    NaoStage stage_(ctx, "backtransform", st, 2);
    e = launch_extract_v(n, nprob, size, A, n, snn, tau, n, ncolv, Vf, n, svf, tauc, off, st);
    if (e == cudaSuccess) e = launch_init_u(n, nprob, size, ncols, Z, n, snn, U, n, snn, lowest, st);
    if (e != cudaSuccess) return e;
  }
  if (q2) {  // U = Q2 Z first (stage 2's reflectors), then stage 1's blocks below
    NaoStage stage_(ctx, "sbr_q2", st, 1);
    e = launch_sbr_q2(q2->B, n, nprob, size, ncols, q2->V2, q2->tau2, q2->sq, U, n, snn, st);
    if (e != cudaSuccess) return e;
  }
  const int nblk = n > off ? (n - off + nb - 1) / nb : 0;
  for (int j = 0; j < nblk; ++j) {  // Gram matrices of all blocks
    const int R0 = j * nb + off, rows = n - R0;
    const z64* Vj = Vf + R0 + (size_t)j * nb * n;  // V_j(r, c) at Vj[r + c n]
    GemmDims dg{nb, nb, rows, nullptr, nullptr, nullptr, 0};
    e = run_zgemm(ctx, "backtransform", nprob, dg, 1.0, GemmOperand{Vj, svf, n, 1, 1, nullptr},
                  GemmOperand{Vj, svf, 1, n, 0, nullptr}, 0.0, G + (size_t)j * nprob * snb2, snb2, nb, 1, ozws,
                  st, digits);
    if (e != cudaSuccess) return e;
  }
  if (nblk > 0) {
    NaoStage stage_(ctx, "backtransform", st, 1);
    e = launch_build_t(nb, nprob, nblk, G, tauc, ncolv, T, st);
    if (e != cudaSuccess) return e;
  }
  for (int j = 0; j < nblk; ++j) {  // VT_j = V_j T_j (rows x nb; T_j upper triangular, row-major)
    const int R0 = j * nb + off, rows = n - R0;
    GemmDims dv{rows, nb, nb, nullptr, nullptr, nullptr, 0};
    e = run_zgemm(ctx, "backtransform", nprob, dv, 1.0, GemmOperand{Vf + R0 + (size_t)j * nb * n, svf, 1, n, 0, nullptr},
                  GemmOperand{T + (size_t)j * nprob * snb2, snb2, nb, 1, 0, nullptr}, 0.0,
                  VT + R0 + (size_t)j * nb * n, svf, 1, n, ozws, st, digits);
    if (e != cudaSuccess) return e;
  }
  for (int j = nblk - 1; j >= 0; --j) {
    const int R0 = j * nb + off, rows = n - R0;
    if (rows <= 0) continue;
    const z64* Vj = Vf + R0 + (size_t)j * nb * n;
    const z64* VTj = VT + R0 + (size_t)j * nb * n;
    GemmDims dw{nb, n, rows, nullptr, ncols, nullptr, 0};
    e = run_zgemm(ctx, "backtransform", nprob, dw, 1.0, GemmOperand{Vj, svf, n, 1, 1, nullptr},
                  GemmOperand{U + R0, snn, 1, n, 0, nullptr}, 0.0, W, snbn, n, 1, ozws, st, digits);
    if (e != cudaSuccess) return e;
    GemmDims du{rows, n, nb, nullptr, ncols, nullptr, 0};
    e = run_zgemm(ctx, "backtransform", nprob, du, -1.0, GemmOperand{VTj, svf, 1, n, 0, nullptr},
                  GemmOperand{W, snbn, n, 1, 0, nullptr}, 1.0, U + R0, snn, 1, n, ozws, st, digits);
    if (e != cudaSuccess) return e;
  }
  NaoStage stage_(ctx, "backtransform", st, 1);
  return launch_normalize_cols(n, nprob, size, ncols, w, n, use_rsqrt, U, n, snn, st);
}

// Eigen_HH step 1, blocked: panels of NAO_HT_NB columns reduced by the cluster kernel, each
// followed by the deferred update A(r0:, r0:) -= V W^H + W V^H of the rest (lower triangle,
// one rank-2 NB product).  VW: [nprob][3 NB][n] workspace (the panel's [V | W | V] columns).  digits: planes of the update
// products; panel_digits: digits of the panel's integer matrix-vector products
// (NAO_HT_DIGITS_FP64, or NAO_HT_DIGITS_MIXED for the H' reduction of the mixed mode).
cudaError_t hetrd_blocked(nao_ctx* ctx, int n, int nprob, const int32_t* size, z64* A, double* d, double* e, z64* tau,
                          z64* VW, void* ozws, cudaStream_t st, int digits, void* dig, int* erow,
                          int panel_digits = NAO_HT_DIGITS_FP64, int cluster_nprob = 0) {
  // exact integer matrix-vector products with the tensor-core method; FP64 FMAs otherwise
  // (up to the order whose digit words still fit in a block's shared memory)
  const bool use_dig = ctx->gemm_method == NAO_GEMM_TC && dig != nullptr && hetrd_digits_fit(n, panel_digits);
  const int pd = use_dig ? panel_digits : 0;
  const int NB = NAO_HT_NB;
  // cluster size from the number of matrices that share the GPU (cluster_nprob: a concurrent
  // launch's matrices included)
  const int cl = hetrd_cluster_size(n, cluster_nprob > 0 ? cluster_nprob : nprob, ctx->num_sms, pd);
  const long long snn = (long long)n * n, svw = (long long)n * 3 * NB;
  for (int i0 = 0; i0 < n; i0 += NB) {
    cudaError_t err = cudaSuccess;
    if (use_dig) {
      NaoStage stage_(ctx, "hetrd_digits", st, 1);
      err = launch_hetrd_digits(n, nprob, size, A, n, snn, i0, dig, erow, pd, st);
    }
    if (err == cudaSuccess) {
      NaoStage stage_(ctx, "hetrd", st, 1);
      err = launch_hetrd_panel(n, nprob, size, A, n, snn, d, e, tau, n, VW, svw, i0, cl, use_dig ? dig : nullptr,
                               erow, pd, VW + (size_t)nprob * svw, st);
    }
    if (err != cudaSuccess) return err;
    const int r0 = i0 + NB;
    if (r0 >= n) break;
    const int rows = n - r0;
    GemmDims dd{rows, rows, 2 * NB, nullptr, nullptr, nullptr, 1};
    // [V | W] (rows r0..) times [W | V]^H; VW holds the panel's columns column-major
    z64* VWr = VW + (size_t)nprob * svw;
    err = run_zgemm(ctx, "hetrd_update", nprob, dd, -1.0, GemmOperand{VWr + (size_t)r0 * 3 * NB, svw, 3 * NB, 1, 0, nullptr},
                    GemmOperand{VWr + (size_t)r0 * 3 * NB + NB, svw, 1, 3 * NB, 1, nullptr}, 1.0,
                    A + r0 + (size_t)r0 * n, snn, 1, n, ozws, st, digits);
    if (err != cudaSuccess) return err;
  }
  return cudaSuccess;
}

// Eigen_HH step 1 in two stages (csrc/sbr.cu): dense -> band of lower bandwidth B, one
// panel of B columns at a time (panel QR, then A22 <- Q^H A22 Q as the tensor-core products
// G = V^H V -> T, X = A22 (V T), M = V^H X, N = T^H M, W = X - V N / 2 and the full rank-2B
// update A22 -= V W^H + W V^H), then band -> tridiagonal by bulge chasing.  Stage 1's
// reflectors stay in A below the band (head of reflector c at row c + B, tau[c]); stage 2's
// go to V2 / tau2.  A must hold the full Hermitian matrix.
struct SbrWork {
  z64 *VW, *VT, *G, *T, *M, *N, *tauc, *AB, *V2, *tau2;
  long long sq;
};

cudaError_t hetrd_two_stage(nao_ctx* ctx, int n, int nprob, const int32_t* size, z64* A, double* d, double* e, z64* tau,
                            const SbrWork& S, int B, void* ozws, cudaStream_t st, int digits) {
  const long long snn = (long long)n * n, svw = (long long)n * 3 * B, svt = (long long)n * B, sbb = (long long)B * B;
  cudaError_t err = cudaSuccess;
  if (size) {  // the products read all n rows and columns
    NaoStage stage_(ctx, "sbr_qr", st, 1);
    err = launch_zero_outside(n, nprob, size, A, snn, st);
    if (err != cudaSuccess) return err;
  }
  for (int c0 = 0; c0 + B < n; c0 += B) {
    const int r0 = c0 + B, rows = n - r0;
    {
      NaoStage stage_(ctx, "sbr_qr", st, 1);
      err = launch_sbr_qr(B, n, nprob, size, A, snn, c0, S.tauc, tau, n, S.VW, svw, st);
      if (err != cudaSuccess) return err;
    }
    const z64* Vp = S.VW + (size_t)r0 * 3 * B;  // V: rows x B, row-major (ld 3B)
    z64* Xp = S.VW + (size_t)r0 * 3 * B + B;    // X, then W, beside it
    z64* A22 = A + r0 + (size_t)r0 * n;
    const GemmOperand opV{Vp, svw, 3 * B, 1, 0, nullptr}, opVh{Vp, svw, 1, 3 * B, 1, nullptr};
    err = run_zgemm(ctx, "sbr_update", nprob, GemmDims{B, B, rows, nullptr, nullptr, nullptr, 0}, 1.0, opVh, opV, 0.0,
                    S.G, sbb, B, 1, ozws, st, digits);  // G = V^H V
    if (err != cudaSuccess) return err;
    {
      NaoStage stage_(ctx, "sbr_update", st, 1);
      err = launch_build_t(B, nprob, 1, S.G, S.tauc, B, S.T, st);
      if (err != cudaSuccess) return err;
    }
    err = run_zgemm(ctx, "sbr_update", nprob, GemmDims{rows, B, B, nullptr, nullptr, nullptr, 0}, 1.0, opV,
                    GemmOperand{S.T, sbb, B, 1, 0, nullptr}, 0.0, S.VT + (size_t)r0 * B, svt, B, 1, ozws, st,
                    digits);  // V T
    if (err == cudaSuccess)
      err = run_zgemm(ctx, "sbr_update", nprob, GemmDims{rows, B, rows, nullptr, nullptr, nullptr, 0}, 1.0,
                      GemmOperand{A22, snn, 1, n, 0, nullptr}, GemmOperand{S.VT + (size_t)r0 * B, svt, B, 1, 0, nullptr},
                      0.0, Xp, svw, 3 * B, 1, ozws, st, digits);  // X = A22 V T
    if (err == cudaSuccess)
      err = run_zgemm(ctx, "sbr_update", nprob, GemmDims{B, B, rows, nullptr, nullptr, nullptr, 0}, 1.0, opVh,
                      GemmOperand{Xp, svw, 3 * B, 1, 0, nullptr}, 0.0, S.M, sbb, B, 1, ozws, st, digits);  // V^H X
    if (err == cudaSuccess)
      err = run_zgemm(ctx, "sbr_update", nprob, GemmDims{B, B, B, nullptr, nullptr, nullptr, 0}, 1.0,
                      GemmOperand{S.T, sbb, 1, B, 1, nullptr}, GemmOperand{S.M, sbb, B, 1, 0, nullptr}, 0.0, S.N, sbb,
                      B, 1, ozws, st, digits);  // T^H M
    if (err == cudaSuccess)
      err = run_zgemm(ctx, "sbr_update", nprob, GemmDims{rows, B, B, nullptr, nullptr, nullptr, 0}, -0.5, opV,
                      GemmOperand{S.N, sbb, B, 1, 0, nullptr}, 1.0, Xp, svw, 3 * B, 1, ozws, st, digits);  // W
    if (err == cudaSuccess)  // A22 -= [V | W] [W | V]^H, both triangles
      err = run_zgemm(ctx, "sbr_update", nprob, GemmDims{rows, rows, 2 * B, nullptr, nullptr, nullptr, 0}, -1.0,
                      GemmOperand{Vp, svw, 3 * B, 1, 0, nullptr}, GemmOperand{Xp, svw, 1, 3 * B, 1, nullptr}, 1.0, A22,
                      snn, 1, n, ozws, st, digits);
    if (err != cudaSuccess) return err;
  }
  NaoStage stage_(ctx, "sbr_chase", st, 2);
  const long long sab = (long long)n * 2 * B;
  err = launch_sbr_band(B, n, nprob, size, A, snn, S.AB, sab, st);
  if (err == cudaSuccess) err = launch_sbr_chase(B, n, nprob, size, S.AB, sab, d, e, n, S.V2, S.tau2, S.sq, st);
  return err;
}

// The second half of the Newton-Schulz step, Z - Z (G - I)/2 with G = Z^T Z given by its
// lower triangle (Z: rows size[p], columns ncols[p]).  Tensor-core method: G - I made full,
// then one five-plane (30-bit) product with alpha = -1/2 and beta = 1 in place on Z (the
// operands are split before the product reads them); the term is ~1e-9 of Z, so 30 bits
// of it are far below Z's own rounding.  Otherwise the FP32 SIMT correction into Z2.
// Returns the array that holds the result.
double* ns_correct(nao_ctx* ctx, int n, int nprob, const int32_t* size, const int32_t* ncols, double* Z, double* G,
                   double* Z2, void* ozws, cudaStream_t st, cudaError_t* err) {
  const long long snn = (long long)n * n;
  const GemmDims d{n, n, n, size, ncols, ncols};
  if (ctx->gemm_method == NAO_GEMM_TC && ozws && dgemm_oz_supported(d)) {
    NaoStage stage_(ctx, "ortho_ns", st, 4);
    *err = launch_sym_minus_identity(n, nprob, ncols, G, n, snn, st);
    if (*err == cudaSuccess)
      *err = launch_dgemm_oz(nprob, d, -0.5, GemmOperand{Z, snn, 1, n, 0, nullptr}, GemmOperand{G, snn, 1, n, 0, nullptr},
                             1.0, Z, snn, 1, n, ozws, ctx->dev_flags, st, NAO_OZ_DIGITS_NS);
    return Z;
  }
  NaoStage stage_(ctx, "ortho_ns", st, 1);
  *err = launch_ns_correct(n, nprob, size, ncols, Z, G, n, snn, Z2, st);
  return Z2;
}

__global__ void ns2_cols_kernel(int nprob, const int* __restrict__ flag, const int32_t* __restrict__ ncols, int n,
                                int32_t* __restrict__ out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < nprob) out[p] = flag[p] ? (ncols ? ncols[p] : n) : 0;
}

// The second Newton-Schulz step, for the problems the tridiagonal solve flagged (ns2) because
// a gap in [1e-11, 1e-9) |T|_1 left overlaps up to ~1e-5 that one step reduces only to ~1e-10.
// Tensor-core method: in place, the other problems' columns counted as zero; FP64 CUDA cores:
// all problems, into the other array.  Returns the array that holds the result.
double* ns_second(nao_ctx* ctx, int n, int nprob, const int32_t* size, const int32_t* ncols, const int* ns2,
                  int32_t* ncols2, double* Zo, double* Z, double* Z2, double* G, void* ozws, cudaStream_t st,
                  cudaError_t* err) {
  const long long snn = (long long)n * n;
  const bool tc = ctx->gemm_method == NAO_GEMM_TC && ozws;
  const int32_t* nc = ncols;
  if (tc) {
    NaoStage stage_(ctx, "ortho_ns", st, 1);
    ns2_cols_kernel<<<(nprob + 127) / 128, 128, 0, st>>>(nprob, ns2, ncols, n, ncols2);
    *err = cudaGetLastError();
    if (*err != cudaSuccess) return Zo;
    nc = ncols2;
  }
  const GemmDims d{n, n, n, nc, nc, size, 1};
  *err = run_dgemm(ctx, "ortho_ns", nprob, d, 1.0, GemmOperand{Zo, snn, n, 1, 0, nullptr},
                   GemmOperand{Zo, snn, 1, n, 0, nullptr}, 0.0, G, snn, 1, n, ozws, st);
  if (*err != cudaSuccess) return Zo;
  return ns_correct(ctx, n, nprob, size, nc, Zo, G, Zo == Z ? Z2 : Z, ozws, st, err);
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

cudaError_t launch_report_timeout(int* flags, int32_t* status, int nstatus, cudaStream_t st) {
  report_timeout_kernel<<<1, 32, 0, st>>>(flags, status, nstatus);
  return cudaGetLastError();
}

static int check_config(const nao_config& c) {
  return (c.f_min >= 0.0 && c.f_min <= 1e-3 && c.inverse_iteration_max >= 0 && c.inverse_iteration_max <= 64 &&
          c.tc_wait_cycles >= 1 && c.tc_wait_cycles <= 1000000000000LL && c.mixed_planes >= 5 && c.mixed_planes <= 7 &&
          (c.overlap_mrrr == 0 || c.overlap_mrrr == 1) && (c.band_width == 0 || c.band_width == 16 || c.band_width == 32) &&
          (c.mrrr_all == 0 || c.mrrr_all == 1) && (c.split_hprime >= 0 && c.split_hprime <= 2))
             ? NAO_OK
             : NAO_E_INVALID;
}

// the wait bound lives in device memory, where the tensor-core kernels read it
static cudaError_t push_wait_bound(nao_ctx* c) {
  const long long w = c->cfg.tc_wait_cycles;
  return cudaMemcpy(c->dev_flags + NAO_FLAG_WAIT, &w, sizeof w, cudaMemcpyHostToDevice);
}

size_t gen_eig_ws_bytes(const nao_ctx* ctx, int n, int nprob, int nSe) {
  const bool use_tc = ctx->gemm_method == NAO_GEMM_TC && zgemm_oz_supported(GemmDims{n, n, n, nullptr, nullptr, nullptr, 0});
  return plan_gen_eig(n, nprob, nSe, use_tc, ctx->cfg.band_width,
                      ctx->cfg.band_width == 0 && nprob >= 2 &&
                          (ctx->cfg.split_hprime == 1 ||
                           (ctx->cfg.split_hprime == 2 && nprob >= NAO_SPLIT_MIN_PROBLEMS))).bytes;
}

size_t density_ws_bytes(const nao_ctx* ctx, int n, int nspin, int nk, int nR, int nb) {
  const bool use_tc =
      ctx->gemm_method == NAO_GEMM_TC && zgemm_oz_supported(GemmDims{n, n, nb, nullptr, nullptr, nullptr, 0});
  return plan_density(n, nspin, nk, nR, nb, ctx->num_sms, use_tc, use_tc && nk >= NAO_PHASE_TC_MIN_NK, false).bytes;
}

size_t bloch_ws_bytes(const nao_ctx* ctx, int n, int nR, int nmat, int nk) {
  return ctx->gemm_method == NAO_GEMM_TC && nk >= NAO_PHASE_TC_MIN_NK ? bloch_tc_ws_bytes(n, nR, nmat, nk) : 0;
}

extern "C" {

void nao_config_defaults(nao_config* cfg) {
  if (!cfg) return;
  cfg->f_min = NAO_F_MIN_DEFAULT;
  cfg->inverse_iteration_max = NAO_INV_ITER_DEFAULT;
  cfg->tc_wait_cycles = NAO_TC_WAIT_DEFAULT;
  cfg->mixed_planes = NAO_MIXED_PLANES_DEFAULT;
  cfg->overlap_mrrr = NAO_OVERLAP_MRRR_DEFAULT;
  cfg->band_width = NAO_BAND_WIDTH_DEFAULT;
  cfg->mrrr_all = NAO_MRRR_ALL_DEFAULT;
  cfg->split_hprime = NAO_SPLIT_HPRIME_DEFAULT;
}

int nao_init(nao_ctx** out, int device, size_t hbm_budget_bytes, const nao_config* cfg) {
  if (!out) return nao_fail(nullptr, NAO_E_INVALID, "nao_init: out is NULL");
  *out = nullptr;
  nao_config conf;
  nao_config_defaults(&conf);
  if (cfg) conf = *cfg;
  if (check_config(conf) != NAO_OK) return nao_fail(nullptr, NAO_E_INVALID, "nao_init: configuration out of range");
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess || count == 0)
    return nao_fail(nullptr, NAO_E_CUDA, "nao_init: no CUDA device (%s)", cudaGetErrorString(e));
  if (device < 0 || device >= count) return nao_fail(nullptr, NAO_E_INVALID, "nao_init: bad device %d", device);
  nao_ctx* c = new nao_ctx();
  c->device = device;
  DeviceGuard g(device);
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, device);
  if (e != cudaSuccess) {
    delete c;
    return nao_fail(nullptr, NAO_E_CUDA, "nao_init: %s", cudaGetErrorString(e));
  }
  c->num_sms = prop.multiProcessorCount;
  c->hbm_budget = hbm_budget_bytes;
  c->cfg = conf;
  e = cudaMalloc(&c->dev_flags, 64 * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(c->dev_flags, 0, 64 * sizeof(int));
  if (e == cudaSuccess) e = push_wait_bound(c);
  if (e != cudaSuccess) {
    if (c->dev_flags) cudaFree(c->dev_flags);
    delete c;
    return nao_fail(nullptr, NAO_E_CUDA, "nao_init: %s", cudaGetErrorString(e));
  }
  *out = c;
  return NAO_OK;
}

void nao_destroy(nao_ctx* ctx) {
  if (!ctx) return;
  serve_shutdown(ctx);
  {
    DeviceGuard g(ctx->device);
    drain_pending(ctx);
    for (auto e : ctx->event_pool) cudaEventDestroy(e);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->dev_flags) cudaFree(ctx->dev_flags);
    if (ctx->aux_stream) cudaStreamDestroy(ctx->aux_stream);
    if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
    if (ctx->join_ev) cudaEventDestroy(ctx->join_ev);
  }
  delete ctx;
}

int nao_get_config(const nao_ctx* ctx, nao_config* cfg) {
  if (!ctx || !cfg) return nao_fail(nullptr, NAO_E_INVALID, "nao_get_config: NULL argument");
  *cfg = ctx->cfg;
  return NAO_OK;
}

int nao_set_config(nao_ctx* ctx, const nao_config* cfg) {
  if (!ctx || !cfg) return nao_fail(nullptr, NAO_E_INVALID, "nao_set_config: NULL argument");
  if (check_config(*cfg) != NAO_OK) return nao_fail(ctx, NAO_E_INVALID, "nao_set_config: configuration out of range");
  DeviceGuard g(ctx->device);
  // the bound is read by kernels at their start: make the change after the work queued so far
  NAO_CUDA_TRY(ctx, cudaDeviceSynchronize());
  ctx->cfg = *cfg;
  NAO_CUDA_TRY(ctx, push_wait_bound(ctx));
  return NAO_OK;
}

int nao_profile_enable(nao_ctx* ctx, int on) {
  if (!ctx) return nao_fail(nullptr, NAO_E_INVALID, "nao_profile_enable: ctx is NULL");
  DeviceGuard g(ctx->device);
  drain_pending(ctx);
  ctx->stages.clear();
  ctx->profiling = on != 0;
  return NAO_OK;
}

int nao_profile_read(nao_ctx* ctx, int max, const char** names, double* ms, int64_t* calls, int64_t* launches) {
  if (!ctx) return nao_fail(nullptr, NAO_E_INVALID, "nao_profile_read: ctx is NULL");
  DeviceGuard g(ctx->device);
  drain_pending(ctx);
  const int n = (int)ctx->stages.size();
  for (int i = 0; i < n && i < max; ++i) {
    if (names) names[i] = ctx->stages[i].name;
    if (ms) ms[i] = ctx->stages[i].ms;
    if (calls) calls[i] = ctx->stages[i].calls;
    if (launches) launches[i] = ctx->stages[i].launches;
  }
  return n;
}

int64_t nao_launch_count(const nao_ctx* ctx) { return ctx ? ctx->launches : 0; }

int nao_set_gemm_method(nao_ctx* ctx, int method) {
  if (!ctx) return nao_fail(nullptr, NAO_E_INVALID, "nao_set_gemm_method: ctx is NULL");
  if (method != NAO_GEMM_FP64 && method != NAO_GEMM_TC)
    return nao_fail(ctx, NAO_E_INVALID, "nao_set_gemm_method: unknown method %d", method);
  ctx->gemm_method = method;
  return NAO_OK;
}

int nao_gen_eig_workspace(nao_ctx* ctx, int n, int nprob, int nS, int precision, size_t* bytes) {
  if (!ctx || !bytes) return nao_fail(ctx, NAO_E_INVALID, "nao_gen_eig_workspace: NULL argument");
  if (n < 1 || nprob < 1 || nS < 1) return nao_fail(ctx, NAO_E_INVALID, "nao_gen_eig_workspace: sizes must be >= 1");
  if (precision != NAO_FP64 && precision != NAO_MIXED_BF16X3)
    return nao_fail(ctx, NAO_E_INVALID, "nao_gen_eig_workspace: precision %d not available", precision);
  const size_t b = gen_eig_ws_bytes(ctx, n, nprob, nS);
  *bytes = b + b / 8;  // the arena keeps 1/8 headroom
  return NAO_OK;
}

int nao_set_refinement(nao_ctx* ctx, int sweeps) {
  if (!ctx) return nao_fail(nullptr, NAO_E_INVALID, "nao_set_refinement: ctx is NULL");
  if (sweeps < -1 || sweeps > 2)
    return nao_fail(ctx, NAO_E_INVALID, "nao_set_refinement: sweeps must be -1, 0, 1 or 2");
  ctx->refine_sweeps = sweeps;
  return NAO_OK;
}

int nao_zgemm(nao_ctx* ctx, int method, int nprob, int M, int N, int K, double alpha, const nao_c128* A, int lda,
              long long strideA, int transA, const nao_c128* B, int ldb, long long strideB, int transB, double beta,
              nao_c128* C, int ldc, long long strideC, void* stream) {
  if (!ctx) return nao_fail(nullptr, NAO_E_INVALID, "nao_zgemm: ctx is NULL");
  if (nprob < 1 || M < 1 || N < 1 || K < 1 || !A || !B || !C) return nao_fail(ctx, NAO_E_INVALID, "nao_zgemm: bad sizes");
  if (transA < 0 || transA > 2 || transB < 0 || transB > 2) return nao_fail(ctx, NAO_E_INVALID, "nao_zgemm: bad trans");
  DeviceGuard g(ctx->device);
  cudaStream_t st = as_stream(stream);
  GemmOperand a{A, strideA, transA ? 1 : lda, transA ? lda : 1, transA == 2, nullptr};
  GemmOperand b{B, strideB, transB ? 1 : ldb, transB ? ldb : 1, transB == 2, nullptr};
  GemmDims d{M, N, K, nullptr, nullptr, nullptr, 0};
  if (method == NAO_GEMM_TC) {
    WsPlan P;
    const size_t o = P.take<char>(zgemm_oz_workspace(nprob, d));
    int rc = nao_ws_reserve(ctx, P.off);
    if (rc) return rc;
    NAO_STAGE("zgemm_tc", 3, launch_zgemm_oz(nprob, d, alpha, a, b, beta, (z64*)C, strideC, ldc, 1,
                                            (char*)ctx->ws + o, ctx->dev_flags, st));
  } else if (method == NAO_GEMM_FP64) {
    NAO_STAGE("zgemm_fp64", 1, launch_zgemm(nprob, d, zmk(alpha, 0.0), a, b, zmk(beta, 0.0), (z64*)C, strideC, ldc, 1, st));
  } else {
    return nao_fail(ctx, NAO_E_INVALID, "nao_zgemm: unknown method %d", method);
  }
  return NAO_OK;
}

const char* nao_last_error(const nao_ctx* ctx) { return ctx ? ctx->last_error.c_str() : g_init_error.c_str(); }

size_t nao_workspace_bytes(const nao_ctx* ctx) { return ctx ? ctx->ws_bytes : 0; }

int nao_bloch_sum(nao_ctx* ctx, int n, int nR, const int32_t* R, int nmat, const double* MR, int nk,
                  const double* kpts, nao_c128* Mk, void* stream) {
  if (!ctx) return nao_fail(nullptr, NAO_E_INVALID, "nao_bloch_sum: ctx is NULL");
  if (n < 1 || nR < 1 || nmat < 1 || nk < 1) return nao_fail(ctx, NAO_E_INVALID, "nao_bloch_sum: sizes must be >= 1");
  if (!R || !MR || !kpts || !Mk) return nao_fail(ctx, NAO_E_INVALID, "nao_bloch_sum: NULL array");
  if ((size_t)8 * nR * 2 > 200 * 1024) return nao_fail(ctx, NAO_E_INVALID, "nao_bloch_sum: nR too large");
  DeviceGuard g(ctx->device);
  cudaStream_t st = as_stream(stream);
  if (ctx->gemm_method == NAO_GEMM_TC && nk >= NAO_PHASE_TC_MIN_NK) {
    const int rc = nao_ws_reserve(ctx, bloch_tc_ws_bytes(n, nR, nmat, nk));
    if (rc) return rc;
    NaoStage stage_(ctx, "bloch_sum", st, 0);
    int nl = 0;
    const cudaError_t e = launch_bloch_sum_tc(n, nR, R, nmat, MR, nk, kpts, (z64*)Mk, ctx->ws, ctx->dev_flags, st, &nl);
    stage_.add_launches(nl);
    NAO_CUDA_TRY(ctx, e);
    return NAO_OK;
  }
  NAO_STAGE("bloch_sum", 1, launch_bloch_sum(n, nR, R, nmat, MR, nk, kpts, (z64*)Mk, st));
  return NAO_OK;
}

int nao_gen_eig(nao_ctx* ctx, int n, int nprob, const nao_c128* H, const nao_c128* S, const int32_t* s_of_prob,
                int nS, double s_cut, int precision, int nb, double* eps, nao_c128* C, int32_t* m_kept,
                int32_t* status, void* stream) {
  return nao_gen_eig_sized(ctx, n, nprob, H, S, s_of_prob, nS, nullptr, s_cut, precision, nb, eps, C, m_kept, status,
                           stream);
}

int nao_gen_eig_sized(nao_ctx* ctx, int n, int nprob, const nao_c128* H, const nao_c128* S, const int32_t* s_of_prob,
                      int nS, const int32_t* s_size, double s_cut, int precision, int nb, double* eps, nao_c128* C,
                      int32_t* m_kept, int32_t* status, void* stream) {
  if (!ctx) return nao_fail(nullptr, NAO_E_INVALID, "nao_gen_eig: ctx is NULL");
  if (n < 1 || nprob < 1) return nao_fail(ctx, NAO_E_INVALID, "nao_gen_eig: n and nprob must be >= 1");
  if (n > 4096) return nao_fail(ctx, NAO_E_INVALID, "nao_gen_eig: n = %d above the supported 4096", n);
  if (!H || !S || !eps || !m_kept || !status) return nao_fail(ctx, NAO_E_INVALID, "nao_gen_eig: NULL array");
  if (precision == NAO_MIXED_TF32)
    return nao_fail(ctx, NAO_E_INVALID,
                    "nao_gen_eig: NAO_MIXED_TF32 not available (12-bit products leave errors one refinement sweep "
                    "does not remove); use NAO_MIXED_BF16X3");
  if (precision != NAO_FP64 && precision != NAO_MIXED_BF16X3)
    return nao_fail(ctx, NAO_E_INVALID, "nao_gen_eig: unknown precision %d", precision);
  if (nb < 1 || nb > n) return nao_fail(ctx, NAO_E_INVALID, "nao_gen_eig: nb must be in [1, n]");
  if (s_of_prob && nS < 1) return nao_fail(ctx, NAO_E_INVALID, "nao_gen_eig: nS must be >= 1 with a map");
  if (!(s_cut >= 0.0)) return nao_fail(ctx, NAO_E_INVALID, "nao_gen_eig: s_cut must be >= 0");
  const int nSe = s_of_prob ? nS : nprob;
  DeviceGuard g(ctx->device);
  cudaStream_t st = as_stream(stream);
  const size_t nn = (size_t)n * n;
  const int nmax = nSe > nprob ? nSe : nprob;

  const bool use_tc = ctx->gemm_method == NAO_GEMM_TC && zgemm_oz_supported(GemmDims{n, n, n, nullptr, nullptr, nullptr, 0});
  const int B2 = ctx->cfg.band_width;  // 0: one-stage reduction
  // Parts 3-4 in two halves on two streams (FP64, one-stage only)
  const bool split = B2 == 0 && precision == NAO_FP64 && nprob >= 2 &&
                     (ctx->cfg.split_hprime == 1 || (ctx->cfg.split_hprime == 2 && nprob >= NAO_SPLIT_MIN_PROBLEMS));
  const GenEigPlan W = plan_gen_eig(n, nprob, nSe, use_tc, B2, split);
  const int ncolv = (n + NAO_WY_NB - 1) / NAO_WY_NB * NAO_WY_NB;
  int rc = nao_ws_reserve(ctx, W.bytes);
  if (rc) return rc;
  char* ws = (char*)ctx->ws;
  z64* AS = (z64*)(ws + W.oAS);
  z64* tauS = (z64*)(ws + W.oTauS);
  double *dS = (double*)(ws + W.odS), *eS = (double*)(ws + W.oeS), *wS = (double*)(ws + W.owS);
  double *Z = (double*)(ws + W.oZ), *Z2 = (double*)(ws + W.oZ2), *G = (double*)(ws + W.oG), *scr = (double*)(ws + W.oScr);
  int32_t *mS = (int32_t*)(ws + W.omS), *stS = (int32_t*)(ws + W.ostS);
  z64* X = (z64*)(ws + W.oX);
  z64 *Hf = (z64*)(ws + W.oHf), *Y = (z64*)(ws + W.oY), *Hp = (z64*)(ws + W.oHp), *V = (z64*)(ws + W.oV);
  z64* tauH = (z64*)(ws + W.oTauH);
  double *dH = (double*)(ws + W.odH), *eH = (double*)(ws + W.oeH), *wH = (double*)(ws + W.owH);
  int32_t *mP = (int32_t*)(ws + W.omP), *nbP = (int32_t*)(ws + W.onbP), *stP = (int32_t*)(ws + W.ostP),
          *stH = (int32_t*)(ws + W.ostH);
  void* ozws = use_tc ? (void*)(ws + W.oOz) : nullptr;
  z64 *Vf = (z64*)(ws + W.oVf), *tauc = (z64*)(ws + W.oTc), *Gw = (z64*)(ws + W.oG2), *Tw = (z64*)(ws + W.oT2),
      *Ww = (z64*)(ws + W.oW), *VTw = (z64*)(ws + W.oW2), *VWp = (z64*)(ws + W.oVW);
  void* digp = use_tc ? (void*)(ws + W.oDig) : nullptr;
  int* erowp = (int*)(ws + W.oErow);
  const SbrWork sbr{VWp, (z64*)(ws + W.oSVT), (z64*)(ws + W.oSG), (z64*)(ws + W.oST), (z64*)(ws + W.oSM),
                    (z64*)(ws + W.oSN), (z64*)(ws + W.oSTc), (z64*)(ws + W.oSAB), (z64*)(ws + W.oSV2),
                    (z64*)(ws + W.oSTau2), B2 > 0 ? sbr_q2_count(n, B2) : 0};
  const Q2Ref q2ref{B2, sbr.V2, sbr.tau2, sbr.sq};
  int* ns2f = (int*)(ws + W.oNs2);
  int32_t* nc2 = (int32_t*)(ws + W.oNc2);
  const Q2Ref* q2 = B2 > 0 ? &q2ref : nullptr;
  const int hoff = B2 > 0 ? B2 : 1;  // head row offset of the reduction's (first-stage) reflectors
  const long long snn = (long long)nn;
  // Mixed mode: the back-transformations, X^H H X, the rank-2k updates of H' and X V run with
  // 30-bit products; the reduction of S, the tridiagonal solves (with their Newton-Schulz
  // step) and s^{-1/2} stay FP64-accurate, and one Ritz refinement sweep with FP64-accurate
  // products follows.
  const bool mixed = precision != NAO_FP64;
  const int dig = mixed ? ctx->cfg.mixed_planes : NAO_OZ_DIGITS_FP64;

  // ---- Part 2: Eigen_HH(S) -> s, U;  X = U_m s_m^{-1/2}
  NAO_STAGE("herm_fill", 1, launch_herm_fill(n, nSe, (const z64*)S, snn, nullptr, AS, n, snn, st));
  // s_size (nullable): the order of each overlap matrix; the leading s_size x s_size block
  // holds it, the rest of the n x n array is zero, and the chain keeps to the block
  if (B2 > 0)
    NAO_CUDA_TRY(ctx, hetrd_two_stage(ctx, n, nSe, s_size, AS, dS, eS, tauS, sbr, B2, ozws, st, NAO_OZ_DIGITS_FP64));
  else
    NAO_CUDA_TRY(ctx, hetrd_blocked(ctx, n, nSe, s_size, AS, dS, eS, tauS, VWp, ozws, st, NAO_OZ_DIGITS_FP64, digp, erowp));
  const int mrrr_s = ctx->cfg.mrrr_all ? 2 : ctx->cfg.overlap_mrrr, mrrr_h = ctx->cfg.mrrr_all ? 2 : 0;
  NAO_STAGE("stein", mrrr_s ? 5 : 4,
            launch_stein(n, nSe, s_size, dS, eS, n, wS, Z, n, snn, scr, stS, nullptr, n,
                         ctx->cfg.inverse_iteration_max, mrrr_s, st, ns2f));
  NAO_STAGE("misc", 1, launch_count_kept(n, nSe, s_size, wS, n, s_cut, mS, stS, st));
  double* Zo = Z2;  // the Newton-Schulz result (Z itself on the tensor-core method)
  {  // one Newton-Schulz step: Z (3I - Z^T Z)/2 = Z - Z (Z^T Z - I)/2
    GemmDims d{n, n, n, s_size, s_size, s_size, 1};
    NAO_CUDA_TRY(ctx, run_dgemm(ctx, "ortho_ns", nSe, d, 1.0, GemmOperand{Z, snn, n, 1, 0, nullptr},
                                GemmOperand{Z, snn, 1, n, 0, nullptr}, 0.0, G, snn, 1, n, ozws, st));
    cudaError_t e = cudaSuccess;
    Zo = ns_correct(ctx, n, nSe, s_size, s_size, Z, G, Z2, ozws, st, &e);
    NAO_CUDA_TRY(ctx, e);
    Zo = ns_second(ctx, n, nSe, s_size, s_size, ns2f, nc2, Zo, Z, Z2, G, ozws, st, &e);
    NAO_CUDA_TRY(ctx, e);
  }
  NAO_CUDA_TRY(ctx, backtransform_blocked(ctx, n, nSe, s_size, mS, AS, tauS, Zo, wS, 1, X, Vf, tauc, Gw, Tw, Ww, VTw,
                                          ozws, st, dig, 0, hoff, q2));
  {
    NaoStage stage_(ctx, "misc", st, 1);
    gather_m_kernel<<<(nprob + 127) / 128, 128, 0, st>>>(nprob, s_of_prob, mS, stS, nb, mP, nbP, stP);
    NAO_CUDA_TRY(ctx, cudaGetLastError());
  }

  if (split) {
    // Parts 3-4 for problems [p0, p0 + np) on stream st, with the workspace slices of that half:
    // per-problem arrays at the half's offset, the arrays laid out by the half's own problem
    // count (the panel's [V | W | V], the WY blocks' G and T, the digit planes) after the first
    // half's, the inverse-iteration scratch and the product workspace in regions of their own
    struct HpHalf {
      const z64* H;
      const z64* X;
      const int32_t* xmap;
      z64 *Hf, *Y, *Hp, *V, *tauH, *Vf, *tauc, *Gw, *Tw, *Ww, *VTw, *VWp, *C;
      double *dH, *eH, *wH, *Z, *Z2, *G, *scr, *eps;
      int32_t *mP, *nbP, *stH, *nc2;
      void *ozws, *digp;
      int *erowp, *ns2;
    };
    auto hp_half = [&](int np, cudaStream_t st, const HpHalf& h, cudaEvent_t part3_done) -> int {
      NAO_STAGE("herm_fill", 1, launch_herm_fill(n, np, h.H, snn, nullptr, h.Hf, n, snn, st));
      {
        GemmDims d{n, n, n, nullptr, h.mP, nullptr};  // Y = Hf X : n x m
        NAO_CUDA_TRY(ctx, run_zgemm(ctx, "zgemm_HX", np, d, 1.0, GemmOperand{h.Hf, snn, 1, n, 0, nullptr},
                                    GemmOperand{h.X, snn, 1, n, 0, h.xmap}, 0.0, h.Y, snn, 1, n, h.ozws, st, dig));
        GemmDims d2{n, n, n, h.mP, h.mP, nullptr, 1};  // Hp = X^H Y : m x m, lower triangle
        NAO_CUDA_TRY(ctx, run_zgemm(ctx, "zgemm_XHY", np, d2, 1.0, GemmOperand{h.X, snn, n, 1, 1, h.xmap},
                                    GemmOperand{h.Y, snn, 1, n, 0, nullptr}, 0.0, h.Hp, snn, 1, n, h.ozws, st, dig));
      }
      NAO_STAGE("misc", 1, launch_hermitize(n, np, h.mP, h.Hp, n, snn, st));
      if (part3_done) NAO_CUDA_TRY(ctx, cudaEventRecord(part3_done, st));
      NAO_CUDA_TRY(ctx, hetrd_blocked(ctx, n, np, h.mP, h.Hp, h.dH, h.eH, h.tauH, h.VWp, h.ozws, st, dig, h.digp,
                                      h.erowp, NAO_HT_DIGITS_FP64, nprob));
      const int nv_max = C ? n : 0;
      NAO_STAGE("stein", mrrr_h ? 5 : 4, launch_stein(n, np, h.mP, h.dH, h.eH, n, h.wH, h.Z, n, snn, h.scr, h.stH,
                                                     h.nbP, nv_max, ctx->cfg.inverse_iteration_max, mrrr_h, st,
                                                     h.ns2));
      if (nv_max > 0) {
        GemmDims d{n, n, n, h.nbP, h.nbP, h.mP, 1};
        NAO_CUDA_TRY(ctx, run_dgemm(ctx, "ortho_ns", np, d, 1.0, GemmOperand{h.Z, snn, n, 1, 0, nullptr},
                                    GemmOperand{h.Z, snn, 1, n, 0, nullptr}, 0.0, h.G, snn, 1, n, h.ozws, st));
        cudaError_t e = cudaSuccess;
        double* Zh = ns_correct(ctx, n, np, h.mP, h.nbP, h.Z, h.G, h.Z2, h.ozws, st, &e);
        NAO_CUDA_TRY(ctx, e);
        Zh = ns_second(ctx, n, np, h.mP, h.nbP, h.ns2, h.nc2, Zh, h.Z, h.Z2, h.G, h.ozws, st, &e);
        NAO_CUDA_TRY(ctx, e);
        NAO_CUDA_TRY(ctx, backtransform_blocked(ctx, n, np, h.mP, h.nbP, h.Hp, h.tauH, Zh, h.wH, 0, h.V, h.Vf, h.tauc,
                                                h.Gw, h.Tw, h.Ww, h.VTw, h.ozws, st, dig, 1));
        GemmDims dc{n, nb, n, nullptr, h.nbP, h.mP};  // C = X V(:, :nb) : n x nb, row-major [n][nb]
        NAO_CUDA_TRY(ctx, run_zgemm(ctx, "zgemm_XV", np, dc, 1.0, GemmOperand{h.X, snn, 1, n, 0, h.xmap},
                                    GemmOperand{h.V, snn, 1, n, 0, nullptr}, 0.0, h.C, (long long)n * nb, nb, 1,
                                    h.ozws, st, dig));
        NAO_STAGE("misc", 1, launch_zero_cols(n, np, nb, h.mP, h.C, st));
      }
      NAO_STAGE("misc", 1, launch_write_eps(n, np, h.mP, h.wH, n, h.eps, st));
      return NAO_OK;
    };
    if (!ctx->aux_stream) {
      NAO_CUDA_TRY(ctx, cudaStreamCreateWithFlags(&ctx->aux_stream, cudaStreamNonBlocking));
      NAO_CUDA_TRY(ctx, cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming));
      NAO_CUDA_TRY(ctx, cudaEventCreateWithFlags(&ctx->join_ev, cudaEventDisableTiming));
    }
    const int np1 = nprob / 2, np2 = nprob - np1;
    const int nblkw = n > 1 ? (n - 1 + NAO_WY_NB - 1) / NAO_WY_NB : 1;
    const long long svf = (long long)n * ncolv, svw = (long long)n * 3 * NAO_HT_NB;
    auto half = [&](int p0, int np, double* scr_h, void* oz_h, char* dig_h) {
      HpHalf h;
      h.H = (const z64*)H + (size_t)p0 * nn;
      h.X = s_of_prob ? X : X + (size_t)p0 * nn;
      h.xmap = s_of_prob ? s_of_prob + p0 : nullptr;
      h.Hf = Hf + (size_t)p0 * nn;
      h.Y = Y + (size_t)p0 * nn;
      h.Hp = Hp + (size_t)p0 * nn;
      h.V = V + (size_t)p0 * nn;
      h.tauH = tauH + (size_t)p0 * n;
      h.Vf = Vf + (size_t)p0 * svf;
      h.tauc = tauc + (size_t)p0 * ncolv;
      h.Gw = Gw + (size_t)nblkw * p0 * NAO_WY_NB * NAO_WY_NB;
      h.Tw = Tw + (size_t)nblkw * p0 * NAO_WY_NB * NAO_WY_NB;
      h.Ww = Ww + (size_t)p0 * NAO_WY_NB * n;
      h.VTw = VTw + (size_t)p0 * svf;
      h.VWp = VWp + (size_t)2 * p0 * svw;
      h.C = C ? (z64*)C + (size_t)p0 * n * nb : nullptr;
      h.dH = dH + (size_t)p0 * n;
      h.eH = eH + (size_t)p0 * n;
      h.wH = wH + (size_t)p0 * n;
      h.Z = Z + (size_t)p0 * nn;
      h.Z2 = use_tc ? Z2 : Z2 + (size_t)p0 * nn;
      h.G = G + (size_t)p0 * nn;
      h.scr = scr_h;
      h.eps = eps + (size_t)p0 * n;
      h.mP = mP + p0;
      h.nbP = nbP + p0;
      h.stH = stH + p0;
      h.ozws = oz_h;
      h.digp = dig_h;
      h.erowp = erowp + (size_t)p0 * (n > 1 ? n - 1 : 1);
      h.ns2 = ns2f + p0;
      h.nc2 = nc2 + p0;
      (void)np;
      return h;
    };
    const HpHalf h1 = half(0, np1, scr, ozws, (char*)digp);
    const HpHalf h2 = half(np1, np2, (double*)(ws + W.oScr2), use_tc ? (void*)(ws + W.oOz2) : nullptr,
                           digp ? (char*)digp + hetrd_digits_bytes(n, np1, NAO_HT_DIGITS_FP64) : nullptr);
    // the second half starts when the first half's Part 3 products are done, so that its
    // products (tensor cores) run beside the first half's Householder panels (integer and
    // FP64 pipes) instead of competing with the same kind of work
    rc = hp_half(np1, st, h1, ctx->fork_ev);
    if (rc) return rc;
    NAO_CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->aux_stream, ctx->fork_ev, 0));
    rc = hp_half(np2, ctx->aux_stream, h2, nullptr);
    if (rc) return rc;
    NAO_CUDA_TRY(ctx, cudaEventRecord(ctx->join_ev, ctx->aux_stream));
    NAO_CUDA_TRY(ctx, cudaStreamWaitEvent(st, ctx->join_ev, 0));
  } else {
  // ---- Part 3: H' = X^H H X
  NAO_STAGE("herm_fill", 1, launch_herm_fill(n, nprob, (const z64*)H, snn, nullptr, Hf, n, snn, st));
  {
    GemmDims d{n, n, n, nullptr, mP, nullptr};  // Y = Hf X : n x m
    NAO_CUDA_TRY(ctx, run_zgemm(ctx, "zgemm_HX", nprob, d, 1.0, GemmOperand{Hf, snn, 1, n, 0, nullptr},
                                GemmOperand{X, snn, 1, n, 0, s_of_prob}, 0.0, Y, snn, 1, n, ozws, st, dig));
    GemmDims d2{n, n, n, mP, mP, nullptr, 1};  // Hp = X^H Y : m x m, lower triangle
    NAO_CUDA_TRY(ctx, run_zgemm(ctx, "zgemm_XHY", nprob, d2, 1.0, GemmOperand{X, snn, n, 1, 1, s_of_prob},
                                GemmOperand{Y, snn, 1, n, 0, nullptr}, 0.0, Hp, snn, 1, n, ozws, st, dig));
  }
  NAO_STAGE("misc", 1, launch_hermitize(n, nprob, mP, Hp, n, snn, st));

  // ---- Part 4: Eigen_HH(H') -> eps, V;  C = X V
  if (B2 > 0)
    NAO_CUDA_TRY(ctx, hetrd_two_stage(ctx, n, nprob, mP, Hp, dH, eH, tauH, sbr, B2, ozws, st, dig));
  else
    NAO_CUDA_TRY(ctx, hetrd_blocked(ctx, n, nprob, mP, Hp, dH, eH, tauH, VWp, ozws, st, dig, digp, erowp,
                                    mixed ? NAO_HT_DIGITS_MIXED : NAO_HT_DIGITS_FP64));
  // Eigenvectors of H' only where they are used (the paper's second pass, dstevx's index
  // range): the lowest nb per problem for C, all m for the mixed-mode refinement, none when
  // the caller asks for eigenvalues only (C = NULL).
  const bool all_vecs = mixed && ctx->refine_sweeps >= 0;
  const int32_t* nvP = all_vecs ? mP : nbP;
  const int nv_max = (C || all_vecs) ? n : 0;
  NAO_STAGE("stein", mrrr_h ? 5 : 4, launch_stein(n, nprob, mP, dH, eH, n, wH, Z, n, snn, scr, stH, nvP, nv_max,
                                                 ctx->cfg.inverse_iteration_max, mrrr_h, st, ns2f));
  if (nv_max > 0) {
    {
      GemmDims d{n, n, n, nvP, nvP, mP, 1};
      NAO_CUDA_TRY(ctx, run_dgemm(ctx, "ortho_ns", nprob, d, 1.0, GemmOperand{Z, snn, n, 1, 0, nullptr},
                                  GemmOperand{Z, snn, 1, n, 0, nullptr}, 0.0, G, snn, 1, n, ozws, st));
      cudaError_t e = cudaSuccess;
      Zo = ns_correct(ctx, n, nprob, mP, nvP, Z, G, Z2, ozws, st, &e);
      NAO_CUDA_TRY(ctx, e);
      Zo = ns_second(ctx, n, nprob, mP, nvP, ns2f, nc2, Zo, Z, Z2, G, ozws, st, &e);
      NAO_CUDA_TRY(ctx, e);
    }
    NAO_CUDA_TRY(ctx, backtransform_blocked(ctx, n, nprob, mP, nvP, Hp, tauH, Zo, wH, 0, V, Vf, tauc, Gw, Tw, Ww, VTw,
                                            ozws, st, dig, 1, hoff, q2));
  }
  if (mixed && ctx->refine_sweeps >= 0) {
    // C^ = X V (all m columns, column-major in Hp), then Ritz refinement sweeps with
    // FP64-accurate products (csrc/refine.cu):  R' = C^H S C^, G = C^H H C^ -> I + F,
    // C = C^ (I + F); after the last sweep (or directly on C^ when there is none) eps =
    // Rayleigh quotients of C from FP64-accurate S C and H C, columns S-normalised, sorted.
    const long long svf = (long long)n * ncolv;
    int32_t* perm = (int32_t*)scr;
    GemmDims dc{n, n, n, nullptr, mP, mP};
    NAO_CUDA_TRY(ctx, run_zgemm(ctx, "zgemm_XV", nprob, dc, 1.0, GemmOperand{X, snn, 1, n, 0, s_of_prob},
                                GemmOperand{V, snn, 1, n, 0, nullptr}, 0.0, Hp, snn, 1, n, ozws, st, dig));
    NAO_STAGE("refine", 1, launch_herm_fill(n, nSe, (const z64*)S, snn, nullptr, AS, n, snn, st));
    const GemmDims dw{n, n, n, nullptr, mP, nullptr};  // n x m, contraction over n
    const GemmDims dr{n, n, n, mP, mP, nullptr, 1};     // m x m lower triangle, contraction over n
    const GemmDims du{n, n, n, nullptr, mP, mP};        // n x m, contraction over m
    for (int sw = 0; sw < ctx->refine_sweeps; ++sw) {
      if (sw > 0) {  // the previous sweep's C (Vf) is the next C^ (Hp)
        NaoStage stage_(ctx, "refine", st, 0);
        NAO_CUDA_TRY(ctx, cudaMemcpy2DAsync(Hp, (size_t)snn * sizeof(z64), Vf, (size_t)svf * sizeof(z64),
                                            nn * sizeof(z64), nprob, cudaMemcpyDeviceToDevice, st));
      }
      NAO_CUDA_TRY(ctx, run_zgemm(ctx, "refine", nprob, dw, 1.0, GemmOperand{AS, snn, 1, n, 0, s_of_prob},
                                  GemmOperand{Hp, snn, 1, n, 0, nullptr}, 0.0, Y, snn, 1, n, ozws, st));
      NAO_CUDA_TRY(ctx, run_zgemm(ctx, "refine", nprob, dw, 1.0, GemmOperand{Hf, snn, 1, n, 0, nullptr},
                                  GemmOperand{Hp, snn, 1, n, 0, nullptr}, 0.0, Vf, svf, 1, n, ozws, st));
      NAO_CUDA_TRY(ctx, run_zgemm(ctx, "refine", nprob, dr, 1.0, GemmOperand{Hp, snn, n, 1, 1, nullptr},
                                  GemmOperand{Y, snn, 1, n, 0, nullptr}, 0.0, V, snn, 1, n, ozws, st));
      NAO_CUDA_TRY(ctx, run_zgemm(ctx, "refine", nprob, dr, 1.0, GemmOperand{Hp, snn, n, 1, 1, nullptr},
                                  GemmOperand{Vf, svf, 1, n, 0, nullptr}, 0.0, Y, snn, 1, n, ozws, st));
      NAO_STAGE("refine", 1, launch_hermitize(n, nprob, mP, V, n, snn, st));
      NAO_STAGE("refine", 1, launch_hermitize(n, nprob, mP, Y, n, snn, st));
      NAO_STAGE("refine", 1, launch_oa_lambda(n, nprob, mP, V, Y, n, snn, wH, n, st));
      NAO_STAGE("refine", 1, launch_oa_f(n, nprob, mP, V, Y, n, snn, wH, n, st));
      NAO_CUDA_TRY(ctx, run_zgemm(ctx, "refine", nprob, du, 1.0, GemmOperand{Hp, snn, 1, n, 0, nullptr},
                                  GemmOperand{Y, snn, 1, n, 0, nullptr}, 0.0, Vf, svf, 1, n, ozws, st));
    }
    // the vectors whose Rayleigh quotients are taken: the last sweep's C (in Vf), or C^
    const bool swept = ctx->refine_sweeps > 0;
    z64* Cf = swept ? Vf : Hp;
    const long long cfs = swept ? svf : snn;
    z64* W2 = swept ? Hp : V;  // H C (V is free once X V has been formed)
    NAO_CUDA_TRY(ctx, run_zgemm(ctx, "refine", nprob, dw, 1.0, GemmOperand{AS, snn, 1, n, 0, s_of_prob},
                                GemmOperand{Cf, cfs, 1, n, 0, nullptr}, 0.0, Y, snn, 1, n, ozws, st));
    NAO_CUDA_TRY(ctx, run_zgemm(ctx, "refine", nprob, dw, 1.0, GemmOperand{Hf, snn, 1, n, 0, nullptr},
                                GemmOperand{Cf, cfs, 1, n, 0, nullptr}, 0.0, W2, snn, 1, n, ozws, st));
    NAO_STAGE("refine", 1, launch_oa_rq(n, nprob, mP, Cf, n, cfs, Y, W2, n, snn, wH, n, st));
    NAO_STAGE("refine", 1, launch_oa_sort(n, nprob, mP, wH, n, eps, perm, st));
    if (C) NAO_STAGE("refine", 1, launch_oa_gather(n, nprob, nb, perm, Cf, n, cfs, (z64*)C, st));
  } else {
    if (C) {
      GemmDims d{n, nb, n, nullptr, nbP, mP};  // C = X V(:, :nb) : n x nb, row-major [n][nb]
      NAO_CUDA_TRY(ctx, run_zgemm(ctx, "zgemm_XV", nprob, d, 1.0, GemmOperand{X, snn, 1, n, 0, s_of_prob},
                                  GemmOperand{V, snn, 1, n, 0, nullptr}, 0.0, (z64*)C, (long long)n * nb, nb, 1, ozws,
                                  st, dig));
      NAO_STAGE("misc", 1, launch_zero_cols(n, nprob, nb, mP, (z64*)C, st));
    }
    NAO_STAGE("misc", 1, launch_write_eps(n, nprob, mP, wH, n, eps, st));
  }
  }  // one pass of Parts 3-4
  {
    NaoStage stage_(ctx, "misc", st, 1);
    finish_status_kernel<<<(nprob + 127) / 128, 128, 0, st>>>(nprob, mP, stP, stH, ctx->dev_flags, m_kept, status);
    NAO_CUDA_TRY(ctx, cudaGetLastError());
  }
  NAO_STAGE("misc", 1, launch_report_timeout(ctx->dev_flags, nullptr, 0, st));  // reported: clear the flag
  return NAO_OK;
}

int nao_density_matrix(nao_ctx* ctx, int n, int nspin, int nk, const double* wk, const double* kpts,
                       const double* eps, const nao_c128* C, int nb, const int32_t* m_kept, double n_electrons,
                       double kT, int nR, const int32_t* R, double* mu_out, double* eband_out, double* f_out,
                       double* rhoR, double* edmR, int32_t* status, void* stream) {
  if (!ctx) return nao_fail(nullptr, NAO_E_INVALID, "nao_density_matrix: ctx is NULL");
  if (n < 1 || nk < 1 || nR < 1 || nb < 1 || nb > n || (nspin != 1 && nspin != 2))
    return nao_fail(ctx, NAO_E_INVALID, "nao_density_matrix: bad sizes");
  if (!wk || !kpts || !eps || !C || !m_kept || !R || !mu_out || !eband_out || !rhoR)
    return nao_fail(ctx, NAO_E_INVALID, "nao_density_matrix: NULL array");
  if (!(kT > 0.0)) return nao_fail(ctx, NAO_E_INVALID, "nao_density_matrix: kT must be > 0");
  if ((size_t)16 * nk * 8 > 200 * 1024) return nao_fail(ctx, NAO_E_INVALID, "nao_density_matrix: nk too large");
  DeviceGuard g(ctx->device);
  cudaStream_t st = as_stream(stream);
  const int nprob = nspin * nk;
  const size_t nn = (size_t)n * n;
  const double gdeg = (nspin == 1) ? 2.0 : 1.0;
  const GemmDims dP{n, n, nb, nullptr, nullptr, nullptr, 0};
  const bool use_tc = ctx->gemm_method == NAO_GEMM_TC && zgemm_oz_supported(dP);
  const bool rho_tc = use_tc && nk >= NAO_PHASE_TC_MIN_NK;
  const DensityPlan W = plan_density(n, nspin, nk, nR, nb, ctx->num_sms, use_tc, rho_tc, edmR != nullptr);
  const size_t of = W.of, onocc = W.onocc, oscr = W.oscr, ost = W.ost, oCs = W.oCs, oP = W.oP, oOz = W.oOz;
  int rc = nao_ws_reserve(ctx, W.bytes);
  if (rc) return rc;
  char* ws = (char*)ctx->ws;
  double* f = f_out ? f_out : (double*)(ws + of);
  int32_t* nocc = (int32_t*)(ws + onocc);
  double* scr = (double*)(ws + oscr);
  int32_t* st_local = (int32_t*)(ws + ost);
  z64* Cs = (z64*)(ws + oCs);
  z64* Pk = (z64*)(ws + oP);
  NAO_STAGE("fermi", 1, launch_fermi(ctx->num_sms, n, nprob, nk, gdeg, wk, eps, m_kept, nb, n_electrons, kT,
                                     ctx->cfg.f_min, f, nocc, mu_out, eband_out, status ? status : st_local, scr, st));
  NAO_STAGE("misc", 1, launch_scale_cols_sqrt(n, nprob, nb, (const z64*)C, f, Cs, st));
  {
    // P(k) = Cs Cs^H over the occupied bands (row-major [n][n])
    GemmDims d{n, n, nb, nullptr, nullptr, nocc};
    NAO_CUDA_TRY(ctx, run_zgemm(ctx, "zgemm_P", nprob, d, 1.0, GemmOperand{Cs, (long long)n * nb, nb, 1, 0, nullptr},
                                GemmOperand{Cs, (long long)n * nb, 1, nb, 1, nullptr}, 0.0, Pk, (long long)nn, n, 1,
                                use_tc ? (void*)(ws + oOz) : nullptr, st));
  }
  auto phase_sum = [&](double* out) -> cudaError_t {
    if (!rho_tc) {
      NaoStage stage_(ctx, "rho_phase", st, 1);
      return launch_rho_phase_sum(n, nspin, nk, nR, R, kpts, wk, gdeg, Pk, out, st);
    }
    NaoStage stage_(ctx, "rho_phase", st, 0);
    int nl = 0;
    const cudaError_t e = launch_rho_phase_tc(n, nspin, nk, nR, R, kpts, wk, gdeg, Pk, out, ws + oOz, ctx->dev_flags,
                                              st, &nl);
    stage_.add_launches(nl);
    return e;
  };
  NAO_CUDA_TRY(ctx, phase_sum(rhoR));
  if (edmR) {  // Part 6's energy density matrix: P_E(k) = Cs diag(eps) Cs^H, the same phase sum
    z64* Ce = (z64*)(ws + W.oCe);
    NAO_STAGE("misc", 1, launch_scale_cols_eps(n, nprob, nb, Cs, f, eps, Ce, st));
    GemmDims d{n, n, nb, nullptr, nullptr, nocc};
    NAO_CUDA_TRY(ctx, run_zgemm(ctx, "zgemm_P", nprob, d, 1.0, GemmOperand{Ce, (long long)n * nb, nb, 1, 0, nullptr},
                                GemmOperand{Cs, (long long)n * nb, 1, nb, 1, nullptr}, 0.0, Pk, (long long)nn, n, 1,
                                use_tc ? (void*)(ws + oOz) : nullptr, st));
    NAO_CUDA_TRY(ctx, phase_sum(edmR));
  }
  NAO_STAGE("misc", 1, launch_report_timeout(ctx->dev_flags, status ? status : st_local, 1, st));
  return NAO_OK;
}

}  // extern "C"
