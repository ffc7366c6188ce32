// FP64-accurate complex GEMM on the BF16 tensor cores (tcgen05), for the GEMM-shaped steps
// of the band step (Sec. 3: Parts 3-4 use ZGEMM; the back-transformation and Part 6 are
// products too).  On this GPU FP64 runs at 1.2 TFLOP/s and BF16 tcgen05 at ~2.4 PFLOP/s, so
// an exact splitting of the FP64 operands into small-integer digit planes (the error-free
// splitting of Ozaki, Ogita, Oishi & Rump, Numer. Algorithms 59, 2012) is ~20x faster than
// FP64 arithmetic while keeping FP64-level accuracy.
//
// Scheme (all my own design choices):
//  * complex -> real: C'' = A' B'' with A' = [Re op(A) | Im op(A)] (M x 2K) and the columns
//    of B'' interleaved, column 2j = (Re b_j ; -Im b_j), 2j+1 = (Im b_j ; Re b_j), so
//    C''(:, 2j) = Re c_j and C''(:, 2j+1) = Im c_j;
//  * every row of A' (column of B'') is scaled by a power of two 2^e so that |x| < 2^e, then
//    q = round(x 2^{60-e}) (int64, exact integer arithmetic on the FP64 bits) is written in
//    ten signed base-64 digits d_1..d_10 (|d_1| <= 64, |d_s| <= 32): 60 bits, so that even
//    entries far below their row's maximum keep FP64-level accuracy in the product;
//  * digit planes are stored as BF16 (exact): A_s = d_s 2^{-6(s-1)}, B_t = d_t 2^{-6(t-6)};
//  * the 55 products A_s B_t with s + t <= 11 run on tcgen05 (M = 128, N = 64, K = 16,
//    FP32 accumulation in TMEM).  Products of one "group" g = s + t share a power-of-two
//    scale, so for g <= 8 their FP32 sums are exact integers while below 2^24 (guaranteed
//    for 2K <= 1792); these seven groups get one TMEM accumulator each.  Groups 9..11 share an
//    eighth (8 x 64 columns = all 512 of TMEM): it is 2^-12 below group 7, so the FP32
//    rounding it collects over thousands of MMAs stays below FP64 rounding of the result
//    (sharing one accumulator from group 7 or 8 on was measured 2-10x less accurate);
//  * epilogue: the exact groups are combined in int64 (units of group 8), the sum of
//    everything converted to FP64 once and scaled by 2^{e_i + f_j - 42}; real alpha, beta.
// Pipeline: the digit tiles of each K step (16) arrive in one of three shared-memory stages
// by bulk asynchronous copies (TMA) issued by one producer thread; one thread issues the
// MMAs and commits them to the stage's barrier.  Every wait is bounded (clock64; the
// pipeline's waits by the context's nao_config.tc_wait_cycles); on timeout the block records
// an error, waits for its issued MMAs and lets its issued copies land (both with the fixed
// long bound), skips its epilogue and still frees its tensor memory.
#include <cuda_bf16.h>

#include "nao_internal.cuh"

namespace {

constexpr int OZ_S = 10;             // digit planes per operand for FP64 accuracy (60 bits); the most
                                     // any product uses (the workspace is sized for it)
constexpr int OZ_BM = 128;           // tile rows (C'' rows)
constexpr int OZ_BN = 64;            // tile columns (C'' columns = 32 complex columns); B plane tile rows
constexpr int OZ_BK = 16;            // K' per MMA step
constexpr int OZ_TILE_A = OZ_BM * OZ_BK * 2;  // bytes of one A plane tile (4096)
constexpr int OZ_TILE_B = OZ_BN * OZ_BK * 2;  // bytes of one B plane tile (2048)
constexpr int OZ_STAGES = 3;
// Short contractions (at most OZ_SHORT_KSTEPS K steps) use tiles of 32 columns, 256 TMEM
// columns and 2 stages (102 KB), so that two CTAs share an SM and one's epilogue overlaps
// the other's MMAs; their B tiles are the contiguous 32-row halves of the 64-row plane tiles.
constexpr int OZ_SHORT_KSTEPS = 16;
constexpr int OZ_THREADS = 256;
constexpr long long OZ_WAIT_CYCLES = NAO_TC_WAIT_DEFAULT;  // ~2 s at 2 GHz
constexpr int OZ_MAX_K2 = 1792;      // 2K bound for exact FP32 group sums (group 8: 9 2^10 per k)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// no-swizzle K-major descriptor: core matrices of 8 rows x 16 bytes; LBO = K-direction core
// stride (128 B), SBO = 8-row-group stride (256 B); version 1 (bit 46).
__device__ __forceinline__ uint64_t oz_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(256 >> 4) << 32) |
         ((uint64_t)1 << 46);
}

// kind::f16 instruction descriptor: F32 accumulate, BF16 A and B, K-major both, M = 128, N = 64.
constexpr uint32_t OZ_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(OZ_BN >> 3) << 17) |
                              ((uint32_t)(OZ_BM >> 4) << 24);

// byte offset of element (row, k) inside a plane tile (rows x 16 K, bf16)
__device__ __forceinline__ int oz_tile_off(int row, int k) {
  return (row >> 3) * 256 + ((k >> 3) & 1) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// biased exponent field of x (0 for zero / subnormal)
__device__ __forceinline__ int exp_field(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7ff); }

// q = round(x * 2^{DB S - e}) for |x| < 2^e (|q| < 2^63), by integer arithmetic on the bits of x
template <int S, int DB>
__device__ __forceinline__ long long oz_fixed(double x, int e) {
  const long long bits = __double_as_longlong(x);
  const int b = (int)((bits >> 52) & 0x7ff);
  if (b == 0) return 0;  // zero (subnormals are far below any row scale used here)
  long long m = (bits & 0xFFFFFFFFFFFFFll) | 0x10000000000000ll;  // 53-bit integer mantissa
  const int sh = b - 1075 + DB * S - e;                             // x 2^{DB S - e} = m 2^{sh}
  long long q;
  if (sh >= 0) q = m << sh;
  else if (sh <= -62) q = 0;
  else q = (m + (1ll << (-sh - 1))) >> (-sh);
  return bits < 0 ? -q : q;
}

// round(x 2^k) for a float x with |x 2^k| < 2^62, by integer arithmetic on the bits of x
__device__ __forceinline__ long long oz_f32_fixed(float x, int k) {
  const int b = __float_as_int(x);
  const int f = (b >> 23) & 0xff;
  if (f == 0) return 0;  // zero (subnormal sums are below any unit used here)
  const long long m = (b & 0x7fffff) | 0x800000;  // x = m 2^{f - 150}
  const int sh = f - 150 + k;
  long long q;
  if (sh >= 0) q = m << sh;
  else if (sh <= -26) q = 0;
  else q = (m + (1ll << (-sh - 1))) >> (-sh);
  return b < 0 ? -q : q;
}

// S signed base-2^DB digits of q (|q| < 2^{DB S}): q = sum_s d_s 2^{DB(S-1-s)}.
// DB = 6: the lower S - 1 in [-32, 31] and |d_0| <= 64, formed from the least significant
// digit up in int32 arithmetic on the two 30-bit halves of q (the carry left by the low half
// is 0 or 1).  DB = 7 (S = 9, 63 bits): the lower eight in [-64, 63] and |d_0| <= 128, from
// three 21-bit parts of q, each leaving a carry of 0 or 1 for the next.
template <int S, int DB>
__device__ __forceinline__ void oz_digits(long long q, int* d) {
  if (DB == 7) {
    static_assert(DB != 7 || S == 9, "base-128 digits come in nines");
    int x = (int)(q & 0x1FFFFF), y = (int)((q >> 21) & 0x1FFFFF), z = (int)(q >> 42);
#pragma unroll
    for (int s = S - 1; s >= S - 3; --s) {
      const int ds = ((x + 64) & 127) - 64;
      d[s] = ds;
      x = (x - ds) >> 7;
    }
    y += x;
#pragma unroll
    for (int s = S - 4; s >= S - 6; --s) {
      const int ds = ((y + 64) & 127) - 64;
      d[s] = ds;
      y = (y - ds) >> 7;
    }
    z += y;
#pragma unroll
    for (int s = S - 7; s >= 1; --s) {
      const int ds = ((z + 64) & 127) - 64;
      d[s] = ds;
      z = (z - ds) >> 7;
    }
    d[0] = z;
  } else if (S <= 5) {
    int x = (int)q;
#pragma unroll
    for (int s = S - 1; s >= 1; --s) {
      const int ds = ((x + 32) & 63) - 32;
      d[s] = ds;
      x = (x - ds) >> 6;
    }
    d[0] = x;
  } else {
    int lo = (int)(q & 0x3FFFFFFF), hi = (int)(q >> 30);  // q = hi 2^30 + lo, 0 <= lo < 2^30
#pragma unroll
    for (int s = S - 1; s >= S - 5; --s) {
      const int ds = ((lo + 32) & 63) - 32;
      d[s] = ds;
      lo = (lo - ds) >> 6;
    }
    hi += lo;
#pragma unroll
    for (int s = S - 6; s >= 1; --s) {
      const int ds = ((hi + 32) & 63) - 32;
      d[s] = ds;
      hi = (hi - ds) >> 6;
    }
    d[0] = hi;
  }
}

// BF16 bits of d 2^k for a digit |d| <= 64 (exact): the top half of the float d, with k
// added to the exponent field (no conversion or multiply instructions)
__device__ __forceinline__ uint32_t oz_bf16_bits(int d, int k) {
  return d ? (__float_as_uint((float)d) >> 16) + (uint32_t)(k << 7) : 0u;
}

// ---------------------------------------------------------------------------- split kernels
// One kernel for both operands, complex or real.  The rows it splits are
//   A (IS_B = false): the M rows of A' = op(A), A' = [Re op(A) | Im op(A)] when complex;
//   B (IS_B = true):  the rows of B''^T, i.e. the columns of B'' (2N interleaved columns when
//                     complex: row 2j = (Re b_j ; -Im b_j), row 2j+1 = (Im b_j ; Re b_j)).
// Plane layout (K-major tiles of TR = 128 (A) or 64 (B) rows x 16 K, bf16):
//   planes[prob][s][row / TR][k' / 16][oz_tile_off(row % TR, k' % 16)].
// Complex operands: K' = 2 Kh with Kh = round_up(K, 8); entries 0..K-1 hold the first
// part (Re op(A); Re b or Im b), entries Kh..Kh+K-1 the second, the rest are zero, so that
// both halves start on an 8-entry (16-byte) boundary.
// A block of 256 threads owns 16 consecutive rows and walks all of K'.  Lane l of a warp
// holds row (l & 7) + 8 (l >> 4) and the 8-element half (l >> 3) & 1 of a 16-wide K step, so
// each of its 16-byte plane chunks is contiguous and a warp stores 512 contiguous bytes per
// plane.  Pass 1 takes the row's largest exponent (the power-of-two row scale), pass 2 writes
// the digits.  Complex rows 2j and 2j+1 of B see the same set of values, hence one scale;
// their second halves repeat the first halves' values (Re b', and -Im b' = -(Im b')), so each
// lane forms the digits of its own first half only and also stores them, negated where the
// value is, as its partner row's second half.
template <bool IS_B, bool REAL, int S, int DB>
__global__ void __launch_bounds__(256) oz_split(int nprob, GemmDims dims, GemmOperand X, int Rp, int K2p,
                                                 __nv_bfloat16* __restrict__ planes, int* __restrict__ xexp) {
  constexpr int TR = IS_B ? OZ_BN : OZ_BM;            // rows per plane tile
  constexpr int TB = TR * OZ_BK * 2;                  // bytes per plane tile
  constexpr int SCALE0 = IS_B ? 30 : 0;               // plane s holds d_s 2^{SCALE0 - DB s}
  const int p = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lr = (lane & 7) + 8 * (lane >> 4);
  const int kh = (lane >> 3) & 1;
  const int row = blockIdx.x * 16 + lr;
  const int R = IS_B ? (dims.Np ? dims.Np[p] : dims.N) : (dims.Mp ? dims.Mp[p] : dims.M);
  const int K = gemm_k(dims, p);
  const int rows_live = (IS_B && !REAL) ? 2 * R : R;
  const bool live = row < rows_live;
  const int x = (IS_B && !REAL) ? row >> 1 : row;  // row (A) or column (B) of op(X)
  const int h = (IS_B && !REAL) ? row & 1 : 0;
  const unsigned char* xb = (const unsigned char*)X.ptr +
                            (size_t)(X.map ? X.map[p] : p) * X.bs * (REAL ? sizeof(double) : sizeof(z64));
  // element k of the row (0 <= k < K): op(X)(x, k) for A, op(X)(k, x) for B
  auto at = [&](int k) -> long long {
    return IS_B ? (long long)k * X.rs + (long long)x * X.cs : (long long)x * X.rs + (long long)k * X.cs;
  };
  // pass 1: largest exponent field over the row's values
  int bmax = 0;
  if (live)
    for (int k = warp * 16 + kh * 8; k < K; k += 8 * 16) {
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        if (k + e >= K) break;
        if (REAL) {
          bmax = max(bmax, exp_field(((const double*)xb)[at(k + e)]));
        } else {
          const z64 v = ((const z64*)xb)[at(k + e)];
          bmax = max(bmax, max(exp_field(v.x), exp_field(v.y)));
        }
      }
    }
  bmax = max(bmax, __shfl_xor_sync(0xffffffffu, bmax, 8));
  __shared__ int s_e[8][16];
  if (kh == 0) s_e[warp][lr] = bmax;
  __syncthreads();
  int bm = 0;
#pragma unroll
  for (int w = 0; w < 8; ++w) bm = max(bm, s_e[w][lr]);
  const int ex = bm == 0 ? -1100 : bm - 1022;  // |value| < 2^ex
  if (warp == 0 && kh == 0 && row < Rp) {
    if (IS_B && !REAL) {
      if (h == 0) xexp[(size_t)p * (Rp / 2) + x] = ex;
    } else {
      xexp[(size_t)p * Rp + row] = ex;
    }
  }
  // pass 2: digits of 8 consecutive K' entries per thread, one 16-byte store per plane
  const int Kh = REAL ? K2p : K2p / 2;  // start of the second half of K' (complex)
  const int nks = K2p / OZ_BK;
  const size_t plane_bytes = (size_t)(Rp / TR) * nks * TB;
  unsigned char* pl0 = (unsigned char*)planes + (size_t)p * S * plane_bytes;
  if (IS_B && !REAL) {
    // 8-groups g of the first half: own row at K' = 8 g, the partner row (same complex
    // column, other part) at K' = Kh + 8 g; both rows lie in the same plane tile
    const int ng = Kh / 8;
    const int prow = row ^ 1;
    unsigned char* rb0 = pl0 + (size_t)(row / TR) * nks * TB;
    const bool cj = X.conj != 0;
    // lane h = 0: Re b' = Re b to both rows; h = 1: Im b' = (cj ? -1 : 1) Im b to its own row
    // and its negation to the partner's second half
    const bool neg = h == 1 && cj;
    const uint32_t pflip = h == 1 ? 0x80008000u : 0u;  // bf16 sign bits (a zero becomes -0)
    for (int g = 2 * warp + kh; g < ng; g += 16) {
      uint32_t pk[S][4];
#pragma unroll
      for (int s2 = 0; s2 < S; ++s2) pk[s2][0] = pk[s2][1] = pk[s2][2] = pk[s2][3] = 0u;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int k = 8 * g + e;
        double v = 0.0;
        if (live && k < K) {
          const z64 z = ((const z64*)xb)[at(k)];
          v = h ? z.y : z.x;
        }
        const long long q = oz_fixed<S, DB>(v, ex);
        int d[S];
        oz_digits<S, DB>(neg ? -q : q, d);
#pragma unroll
        for (int s2 = 0; s2 < S; ++s2) pk[s2][e >> 1] |= oz_bf16_bits(d[s2], SCALE0 - DB * s2) << (16 * (e & 1));
      }
      const int g2 = ng + g;
      unsigned char* own = rb0 + (size_t)(g >> 1) * TB + oz_tile_off(row % TR, (g & 1) * 8);
      unsigned char* par = rb0 + (size_t)(g2 >> 1) * TB + oz_tile_off(prow % TR, (g2 & 1) * 8);
#pragma unroll
      for (int s2 = 0; s2 < S; ++s2) {
        *(uint4*)(own + (size_t)s2 * plane_bytes) = make_uint4(pk[s2][0], pk[s2][1], pk[s2][2], pk[s2][3]);
        *(uint4*)(par + (size_t)s2 * plane_bytes) =
            make_uint4(pk[s2][0] ^ pflip, pk[s2][1] ^ pflip, pk[s2][2] ^ pflip, pk[s2][3] ^ pflip);
      }
    }
    return;
  }
  unsigned char* base = pl0 + (size_t)(row / TR) * nks * TB + oz_tile_off(row % TR, kh * 8);
  for (int c = warp; c < nks; c += 8) {
    uint32_t pk[S][4];
#pragma unroll
    for (int s = 0; s < S; ++s) pk[s][0] = pk[s][1] = pk[s][2] = pk[s][3] = 0u;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int kk = c * OZ_BK + kh * 8 + e;
      double v = 0.0;
      bool neg = false;  // negations are applied to the exact integer, not as FP64 instructions
      if (REAL) {
        if (live && kk < K) v = ((const double*)xb)[at(kk)];
      } else {  // A' = [Re op(A) | Im op(A)], the second half from K' = Kh on
        const bool hi = kk >= Kh;
        const int k = hi ? kk - Kh : kk;
        if (live && k < K) {
          const z64 z = ((const z64*)xb)[at(k)];
          v = hi ? z.y : z.x;
          neg = hi && X.conj != 0;  // conj: Im z enters with the opposite sign
        }
      }
      const long long q = oz_fixed<S, DB>(v, ex);
      int d[S];
      oz_digits<S, DB>(neg ? -q : q, d);
#pragma unroll
      for (int s = 0; s < S; ++s) pk[s][e >> 1] |= oz_bf16_bits(d[s], SCALE0 - DB * s) << (16 * (e & 1));
    }
#pragma unroll
    for (int s = 0; s < S; ++s)
      *(uint4*)(base + (size_t)s * plane_bytes + (size_t)c * TB) = make_uint4(pk[s][0], pk[s][1], pk[s][2], pk[s][3]);
  }
}

// ---------------------------------------------------------------------------- tensor kernel
// instruction descriptor for N = nn output columns (a multiple of 16, <= 256)
__device__ __forceinline__ uint32_t oz_idesc(int nn) {
  return (OZ_IDESC & ~(0x3Fu << 17)) | ((uint32_t)(nn >> 3) << 17);
}

__device__ __forceinline__ void oz_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
               "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
               :: "r"(dtmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

// A bound below OZ_PROBE_CYCLES makes the wait one non-blocking test (try_wait may suspend
// the thread for a while on its own, so a short bound would otherwise expire or not
// depending on that suspension).
constexpr long long OZ_PROBE_CYCLES = 1024;

__device__ __forceinline__ bool oz_wait(uint64_t* mbar, uint32_t parity, long long limit = OZ_WAIT_CYCLES) {
  if (limit < OZ_PROBE_CYCLES) {
    uint32_t ok;
    asm volatile("{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(smem_u32(mbar)), "r"(parity));
    return ok != 0;
  }
  const long long t0 = clock64();
  while (true) {
    uint32_t ok;
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(smem_u32(mbar)), "r"(parity));
    if (ok) return true;
    if (clock64() - t0 > limit) return false;
  }
}

__device__ __forceinline__ void oz_expect_tx(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(smem_u32(mbar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void oz_bulk_copy(void* dst_smem, const void* src_gmem, uint32_t bytes, uint64_t* mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               :: "r"(smem_u32(dst_smem)), "l"(src_gmem), "r"(bytes), "r"(smem_u32(mbar)) : "memory");
}

// Warp-specialised pipeline over OZ_STAGES shared-memory stages:
//   warp 0 / lane 0 (producer): waits until a stage is free (its "empty" barrier, arrived
//     by the MMA commit), then loads it with 20 bulk copies (cp.async.bulk, the 1-D TMA)
//     that complete on the stage's "full" barrier;
//   warp 1 / lane 0 (MMA issuer): waits for a full stage, issues the MMAs of its digit products, commits them
//     to the stage's empty barrier, and after the last stage to the "done" barrier;
//   all 8 warps: wait for "done", then run the epilogue from TMEM.
template <bool REAL, int S, int DB, int BN, int NST>
__global__ void __launch_bounds__(OZ_THREADS, BN == OZ_BN ? 1 : 2)
oz_gemm_kernel(int nprob, GemmDims dims, double alpha, double beta, const __nv_bfloat16* __restrict__ Ap,
               const __nv_bfloat16* __restrict__ Bp, const int* __restrict__ rexp, const int* __restrict__ cexp, int Mp,
               int N2p, int K2p, void* __restrict__ Cv, long long Cbs, long long Crs, long long Ccs, int* __restrict__ err) {
  // Accumulator a holds the digit group s + t = a (0-based; G_a = n_a 2^{30 - DB a}), the last
  // one also every group beyond it (MERGED).  The first NEX accumulators are combined exactly
  // (their FP32 sums are exact integers: DB = 6 while 2K' <= 1792, DB = 7 while K' <= 512);
  // the rest lie at least 2^-35 below the first group and enter rounded.
  constexpr int NACC = S < 8 ? S : 8;
  constexpr bool MERGED = S > NACC;
  constexpr int NEX = DB == 7 ? 6 : (MERGED ? NACC - 1 : NACC);
  constexpr int TMEM_COLS = NACC * BN <= 128 ? 128 : (NACC * BN <= 256 ? 256 : 512);
  constexpr int TILE_B = BN * OZ_BK * 2;              // bytes of one B tile in shared memory
  constexpr int STAGE = S * (OZ_TILE_A + TILE_B);     // bytes per pipeline stage
  constexpr int kUnitExp = DB * (NEX - 1) - 30;       // an accumulator's value in units of the last exact
                                                      // group: v 2^kUnitExp
  constexpr int kExp = -DB * (NEX + 1);               // the output is t 2^{e_i + f_j + kExp}
  extern __shared__ __align__(1024) unsigned char oz_smem[];
  __shared__ uint64_t full_bar[NST], empty_bar[NST], done_bar;
  __shared__ uint32_t tbase;
  __shared__ volatile int s_fail;
  __shared__ int s_issued;
  const int p = blockIdx.z;
  const int rb = blockIdx.y, cb = blockIdx.x;
  const int M = dims.Mp ? dims.Mp[p] : dims.M;
  const int N = dims.Np ? dims.Np[p] : dims.N;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // uniform early exits (before any barrier or allocation)
  const int CPT = REAL ? BN : BN / 2;  // output columns per tile
  if (rb * OZ_BM >= M || cb * CPT >= N) return;
  if (dims.lower && cb * CPT > rb * OZ_BM + OZ_BM - 1) return;
  unsigned char* stage0 = (unsigned char*)(((uintptr_t)oz_smem + 1023) & ~(uintptr_t)1023);
  const int nks = K2p / OZ_BK;  // plane layout (all problems)
  // this problem's digit planes hold data in the K steps [0, s1) and (complex) [s2a, s2b), the
  // second half K2p / 2 .. K2p / 2 + K_p; the loop runs over those steps only (one range when
  // they meet, as for K_p = K)
  const int Kprob = gemm_k(dims, p);
  int s1 = min(nks, (Kprob + OZ_BK - 1) / OZ_BK), s2a = s1, s2b = s1;
  if (!REAL) {
    s2a = (K2p / 2) / OZ_BK;
    s2b = min(nks, (K2p / 2 + Kprob + OZ_BK - 1) / OZ_BK);
    if (s2a <= s1) s1 = s2a = s2b;
  }
  const int nks_p = max(1, s1 + (s2b - s2a));
  const size_t aplane = (size_t)(Mp / OZ_BM) * nks * (OZ_TILE_A / 2);
  const size_t bplane = (size_t)(N2p / OZ_BN) * nks * (OZ_TILE_B / 2);
  const unsigned char* Abase = (const unsigned char*)(Ap + (size_t)p * S * aplane) + (size_t)rb * nks * OZ_TILE_A;
  // B rows cb BN .. +BN-1: plane tile (cb BN) / 64, from its row (cb BN) % 64 on (contiguous)
  const unsigned char* Bbase = (const unsigned char*)(Bp + (size_t)p * S * bplane) +
                               (size_t)((cb * BN) / OZ_BN) * nks * OZ_TILE_B + (((cb * BN) % OZ_BN) >> 3) * 256;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tbase)), "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    s_fail = 0;
    s_issued = 0;
    for (int st = 0; st < NST; ++st) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&full_bar[st])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&empty_bar[st])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&done_bar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tbase;

  // the pipeline's waits take the context's bound (nao_config.tc_wait_cycles); the wait for
  // the issued MMAs and the drain of issued copies after a failure keep the fixed long bound,
  // so that no copy or MMA is still in flight when the block frees its memory
  long long wait_lim = err ? *(const volatile long long*)(err + NAO_FLAG_WAIT) : OZ_WAIT_CYCLES;
  if (wait_lim <= 0) wait_lim = OZ_WAIT_CYCLES;
  if (warp == 0 && lane == 0) {
    // ---------------- producer
    int ks = 0;
    for (; ks < nks_p; ++ks) {
      const int st = ks % NST;
      if (ks >= NST && !oz_wait(&empty_bar[st], ((ks / NST) - 1) & 1, wait_lim)) {
        s_fail = 1;
        break;
      }
      if (s_fail) break;
      const int kst = ks < s1 ? ks : s2a + (ks - s1);  // K step of the planes
      unsigned char* sdst = stage0 + st * STAGE;
      oz_expect_tx(&full_bar[st], STAGE);
#pragma unroll
      for (int s = 0; s < S; ++s)
        oz_bulk_copy(sdst + s * OZ_TILE_A, Abase + (size_t)s * aplane * 2 + (size_t)kst * OZ_TILE_A, OZ_TILE_A,
                     &full_bar[st]);
#pragma unroll
      for (int t = 0; t < S; ++t)
        oz_bulk_copy(sdst + S * OZ_TILE_A + t * TILE_B, Bbase + (size_t)t * bplane * 2 + (size_t)kst * OZ_TILE_B,
                     TILE_B, &full_bar[st]);
    }
    s_issued = ks;
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    uint32_t init_mask = 0;  // accumulators written at least once
    int ks = 0;
    for (; ks < nks_p; ++ks) {
      const int st = ks % NST;
      if (!oz_wait(&full_bar[st], (ks / NST) & 1, wait_lim)) {
        s_fail = 1;
        break;
      }
      if (s_fail) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      unsigned char* ssrc = stage0 + st * STAGE;
      const uint32_t sa = smem_u32(ssrc), sb = smem_u32(ssrc + S * OZ_TILE_A);
      // Digit products A_s B_t (0-based, s + t <= S - 1) into accumulator min(s + t, NACC - 1).
      // The accumulators are adjacent and so are the B planes, so for each s the planes
      // t = 0 .. NACC - 1 - s stack into one operand of BN w rows: one MMA with N = BN w
      // (<= 256) feeds w accumulators (the last one the merged groups' first product) and
      // reads A_s from shared memory once instead of w times.  The merged groups' other
      // products take one N = BN MMA each.  A window's accumulators are all fresh or all
      // written (s = 0 writes all of them first), so one accumulate flag serves it.
      constexpr int WMAX = 256 / BN;
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const uint64_t ad = oz_desc(sa + s * OZ_TILE_A);
        const int tlast = min(NACC - 1 - s, S - 1 - s);  // last t of the window (< 0: none)
#pragma unroll
        for (int t0 = 0; t0 <= tlast; t0 += WMAX) {
          const int w = min(WMAX, tlast - t0 + 1), acc0 = s + t0;
          const uint32_t on = (init_mask >> acc0) & 1u;
          oz_mma(tmem + acc0 * BN, ad, oz_desc(sb + t0 * TILE_B), oz_idesc(w * BN), on);
          init_mask |= ((1u << w) - 1u) << acc0;
        }
        if (MERGED) {
#pragma unroll
          for (int t = (tlast + 1 > 0 ? tlast + 1 : 0); t < S && s + t <= S - 1; ++t) {
            const uint32_t on = (init_mask >> (NACC - 1)) & 1u;
            oz_mma(tmem + (NACC - 1) * BN, ad, oz_desc(sb + t * TILE_B), oz_idesc(BN), on);
            init_mask |= 1u << (NACC - 1);
          }
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   :: "r"(smem_u32(&empty_bar[st])));
    }
    // "done" arrives when every MMA issued above has completed (also after a failure)
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_u32(&done_bar)));
  }
  // everyone: wait for the MMAs (bounded), then the epilogue
  const bool done_ok = oz_wait(&done_bar, 0);
  if (!done_ok && tid == 0) s_fail = 1;
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (s_fail) {
    if (tid == 0) {
      atomicExch(err + NAO_FLAG_TIMEOUT, 1);
      // let every bulk copy that was issued land before the block (and its shared memory) goes
      const int issued = s_issued;
      for (int ks = (issued > NST ? issued - NST : 0); ks < issued; ++ks)
        oz_wait(&full_bar[ks % NST], (ks / NST) & 1);
    }
  } else {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 (tile rows); warps 0-3 take
    // complex columns 0..15 of the tile, warps 4-7 columns 16..31.
    const int row = 32 * (warp & 3) + lane;
    const int gi = rb * OZ_BM + row;
    const int half = warp >> 2;
    const int erow = (gi < M) ? rexp[(size_t)p * Mp + gi] : 0;
    // alpha = +-2^ae goes into the exponent; any other alpha takes one FP64 multiply
    const long long abits = __double_as_longlong(alpha);
    const int afield = (int)((abits >> 52) & 0x7ff);
    const bool amul = (abits & 0xFFFFFFFFFFFFFll) != 0 || afield == 0 || afield == 0x7ff;
    const int ae = amul ? 0 : afield - 1023;
    const bool aneg = !amul && abits < 0;
    for (int cc = 0; cc < BN / 4; cc += 4) {  // 8 C'' columns per round
      const int col0 = half * (BN / 2) + 2 * cc;
      uint32_t v[NACC][8];
#pragma unroll
      for (int a = 0; a < NACC; ++a) {
        const uint32_t taddr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + a * BN + col0;
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(v[a][0]), "=r"(v[a][1]), "=r"(v[a][2]), "=r"(v[a][3]), "=r"(v[a][4]), "=r"(v[a][5]),
                       "=r"(v[a][6]), "=r"(v[a][7])
                     : "r"(taddr));
      }
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (gi >= M) continue;
      // every output as one fixed-point integer t (value t 2^{e_i + f_j + kExp - sh}), turned
      // into a double by integer operations: no FP64 instruction unless beta != 0
      long long t[8];
      int sh[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        // exact groups a < NEX: G_a = n_a 2^{30 - DB a} with integer n_a;
        // hi = sum_a n_a 2^{DB (NEX - 1 - a)} counts in units of the last exact group
        long long hi = 0;
#pragma unroll
        for (int a = 0; a < NEX; ++a) {
          const float gv = __uint_as_float(v[a][c]);
          const long long ng = (long long)__float2int_rn(ldexpf(gv, DB * a - 30));
          hi += ng * (1ll << (DB * (NEX - 1 - a)));
        }
        if (NEX < NACC) {
          // |hi| < 2^59; shift it up to just below 2^60 and add the other accumulators
          // (|.| < 2^18 in units of 1) rounded to the new unit, which stays below 2^62
          const unsigned long long ah = hi < 0 ? 0ull - (unsigned long long)hi : (unsigned long long)hi;
          const int s = min(max(__clzll((long long)ah) - 4, 0), 40);
          long long tt = (long long)((unsigned long long)hi << s);
#pragma unroll
          for (int a = NEX; a < NACC; ++a) tt += oz_f32_fixed(__uint_as_float(v[a][c]), s + kUnitExp);
          t[c] = tt;
          sh[c] = s;
        } else {
          t[c] = hi;
          sh[c] = 0;
        }
      }
      if (REAL) {
        double* Cp = (double*)Cv + (size_t)p * Cbs;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int gj = cb * BN + col0 + c;
          if (gj >= N) continue;
          const int ex = erow + cexp[(size_t)p * N2p + gj] + kExp + ae;
          double* cp = Cp + (long long)gi * Crs + (long long)gj * Ccs;
          double r = fix_to_double(t[c], ex - sh[c], aneg);
          if (amul) r *= alpha;
          if (beta != 0.0) r = fma(beta, *cp, r);
          *cp = r;
        }
      } else {
        z64* Cp = (z64*)Cv + (size_t)p * Cbs;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int gj = cb * (BN / 2) + half * (BN / 4) + cc + q;  // complex column
          if (gj >= N) continue;
          const int ex = erow + cexp[(size_t)p * (N2p / 2) + gj] + kExp + ae;
          z64* cp = Cp + (long long)gi * Crs + (long long)gj * Ccs;
          z64 r = zmk(fix_to_double(t[2 * q], ex - sh[2 * q], aneg),
                      fix_to_double(t[2 * q + 1], ex - sh[2 * q + 1], aneg));
          if (amul) {
            r.x *= alpha;
            r.y *= alpha;
          }
          if (beta != 0.0) {
            const z64 old = *cp;
            r.x = fma(beta, old.x, r.x);
            r.y = fma(beta, old.y, r.y);
          }
          *cp = r;
        }
      }
    }
  }
  __syncthreads();
  asm volatile("tcgen05.fence::before_thread_sync;");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TMEM_COLS));
}

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Split both operands into S digit planes of DB bits and run the tensor kernel.  The plane
// buffers are laid out for OZ_S planes (the workspace size), whatever S is used.  Base-128
// digits (DB = 7) always take the 32-column tiles: their contractions are at most 32 K steps.
template <bool REAL, int S, int DB>
cudaError_t launch_oz(int nprob, GemmDims dims, double alpha, GemmOperand A, GemmOperand B, double beta, void* C,
                      long long Cbs, long long Crs, long long Ccs, void* ws, int* err, cudaStream_t st) {
  if (nprob <= 0 || dims.M <= 0 || dims.N <= 0) return cudaSuccess;
  const int w2 = REAL ? 1 : 2;
  const int Mp = round_up(dims.M, OZ_BM), N2p = round_up(w2 * dims.N, OZ_BN), K2p = round_up(w2 * dims.K, OZ_BK);
  unsigned char* w = (unsigned char*)ws;
  __nv_bfloat16* Apl = (__nv_bfloat16*)w;
  w += (size_t)nprob * OZ_S * Mp * K2p * 2;
  __nv_bfloat16* Bpl = (__nv_bfloat16*)w;
  w += (size_t)nprob * OZ_S * N2p * K2p * 2;
  int* rexp = (int*)w;
  int* cexp = rexp + (size_t)nprob * Mp;
  oz_split<false, REAL, S, DB><<<dim3(Mp / 16, nprob), 256, 0, st>>>(nprob, dims, A, Mp, K2p, Apl, rexp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  oz_split<true, REAL, S, DB><<<dim3(N2p / 16, nprob), 256, 0, st>>>(nprob, dims, B, N2p, K2p, Bpl, cexp);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (DB == 7 || K2p / OZ_BK <= OZ_SHORT_KSTEPS) {
    constexpr int BN = OZ_BN / 2, NST = 2;
    const size_t smem = NST * (size_t)S * (OZ_TILE_A + BN * OZ_BK * 2) + 1024;
    e = cudaFuncSetAttribute(oz_gemm_kernel<REAL, S, DB, BN, NST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(N2p / BN, Mp / OZ_BM, nprob);
    oz_gemm_kernel<REAL, S, DB, BN, NST><<<grid, OZ_THREADS, smem, st>>>(nprob, dims, alpha, beta, Apl, Bpl, rexp,
                                                                         cexp, Mp, N2p, K2p, C, Cbs, Crs, Ccs, err);
    return cudaGetLastError();
  }
  if constexpr (DB == 6) {
    const size_t smem = OZ_STAGES * (size_t)S * (OZ_TILE_A + OZ_TILE_B) + 1024;
    e = cudaFuncSetAttribute(oz_gemm_kernel<REAL, S, DB, OZ_BN, OZ_STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(N2p / OZ_BN, Mp / OZ_BM, nprob);
    oz_gemm_kernel<REAL, S, DB, OZ_BN, OZ_STAGES><<<grid, OZ_THREADS, smem, st>>>(
        nprob, dims, alpha, beta, Apl, Bpl, rexp, cexp, Mp, N2p, K2p, C, Cbs, Crs, Ccs, err);
  }
  return cudaGetLastError();
}

// Longest contraction of one exact chunk: base-64 digits 2K' <= OZ_MAX_K2 (complex) or
// K' <= OZ_MAX_K2 (real); base-128 digits K' <= 512.
constexpr int OZ_CHUNK_C = OZ_MAX_K2 / 2, OZ_CHUNK_R = OZ_MAX_K2;
constexpr int OZ7_CHUNK_C = 256, OZ7_CHUNK_R = 512;

// Products longer than one chunk: C = alpha sum_c op(A)(:, c) op(B)(c, :) + beta C, every
// chunk FP64-accurate, the sum accumulated in FP64 through beta = 1.  digits: 5, 6, 7 or 10
// base-64 planes, or NAO_OZ_DIGITS_B128 (nine base-128 planes, 63 bits).
template <bool REAL>
cudaError_t launch_oz_chunked(int nprob, GemmDims dims, double alpha, GemmOperand A, GemmOperand B, double beta,
                              void* C, long long Cbs, long long Crs, long long Ccs, void* ws, int* err,
                              cudaStream_t st, int digits) {
  // FP64-accurate contractions that fit one base-128 chunk take the nine base-128 planes: as
  // accurate (63 bits) and fewer, wider MMAs
  if (digits == NAO_OZ_DIGITS_FP64 && dims.K <= (REAL ? OZ7_CHUNK_R : OZ7_CHUNK_C)) digits = NAO_OZ_DIGITS_B128;
  const bool b128 = digits == NAO_OZ_DIGITS_B128;
  const int chunk = b128 ? (REAL ? OZ7_CHUNK_R : OZ7_CHUNK_C) : (REAL ? OZ_CHUNK_R : OZ_CHUNK_C);
  const size_t esz = REAL ? sizeof(double) : sizeof(z64);
  for (int k0 = 0; k0 < dims.K || k0 == 0; k0 += chunk) {
    GemmDims d = dims;
    d.K = dims.K - k0 < chunk ? dims.K - k0 : chunk;
    d.k0 = dims.k0 + k0;
    GemmOperand a = A, b = B;
    a.ptr = (const char*)A.ptr + (long long)k0 * A.cs * (long long)esz;  // op(A)(i, k) at i rs + k cs
    b.ptr = (const char*)B.ptr + (long long)k0 * B.rs * (long long)esz;  // op(B)(k, j) at k rs + j cs
    const double bt = k0 == 0 ? beta : 1.0;
    cudaError_t e;
    switch (digits) {
      case 5: e = launch_oz<REAL, 5, 6>(nprob, d, alpha, a, b, bt, C, Cbs, Crs, Ccs, ws, err, st); break;
      case 6: e = launch_oz<REAL, 6, 6>(nprob, d, alpha, a, b, bt, C, Cbs, Crs, Ccs, ws, err, st); break;
      case 7: e = launch_oz<REAL, 7, 6>(nprob, d, alpha, a, b, bt, C, Cbs, Crs, Ccs, ws, err, st); break;
      case OZ_S: e = launch_oz<REAL, OZ_S, 6>(nprob, d, alpha, a, b, bt, C, Cbs, Crs, Ccs, ws, err, st); break;
      case NAO_OZ_DIGITS_B128: e = launch_oz<REAL, 9, 7>(nprob, d, alpha, a, b, bt, C, Cbs, Crs, Ccs, ws, err, st); break;
      default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    if (dims.K <= chunk) break;
  }
  return cudaSuccess;
}

}  // namespace

bool zgemm_oz_supported(GemmDims dims) { return dims.M > 0 && dims.N > 0 && dims.K > 0; }

size_t zgemm_oz_workspace(int nprob, GemmDims dims) {
  const int Kc = dims.K < OZ_CHUNK_C ? dims.K : OZ_CHUNK_C;
  const int Mp = round_up(dims.M, OZ_BM), N2p = round_up(2 * dims.N, OZ_BN), K2p = round_up(2 * Kc, OZ_BK);
  const size_t a = (size_t)nprob * OZ_S * Mp * K2p * 2, b = (size_t)nprob * OZ_S * N2p * K2p * 2;
  return a + b + (size_t)nprob * (Mp + N2p) * sizeof(int) + 4096;
}

cudaError_t launch_zgemm_oz(int nprob, GemmDims dims, double alpha, GemmOperand A, GemmOperand B, double beta, z64* C,
                            long long Cbs, long long Crs, long long Ccs, void* ws, int* err, cudaStream_t st,
                            int digits) {
  return launch_oz_chunked<false>(nprob, dims, alpha, A, B, beta, (void*)C, Cbs, Crs, Ccs, ws, err, st, digits);
}

bool dgemm_oz_supported(GemmDims dims) { return dims.M > 0 && dims.N > 0 && dims.K > 0; }

size_t dgemm_oz_workspace(int nprob, GemmDims dims) {
  const int Kc = dims.K < OZ_CHUNK_R ? dims.K : OZ_CHUNK_R;
  const int Mp = round_up(dims.M, OZ_BM), Np = round_up(dims.N, OZ_BN), Kp = round_up(Kc, OZ_BK);
  return (size_t)nprob * OZ_S * ((size_t)Mp + Np) * Kp * 2 + (size_t)nprob * ((size_t)Mp + Np) * sizeof(int) + 4096;
}

cudaError_t launch_dgemm_oz(int nprob, GemmDims dims, double alpha, GemmOperand A, GemmOperand B, double beta, double* C,
                            long long Cbs, long long Crs, long long Ccs, void* ws, int* err, cudaStream_t st,
                            int digits) {
  return launch_oz_chunked<true>(nprob, dims, alpha, A, B, beta, (void*)C, Cbs, Crs, Ccs, ws, err, st, digits);
}
