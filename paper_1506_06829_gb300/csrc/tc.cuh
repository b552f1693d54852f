// FP64 block combinations Y = beta Y + sum_t alpha_t X_t C_t and Gram products C = X^* Y on
// GB300's tensor cores (tcgen05, bf16 operands, FP32 accumulators in tensor memory),
// accurate to FP64 working precision by splitting every double into small integer digits.
//
// Scheme (per tile of 128 rows; K' = 2 sum w_t real columns, N' = 2 c real columns):
// * complex to real: a row of [X_0 X_1 ...] is the K' doubles (Re, Im, Re, Im, ...),
//   C' (K' x N') = [[Re c, Im c], [-Im c, Re c]] per complex entry, so Y' = X' C' is the
//   interleaved complex result;
// * row r of X' shares one exponent bound T_r (every |x| < 2^(T_r + 1)); each x becomes
//   the integer S = round(x 2^(54 - T_r)), |S| <= 2^55, written in 7 balanced base-256
//   digits, S = sum_{a=0..6} s_a 256^(6 - a) with s_1..s_6 in [-128, 127] and
//   |s_0| <= 128 (exact in bf16); column n of C' likewise with its bound G_n;
// * the tensor core forms the digit diagonals D_d = sum_{a + b = d} X'_a C'_b for
//   d = 0..7 (34 digit-pair products).  The 7 digit planes of C' and a zero plane are
//   stacked along N, so one MMA of X'_a against planes b = 0..7-a, written at accumulator
//   column a N', lands each product X'_a C'_b on diagonal a + b: 7 MMAs per K step (N
//   split at 256).  |s_a s_b| <= 2^14, at most 7 pairs per diagonal and K' <= 64, so
//   |D_d| < 7 2^20: every FP32 partial sum is an exact integer;
// * y = 2^(T_r + G_n - 68) Z, Z = sum_d D_d 256^(7 - d) formed exactly in 96-bit
//   integer arithmetic and rounded once to double (nearest, ties to even).
// The Gram products C = X^* Y use the same digits with the contraction over the rows (per-
// column exponent bounds over 128-row windows); see the Gram kernels below.
//
// Kernels in this file, all persistent with one (or two) CTAs per SM and every wait on an
// mbarrier bounded:
// * tc_combine_kernel<K'/8, CTAs per SM>: the combination, digit warps + epilogue warps;
// * tc_gram_narrow_kernel<tasks>: Gram products of narrow blocks (digit planes stacked
//   along M and N, exact integer diagonal sums in shared memory), with an MMA-issue warp;
// * tc_gram_wide_kernel: wider Gram products (the combination's layout, diagonals formed
//   by the MMA), with an MMA-issue warp;
// * tc_gram_kernel: the first, serial Gram form, for X up to 128 columns.
// Error per output: input rounding <= 2^-55 (max_k |x_rk| sum_k |c_kn| + K' max_k |x_rk|
// max_k |c_kn|), the dropped pairs a + b >= 8 (weight <= 2^-62 K' 2^(T_r + G_n) in all),
// and the final rounding: at most (K'/4 + 2) u max_k |x_rk| sum_k |c_kn| with u = 2^-53.
// This bound is the scheme's own: it is not ordered against the classical bound
// K' u sum_k |x_rk| |c_kn| of a DFMA dot product, which is the smaller one when a row's
// entries span decades.  Results below 2^-1022 (subnormal) take a second rounding.
#pragma once
#include <climits>
#include <cstdint>

namespace gplhr {

// ------------------------------------------------------------- tcgen05 PTX --
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory operand descriptor, K-major without swizzle: core matrices of 8 rows x
// 16 bytes stored as 128 contiguous bytes; lbo = byte step between cores along K, sbo =
// between cores along M (or N).
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}
// Instruction descriptor, kind::f16: bf16 A and B (both K-major), f32 accumulator, M x N.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                          int accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
               : "memory");
}
// One test of the phase; a thread whose phase is not complete sleeps until it completes
// or for at most TC_WAIT_NS (it does not spin and take issue slots from working warps).
constexpr uint32_t TC_WAIT_NS = 20000;
constexpr int TC_WAIT_TRIES = 1 << 16;  // at most ~1.3 s in all
__device__ __forceinline__ bool mbar_try_wait(uint64_t* mbar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_u32(mbar)), "r"(parity), "r"(TC_WAIT_NS)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&r)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ------------------------------------------------------------ digit algebra --
constexpr int TC_DIGITS = 7;     // balanced base-256 digits of a 55-bit integer
constexpr int TC_DIAG = 8;       // accumulated digit diagonals a + b = 0..7
constexpr int TC_ROWS = 128;     // rows per tile = tensor-memory lanes (M)
constexpr int TC_KMAX = 64;      // K' per tile (complex inputs: 32 columns)
constexpr int TC_NMAX = 64;      // N' (complex outputs: 32 columns)
constexpr int TC_NOEXP = -100000;

// Exponent bound of a double: |v| < 2^(e + 1) with e = ee + 52, |v| = M 2^ee; the
// largest finite bound for Inf / NaN (their rows and columns come out as NaN).
__device__ __forceinline__ int tc_top(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int eb = (int)((b >> 52) & 0x7FF);
  if ((b << 1) == 0) return TC_NOEXP;
  return (eb ? eb - 1075 : -1074) + 52;
}
__device__ __forceinline__ bool tc_nonfinite(double v) {
  return (((unsigned long long)__double_as_longlong(v) >> 52) & 0x7FF) == 0x7FF;
}

// The digits of v against the exponent bound T (T >= tc_top(v)) as floats holding small
// integers: F = round(|v| 2^(54 - T)) < 2^55 (half up); F + 0x808080808080 carries the
// balancing, so digit a >= 1 is byte (6 - a) of that sum minus 128 and digit 0 its
// bits 48..55; every digit takes v's sign.
__device__ __forceinline__ void tc_digits(double v, int T, float (&f)[TC_DIGITS]) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int eb = (int)((b >> 52) & 0x7FF);
  const unsigned long long M =
      eb == 0x7FF ? 0ull : ((b & 0x000FFFFFFFFFFFFFull) | (eb ? (1ull << 52) : 0ull));
  const int sh = (eb ? eb - 1075 : -1074) + 54 - T;  // <= 2
  unsigned long long F = 0;
  if (sh >= 0)
    F = M << (sh & 3);
  else if (sh > -60)
    F = (M + (1ull << (-sh - 1))) >> (-sh);
  const unsigned long long S = F + 0x0000808080808080ull;
  const uint32_t lo = (uint32_t)S, hi = (uint32_t)(S >> 32);
  const float sg = (b >> 63) ? -1.0f : 1.0f;
  // 0x4B0000xx as a float is 2^23 + xx; sg (2^23 + xx) - sg (2^23 + 128) is exact
  const float m0 = sg * 8388608.0f, m1 = sg * 8388736.0f;
  f[0] = fmaf(sg, __uint_as_float(__byte_perm(hi, 0x4B000000u, 0x7442)), -m0);
  f[1] = fmaf(sg, __uint_as_float(__byte_perm(hi, 0x4B000000u, 0x7441)), -m1);
  f[2] = fmaf(sg, __uint_as_float(__byte_perm(hi, 0x4B000000u, 0x7440)), -m1);
  f[3] = fmaf(sg, __uint_as_float(__byte_perm(lo, 0x4B000000u, 0x7443)), -m1);
  f[4] = fmaf(sg, __uint_as_float(__byte_perm(lo, 0x4B000000u, 0x7442)), -m1);
  f[5] = fmaf(sg, __uint_as_float(__byte_perm(lo, 0x4B000000u, 0x7441)), -m1);
  f[6] = fmaf(sg, __uint_as_float(__byte_perm(lo, 0x4B000000u, 0x7440)), -m1);
}

// Two bf16 halves packed from floats that hold bf16-exact values (their top 16 bits).
__device__ __forceinline__ uint32_t tc_pack2(float lo, float hi) {
  return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632);
}

// 2^p (hi 2^32 + lo) for |hi|, |lo| < 2^48, rounded once to the nearest double (ties
// to even); a result below 2^-1022 takes a second rounding to the subnormal grid.
// The magnitude (< 2^81) is brought to at most 63 bits: exactly when it is below 2^63,
// else shifted right by s with the dropped bits collapsed into a sticky lowest bit; the
// integer-to-double conversion then rounds once (the sticky bit lies below its rounding
// point), and 2^(s + p) is applied to the exponent field, exactly while it stays normal.
__device__ __forceinline__ double tc_round96(long long hi, long long lo, int p) {
  long long zh = hi + (lo >> 32);  // value = zh 2^32 + zl, zl in [0, 2^32)
  uint32_t zl = (uint32_t)lo;
  const bool neg = zh < 0;
  if (neg) {  // 96-bit negation
    zh = -zh - (zl != 0u ? 1 : 0);
    zl = 0u - zl;
  }
  const uint64_t uh = (uint64_t)zh;  // < 2^49
  uint64_t W;
  int s = 0;
  if (uh < (1ull << 31)) {
    W = (uh << 32) | zl;
  } else {
    s = 33 - __clzll((long long)uh);  // 1..18: the magnitude has 63 + s bits
    W = (uh << (32 - s)) | (zl >> s) | ((zl << (32 - s)) != 0u ? 1ull : 0ull);
  }
  if (W == 0) return 0.0;
  unsigned long long bits = (unsigned long long)__double_as_longlong(__ull2double_rn(W));
  const int e = s + p;
  const int nb = (int)(bits >> 52) + e;  // the result's biased exponent
  if (nb >= 1 && nb <= 2046)
    bits += (unsigned long long)(long long)e << 52;
  else if (nb > 2046)
    bits = 0x7FF0000000000000ull;
  else
    bits = (unsigned long long)__double_as_longlong(scalbn(__longlong_as_double((long long)bits), e));
  return __longlong_as_double((long long)(bits | (neg ? (1ull << 63) : 0ull)));
}

// The eight digit diagonals D_0..D_7 of the combination (FP32 accumulators holding
// integers of magnitude <= 7 2^20, K' <= 64) as Z = hi 2^32 + lo = sum_d D_d 256^(7 - d):
// pairs first in 32 bits (|256 D_2k + D_2k+1| < 2^31), then two 48-bit halves.
// SMALL: |D_d| < 2^22 (K' <= 32), so 1.5 2^23 + D_d is exact in FP32 and its low bits give
// D_d + 2^22 (an FP32 addition and an integer one instead of a conversion).
template <bool SMALL>
__device__ __forceinline__ void tc_diag_sum(const uint32_t (&D)[TC_DIAG], long long& hi, long long& lo) {
  int I[TC_DIAG];
#pragma unroll
  for (int d = 0; d < TC_DIAG; ++d)
    I[d] = SMALL ? __float_as_int(__uint_as_float(D[d]) + 12582912.0f) - 0x4B400000
                 : __float2int_rn(__uint_as_float(D[d]));
  int P[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) P[k] = I[2 * k] * 256 + I[2 * k + 1];
  hi = (long long)P[0] * 65536ll + (long long)P[1];
  lo = (long long)P[2] * 65536ll + (long long)P[3];
}

// Exact integer value of an FP32 accumulator holding an integer of magnitude < 2^24.
__device__ __forceinline__ int tc_f2i(uint32_t u) { return __float2int_rn(__uint_as_float(u)); }

// Named barrier over the first `count` threads of the CTA (barrier 0 is __syncthreads),
// with an AND vote: every participating thread gets the same answer.
__device__ __forceinline__ bool bar_and(int id, int count, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.b32 p, %1, 0;\n bar.red.and.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)pred), "r"(id), "r"(count)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_u32(bar)) : "memory");
}
// Bounded wait for the phase of the given parity: false after `tries` tests, or as soon
// as another role has raised *abort.  The pipeline's waits on other roles take the
// limit from the kernel arguments (a context option lowers it to test the time-out
// path); the final wait for the CTA's own products before tensor memory is freed always
// takes the full TC_WAIT_TRIES.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, volatile int* abort,
                                                  int tries) {
  for (int it = 0; it < tries; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort) return false;
  }
  return false;
}

struct TcCombArgs {
  CombArgs a;
  int kp;          // K' padded to a multiple of 16 (<= TC_KMAX)
  int np;          // N' padded to a multiple of 16 (<= TC_NMAX)
  int ds;          // A digit stages in shared memory (1 or 2)
  int ts;          // accumulator buffers in tensor memory (1 or 2)
  int tmem_cols;   // power of two >= max(32, ts TC_DIAG np)
  int* err;        // set to 1 if a wait gave up
  int wait_tries;    // limit of the pipeline's mbarrier waits (tests lower it)
  int probe;         // test hook: the epilogue also waits on a barrier nothing completes
};

__host__ __device__ constexpr size_t tc_comb_smem_bytes(int kp, int np, int ds) {
  return (size_t)ds * TC_DIGITS * TC_ROWS * kp * 2 + (size_t)TC_DIAG * np * kp * 2;
}

__device__ __forceinline__ int tc_off(int row, int k, int KC) {  // element offset in a core-matrix tile
  return ((row >> 3) * KC + (k >> 3)) * 64 + (row & 7) * 8 + (k & 7);
}

// The value of C' at (kk, nn): stacked alpha_t C_t (staged in shared memory as sCv[j c + l]),
// complex entries as 2 x 2 real blocks.
__device__ __forceinline__ double tc_cval(const double2* sCv, int wsum, int c, int kk, int nn) {
  const int j = kk >> 1, p = kk & 1, l = nn >> 1, q = nn & 1;
  if (j >= wsum || l >= c) return 0.0;
  const double2 cv = sCv[j * c + l];
  return p == 0 ? (q == 0 ? cv.x : cv.y) : (q == 0 ? -cv.y : cv.x);
}

// The combination as a pipeline of two roles in one persistent CTA per SM, so that the
// loads and digit splitting of one tile, the MMAs of the tile before and the epilogue of
// the one before that run at the same time (tile i uses A stage i % ds and accumulator
// buffer i % ts; mbarriers pass the stages and buffers between the roles):
// * warps 0-7 (digits): thread (row, half) = (tid % 128, tid / 128) loads the row's
//   k-chunks kc = half, half + 2, ... (4 complex values each); the two halves agree on
//   the row's exponent bound (named barrier 1); once the stage is free the row's digits
//   are written to it, 8 consecutive k of one digit per 16-byte store.  When all are
//   written, thread 0 waits for the buffer to be free and issues the MMAs: plane da of
//   X' against C' planes 0 .. 7 - da (stack rows 0 .. (8 - da) np) at accumulator
//   column da np; the first MMA (ks = 0, da = 0, all 8 planes) initialises every
//   diagonal; commits free the stage and fill the buffer;
// * warps 8-15 (epilogue): warp 8 + 4 e + q reads tensor-memory lanes 32 q .. 32 q + 31
//   (rows 32 q .. of the tile) and the column groups nb = 4 e, 4 e + 8, ...; it forms,
//   rounds and stores those outputs, then frees the buffer.
// 16 warps, so that every SM sub-partition holds 4 of them and each thread may use 128
// registers.  The row exponent bounds and non-finite flags go through a ring of TC_RING
// slots (a slot is rewritten only after its tile's buffer was freed: TC_RING >= ds + ts).
// Every wait has an iteration limit; a role that gives up raises the abort flag, which
// ends the other role's waits; thread 0 waits (bounded) for its last products, and the CTA
// frees its tensor memory and returns with *err = 1.
constexpr int TC_DWARPS = 8, TC_EWARPS = 8;
constexpr int TC_PIPE_THREADS = (TC_DWARPS + TC_EWARPS) * 32;
constexpr int TC_RING = 4;

// Thread (row r, half h)'s k-chunks kc = h, h + 2, ... of the stacked row: 4 complex
// values each, as (Re, Im) pairs; zeros when the row is not valid or the column is padding.
template <int KC>
__device__ __forceinline__ void tc_row_load(const double2* const* colp, const int* coll, int wsum, bool valid, int r,
                                            int h, double (&xv)[4 * KC]) {
#pragma unroll
  for (int i = 0; i < KC / 2; ++i) {
    const int kc = 2 * i + h;
#pragma unroll
    for (int uu = 0; uu < 4; ++uu) {
      const int j = kc * 4 + uu;
      double2 v = make_double2(0.0, 0.0);
      if (valid && j < wsum) v = colp[j][(size_t)r * coll[j]];
      xv[8 * i + 2 * uu] = v.x;
      xv[8 * i + 2 * uu + 1] = v.y;
    }
  }
}

// CPS: CTAs per SM (2 only at K' <= 32, N' = 16: 64 registers per thread, 4-column
// epilogue groups; twice the warps to hide latency).
template <int KC, int CPS = 1>  // K' / 8 (2, 4, 6 or 8)
__global__ void __launch_bounds__(TC_PIPE_THREADS, CPS) tc_combine_kernel(int n, TcCombArgs ta) {
  const CombArgs& a = ta.a;
  if (a.skip && *a.skip == 0) return;
  extern __shared__ __align__(128) unsigned char tc_smem[];
  constexpr int kp = 8 * KC;
  const int np = ta.np, ds = ta.ds, ts = ta.ts;
  uint16_t* sB = reinterpret_cast<uint16_t*>(tc_smem);        // 8 np x kp: plane b, column n at row b np + n
  uint16_t* sA = sB + TC_DIAG * np * kp;                       // ds stages of TC_DIGITS x 128 x kp
  __shared__ __align__(8) uint64_t bar_dempty[2], bar_tfull[2], bar_tempty[2], bar_row[TC_RING];
  __shared__ __align__(8) uint64_t bar_never;  // test hook: nothing ever completes its phase 0
  __shared__ uint32_t taddr_s;
  __shared__ volatile int abort_s;
  __shared__ double nwarp[TC_EWARPS][COMB_MAX_NORMS];  // norm columns: one partial per epilogue warp
  __shared__ const double2* colp[TC_KMAX / 2];
  __shared__ int coll[TC_KMAX / 2];
  __shared__ int sG[TC_NMAX], sBadC[TC_NMAX];
  __shared__ int sX[2][2][TC_ROWS], sXb[2][2][TC_ROWS];       // exponent exchange between the halves
  __shared__ int sRowT[TC_RING][TC_ROWS], sRowBad[TC_RING][TC_ROWS];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int wsum = 0;
  for (int t = 0; t < a.nin; ++t) wsum += a.in[t].w;
  const int nnorm = a.c - a.c_store;
  for (int e = tid; e < TC_EWARPS * nnorm; e += TC_PIPE_THREADS) nwarp[e / nnorm][e % nnorm] = 0.0;
  if (tid < TC_KMAX / 2) {  // where input column j of the stacked row lives
    const double2* p = nullptr;
    int ld = 0;
    if (tid < wsum) {
      int t = 0, jj = tid;
      while (jj >= a.in[t].w) {
        jj -= a.in[t].w;
        ++t;
      }
      p = a.in[t].X + jj;
      ld = a.in[t].ldx;
    }
    colp[tid] = p;
    coll[tid] = ld;
  }
  // B operand (C' digits): alpha_t C_t staged in shared memory (the A stages are free until
  // the roles start; all threads load at once), column exponents, then the digits of all
  // kp x np entries
  double2* sCv = reinterpret_cast<double2*>(sA);
  for (int e = tid; e < wsum * a.c; e += TC_PIPE_THREADS) {
    const int j = e / a.c, l = e - j * a.c;
    int t = 0, jj = j;
    while (jj >= a.in[t].w) {
      jj -= a.in[t].w;
      ++t;
    }
    sCv[e] = cmul(a.in[t].alpha, a.in[t].C[(size_t)jj * a.in[t].ldc + l]);
  }
  __syncthreads();
  if (tid < np) {
    int G = TC_NOEXP, bad = 0;
    for (int kk = 0; kk < kp; ++kk) {
      const double v = tc_cval(sCv, wsum, a.c, kk, tid);
      G = max(G, tc_top(v));
      bad |= tc_nonfinite(v);
    }
    sG[tid] = G;
    sBadC[tid] = bad;
  }
  if (tid == 0) {
    abort_s = 0;
    for (int i = 0; i < 2; ++i) {
      mbar_init(&bar_dempty[i], 1);
      mbar_init(&bar_tfull[i], 1);
      mbar_init(&bar_tempty[i], TC_EWARPS * 32);
    }
    for (int i = 0; i < TC_RING; ++i) mbar_init(&bar_row[i], TC_ROWS);
    mbar_init(&bar_never, 1);
  }
  __syncthreads();
  for (int e = tid; e < kp * np; e += TC_PIPE_THREADS) {
    const int nn = e / kp, kk = e - nn * kp;
    float dg[TC_DIGITS];
    tc_digits(tc_cval(sCv, wsum, a.c, kk, nn), sG[nn], dg);
#pragma unroll
    for (int d = 0; d < TC_DIGITS; ++d)
      sB[tc_off(d * np + nn, kk, KC)] = (uint16_t)(__float_as_uint(dg[d]) >> 16);
    sB[tc_off(TC_DIGITS * np + nn, kk, KC)] = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&taddr_s)),
                 "r"(ta.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = taddr_s;
  const uint32_t a_slice = TC_ROWS * kp * 2;              // bytes per digit plane
  const uint32_t a_stage = TC_DIGITS * a_slice;           // bytes per stage
  const int ntiles = (n + TC_ROWS - 1) / TC_ROWS;

  if (warp < TC_DWARPS) {
    // ------------------------------------------------------------ digits role --
    const int rl = tid & (TC_ROWS - 1), h = tid >> 7;
    const uint32_t sA_addr = smem_u32(sA), sB_addr = smem_u32(sB);
    int it = 0, last_b = -1;
    uint32_t last_v = 0;
    bool mma_ok = true;  // thread 0: its last wait for a buffer succeeded
    constexpr bool PF = KC == 2 && CPS == 1;  // registers allow the next tile's values ahead
    double xn[PF ? 4 * KC : 1];
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
      const int s = it % ds;
      const uint32_t u = (uint32_t)(it / ds);
      const int r = tile * TC_ROWS + rl;
      const bool valid = r < n;
      if (h == 0) {  // into L2: this row of the next tile's inputs, this row's old outputs
        const int r2 = r + gridDim.x * TC_ROWS;
        if (r2 < n)
          for (int t = 0; t < a.nin; ++t)
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.in[t].X + (size_t)r2 * a.in[t].ldx),
                         "r"((uint32_t)(a.in[t].w * 16))
                         : "memory");
        if (valid && a.beta_one) {
          if (a.c_split > 0)
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.Y + (size_t)r * a.ldy),
                         "r"((uint32_t)(a.c_split * 16))
                         : "memory");
          if (a.c_store > a.c_split)
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.Y2 + (size_t)r * a.ldy2),
                         "r"((uint32_t)((a.c_store - a.c_split) * 16))
                         : "memory");
        }
      }
      double xv[4 * KC];
      if constexpr (PF) {  // this tile's values were loaded one tile ahead
        if (it == 0) tc_row_load<KC>(colp, coll, wsum, valid, r, h, xv);
        else
#pragma unroll
          for (int e = 0; e < 4 * KC; ++e) xv[e] = xn[e];
        const int r2 = r + gridDim.x * TC_ROWS;
        tc_row_load<KC>(colp, coll, wsum, r2 < n, r2, h, xn);
      } else {
        tc_row_load<KC>(colp, coll, wsum, valid, r, h, xv);
      }
      int T = TC_NOEXP, bad = 0;
#pragma unroll
      for (int e = 0; e < 4 * KC; ++e) {
        T = max(T, tc_top(xv[e]));
        bad |= tc_nonfinite(xv[e]);
      }
      sX[it & 1][h][rl] = T;
      sXb[it & 1][h][rl] = bad;
      // both halves' bounds, and the stage free (the same decision in every thread)
      bool ok = bar_and(1, TC_DWARPS * 32, true);
      T = max(sX[it & 1][0][rl], sX[it & 1][1][rl]);
      bad = sXb[it & 1][0][rl] | sXb[it & 1][1][rl];
      ok = bar_and(1, TC_DWARPS * 32, mma_ok && mbar_wait_bounded(&bar_dempty[s], (u & 1) ^ 1, &abort_s, ta.wait_tries));
      if (!ok) {
        if (tid == 0) {
          abort_s = 1;
          atomicExch(ta.err, 1);
        }
        break;
      }
      if (h == 0) {
        const int slot = it % TC_RING;
        sRowT[slot][rl] = T;
        sRowBad[slot][rl] = bad;
        mbar_arrive(&bar_row[slot]);
      }
      uint16_t* sAs = sA + (size_t)s * (a_stage / 2);
#pragma unroll
      for (int i = 0; i < KC / 2; ++i) {
        const int kc = 2 * i + h;
        {
          uint32_t wv[TC_DIGITS][4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            float d0[TC_DIGITS], d1[TC_DIGITS];
            tc_digits(xv[8 * i + 2 * q], T, d0);
            tc_digits(xv[8 * i + 2 * q + 1], T, d1);
#pragma unroll
            for (int d = 0; d < TC_DIGITS; ++d) wv[d][q] = tc_pack2(d0[d], d1[d]);
          }
#pragma unroll
          for (int d = 0; d < TC_DIGITS; ++d)
            *reinterpret_cast<uint4*>(sAs + d * TC_ROWS * kp + tc_off(rl, kc * 8, KC)) =
                make_uint4(wv[d][0], wv[d][1], wv[d][2], wv[d][3]);
        }
      }
      fence_async_smem();
      bar_and(1, TC_DWARPS * 32, true);  // the stage is complete
      if (tid == 0) {
        const int b = it % ts;
        const uint32_t v = (uint32_t)(it / ts);
        mma_ok = mbar_wait_bounded(&bar_tempty[b], (v & 1) ^ 1, &abort_s, ta.wait_tries);
        if (mma_ok) {
          tc_fence_after();
          const uint32_t a0 = sA_addr + (uint32_t)s * a_stage;
          const uint32_t d0 = tmem + (uint32_t)(b * TC_DIAG * np);
          for (int ks = 0; ks < kp / 16; ++ks)
            for (int da = 0; da < TC_DIGITS; ++da) {
              const uint64_t ad = umma_desc(a0 + da * a_slice + ks * 256, 128, KC * 128);
              const int ntot = (TC_DIAG - da) * np;
              for (int c0 = 0; c0 < ntot; c0 += 256) {
                const int nc = min(256, ntot - c0);
                const uint64_t bd =
                    umma_desc(sB_addr + (uint32_t)(c0 >> 3) * (uint32_t)(KC * 128) + ks * 256, 128, KC * 128);
                umma_bf16(d0 + (uint32_t)(da * np + c0), ad, bd, umma_idesc_bf16(TC_ROWS, nc),
                          (ks > 0 || da > 0) ? 1 : 0);
              }
            }
          umma_commit(&bar_dempty[s]);
          umma_commit(&bar_tfull[b]);
          last_b = b;
          last_v = v;
        } else {
          abort_s = 1;
          atomicExch(ta.err, 1);
        }
      }
    }
    if (tid == 0 && last_b >= 0) {  // the last products complete before the tensor memory is freed
      volatile int never = 0;
      if (!mbar_wait_bounded(&bar_tfull[last_b], last_v & 1, &never, TC_WAIT_TRIES)) atomicExch(ta.err, 1);
    }
  } else if (warp < TC_DWARPS + TC_EWARPS) {
    // ---------------------------------------------------------- epilogue role --
    const int ew = warp - TC_DWARPS, q4 = warp & 3, eh = ew >> 2;
    const int row_in = q4 * 32 + lane;
    const uint32_t lane_base = (uint32_t)(q4 * 32) << 16;
    constexpr int CW = CPS == 1 ? 8 : 4;  // columns per chunk
    // |y|^2 of this thread's rows in its norm columns, summed over its tiles (column
    // index: chunk (nb - CW eh) / (2 CW), complex column within it; <= 16 at N' <= 64)
    double nacc[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) nacc[i] = 0.0;
    int it = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
      const int b = it % ts, slot = it % TC_RING;
      const uint32_t v = (uint32_t)(it / ts);
      bool ok = mbar_wait_bounded(&bar_row[slot], (uint32_t)(it / TC_RING) & 1, &abort_s, ta.wait_tries) &&
                mbar_wait_bounded(&bar_tfull[b], v & 1, &abort_s, ta.wait_tries) &&
                (!ta.probe || mbar_wait_bounded(&bar_never, 0, &abort_s, ta.wait_tries));
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) {
        if (lane == 0) {
          abort_s = 1;
          atomicExch(ta.err, 1);
        }
        break;
      }
      tc_fence_after();
      const int r = tile * TC_ROWS + row_in;
      const bool valid = r < n;
      const int T = sRowT[slot][row_in], bad = sRowBad[slot][row_in];
      const uint32_t tb = tmem + lane_base + (uint32_t)(b * TC_DIAG * np);
      for (int nb = CW * eh; nb < np; nb += 2 * CW) {  // chunks of CW real columns, alternating halves
        uint32_t acc[TC_DIAG][CW];
#pragma unroll
        for (int d = 0; d < TC_DIAG; ++d) {
          if constexpr (CW == 8)
            tmem_ld8(tb + (uint32_t)(d * np + nb), acc[d]);
          else
            tmem_ld4(tb + (uint32_t)(d * np + nb), acc[d]);
        }
        tmem_wait_ld();
        if (!valid) continue;
#pragma unroll
        for (int uu = 0; uu < CW; uu += 2) {
          const int nn = nb + uu, l = nn >> 1;
          if (l >= a.c) continue;
          double yv[2];
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            uint32_t dg[TC_DIAG];
#pragma unroll
            for (int d = 0; d < TC_DIAG; ++d) dg[d] = acc[d][uu + q];
            long long hi, lo;
            tc_diag_sum<(KC <= 4)>(dg, hi, lo);
            yv[q] = tc_round96(hi, lo, T + sG[nn + q] - 68);
            if (bad || sBadC[nn + q]) yv[q] = __longlong_as_double(0x7FF8000000000000ll);
          }
          double2 y = make_double2(yv[0], yv[1]);
          if (l < a.c_store) {
            double2* dst = comb_out(a, r, l);
            if (a.beta_one) {
              const double2 o = *dst;
              y.x += o.x;
              y.y += o.y;
            }
            *dst = y;
          } else {
            nacc[((nb - CW * eh) / (2 * CW)) * (CW / 2) + uu / 2] += y.x * y.x + y.y * y.y;
          }
        }
      }
      tc_fence_before();
      mbar_arrive(&bar_tempty[b]);
    }
    // norm columns: the warp's rows summed by a fixed shuffle tree into the warp's slot
    if (nnorm > 0)
      for (int ci = 0; ci < 16; ++ci) {
        const int nb = CW * eh + 2 * CW * (ci / (CW / 2)), l = (nb >> 1) + ci % (CW / 2);
        if (nb >= np || l < a.c_store || l >= a.c) continue;  // the same in the whole warp
        double sv = nacc[ci];
        for (int off = 16; off > 0; off >>= 1) sv += __shfl_xor_sync(0xffffffffu, sv, off);
        if (lane == 0) nwarp[ew][l - a.c_store] = sv;
      }
  }
  __syncthreads();
  tc_fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ta.tmem_cols)
                              : "memory");
  if (a.normpart)  // the epilogue warps' partials, added in a fixed order
    for (int e = tid; e < nnorm; e += TC_PIPE_THREADS) {
      double sv = 0.0;
      for (int w = 0; w < TC_EWARPS; ++w) sv += nwarp[w][e];
      a.normpart[(size_t)blockIdx.x * nnorm + e] = sv;
    }
}

// ------------------------------------------------ Gram products on the tensor cores --
// C = X^* [Y0 Y1] (wx x wy, wy = wy0 + wy1) with the digit scheme of the combination, the
// contraction now over the rows.  Real form: X' (n x 2wx) and Y' (n x 2wy) hold the real
// and imaginary parts as columns; G = X'^T Y' gives the four real products of every
// complex pair, Re C(j,l) = G(2j,2l) + G(2j+1,2l+1), Im C(j,l) = G(2j,2l+1) - G(2j+1,2l).
// * The rows are taken in windows of 128.  Every real column c of X' and of Y' gets its
//   exponent bound E_c over the window's rows (a first pass); each value becomes the
//   integer round(v 2^(54 - E_c)) in 7 balanced base-256 digits.
// * A = X'^T (M = real column of X, up to two 128-row tiles; K = row), B = Y'^T with the
//   digit planes stacked along N as in the combination; per 16-row K step 7 MMAs per M
//   tile.  Over a window |D_d| <= 7 * 128 * 2^14 < 2^24: exact FP32 accumulation.
// * After a window every G entry is formed exactly and rounded once to double
//   (2^(E_m + E_n - 68) Z), then added to FP64 accumulators in registers; the CTA's
//   partial C goes to partial[blockIdx.x][j wy + l] for the deterministic reduction.
// Error: per window as for the combination, plus one FP64 addition per window.
constexpr int TG_WIN = 128;   // rows per window (exact accumulation bound)
constexpr int TG_SUB = 32;    // rows per shared-memory pass (two 16-row K steps)
constexpr int TG_THREADS = 256;
constexpr int TG_AMAX = 128;  // complex columns of X (2 M tiles)
constexpr int TG_BMAX = 32;   // complex columns of [Y0 Y1]

struct TcGramArgs {
  int n;
  const double2* X;
  int ldx, wx;
  const double2* Y0;
  int ldy0, wy0;
  const double2* Y1;
  int ldy1, wy1;
  double2* partial;  // [gridDim.x][wx * (wy0 + wy1)]
  const int* skip;   // nothing happens when non-null and *skip == 0
  int* err;          // set to 1 if a wait on the tensor core gave up
  int wait_tries;    // limit of the pipeline's mbarrier waits (tests lower it)
  int np;            // 2 cbw rounded up to a multiple of 16 (<= 64)
  int mt;            // M tiles: 2 wx <= 128 mt (1 or 2; 2 needs np <= 32)
  int tmem_cols;     // power of two >= mt * 8 * np
  int cbw;           // columns of [Y0 Y1] per column block: CTA (x, y) takes block y
};

// Dynamic shared memory: A digits (7 planes x mt x 128 x TG_SUB) and B digits (8 planes x
// np x TG_SUB), bf16.  Column blocks: the grid's y index selects columns [y cbw, y cbw + cbw)
// of [Y0 Y1], and its x CTAs share that block's windows; block y's partials lie at
// partial + y gridDim.x wx cbw, CTA x's at x wx wyb after that (wyb = the block's width).
__host__ __device__ constexpr size_t tg_smem_bytes(int mt, int np) {
  return (size_t)TC_DIGITS * mt * 128 * TG_SUB * 2 + (size_t)TC_DIAG * np * TG_SUB * 2;
}

__global__ void __launch_bounds__(TG_THREADS, 1) tc_gram_kernel(TcGramArgs ta) {
  if (ta.skip && *ta.skip == 0) return;
  extern __shared__ __align__(1024) unsigned char tg_smem[];
  const int c0 = blockIdx.y * ta.cbw;
  const int np = ta.np, mt = ta.mt, wx = ta.wx, wy = min(ta.cbw, ta.wy0 + ta.wy1 - c0), n = ta.n;
  constexpr int KC = TG_SUB / 8;
  uint16_t* sA = reinterpret_cast<uint16_t*>(tg_smem);           // [7][mt][128 x TG_SUB]
  uint16_t* sB = sA + (size_t)TC_DIGITS * mt * 128 * TG_SUB;     // [8 np x TG_SUB]
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t taddr_s;
  __shared__ int sE[2 * TG_AMAX], sF[2 * TG_BMAX], sBadE[2 * TG_AMAX], sBadF[2 * TG_BMAX];
  __shared__ const double2* colY[TG_BMAX];
  __shared__ int ldY[TG_BMAX];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid < wy) {
    const int cc = c0 + tid;
    colY[tid] = cc < ta.wy0 ? ta.Y0 + cc : ta.Y1 + (cc - ta.wy0);
    ldY[tid] = cc < ta.wy0 ? ta.ldy0 : ta.ldy1;
  }
  // zero digits once: padding rows of A and B and B's zero plane are never rewritten
  {
    const size_t words = tg_smem_bytes(mt, np) / 16;
    for (size_t e = tid; e < words; e += TG_THREADS) reinterpret_cast<uint4*>(tg_smem)[e] = make_uint4(0, 0, 0, 0);
  }
  if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)) : "memory");
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&taddr_s)),
                 "r"(ta.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = taddr_s;
  // this thread's accumulators: one M row, CP consecutive real columns of Y'
  const int half = tid >> 7;                      // warps 0-3 / 4-7
  const int tile = mt == 2 ? half : 0;            // M tile of this thread's TMEM lanes
  const int CP = mt == 2 ? np : np / 2;           // real columns per thread (<= 32)
  const int col0 = mt == 2 ? 0 : half * (np / 2);
  const int mrow = tile * 128 + (warp & 3) * 32 + lane;
  const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
  double acc[32];
#pragma unroll
  for (int q = 0; q < 32; ++q) acc[q] = 0.0;
  bool bad_row = false;
  uint32_t bad_cols = 0;
  const int nwin = (n + TG_WIN - 1) / TG_WIN;
  const int W = wx + wy, R = TG_THREADS / W;
  uint32_t parity = 0;
  bool ok = true;
  for (int win = blockIdx.x; win < nwin && ok; win += gridDim.x) {
    const int r0 = win * TG_WIN, nr = min(TG_WIN, n - r0);
    // pass 1: exponent bound of every real column over the window's rows
    for (int c = tid; c < 2 * TG_AMAX; c += TG_THREADS) { sE[c] = TC_NOEXP; sBadE[c] = 0; }
    if (tid < 2 * TG_BMAX) { sF[tid] = TC_NOEXP; sBadF[tid] = 0; }
    __syncthreads();
    if (tid < R * W) {
      const int col = tid % W, rg = tid / W;
      int tre = TC_NOEXP, tim = TC_NOEXP, bre = 0, bim = 0;
      const double2* base = col < wx ? ta.X + col : colY[col - wx];
      const size_t ld = col < wx ? (size_t)ta.ldx : (size_t)ldY[col - wx];
      for (int r = rg; r < nr; r += R) {
        const double2 v = base[(size_t)(r0 + r) * ld];
        tre = max(tre, tc_top(v.x));
        tim = max(tim, tc_top(v.y));
        bre |= tc_nonfinite(v.x);
        bim |= tc_nonfinite(v.y);
      }
      int* E = col < wx ? sE + 2 * col : sF + 2 * (col - wx);
      int* Bf = col < wx ? sBadE + 2 * col : sBadF + 2 * (col - wx);
      atomicMax(E, tre);
      atomicMax(E + 1, tim);
      if (bre) atomicOr(Bf, 1);
      if (bim) atomicOr(Bf + 1, 1);
    }
    __syncthreads();
    for (int sc = 0; sc < TG_WIN / TG_SUB && ok; ++sc) {
      const int rs = r0 + sc * TG_SUB;
      // A digits: task (group g of 8 rows, complex column j), 2 real columns of X'
      for (int a = tid; a < 4 * wx; a += TG_THREADS) {
        const int j = a % wx, g = a / wx;
        double re[8], im[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int r = rs + 8 * g + u;
          const double2 v = r < n ? ta.X[(size_t)r * ta.ldx + j] : make_double2(0.0, 0.0);
          re[u] = v.x;
          im[u] = v.y;
        }
#pragma unroll
        for (int p = 0; p < 2; ++p) {
          const int m = 2 * j + p, T = sE[m];
          uint32_t wv[TC_DIGITS][4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            float d0[TC_DIGITS], d1[TC_DIGITS];
            tc_digits(p ? im[2 * q] : re[2 * q], T, d0);
            tc_digits(p ? im[2 * q + 1] : re[2 * q + 1], T, d1);
#pragma unroll
            for (int d = 0; d < TC_DIGITS; ++d) wv[d][q] = tc_pack2(d0[d], d1[d]);
          }
          const int t = m >> 7, ml = m & 127;
#pragma unroll
          for (int d = 0; d < TC_DIGITS; ++d)
            *reinterpret_cast<uint4*>(sA + ((size_t)(d * mt + t) * 128 * TG_SUB) + tc_off(ml, 8 * g, KC)) =
                make_uint4(wv[d][0], wv[d][1], wv[d][2], wv[d][3]);
        }
      }
      // B digits: task (group g, complex column l), planes stacked along N
      for (int b = tid; b < 4 * wy; b += TG_THREADS) {
        const int l = b % wy, g = b / wy;
        double re[8], im[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int r = rs + 8 * g + u;
          const double2 v = r < n ? colY[l][(size_t)r * ldY[l]] : make_double2(0.0, 0.0);
          re[u] = v.x;
          im[u] = v.y;
        }
#pragma unroll
        for (int p = 0; p < 2; ++p) {
          const int nn = 2 * l + p, T = sF[nn];
          uint32_t wv[TC_DIGITS][4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            float d0[TC_DIGITS], d1[TC_DIGITS];
            tc_digits(p ? im[2 * q] : re[2 * q], T, d0);
            tc_digits(p ? im[2 * q + 1] : re[2 * q + 1], T, d1);
#pragma unroll
            for (int d = 0; d < TC_DIGITS; ++d) wv[d][q] = tc_pack2(d0[d], d1[d]);
          }
#pragma unroll
          for (int d = 0; d < TC_DIGITS; ++d)
            *reinterpret_cast<uint4*>(sB + tc_off(d * np + nn, 8 * g, KC)) =
                make_uint4(wv[d][0], wv[d][1], wv[d][2], wv[d][3]);
        }
      }
      fence_async_smem();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
        for (int ks = 0; ks < TG_SUB / 16; ++ks)
          for (int t = 0; t < mt; ++t)
            for (int da = 0; da < TC_DIGITS; ++da) {
              const uint64_t ad = umma_desc(a0 + (uint32_t)((da * mt + t) * 128 * TG_SUB * 2) + ks * 256, 128, KC * 128);
              const int ntot = (TC_DIAG - da) * np;
              for (int c0 = 0; c0 < ntot; c0 += 256) {
                const int nc = min(256, ntot - c0);
                const uint64_t bd = umma_desc(b0 + (uint32_t)(c0 >> 3) * (KC * 128) + ks * 256, 128, KC * 128);
                umma_bf16(tmem + (uint32_t)(t * TC_DIAG * np + da * np + c0), ad, bd, umma_idesc_bf16(128, nc),
                          (sc > 0 || ks > 0 || da > 0) ? 1 : 0);
              }
            }
        umma_commit(&mbar);
      }
      bool done = false;
      for (int it = 0; it < TC_WAIT_TRIES && !done; ++it) done = mbar_try_wait(&mbar, parity);
      parity ^= 1;
      if (!__syncthreads_and(done)) {
        if (tid == 0) atomicExch(ta.err, 1);
        ok = false;
      }
      tc_fence_after();
    }
    if (!ok) break;
    // flush: every G entry of the window exactly, rounded once, into the FP64 accumulators
    const bool vrow = mrow < 2 * wx;
    if (vrow && sBadE[mrow]) bad_row = true;
#pragma unroll
    for (int g4 = 0; g4 < 8; ++g4) {
      if (4 * g4 < CP) {
        uint32_t dg[TC_DIAG][4];
#pragma unroll
        for (int d = 0; d < TC_DIAG; ++d)
          tmem_ld4(tmem + lane_base + (uint32_t)(tile * TC_DIAG * np + d * np + col0 + 4 * g4), dg[d]);
        tmem_wait_ld();
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int q = 4 * g4 + u, nn = col0 + q;
          if (!vrow || nn >= 2 * wy) continue;
          if (sBadF[nn]) bad_cols |= 1u << q;
          const long long hi = (long long)tc_f2i(dg[0][u]) * 16777216ll + (long long)tc_f2i(dg[1][u]) * 65536ll +
                               (long long)tc_f2i(dg[2][u]) * 256ll + (long long)tc_f2i(dg[3][u]);
          const long long lo = (long long)tc_f2i(dg[4][u]) * 16777216ll + (long long)tc_f2i(dg[5][u]) * 65536ll +
                               (long long)tc_f2i(dg[6][u]) * 256ll + (long long)tc_f2i(dg[7][u]);
          acc[q] += tc_round96(hi, lo, sE[mrow] + sF[nn] - 68);
        }
      }
    }
    tc_fence_before();
    __syncthreads();  // the next window's first products overwrite the accumulators
  }
  // complex result from the four real products (rows 2j, 2j+1 are adjacent lanes)
  const bool ev = (lane & 1) == 0;
  const int j = mrow >> 1;
  const bool pbad = __shfl_down_sync(0xffffffffu, (int)bad_row, 1) != 0;
  const double qnan = __longlong_as_double(0x7FF8000000000000ll);
#pragma unroll
  for (int q = 0; q < 32; q += 2) {
    const double o0 = __shfl_down_sync(0xffffffffu, acc[q], 1);
    const double o1 = __shfl_down_sync(0xffffffffu, acc[q + 1], 1);
    const int l = (col0 + q) >> 1;
    if (ev && q < CP && j < wx && l < wy) {
      double2 v = make_double2(acc[q] + o1, acc[q + 1] - o0);
      if (bad_row || pbad || ((bad_cols >> q) & 3u)) v = make_double2(qnan, qnan);
      ta.partial[((size_t)blockIdx.y * gridDim.x * ta.cbw + (size_t)blockIdx.x * wy) * wx + (size_t)j * wy + l] = v;
    }
  }
  __syncthreads();
  tc_fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ta.tmem_cols)
                              : "memory");
}

// ------------------------------------------- narrow Gram products, pipelined --
// C = X^* [Y0 Y1] for narrow blocks (wx <= 24, wy <= 16), the digit scheme of the
// combination with the contraction over the rows, laid out so that nothing is padded:
// * A = the 7 digit planes of X' stacked along M: lane L = a (2 wx) + m holds plane a of
//   real column m (mt = ceil(14 wx / 128) tiles of 128 lanes); B = the 7 planes of Y'
//   stacked along N: row b np + n.  One MMA per 16-row K step and M tile forms every
//   plane product P_ab(m, n) = sum_r X'_a(r, m) Y'_b(r, n) at lane (a, m), column b np + n.
// * Each CTA takes a contiguous range of 64-row halves (CTA b: halves [b H / G, (b+1) H / G),
//   H = ceil(n / 64), G CTAs) and cuts it into pieces of up to TN_PIECE = 8 halves (512
//   rows) from its start.  A piece has per-column exponent bounds (a first pass over the
//   piece) and accumulates every P_ab in tensor memory over all its rows (|P_ab| <=
//   512 2^14 = 2^23, exact in FP32).  After a piece the diagonals
//   D_d(m, n) = sum_{a+b=d} P_ab(m, n), d = 0..7, are summed across lanes in shared
//   memory with integer additions (each P_ab taken exactly to int32), which are exact
//   and so independent of their order; every G(m, n) is then formed and rounded once
//   (tc_round96) and added to FP64 accumulators, and the CTA's partial C goes to
//   partial[blockIdx.x][j wy + l].  One rounding per 512 rows instead of per 128: the
//   epilogue's lane sums and roundings are what bounds this kernel.
// * Pipeline: warps 0-7 (digits) take a piece 128 rows at a time for the exponent pass
//   (task (row pair, complex column) = two loads, shared atomicMax), then half by half
//   (the two shared-memory stages alternate) for the digits, and each half is marked full.  Warp 12 (one thread) issues each full half's MMAs into accumulator
//   buffer (window % ts), so that the digit warps never wait for the issue.  Warps 8-11
//   (epilogue) read the buffer (warp 8 + q: lanes 32 q .. 32 q + 31 of every tile), free
//   it, and form the window's products.  X^* X (self) splits X once and writes both
//   operands.  13 warps: at most 4 per SM sub-partition, 128 registers per thread.
// Every wait has an iteration limit, as in the combination.
constexpr int TN_WIN = 128;   // rows of one task sweep of the digit warps
constexpr int TN_HALF = 64;   // rows per shared-memory stage
constexpr int TN_PIECE = 8;   // halves per piece (one exponent pass, one epilogue)
constexpr int TN_DWARPS = 8, TN_EWARPS = 4;
constexpr int TN_THREADS = (TN_DWARPS + TN_EWARPS + 1) * 32;
constexpr int TN_XMAX = 24, TN_YMAX = 16;
constexpr int TN_TASKS = 8;                          // tasks per digits thread, at most: 64 W <= 256 TN_TASKS
constexpr int TN_OUT = (TN_XMAX * TN_YMAX + TN_EWARPS * 32 - 1) / (TN_EWARPS * 32);
constexpr int TN_RING = 4;

struct TcGramNArgs {
  int n;
  const double2* X;
  int ldx, wx;
  const double2* Y0;
  int ldy0, wy0;
  const double2* Y1;
  int ldy1, wy1;
  int self;          // Y0 == X, wy1 == 0
  double2* partial;  // [gridDim.x][wx * (wy0 + wy1)]
  const int* skip;
  int* err;
  int wait_tries;    // limit of the pipeline's mbarrier waits (tests lower it)
  int mt;            // M tiles: 14 wx <= 128 mt (<= 3)
  int np;            // 2 wy rounded up to 16 (16 or 32)
  int ts;            // accumulator buffers (1 or 2)
  int tmem_cols;     // power of two >= ts mt 7 np
};

// Shared memory: two stages of (A: mt x 128 lanes, B: 7 np rows) x 64 rows of bf16, then
// the diagonal sums: 8 x 2 wx x (2 wy + 1) int32.
__host__ __device__ constexpr size_t tn_stage_bytes(int mt, int np) {
  return ((size_t)mt * 128 + 7 * (size_t)np) * TN_HALF * 2;
}
__host__ __device__ constexpr size_t tn_smem_bytes(int mt, int np, int wx, int wy) {
  return 2 * tn_stage_bytes(mt, np) + (size_t)TC_DIAG * 2 * wx * (2 * wy + 1) * 4;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

// Rows r, r + 1 of complex column j of [X Y0 Y1] as (Re r, Re r+1, Im r, Im r+1); rows
// at or beyond rlim (the end of the piece, at most n) read as zero.
__device__ __forceinline__ void tn_load1(const TcGramNArgs& ta, int r, int rlim, int j, double (&v)[4]) {
  const int wx = ta.wx;
  const double2* base;
  size_t ld;
  if (j < wx) {
    base = ta.X + j;
    ld = (size_t)ta.ldx;
  } else if (j - wx < ta.wy0) {
    base = ta.Y0 + (j - wx);
    ld = (size_t)ta.ldy0;
  } else {
    base = ta.Y1 + (j - wx - ta.wy0);
    ld = (size_t)ta.ldy1;
  }
  double2 x0 = make_double2(0.0, 0.0), x1 = x0;
  if (r < rlim) x0 = base[(size_t)r * ld];
  if (r + 1 < rlim) x1 = base[(size_t)(r + 1) * ld];
  v[0] = x0.x;
  v[1] = x1.x;
  v[2] = x0.y;
  v[3] = x1.y;
}

template <int NT>  // tasks per digits thread (4: W <= 16 loaded columns, 8: W <= 32)
__global__ void __launch_bounds__(TN_THREADS, 1) tc_gram_narrow_kernel(TcGramNArgs ta) {
  if (ta.skip && *ta.skip == 0) return;
  extern __shared__ __align__(1024) unsigned char tn_smem[];
  const int n = ta.n, wx = ta.wx, wy = ta.wy0 + ta.wy1, mt = ta.mt, np = ta.np, ts = ta.ts;
  const int W = ta.self ? wx : wx + wy;              // complex columns loaded per row
  const int MX = 2 * wx, NY = 2 * wy, SP = NY + 1;   // real columns; diagonal-sum row stride
  const size_t stage = tn_stage_bytes(mt, np);
  uint16_t* sA0 = reinterpret_cast<uint16_t*>(tn_smem);                       // stage h: + h stage
  int* sD = reinterpret_cast<int*>(tn_smem + 2 * stage);                      // [8][MX][SP]
  __shared__ __align__(8) uint64_t bar_dfull[2], bar_dempty[2], bar_tfull[2], bar_tempty[2], bar_exp[TN_RING],
      bar_expfree[TN_RING];
  __shared__ uint32_t taddr_s;
  __shared__ volatile int abort_s;
  __shared__ int sE[TN_RING][2 * (TN_XMAX + TN_YMAX)], sBad[TN_RING][2 * (TN_XMAX + TN_YMAX)];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  {  // zero the stages (padding lanes and rows stay zero) and the diagonal sums
    const size_t words = tn_smem_bytes(mt, np, wx, wy) / 4;
    for (size_t e = tid; e < words; e += TN_THREADS) reinterpret_cast<uint32_t*>(tn_smem)[e] = 0u;
  }
  if (tid == 0) {
    abort_s = 0;
    for (int i = 0; i < 2; ++i) {
      mbar_init(&bar_dfull[i], TN_DWARPS * 32);
      mbar_init(&bar_dempty[i], 1);
      mbar_init(&bar_tfull[i], 1);
      mbar_init(&bar_tempty[i], TN_EWARPS * 32);
    }
    for (int i = 0; i < TN_RING; ++i) {
      mbar_init(&bar_exp[i], TN_DWARPS * 32);
      mbar_init(&bar_expfree[i], TN_EWARPS * 32);
    }
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&taddr_s)),
                 "r"(ta.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = taddr_s;
  const int bufcols = mt * 7 * np;
  const int ncol = ta.self ? MX : MX + NY;  // real columns with an exponent (Y' after X')
  // this CTA's halves [h0, h1), cut into pieces of TN_PIECE halves from h0
  const int H = (n + TN_HALF - 1) / TN_HALF;
  const int h0 = (int)((long long)H * blockIdx.x / gridDim.x);
  const int h1 = (int)((long long)H * (blockIdx.x + 1) / gridDim.x);

  if (warp < TN_DWARPS) {
    // ------------------------------------------------------------ digits role --
    int trp[NT], tj[NT];  // this thread's tasks t = tid + 256 i: (row pair of a 128-row sweep, complex column)
#pragma unroll
    for (int i = 0; i < NT; ++i) {
      const int t = tid + 256 * i;
      trp[i] = t / W;
      tj[i] = t - trp[i] * W;
    }
    // A lane a 2 wx + c of plane a lies a 2 wx 64 elements after lane c when 2 wx is a
    // multiple of 8 (the core-matrix layout runs on across the 128-lane tiles)
    const bool alin = (MX & 7) == 0;
    int it = 0, hc = 0;  // pieces, halves written
    bool ok = true;
    for (int ph = h0; ph < h1 && ok; ph += TN_PIECE, ++it) {
      const int pe = min(h1, ph + TN_PIECE);
      const int slot = it % TN_RING;
      const int rlim = min(n, pe * TN_HALF);
      // the exponent slot is free once the epilogue of piece it - TN_RING has rounded
      ok = bar_and(1, TN_DWARPS * 32,
                   mbar_wait_bounded(&bar_expfree[slot], ((uint32_t)(it / TN_RING) & 1) ^ 1, &abort_s, ta.wait_tries));
      if (!ok) break;
      for (int c = tid; c < ncol; c += TN_DWARPS * 32) {
        sE[slot][c] = TC_NOEXP;
        sBad[slot][c] = 0;
      }
      bar_and(1, TN_DWARPS * 32, true);
      // exponent pass over the piece, a 128-row sweep at a time (tasks four at a time)
      for (int r0 = ph * TN_HALF; r0 < rlim; r0 += TN_WIN) {
#pragma unroll
        for (int i0 = 0; i0 < NT; i0 += 4) {
          double v[4][4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            if (trp[i0 + i] < TN_WIN / 2) {
              tn_load1(ta, r0 + 2 * trp[i0 + i], rlim, tj[i0 + i], v[i]);
            } else {
#pragma unroll
              for (int c = 0; c < 4; ++c) v[i][c] = 0.0;
            }
          }
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int rp = trp[i0 + i], j = tj[i0 + i];
            if (rp < TN_WIN / 2) {
              const int c = (j < wx ? 2 * j : MX + 2 * (j - wx));  // real columns c (Re), c + 1 (Im)
              const int tre = max(tc_top(v[i][0]), tc_top(v[i][1])), tim = max(tc_top(v[i][2]), tc_top(v[i][3]));
              if (tre > TC_NOEXP) atomicMax(&sE[slot][c], tre);
              if (tim > TC_NOEXP) atomicMax(&sE[slot][c + 1], tim);
              if (tc_nonfinite(v[i][0]) | tc_nonfinite(v[i][1])) sBad[slot][c] = 1;
              if (tc_nonfinite(v[i][2]) | tc_nonfinite(v[i][3])) sBad[slot][c + 1] = 1;
            }
          }
        }
      }
      bar_and(1, TN_DWARPS * 32, true);
      mbar_arrive(&bar_exp[slot]);
      // digits, half by half, into the two stages in turn
      for (int hh = ph; hh < pe; ++hh, ++hc) {
        const int s = hc & 1;
        ok = bar_and(1, TN_DWARPS * 32,
                     mbar_wait_bounded(&bar_dempty[s], ((uint32_t)(hc >> 1) & 1) ^ 1, &abort_s, ta.wait_tries));
        if (!ok) break;
        uint16_t* sA = sA0 + (size_t)s * (stage / 2);
        uint16_t* sB = sA + (size_t)mt * 128 * TN_HALF;
        const int hb = (hh - ph) & 1;                       // half of its 128-row sweep
        const int rs = (ph + ((hh - ph) & ~1)) * TN_HALF;   // first row of that sweep
#pragma unroll
        for (int i = 0; i < NT; ++i) {
          const int rp = trp[i], j = tj[i];
          if (rp < TN_WIN / 2 && (rp >> 5) == hb) {
            const int kk = 2 * (rp & 31);  // row within the half (even)
            double vv[4];
            tn_load1(ta, rs + 2 * rp, rlim, j, vv);
#pragma unroll
            for (int p = 0; p < 2; ++p) {  // Re, Im
              const int c = (j < wx ? 2 * j : MX + 2 * (j - wx)) + p;
              float d0[TC_DIGITS], d1[TC_DIGITS];
              const int T = sE[slot][c];
              tc_digits(vv[2 * p], T, d0);
              tc_digits(vv[2 * p + 1], T, d1);
              if (j < wx) {  // lanes a 2 wx + c across the tiles: tc_off runs on past lane 127
                const int base = tc_off(c, kk, 8);
#pragma unroll
                for (int a = 0; a < TC_DIGITS; ++a)
                  *reinterpret_cast<uint32_t*>(sA + (alin ? base + a * MX * 64 : tc_off(a * MX + c, kk, 8))) =
                      tc_pack2(d0[a], d1[a]);
              }
              if (j >= wx || ta.self) {  // rows b np + nn, np a multiple of 16
                const int nn = j < wx ? c : c - MX;
                const int base = tc_off(nn, kk, 8);
#pragma unroll
                for (int b = 0; b < TC_DIGITS; ++b)
                  *reinterpret_cast<uint32_t*>(sB + base + b * np * 64) = tc_pack2(d0[b], d1[b]);
              }
            }
          }
        }
        fence_async_smem();
        mbar_arrive(&bar_dfull[s]);
      }
    }
    if (!ok && tid == 0) {
      abort_s = 1;
      atomicExch(ta.err, 1);
    }
  } else if (warp == TN_DWARPS + TN_EWARPS) {
    // --------------------------------------------------------------- MMA role --
    if (lane == 0) {
      const uint32_t sbase = smem_u32(tn_smem);
      const uint32_t idesc = umma_idesc_bf16(128, 7 * np);
      int it = 0, hc = 0, last_b = -1;
      uint32_t last_v = 0;
      bool ok = true;
      for (int ph = h0; ph < h1 && ok; ph += TN_PIECE, ++it) {
        const int pe = min(h1, ph + TN_PIECE);
        const int b = it % ts;
        const uint32_t vv = (uint32_t)(it / ts);
        for (int hh = ph; hh < pe; ++hh, ++hc) {
          const int s = hc & 1;
          ok = mbar_wait_bounded(&bar_dfull[s], (uint32_t)(hc >> 1) & 1, &abort_s, ta.wait_tries) &&
               (hh > ph || mbar_wait_bounded(&bar_tempty[b], (vv & 1) ^ 1, &abort_s, ta.wait_tries));
          if (!ok) break;
          tc_fence_after();
          const uint32_t a0 = sbase + (uint32_t)(s * stage);
          const uint32_t b0 = a0 + (uint32_t)(mt * 128 * TN_HALF * 2);
          for (int ks = 0; ks < TN_HALF / 16; ++ks)
            for (int t = 0; t < mt; ++t)
              umma_bf16(tmem + (uint32_t)(b * bufcols + t * 7 * np),
                        umma_desc(a0 + (uint32_t)(t * 128 * TN_HALF * 2) + ks * 256, 128, 8 * 128),
                        umma_desc(b0 + ks * 256, 128, 8 * 128), idesc, (hh > ph || ks > 0) ? 1 : 0);
          umma_commit(&bar_dempty[s]);
          if (hh == pe - 1) {
            umma_commit(&bar_tfull[b]);
            last_b = b;
            last_v = vv;
          }
        }
      }
      if (!ok) {
        abort_s = 1;
        atomicExch(ta.err, 1);
      }
      if (last_b >= 0) {  // the last products complete before the tensor memory is freed
        volatile int never = 0;
        if (!mbar_wait_bounded(&bar_tfull[last_b], last_v & 1, &never, TC_WAIT_TRIES)) atomicExch(ta.err, 1);
      }
    }
  } else {
    // ---------------------------------------------------------- epilogue role --
    const int etid = tid - TN_DWARPS * 32, q4 = warp & 3;
    const uint32_t lane_base = (uint32_t)(q4 * 32) << 16;
    double acc[TN_OUT][4];
    uint32_t badmask = 0;
#pragma unroll
    for (int i = 0; i < TN_OUT; ++i)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][q] = 0.0;
    int it = 0;
    for (int ph = h0; ph < h1; ph += TN_PIECE, ++it) {
      const int b = it % ts, slot = it % TN_RING;
      const uint32_t vv = (uint32_t)(it / ts);
      // one decision for all epilogue warps (they share the named barrier below)
      const bool ok = bar_and(
          2, TN_EWARPS * 32,
          mbar_wait_bounded(&bar_exp[slot], (uint32_t)(it / TN_RING) & 1, &abort_s, ta.wait_tries) &&
              mbar_wait_bounded(&bar_tfull[b], vv & 1, &abort_s, ta.wait_tries));
      if (!ok) {
        if (etid == 0) {
          abort_s = 1;
          atomicExch(ta.err, 1);
        }
        break;
      }
      tc_fence_after();
      // plane products -> diagonal sums (exact integer additions; |P_ab| <= 2^23)
      for (int t = 0; t < mt; ++t) {
        const int L = t * 128 + q4 * 32 + lane, a = L / MX, m = L - a * MX;
        const bool vl = a < TC_DIGITS;
        for (int bp0 = 0; bp0 < TC_DIGITS; bp0 += 2) {  // two planes of 16 columns per round trip
          for (int n0 = 0; n0 < np; n0 += 16) {
            uint32_t r[2][16];
#pragma unroll
            for (int e = 0; e < 2; ++e)
              if (bp0 + e < TC_DIGITS)
                tmem_ld16(tmem + lane_base + (uint32_t)(b * bufcols + t * 7 * np + (bp0 + e) * np + n0), r[e]);
            tmem_wait_ld();
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              const int bp = bp0 + e;
              if (bp < TC_DIGITS && vl && a + bp < TC_DIAG) {
                int* dst = sD + ((size_t)(a + bp) * MX + m) * SP + n0;
#pragma unroll
                for (int u = 0; u < 16; ++u)
                  if (n0 + u < NY) atomicAdd(dst + u, tc_f2i(r[e][u]));
              }
            }
          }
        }
      }
      tc_fence_before();
      mbar_arrive(&bar_tempty[b]);
      bar_and(2, TN_EWARPS * 32, true);
      // this thread's outputs: every G(m, n) of the piece, rounded once, into FP64
#pragma unroll
      for (int i = 0; i < TN_OUT; ++i) {
        const int o = etid + TN_EWARPS * 32 * i;
        if (o < wx * wy) {
          const int j = o / wy, l = o - j * wy;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int m = 2 * j + (q >> 1), nn = 2 * l + (q & 1);
            const int cy = ta.self ? nn : MX + nn;
            int* src = sD + (size_t)m * SP + nn;
            long long hi = 0, lo = 0;
#pragma unroll
            for (int d = 0; d < TC_DIAG; ++d) {
              const long long Dd = (long long)src[(size_t)d * MX * SP];
              src[(size_t)d * MX * SP] = 0;
              if (d < 4)
                hi += Dd << (8 * (3 - d));
              else
                lo += Dd << (8 * (7 - d));
            }
            acc[i][q] += tc_round96(hi, lo, sE[slot][m] + sE[slot][cy] - 68);
            if (sBad[slot][m] | sBad[slot][cy]) badmask |= 1u << (4 * i + q);
          }
        }
      }
      bar_and(2, TN_EWARPS * 32, true);  // the sums are zero again
      mbar_arrive(&bar_expfree[slot]);
    }
    // G(2j, 2l) = Re x Re, (2j, 2l+1) = Re x Im, (2j+1, 2l) = Im x Re, (2j+1, 2l+1) = Im x Im
#pragma unroll
    for (int i = 0; i < TN_OUT; ++i) {
      const int o = etid + TN_EWARPS * 32 * i;
      if (o < wx * wy) {
        double2 cz = make_double2(acc[i][0] + acc[i][3], acc[i][1] - acc[i][2]);
        if ((badmask >> (4 * i)) & 0xFu) cz = make_double2(__longlong_as_double(0x7FF8000000000000ll),
                                                           __longlong_as_double(0x7FF8000000000000ll));
        ta.partial[(size_t)blockIdx.x * wx * wy + o] = cz;
      }
    }
  }
  __syncthreads();
  tc_fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ta.tmem_cols)
                              : "memory");
}

// ---------------------------------------------- wide Gram products, pipelined --
// C = X^* [Y0 Y1] for wx <= 64, wy <= 32 (2 wx real columns on the 128 tensor-memory
// lanes, N' = 2 wy): the combination's layout with the contraction over the rows.
// * A = X'^T, one 128-lane slab per digit plane; B = Y'^T with its 7 digit planes and a
//   zero plane stacked along N (row b np + n).  Per 16-row K step, plane a of A against B
//   planes 0 .. 7 - a, written at accumulator column a np, lands every product on its
//   diagonal: the MMAs form D_d(m, n), d = 0..7, directly (|D_d| <= 7 2^21 over a 128-row
//   window: exact in FP32).
// * Windows of 128 rows with per-column exponent bounds (a first pass over the window),
//   written to shared memory in four stages of 32 rows (two stage buffers).
// * Roles: warps 0-5 (digits, 192 threads) run the exponent pass and write the stages;
//   warp 14 (one thread) issues each full stage's MMAs; warps 6-13 (epilogue: two per
//   lane quarter, alternate 8-column chunks) form every G(m, n) of the window,
//   round it once (tc_round96) and add it to an FP64 accumulator in shared memory that
//   the thread owns.  At the end the CTA's complex partial C goes to
//   partial[blockIdx.x][j wy + l].  15 warps: 128 registers per thread.
// Every wait has an iteration limit, as in the combination.
constexpr int TW_WIN = 128, TW_STAGE = 32;
constexpr int TW_DWARPS = 6, TW_EWARPS = 8;
constexpr int TW_THREADS = (TW_DWARPS + TW_EWARPS + 1) * 32;
constexpr int TW_XMAX = 64, TW_YMAX = 32;
constexpr int TW_RING = 4;

struct TcGramWArgs {
  int n;
  const double2* X;
  int ldx, wx;
  const double2* Y0;
  int ldy0, wy0;
  const double2* Y1;
  int ldy1, wy1;
  int self;          // Y0 == X, wy1 == 0
  double2* partial;  // [gridDim.x][wx * (wy0 + wy1)]
  const int* skip;
  int* err;
  int wait_tries;    // limit of the pipeline's mbarrier waits (tests lower it)
  int np;            // 2 wy rounded up to 16 (<= 64)
  int ts;            // accumulator buffers (1 or 2)
  int tmem_cols;     // power of two >= ts 8 np
};

__host__ __device__ constexpr size_t tw_stage_bytes(int np) {
  return ((size_t)TC_DIGITS * 128 + (size_t)TC_DIAG * np) * TW_STAGE * 2;
}
// two stages, then the FP64 accumulators [2 wx][2 wy] and their non-finite flags
__host__ __device__ constexpr size_t tw_smem_bytes(int np, int wx, int wy) {
  return 2 * tw_stage_bytes(np) + (size_t)4 * wx * wy * 8 + (size_t)4 * wx * wy;
}

__global__ void __launch_bounds__(TW_THREADS, 1) tc_gram_wide_kernel(TcGramWArgs ta) {
  if (ta.skip && *ta.skip == 0) return;
  extern __shared__ __align__(1024) unsigned char tw_smem[];
  const int n = ta.n, wx = ta.wx, wy = ta.wy0 + ta.wy1, np = ta.np, ts = ta.ts;
  const int W = ta.self ? wx : wx + wy;
  const int MX = 2 * wx, NY = 2 * wy;
  const size_t stage = tw_stage_bytes(np);
  double* sAcc = reinterpret_cast<double*>(tw_smem + 2 * stage);             // [MX][NY]
  unsigned char* sBadAcc = reinterpret_cast<unsigned char*>(sAcc + (size_t)MX * NY);
  __shared__ __align__(8) uint64_t bar_dfull[2], bar_dempty[2], bar_tfull[2], bar_tempty[2], bar_exp[TW_RING];
  __shared__ uint32_t taddr_s;
  __shared__ volatile int abort_s;
  __shared__ int sE[TW_RING][2 * (TW_XMAX + TW_YMAX)], sBad[TW_RING][2 * (TW_XMAX + TW_YMAX)];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  {  // zero the stages (padding lanes, rows and the zero plane stay zero) and the accumulators
    const size_t words = tw_smem_bytes(np, wx, wy) / 4;
    for (size_t e = tid; e < words; e += TW_THREADS) reinterpret_cast<uint32_t*>(tw_smem)[e] = 0u;
  }
  if (tid == 0) {
    abort_s = 0;
    for (int i = 0; i < 2; ++i) {
      mbar_init(&bar_dfull[i], TW_DWARPS * 32);
      mbar_init(&bar_dempty[i], 1);
      mbar_init(&bar_tfull[i], 1);
      mbar_init(&bar_tempty[i], TW_EWARPS * 32);
    }
    for (int i = 0; i < TW_RING; ++i) mbar_init(&bar_exp[i], TW_DWARPS * 32);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&taddr_s)),
                 "r"(ta.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = taddr_s;
  const int nwin = (n + TW_WIN - 1) / TW_WIN;
  const int ncol = ta.self ? MX : MX + NY;
  constexpr int DT = TW_DWARPS * 32;

  if (warp < TW_DWARPS) {
    // ------------------------------------------------------------ digits role --
    int it = 0;
    // task t = tid + k DT is (row pair t / W, column t % W); when W divides DT the column is
    // tid % W for every k and the row pair advances by DT / W
    const bool wdiv = DT % W == 0;
    const int jw = tid % W, rpw = tid / W, rstep = DT / W;
    for (int win = blockIdx.x; win < nwin; win += gridDim.x, ++it) {
      const int slot = it % TW_RING, r0 = win * TW_WIN, nr = min(TW_WIN, n - r0);
      // the exponent slot is free once the previous window's first stage was consumed
      // (that window's MMAs began after the epilogue of the one before it had finished)
      bool ok = bar_and(1, DT, mbar_wait_bounded(&bar_dempty[0], ((uint32_t)(2 * it) & 1u) ^ 1u, &abort_s, ta.wait_tries));
      if (!ok) {
        if (tid == 0) {
          abort_s = 1;
          atomicExch(ta.err, 1);
        }
        break;
      }
      for (int c = tid; c < ncol; c += DT) {
        sE[slot][c] = TC_NOEXP;
        sBad[slot][c] = 0;
      }
      bar_and(1, DT, true);
      {  // exponent pass: thread (column j, row phase) over rows rg, rg + R, ...
        const int R = DT / W;
        if (tid < R * W) {
          const int j = tid % W, rg = tid / W;
          const double2* base;
          size_t ld;
          if (j < wx) {
            base = ta.X + j;
            ld = (size_t)ta.ldx;
          } else if (j - wx < ta.wy0) {
            base = ta.Y0 + (j - wx);
            ld = (size_t)ta.ldy0;
          } else {
            base = ta.Y1 + (j - wx - ta.wy0);
            ld = (size_t)ta.ldy1;
          }
          int tre = TC_NOEXP, tim = TC_NOEXP, bre = 0, bim = 0;
#pragma unroll 8
          for (int r = rg; r < nr; r += R) {
            const double2 v = base[(size_t)(r0 + r) * ld];
            tre = max(tre, tc_top(v.x));
            tim = max(tim, tc_top(v.y));
            bre |= tc_nonfinite(v.x);
            bim |= tc_nonfinite(v.y);
          }
          const int c = j < wx ? 2 * j : MX + 2 * (j - wx);
          if (tre > TC_NOEXP) atomicMax(&sE[slot][c], tre);
          if (tim > TC_NOEXP) atomicMax(&sE[slot][c + 1], tim);
          if (bre) sBad[slot][c] = 1;
          if (bim) sBad[slot][c + 1] = 1;
        }
      }
      bar_and(1, DT, true);
      mbar_arrive(&bar_exp[slot]);
      for (int sc = 0; sc < TW_WIN / TW_STAGE; ++sc) {
        const int st = sc & 1;
        const uint32_t u = (uint32_t)(2 * it + (sc >> 1));
        if (sc > 0) {
          ok = bar_and(1, DT, mbar_wait_bounded(&bar_dempty[st], (u & 1) ^ 1, &abort_s, ta.wait_tries));
          if (!ok) break;
        }
        uint16_t* sA = reinterpret_cast<uint16_t*>(tw_smem + st * stage);
        uint16_t* sB = sA + (size_t)TC_DIGITS * 128 * TW_STAGE;
        // tasks: (row pair, complex column), 16 W of them, four at a time: the loads of a
        // batch are all in flight before its digits are formed
        constexpr int TB = 4;
        for (int t0 = tid, kq = 0; t0 < (TW_STAGE / 2) * W; t0 += TB * DT, kq += TB) {
          double vv[TB][4];
#pragma unroll
          for (int q = 0; q < TB; ++q) {
            const int t = t0 + q * DT;
            const int rp = wdiv ? rpw + (kq + q) * rstep : t / W, j = wdiv ? jw : t - rp * W;
            const int r = r0 + sc * TW_STAGE + 2 * rp;
            double2 x0 = make_double2(0.0, 0.0), x1 = x0;
            if (t < (TW_STAGE / 2) * W) {
              const double2* base;
              size_t ld;
              if (j < wx) {
                base = ta.X + j;
                ld = (size_t)ta.ldx;
              } else if (j - wx < ta.wy0) {
                base = ta.Y0 + (j - wx);
                ld = (size_t)ta.ldy0;
              } else {
                base = ta.Y1 + (j - wx - ta.wy0);
                ld = (size_t)ta.ldy1;
              }
              if (r < n) x0 = base[(size_t)r * ld];
              if (r + 1 < n) x1 = base[(size_t)(r + 1) * ld];
            }
            vv[q][0] = x0.x;
            vv[q][1] = x1.x;
            vv[q][2] = x0.y;
            vv[q][3] = x1.y;
          }
#pragma unroll
          for (int q = 0; q < TB; ++q) {
            const int t = t0 + q * DT;
            const int rp = wdiv ? rpw + (kq + q) * rstep : t / W, j = wdiv ? jw : t - rp * W;
            if (t >= (TW_STAGE / 2) * W) break;
            const int kk = 2 * rp;
#pragma unroll
            for (int p = 0; p < 2; ++p) {
              const int c = (j < wx ? 2 * j : MX + 2 * (j - wx)) + p;
              float d0[TC_DIGITS], d1[TC_DIGITS];
              const int T = sE[slot][c];
              tc_digits(vv[q][2 * p], T, d0);
              tc_digits(vv[q][2 * p + 1], T, d1);
              if (j < wx) {
#pragma unroll
                for (int a = 0; a < TC_DIGITS; ++a)
                  *reinterpret_cast<uint32_t*>(sA + (size_t)a * 128 * TW_STAGE + tc_off(c, kk, TW_STAGE / 8)) =
                      tc_pack2(d0[a], d1[a]);
              }
              if (j >= wx || ta.self) {  // rows b np + nn, np a multiple of 16
                const int nn = j < wx ? c : c - MX;
                const int base = tc_off(nn, kk, TW_STAGE / 8);
#pragma unroll
                for (int b = 0; b < TC_DIGITS; ++b)
                  *reinterpret_cast<uint32_t*>(sB + base + b * np * (TW_STAGE / 8) * 8) = tc_pack2(d0[b], d1[b]);
              }
            }
          }
        }
        fence_async_smem();
        mbar_arrive(&bar_dfull[st]);
      }
      if (!ok) {
        if (tid == 0) {
          abort_s = 1;
          atomicExch(ta.err, 1);
        }
        break;
      }
    }
  } else if (warp == TW_DWARPS + TW_EWARPS) {
    // --------------------------------------------------------------- MMA role --
    if (lane == 0) {
      const uint32_t sbase = smem_u32(tw_smem);
      constexpr uint32_t KCB = (TW_STAGE / 8) * 128;  // bytes between 8-row groups
      int it = 0, last_b = -1;
      uint32_t last_v = 0;
      for (int win = blockIdx.x; win < nwin; win += gridDim.x, ++it) {
        const int b = it % ts;
        const uint32_t vv = (uint32_t)(it / ts);
        bool ok = true;
        for (int sc = 0; sc < TW_WIN / TW_STAGE && ok; ++sc) {
          const int st = sc & 1;
          const uint32_t u = (uint32_t)(2 * it + (sc >> 1));
          ok = mbar_wait_bounded(&bar_dfull[st], u & 1, &abort_s, ta.wait_tries) &&
               (sc > 0 || mbar_wait_bounded(&bar_tempty[b], (vv & 1) ^ 1, &abort_s, ta.wait_tries));
          if (!ok) break;
          tc_fence_after();
          const uint32_t a0 = sbase + (uint32_t)(st * stage);
          const uint32_t b0 = a0 + (uint32_t)(TC_DIGITS * 128 * TW_STAGE * 2);
          for (int ks = 0; ks < TW_STAGE / 16; ++ks)
            for (int da = 0; da < TC_DIGITS; ++da) {
              const uint64_t ad = umma_desc(a0 + (uint32_t)(da * 128 * TW_STAGE * 2) + ks * 256, 128, KCB);
              const int ntot = (TC_DIAG - da) * np;
              for (int c0 = 0; c0 < ntot; c0 += 256) {
                const int nc = min(256, ntot - c0);
                const uint64_t bd = umma_desc(b0 + (uint32_t)(c0 >> 3) * KCB + ks * 256, 128, KCB);
                umma_bf16(tmem + (uint32_t)(b * TC_DIAG * np + da * np + c0), ad, bd, umma_idesc_bf16(128, nc),
                          (sc > 0 || ks > 0 || da > 0) ? 1 : 0);
              }
            }
          umma_commit(&bar_dempty[st]);
          if (sc == TW_WIN / TW_STAGE - 1) {
            umma_commit(&bar_tfull[b]);
            last_b = b;
            last_v = vv;
          }
        }
        if (!ok) {
          abort_s = 1;
          atomicExch(ta.err, 1);
          break;
        }
      }
      if (last_b >= 0) {  // the last products complete before the tensor memory is freed
        volatile int never = 0;
        if (!mbar_wait_bounded(&bar_tfull[last_b], last_v & 1, &never, TC_WAIT_TRIES)) atomicExch(ta.err, 1);
      }
    }
  } else {
    // ---------------------------------------------------------- epilogue role --
    const int ew = warp - TW_DWARPS, q4 = warp & 3, eh = ew >> 2;
    const int m = q4 * 32 + lane;  // this thread's lane: real column m of X'
    const bool vm = m < MX;
    const uint32_t lane_base = (uint32_t)(q4 * 32) << 16;
    int it = 0;
    for (int win = blockIdx.x; win < nwin; win += gridDim.x, ++it) {
      const int b = it % ts, slot = it % TW_RING;
      const uint32_t vv = (uint32_t)(it / ts);
      bool ok = mbar_wait_bounded(&bar_exp[slot], (uint32_t)(it / TW_RING) & 1, &abort_s, ta.wait_tries) &&
                mbar_wait_bounded(&bar_tfull[b], vv & 1, &abort_s, ta.wait_tries);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) {
        if (lane == 0) {
          abort_s = 1;
          atomicExch(ta.err, 1);
        }
        break;
      }
      tc_fence_after();
      const int Em = vm ? sE[slot][m] : 0;
      const int bm = vm ? sBad[slot][m] : 0;
      const uint32_t tb = tmem + lane_base + (uint32_t)(b * TC_DIAG * np);
      for (int nb = 8 * eh; nb < np; nb += 16) {  // 8-column chunks: the 8 diagonals in one round trip
        uint32_t acc[TC_DIAG][8];
#pragma unroll
        for (int d = 0; d < TC_DIAG; ++d) tmem_ld8(tb + (uint32_t)(d * np + nb), acc[d]);
        tmem_wait_ld();
        if (!vm) continue;
#pragma unroll
        for (int uu = 0; uu < 8; ++uu) {
          const int nn = nb + uu;
          if (nn >= NY) continue;
          const int cy = ta.self ? nn : MX + nn;
          long long hi = 0, lo = 0;
#pragma unroll
          for (int d = 0; d < TC_DIAG; ++d) {
            const long long Dd = (long long)__float2int_rn(__uint_as_float(acc[d][uu]));
            if (d < 4)
              hi += Dd << (8 * (3 - d));
            else
              lo += Dd << (8 * (7 - d));
          }
          sAcc[(size_t)m * NY + nn] += tc_round96(hi, lo, Em + sE[slot][cy] - 68);
          if (bm | sBad[slot][cy]) sBadAcc[(size_t)m * NY + nn] = 1;
        }
      }
      tc_fence_before();
      mbar_arrive(&bar_tempty[b]);
    }
    bar_and(2, TW_EWARPS * 32, true);
    // G(2j, 2l) = Re x Re, (2j, 2l+1) = Re x Im, (2j+1, 2l) = Im x Re, (2j+1, 2l+1) = Im x Im
    const int etid = tid - TW_DWARPS * 32;
    for (int o = etid; o < wx * wy; o += TW_EWARPS * 32) {
      const int j = o / wy, l = o - j * wy;
      const size_t i00 = (size_t)(2 * j) * NY + 2 * l, i10 = i00 + NY;
      double2 cz = make_double2(sAcc[i00] + sAcc[i10 + 1], sAcc[i00 + 1] - sAcc[i10]);
      if (sBadAcc[i00] | sBadAcc[i00 + 1] | sBadAcc[i10] | sBadAcc[i10 + 1])
        cz = make_double2(__longlong_as_double(0x7FF8000000000000ll), __longlong_as_double(0x7FF8000000000000ll));
      ta.partial[(size_t)blockIdx.x * wx * wy + o] = cz;
    }
  }
  __syncthreads();
  tc_fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ta.tmem_cols)
                              : "memory");
}

}  // namespace gplhr
