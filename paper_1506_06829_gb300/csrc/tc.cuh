// FP64 block combination Y = beta Y + sum_t alpha_t X_t C_t on GB300's tensor cores
// (tcgen05, bf16 operands, FP32 accumulators in tensor memory), accurate to FP64 working
// precision by splitting every double into small integer digits.
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
// Error per output: input rounding <= 2^-55 (max_k |x_rk| sum_k |c_kn| + K' max_k |x_rk|
// max_k |c_kn|), the dropped pairs a + b >= 8 (weight <= 2^-62 K' 2^(T_r + G_n) in all),
// and the final rounding: at most (K'/4 + 2) u max_k |x_rk| sum_k |c_kn| with u = 2^-53,
// a quarter of the classical bound K' u sum_k |x_rk| |c_kn| <= K' u max|x| sum|c| of a
// DFMA dot product.  Results below 2^-1022 (subnormal) take a second rounding.
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
__device__ __forceinline__ bool mbar_try_wait(uint64_t* mbar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_u32(mbar)), "r"(parity)
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
constexpr int TC_THREADS = 256;  // two threads per row: each loads half of the row
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
// to even), in integer arithmetic; a result below 2^-1022 takes a second rounding to the
// subnormal grid.
__device__ __forceinline__ double tc_round96(long long hi, long long lo, int p) {
  long long zh = hi + (lo >> 32);  // value = zh 2^32 + zl, zl in [0, 2^32)
  uint32_t zl = (uint32_t)lo;
  const bool neg = zh < 0;
  if (neg) {  // 96-bit negation
    zh = -zh - (zl != 0u ? 1 : 0);
    zl = 0u - zl;
  }
  const uint64_t uh = (uint64_t)zh;  // < 2^49
  if (uh == 0 && zl == 0) return 0.0;
  uint64_t mant;  // 53 bits, leading one at bit 52
  int e;          // exponent of the leading one
  if (uh < (1ull << 21)) {  // below 2^53: exact
    const uint64_t v = (uh << 32) | zl;
    const int lz = __clzll((long long)v);
    mant = v << (lz - 11);
    e = 63 - lz;
  } else {
    const int L = 64 - __clzll((long long)uh);  // 22..49 bits above zl
    const int sh = L - 21;                       // 1..28 bits of zl dropped
    mant = (uh << (32 - sh)) | (zl >> sh);
    const uint32_t rem = zl << (32 - sh);        // the dropped bits, left-aligned
    if (rem > 0x80000000u || (rem == 0x80000000u && (mant & 1))) ++mant;
    e = L + 31;
    if (mant >> 53) {
      mant >>= 1;
      ++e;
    }
  }
  e += p;
  const uint64_t sgn = neg ? (1ull << 63) : 0ull;
  if (e > 1023) return __longlong_as_double((long long)(sgn | 0x7FF0000000000000ull));
  if (e >= -1022)
    return __longlong_as_double((long long)(sgn | ((uint64_t)(e + 1023) << 52) | (mant & 0xFFFFFFFFFFFFFull)));
  const double d = scalbn((double)mant, e - 52);
  return neg ? -d : d;
}

// Exact integer value of an FP32 accumulator holding an integer of magnitude < 2^24.
__device__ __forceinline__ int tc_f2i(uint32_t u) { return __float2int_rn(__uint_as_float(u)); }

struct TcCombArgs {
  CombArgs a;
  int kp;          // K' padded to a multiple of 16 (<= TC_KMAX)
  int np;          // N' padded to a multiple of 16 (<= TC_NMAX)
  int tmem_cols;   // power of two >= max(32, TC_DIAG np)
  int* err;        // set to 1 if a wait on the tensor core gave up
};

__device__ __forceinline__ int tc_off(int row, int k, int KC) {  // element offset in a core-matrix tile
  return ((row >> 3) * KC + (k >> 3)) * 64 + (row & 7) * 8 + (k & 7);
}

// The value of C' at (kk, nn): stacked alpha_t C_t, complex entries as 2 x 2 real blocks.
__device__ __forceinline__ double tc_cval(const CombArgs& a, int wsum, int kk, int nn) {
  const int j = kk >> 1, p = kk & 1, l = nn >> 1, q = nn & 1;
  if (j >= wsum || l >= a.c) return 0.0;
  int t = 0, jj = j;
  while (jj >= a.in[t].w) {
    jj -= a.in[t].w;
    ++t;
  }
  const double2 cv = cmul(a.in[t].alpha, a.in[t].C[(size_t)jj * a.c + l]);
  return p == 0 ? (q == 0 ? cv.x : cv.y) : (q == 0 ? -cv.y : cv.x);
}

// One persistent CTA per (SM, slot); 128 rows per tile, thread (r, h) = (tid % 128,
// tid / 128) loads and splits the row's k-chunks kc = h, h + 2, ... (8 reals each) and
// writes the output column groups nb = 4 h, 4 h + 8, ...  Warp w reads tensor-memory
// lanes 32 (w % 4) .. +31, which hold rows 32 (w % 4) .. +31 of the tile.
__global__ void __launch_bounds__(TC_THREADS, 2) tc_combine_kernel(int n, TcCombArgs ta) {
  const CombArgs& a = ta.a;
  if (a.skip && *a.skip == 0) return;
  extern __shared__ __align__(128) unsigned char tc_smem[];
  const int kp = ta.kp, np = ta.np, KC = kp >> 3;
  uint16_t* sA = reinterpret_cast<uint16_t*>(tc_smem);         // TC_DIGITS x 128 x kp
  uint16_t* sB = sA + TC_DIGITS * TC_ROWS * kp;                // 8 np x kp: plane b, column n
  int* sG = reinterpret_cast<int*>(sB + TC_DIAG * np * kp);    // at row b np + n; plane 7 zero
  int* sBadC = sG + np;                                        // np non-finite flags
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t taddr_s;
  __shared__ double nsum[COMB_MAX_NORMS];
  __shared__ const double2* colp[TC_KMAX / 2];
  __shared__ int coll[TC_KMAX / 2];
  __shared__ int sT[2][TC_ROWS];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int rl = tid & (TC_ROWS - 1), h = tid >> 7;
  int wsum = 0;
  for (int t = 0; t < a.nin; ++t) wsum += a.in[t].w;
  const int nnorm = a.c - a.c_store;
  for (int e = tid; e < nnorm; e += TC_THREADS) nsum[e] = 0.0;
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
  // B operand (C' digits): column exponents, then the digits of all kp x np entries
  if (tid < np) {
    int G = TC_NOEXP, bad = 0;
    for (int kk = 0; kk < kp; ++kk) {
      const double v = tc_cval(a, wsum, kk, tid);
      G = max(G, tc_top(v));
      bad |= tc_nonfinite(v);
    }
    sG[tid] = G;
    sBadC[tid] = bad;
  }
  __syncthreads();
  for (int e = tid; e < kp * np; e += TC_THREADS) {
    const int nn = e / kp, kk = e - nn * kp;
    float dg[TC_DIGITS];
    tc_digits(tc_cval(a, wsum, kk, nn), sG[nn], dg);
#pragma unroll
    for (int d = 0; d < TC_DIGITS; ++d)
      sB[tc_off(d * np + nn, kk, KC)] = (uint16_t)(__float_as_uint(dg[d]) >> 16);
    sB[tc_off(TC_DIGITS * np + nn, kk, KC)] = 0;
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
  const uint32_t a_slice = TC_ROWS * kp * 2;  // bytes
  const uint32_t sA_addr = smem_u32(sA), sB_addr = smem_u32(sB);
  const int ntiles = (n + TC_ROWS - 1) / TC_ROWS;
  const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
  bool ok = true;
  uint32_t parity = 0;
  for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, parity ^= 1) {
    const int r = tile * TC_ROWS + rl;
    const bool valid = r < n;
    {  // this row of the CTA's next tile into L2 while this tile is processed
      const int r2 = r + gridDim.x * TC_ROWS;
      if (h == 0 && r2 < n)
        for (int t = 0; t < a.nin; ++t)
          asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.in[t].X + (size_t)r2 * a.in[t].ldx),
                       "r"((uint32_t)(a.in[t].w * 16))
                       : "memory");
    }
    // this thread's k-chunks of the row: 4 complex values each, in registers
    double xv[TC_KMAX / 2];
    int T = TC_NOEXP, bad = 0;
#pragma unroll
    for (int i = 0; i < TC_KMAX / 16; ++i) {
      const int kc = 2 * i + h;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int j = kc * 4 + u;
        double2 v = make_double2(0.0, 0.0);
        if (valid && kc < KC && j < wsum) v = colp[j][(size_t)r * coll[j]];
        xv[8 * i + 2 * u] = v.x;
        xv[8 * i + 2 * u + 1] = v.y;
        T = max(T, max(tc_top(v.x), tc_top(v.y)));
        bad |= tc_nonfinite(v.x) | tc_nonfinite(v.y);
      }
    }
    sT[h][rl] = T;
    __syncthreads();
    T = max(sT[0][rl], sT[1][rl]);
    __syncthreads();
    sT[h][rl] = bad;
    // A operand: 8 consecutive k of one digit per 16-byte store
#pragma unroll
    for (int i = 0; i < TC_KMAX / 16; ++i) {
      const int kc = 2 * i + h;
      if (kc < KC) {
        // two values at a time (few live registers, so the compiler can interleave)
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
          *reinterpret_cast<uint4*>(sA + d * TC_ROWS * kp + tc_off(rl, kc * 8, KC)) =
              make_uint4(wv[d][0], wv[d][1], wv[d][2], wv[d][3]);
      }
    }
    fence_async_smem();
    __syncthreads();
    bad = sT[0][rl] | sT[1][rl];
    if (tid == 0) {
      tc_fence_after();
      // plane da of X' against C' planes 0 .. 7 - da (stack rows 0 .. (8 - da) np) at
      // accumulator column da np; the first MMA (ks = 0, da = 0, all 8 planes)
      // initialises every diagonal
      for (int ks = 0; ks < kp / 16; ++ks)
        for (int da = 0; da < TC_DIGITS; ++da) {
          const uint64_t ad = umma_desc(sA_addr + da * a_slice + ks * 256, 128, KC * 128);
          const int ntot = (TC_DIAG - da) * np;
          for (int c0 = 0; c0 < ntot; c0 += 256) {
            const int nc = min(256, ntot - c0);
            const uint64_t bd = umma_desc(sB_addr + (uint32_t)(c0 >> 3) * (uint32_t)(KC * 128) + ks * 256, 128, KC * 128);
            umma_bf16(tmem + (uint32_t)(da * np + c0), ad, bd, umma_idesc_bf16(TC_ROWS, nc), (ks > 0 || da > 0) ? 1 : 0);
          }
        }
      umma_commit(&mbar);
    }
    // wait for the products (bounded)
    bool done = false;
    for (int it = 0; it < (1 << 22) && !done; ++it) done = mbar_try_wait(&mbar, parity);
    if (!__syncthreads_and(done)) {  // the same decision in every thread
      if (tid == 0) atomicExch(ta.err, 1);
      ok = false;
      break;
    }
    tc_fence_after();
    for (int nb = 4 * h; nb < np; nb += 8) {  // groups of 4 real columns, alternating halves
      uint32_t acc[TC_DIAG][4];
#pragma unroll
      for (int d = 0; d < TC_DIAG; ++d) tmem_ld4(tmem + lane_base + (uint32_t)(d * np + nb), acc[d]);
      tmem_wait_ld();
      if (!valid) continue;
#pragma unroll
      for (int u = 0; u < 4; u += 2) {
        const int nn = nb + u, l = nn >> 1;
        if (l >= a.c) continue;
        double yv[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const long long hi = (long long)tc_f2i(acc[0][u + q]) * 16777216ll +
                               (long long)tc_f2i(acc[1][u + q]) * 65536ll +
                               (long long)tc_f2i(acc[2][u + q]) * 256ll + (long long)tc_f2i(acc[3][u + q]);
          const long long lo = (long long)tc_f2i(acc[4][u + q]) * 16777216ll +
                               (long long)tc_f2i(acc[5][u + q]) * 65536ll +
                               (long long)tc_f2i(acc[6][u + q]) * 256ll + (long long)tc_f2i(acc[7][u + q]);
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
          atomicAdd(&nsum[l - a.c_store], y.x * y.x + y.y * y.y);
        }
      }
    }
    tc_fence_before();
    __syncthreads();
  }
  __syncthreads();
  tc_fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ta.tmem_cols)
                              : "memory");
  if (a.normpart)
    for (int e = tid; e < nnorm; e += TC_THREADS) a.normpart[(size_t)blockIdx.x * nnorm + e] = nsum[e];
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
  int np;            // 2 (wy0 + wy1) rounded up to a multiple of 16 (<= 64)
  int mt;            // M tiles: 2 wx <= 128 mt (1 or 2; 2 needs np <= 32)
  int tmem_cols;     // power of two >= mt * 8 * np
};

// Dynamic shared memory: A digits (7 planes x mt x 128 x TG_SUB) and B digits (8 planes x
// np x TG_SUB), bf16.
__host__ __device__ constexpr size_t tg_smem_bytes(int mt, int np) {
  return (size_t)TC_DIGITS * mt * 128 * TG_SUB * 2 + (size_t)TC_DIAG * np * TG_SUB * 2;
}

__global__ void __launch_bounds__(TG_THREADS, 1) tc_gram_kernel(TcGramArgs ta) {
  if (ta.skip && *ta.skip == 0) return;
  extern __shared__ __align__(1024) unsigned char tg_smem[];
  const int np = ta.np, mt = ta.mt, wx = ta.wx, wy = ta.wy0 + ta.wy1, n = ta.n;
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
    colY[tid] = tid < ta.wy0 ? ta.Y0 + tid : ta.Y1 + (tid - ta.wy0);
    ldY[tid] = tid < ta.wy0 ? ta.ldy0 : ta.ldy1;
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
      for (int it = 0; it < (1 << 22) && !done; ++it) done = mbar_try_wait(&mbar, parity);
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
      ta.partial[(size_t)blockIdx.x * wx * wy + (size_t)j * wy + l] = v;
    }
  }
  __syncthreads();
  tc_fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ta.tmem_cols)
                              : "memory");
}

}  // namespace gplhr
