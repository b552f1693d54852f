// Device kernels of the GPLHR block iteration (FP64 / complex128).
//
// Dense n x w blocks are row-major with leading dimension ld (elements): row i of
// a block is w contiguous double2 values, so a sparse row gathers whole block rows
// with coalesced 16*w-byte loads.  Small coefficient matrices (w x c) are row-major.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace gplhr {

// Block index of a kernel body: the hardware one, or a virtual one when the persistent
// kernel of the batched iteration runs the body for a recorded launch (block (x, y) of a
// gx x gy grid).  Every body here runs with 256 threads per CTA.
struct Cta {
  int x, y, gx, gy;
  static __device__ __forceinline__ Cta hw() {
    return Cta{(int)blockIdx.x, (int)blockIdx.y, (int)gridDim.x, (int)gridDim.y};
  }
};

// ----------------------------------------------------------------- complex ----
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// c + a * b
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {
  c.x = fma(a.x, b.x, c.x);
  c.x = fma(-a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y);
  c.y = fma(a.y, b.x, c.y);
  return c;
}
// c + conj(a) * b
__device__ __forceinline__ double2 cfmaconj(double2 a, double2 b, double2 c) {
  c.x = fma(a.x, b.x, c.x);
  c.x = fma(a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y);
  c.y = fma(-a.y, b.x, c.y);
  return c;
}
// c + v * b for a real v
__device__ __forceinline__ double2 rfma(double v, double2 b, double2 c) {
  c.x = fma(v, b.x, c.x);
  c.y = fma(v, b.y, c.y);
  return c;
}
__device__ __forceinline__ double2 vfma(double v, double2 b, double2 c) { return rfma(v, b, c); }
__device__ __forceinline__ double2 vfma(double2 v, double2 b, double2 c) { return cfma(v, b, c); }

__device__ __forceinline__ double2 shfl_xor2(double2 v, int m) {
  v.x = __shfl_xor_sync(0xffffffffu, v.x, m);
  v.y = __shfl_xor_sync(0xffffffffu, v.y, m);
  return v;
}

// Single-precision complex (the FP32 bulk phase of the mixed-precision mode computes
// on GB300's FFMA pipe; storage stays complex128 and is converted on load and store).
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {
  c.x = fmaf(a.x, b.x, c.x);
  c.x = fmaf(-a.y, b.y, c.x);
  c.y = fmaf(a.x, b.y, c.y);
  c.y = fmaf(a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ float2 cfmaconj(float2 a, float2 b, float2 c) {
  c.x = fmaf(a.x, b.x, c.x);
  c.x = fmaf(a.y, b.y, c.x);
  c.y = fmaf(a.x, b.y, c.y);
  c.y = fmaf(-a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ float2 shfl_xor2(float2 v, int m) {
  v.x = __shfl_xor_sync(0xffffffffu, v.x, m);
  v.y = __shfl_xor_sync(0xffffffffu, v.y, m);
  return v;
}

// Compute-type traits: T = double (FP64) or float (FP32).
template <typename T> struct Cx;
template <> struct Cx<double> { using t = double2; };
template <> struct Cx<float> { using t = float2; };
template <typename T> using cplx = typename Cx<T>::t;

template <typename T> __device__ __forceinline__ cplx<T> to_t(double2 v);
template <> __device__ __forceinline__ double2 to_t<double>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 to_t<float>(double2 v) {
  return make_float2((float)v.x, (float)v.y);
}
template <typename T> __device__ __forceinline__ cplx<T> to_t(float2 v);
template <> __device__ __forceinline__ double2 to_t<double>(float2 v) { return make_double2(v.x, v.y); }
template <> __device__ __forceinline__ float2 to_t<float>(float2 v) { return v; }
__device__ __forceinline__ double2 to_d(double2 v) { return v; }
__device__ __forceinline__ double2 to_d(float2 v) { return make_double2(v.x, v.y); }
template <typename T> __device__ __forceinline__ cplx<T> czero() {
  cplx<T> z;
  z.x = 0;
  z.y = 0;
  return z;
}
// acc + v * x for a sparse-matrix value v (real double or complex double2)
template <typename T> __device__ __forceinline__ cplx<T> mfma(double v, cplx<T> x, cplx<T> acc) {
  const T r = (T)v;
  acc.x = fma(r, x.x, acc.x);
  acc.y = fma(r, x.y, acc.y);
  return acc;
}
template <typename T> __device__ __forceinline__ cplx<T> mfma(double2 v, cplx<T> x, cplx<T> acc) {
  return cfma(to_t<T>(v), x, acc);
}
template <typename T> __device__ __forceinline__ cplx<T> mfma(float v, cplx<T> x, cplx<T> acc) {
  const T r = (T)v;
  acc.x = fma(r, x.x, acc.x);
  acc.y = fma(r, x.y, acc.y);
  return acc;
}
template <typename T> __device__ __forceinline__ cplx<T> mfma(float2 v, cplx<T> x, cplx<T> acc) {
  return cfma(to_t<T>(v), x, acc);
}

// ------------------------------------------------------------------- SpMM -----
// Y = M X for up to two CSR matrices sharing the input block (A and B of the pencil).
// A warp works on 32/G rows at once, a group of G lanes per row; lane c of a group
// holds V consecutive columns of the block (c V .. c V + V - 1), so the group's gather
// of one block row X[col, :] is one coalesced 16 G-byte access (complex128, V = 1, or
// complex64, V = 2).  The group first loads up to 32 (column, value) pairs of its row,
// spread over its lanes, then walks them in batches of 8: column indices by shuffle,
// 8 independent block-row gathers in flight per lane, then the multiply-adds.  A row
// longer than 32 entries takes several rounds (a warp runs as many rounds as its
// longest row needs).  Each output row is written once, by its group.
template <typename VT>
struct CsrDev {
  const int* rowptr;
  const int* col;
  const VT* val;
};

__device__ __forceinline__ double shfl_val(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ float shfl_val(float v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ float2 shfl_val(float2 v, int src) {
  v.x = __shfl_sync(0xffffffffu, v.x, src);
  v.y = __shfl_sync(0xffffffffu, v.y, src);
  return v;
}
__device__ __forceinline__ double2 shfl_val(double2 v, int src) {
  v.x = __shfl_sync(0xffffffffu, v.x, src);
  v.y = __shfl_sync(0xffffffffu, v.y, src);
  return v;
}
template <typename VT> __device__ __forceinline__ VT zero_val();
template <> __device__ __forceinline__ double zero_val<double>() { return 0.0; }
template <> __device__ __forceinline__ double2 zero_val<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float zero_val<float>() { return 0.0f; }
template <> __device__ __forceinline__ float2 zero_val<float2>() { return make_float2(0.0f, 0.0f); }

// V consecutive complex values of the block row at p (V = 2: one 16-byte load).
// NC: through the read-only (non-coherent) data path.  Only a kernel that never writes
// the block during its lifetime may use it; the persistent kernel of the batched
// iteration, which writes blocks in one step and reads them in a later one, does not.
template <typename T, int V, bool NC>
__device__ __forceinline__ void load_xv(const cplx<T>* p, cplx<T> (&x)[V]) {
  if constexpr (V == 1) {
    x[0] = NC ? __ldg(p) : *p;
  } else {
    static_assert(V == 2 && sizeof(cplx<T>) == 8, "V = 2 loads two complex64 values");
    const float4* q4 = reinterpret_cast<const float4*>(p);
    const float4 q = NC ? __ldg(q4) : *q4;
    x[0] = make_float2(q.x, q.y);
    x[1] = make_float2(q.z, q.w);
  }
}

constexpr int SPMM_THREADS = 256;
constexpr int SPMM_BATCH = 8;

template <typename VT, typename T, int G, int V, bool NC>
__device__ __forceinline__ void spmm_group_row(const CsrDev<VT>& M, int r, int n, const cplx<T>* X,
                                               int ldx, int w, int c, int lane, double2* Y, int ldy) {
  constexpr int PER = 32 / G;  // (column, value) pairs each lane loads per round
  const bool active = r < n;
  const int j0 = active ? M.rowptr[r] : 0;
  const int j1 = active ? M.rowptr[r + 1] : 0;
  const int c0 = c * V;
  const bool colok = c0 < w;
  const int gbase = lane & ~(G - 1);
  cplx<T> acc[V];
#pragma unroll
  for (int v = 0; v < V; ++v) acc[v] = czero<T>();
  for (int base = j0; __any_sync(0xffffffffu, base < j1); base += 32) {
    const int cnt = max(0, min(32, j1 - base));
    const int wcnt = (int)__reduce_max_sync(0xffffffffu, (unsigned)cnt);
    int colr[PER];
    VT valr[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int e = c + G * q;
      colr[q] = e < cnt ? M.col[base + e] : 0;
      valr[q] = e < cnt ? M.val[base + e] : zero_val<VT>();
    }
#pragma unroll
    for (int tb = 0; tb < 32; tb += SPMM_BATCH) {
      if (tb >= wcnt) break;
      int cc[SPMM_BATCH];
      VT vv[SPMM_BATCH];
#pragma unroll
      for (int u = 0; u < SPMM_BATCH; ++u) {
        const int t = tb + u;
        cc[u] = __shfl_sync(0xffffffffu, colr[t / G], gbase + t % G);
        vv[u] = shfl_val(valr[t / G], gbase + t % G);
      }
      cplx<T> xv[SPMM_BATCH][V];
#pragma unroll
      for (int u = 0; u < SPMM_BATCH; ++u) {
        if (tb + u < cnt && colok) {
          load_xv<T, V, NC>(X + (size_t)cc[u] * ldx + c0, xv[u]);
        } else {
#pragma unroll
          for (int v = 0; v < V; ++v) xv[u][v] = czero<T>();
        }
      }
#pragma unroll
      for (int u = 0; u < SPMM_BATCH; ++u)
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = mfma<T>(vv[u], xv[u][v], acc[v]);
    }
  }
  if (active) {
#pragma unroll
    for (int v = 0; v < V; ++v)
      if (c0 + v < w) Y[(size_t)r * ldy + c0 + v] = to_d(acc[v]);
  }
}

// T is the arithmetic (double, or float in the FP32 bulk phase; X is then the
// complex64 copy of the block); the outputs are complex128.  Requires w <= G V; with
// V = 2 the rows of X must be 16-byte aligned (ldx even).
template <typename VTA, typename VTB, typename T, int G, int V, bool NC = true>
__device__ __forceinline__ void spmm_body(const Cta& cta, int n, CsrDev<VTA> A, CsrDev<VTB> B, int hasB,
                                                            const cplx<T>* X, int ldx, int w,
                                                            double2* AX, int ldax,
                                                            double2* BX, int ldbx) {
  constexpr int RPW = 32 / G;
  const int lane = threadIdx.x & 31;
  const int g = lane / G, c = lane - g * G;
  const int warp = (cta.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (cta.gx * blockDim.x) >> 5;
  for (int rb = warp * RPW; rb < n; rb += nwarps * RPW) {
    spmm_group_row<VTA, T, G, V, NC>(A, rb + g, n, X, ldx, w, c, lane, AX, ldax);
    if (hasB) spmm_group_row<VTB, T, G, V, NC>(B, rb + g, n, X, ldx, w, c, lane, BX, ldbx);
  }
}
template <typename VTA, typename VTB, typename T, int G, int V>
__global__ void __launch_bounds__(SPMM_THREADS) spmm_kernel(int n, CsrDev<VTA> A, CsrDev<VTB> B, int hasB,
                                                            const cplx<T>* __restrict__ X, int ldx, int w,
                                                            double2* __restrict__ AX, int ldax,
                                                            double2* __restrict__ BX, int ldbx) {
  spmm_body<VTA, VTB, T, G, V>(Cta::hw(), n, A, B, hasB, X, ldx, w, AX, ldax, BX, ldbx);
}

// ------------------------------------------------------------------- Gram -----
// Split-n Gram product over the rows:  partial[b][o] = sum over rows of chunk b of
// conj(X[r][i_o]) Y[r][j_o], Y the column concatenation of Y0 (wy0 cols) and Y1.
// Outputs o enumerate the wx x wy result row-major, or only its upper triangle
// (i <= j) when herm = 1 (X^* X, whose lower triangle is the conjugate transpose).
//
// FP64 on GB300 issues at ~2 DFMA/clk/SM, so every issued DFMA must be useful:
// thread g of a CTA owns ACC consecutive outputs (all valid except possibly in the
// very last thread, which computes padding it then discards), and when the CTA has
// fewer than 256 output groups the threads split the staged rows into RG row
// groups whose partial sums are added in shared memory at the end.  The grid is
// (nchunk, ntile): chunk b of rows, tile t of G*ACC outputs.
constexpr int GRAM_THREADS = 256;
constexpr int GRAM_ROWS = 16;

__device__ __forceinline__ void gram_index(int o, int wx, int wy, int herm, int& i, int& j) {
  if (!herm) {
    i = o / wy;
    j = o - i * wy;
    return;
  }
  // upper triangle, row-major: row i starts at i*wx - i*(i-1)/2
  int r = 0, off = 0;
  while (r + 1 < wx && off + (wx - r) <= o) {
    off += wx - r;
    ++r;
  }
  i = r;
  j = r + (o - off);
}

template <int ACC, typename T = double>
__device__ __forceinline__ void gram_partial_body(const Cta& cta,
    int n, int rows_per_chunk, const double2* X, int ldx, int wx,
                    const double2* Y0, int ldy0, int wy0, const double2* Y1,
                    int ldy1, int wy1, int herm, int nout, int G, int RG, double2* partial,
                    const int* skip) {
  if (skip && *skip == 0) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  using C2 = cplx<T>;
  C2* sm = reinterpret_cast<C2*>(smraw);
  const int wy = wy0 + wy1;
  C2* xs = sm;                         // GRAM_ROWS x wx
  C2* ys = sm + GRAM_ROWS * wx;        // GRAM_ROWS x wy
  const int tid = threadIdx.x;
  const int g = tid % G, rg = tid / G;
  const int tile0 = cta.y * G * ACC;
  const int o0 = tile0 + g * ACC;
  const bool active = rg < RG && o0 < nout;
  const int r0 = cta.x * rows_per_chunk;
  const int r1 = min(n, r0 + rows_per_chunk);
  C2 acc[ACC];
  int oi[ACC], oj[ACC];
#pragma unroll
  for (int t = 0; t < ACC; ++t) {
    acc[t] = czero<T>();
    const int o = min(o0 + t, nout - 1);
    gram_index(o, wx, wy, herm, oi[t], oj[t]);
  }
  for (int rb = r0; rb < r1; rb += GRAM_ROWS) {
    const int nr = min(GRAM_ROWS, r1 - rb);
    __syncthreads();
    for (int e = tid; e < nr * wx; e += blockDim.x) {
      const int rr = e / wx, cc = e - rr * wx;
      xs[rr * wx + cc] = to_t<T>(X[(size_t)(rb + rr) * ldx + cc]);
    }
    for (int e = tid; e < nr * wy; e += blockDim.x) {
      const int rr = e / wy, cc = e - rr * wy;
      ys[rr * wy + cc] = to_t<T>(cc < wy0 ? Y0[(size_t)(rb + rr) * ldy0 + cc]
                                          : Y1[(size_t)(rb + rr) * ldy1 + (cc - wy0)]);
    }
    __syncthreads();
    if (active) {
      for (int rr = rg; rr < nr; rr += RG) {
        const C2* xr = xs + rr * wx;
        const C2* yr = ys + rr * wy;
#pragma unroll
        for (int t = 0; t < ACC; ++t) acc[t] = cfmaconj(xr[oi[t]], yr[oj[t]], acc[t]);
      }
    }
  }
  // add the RG row-group partials: red[rg][g*ACC + t]
  __syncthreads();
  C2* red = sm;
  const int per = G * ACC;
  if (rg < RG) {
#pragma unroll
    for (int t = 0; t < ACC; ++t) red[rg * per + g * ACC + t] = acc[t];
  }
  __syncthreads();
  double2* out = partial + (size_t)cta.x * nout;
  for (int e = tid; e < per; e += blockDim.x) {
    const int o = tile0 + e;
    if (o >= nout) break;
    double2 s = to_d(red[e]);
    for (int q = 1; q < RG; ++q) s = cadd(s, to_d(red[q * per + e]));
    out[o] = s;
  }
}
template <int ACC, typename T = double>
__global__ void __launch_bounds__(GRAM_THREADS)
gram_partial_kernel(int n, int rows_per_chunk, const double2* __restrict__ X, int ldx, int wx,
                    const double2* __restrict__ Y0, int ldy0, int wy0, const double2* __restrict__ Y1,
                    int ldy1, int wy1, int herm, int nout, int G, int RG, double2* __restrict__ partial,
                    const int* skip) {
  gram_partial_body<ACC, T>(Cta::hw(), n, rows_per_chunk, X, ldx, wx, Y0, ldy0, wy0, Y1, ldy1, wy1, herm,
      nout, G, RG, partial, skip);
}

// Gram of FP32-valued blocks with exact products (bulk phase of the mixed mode, whose
// blocks hold FP32 values in complex128 storage).  Each real product a*b is formed
// exactly as the float pair (p, e) = (a*b, fma(a, b, -a*b)) on the FP32 pipe; a tile of
// rows is summed in a compensated float pair (TwoSum on the high parts, the low parts
// and rounding errors added into a second float), and each tile's pair is added into
// FP64 accumulators.  The FP64 pipe (about 2 DFMA per clock per SM on GB300) sees only
// the conversions and the per-tile additions.
// Error-free transformations written with the _rn intrinsics, which the compiler never
// contracts into FMAs (a contracted a*b + s would break the exact product / TwoSum).
__device__ __forceinline__ void two_sum_acc(float& sh, float& sl, float p, float pe) {
  const float s = __fadd_rn(sh, p);
  const float bb = __fsub_rn(s, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(err, pe));
}
__device__ __forceinline__ void exact_prod_acc(float& sh, float& sl, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float pe = __fmaf_rn(a, b, -p);  // exact: a*b = p + pe for float a, b
  two_sum_acc(sh, sl, p, pe);
}

// Rows per staged tile of the exact-product Gram, and rows a thread sums in its float
// pair between flushes to FP64 (compensated-sum error <= X32_FLUSH * 2^-48 * sum |p|).
constexpr int X32_ROWS = 32;
constexpr int X32_FLUSH = 32;

template <int ACC>
__device__ __forceinline__ void gram_partial_x32_body(const Cta& cta,
    int n, int rows_per_chunk, const double2* X, int ldx, int wx,
                        const double2* Y0, int ldy0, int wy0, const double2* Y1,
                        int ldy1, int wy1, int herm, int nout, int G, int RG, double2* partial,
                        const int* skip) {
  if (skip && *skip == 0) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* xs = reinterpret_cast<float2*>(smraw);  // X32_ROWS x wx
  const int wy = wy0 + wy1;
  float2* ys = xs + X32_ROWS * wx;                 // X32_ROWS x wy
  const int tid = threadIdx.x;
  const int g = tid % G, rg = tid / G;
  const int tile0 = cta.y * G * ACC;
  const int o0 = tile0 + g * ACC;
  const bool active = rg < RG && o0 < nout;
  const int r0 = cta.x * rows_per_chunk;
  const int r1 = min(n, r0 + rows_per_chunk);
  double2 acc[ACC];
  int oi[ACC], oj[ACC];
#pragma unroll
  for (int t = 0; t < ACC; ++t) {
    acc[t] = make_double2(0.0, 0.0);
    const int o = min(o0 + t, nout - 1);
    gram_index(o, wx, wy, herm, oi[t], oj[t]);
  }
  // float-pair accumulators, flushed to FP64 after about X32_FLUSH rows of this thread
  float rh[ACC], rl[ACC], ih[ACC], il[ACC];
#pragma unroll
  for (int t = 0; t < ACC; ++t) rh[t] = rl[t] = ih[t] = il[t] = 0.0f;
  const int tiles_per_flush = max(1, (X32_FLUSH * RG) / X32_ROWS);
  int tile = 0;
  for (int rb = r0; rb < r1; rb += X32_ROWS, ++tile) {
    const int nr = min(X32_ROWS, r1 - rb);
    __syncthreads();
    for (int e = tid; e < nr * wx; e += blockDim.x) {
      const int rr = e / wx, cc = e - rr * wx;
      xs[rr * wx + cc] = to_t<float>(X[(size_t)(rb + rr) * ldx + cc]);
    }
    for (int e = tid; e < nr * wy; e += blockDim.x) {
      const int rr = e / wy, cc = e - rr * wy;
      ys[rr * wy + cc] = to_t<float>(cc < wy0 ? Y0[(size_t)(rb + rr) * ldy0 + cc]
                                              : Y1[(size_t)(rb + rr) * ldy1 + (cc - wy0)]);
    }
    __syncthreads();
    if (active) {
      for (int rr = rg; rr < nr; rr += RG) {
        const float2* xr = xs + rr * wx;
        const float2* yr = ys + rr * wy;
#pragma unroll
        for (int t = 0; t < ACC; ++t) {
          const float2 a = xr[oi[t]], b = yr[oj[t]];
          // conj(a) b = (ar br + ai bi) + i (ar bi - ai br)
          exact_prod_acc(rh[t], rl[t], a.x, b.x);
          exact_prod_acc(rh[t], rl[t], a.y, b.y);
          exact_prod_acc(ih[t], il[t], a.x, b.y);
          exact_prod_acc(ih[t], il[t], -a.y, b.x);
        }
      }
      if ((tile + 1) % tiles_per_flush == 0 || rb + X32_ROWS >= r1) {
#pragma unroll
        for (int t = 0; t < ACC; ++t) {
          acc[t].x += (double)rh[t] + (double)rl[t];
          acc[t].y += (double)ih[t] + (double)il[t];
          rh[t] = rl[t] = ih[t] = il[t] = 0.0f;
        }
      }
    }
  }
  __syncthreads();
  double2* red = reinterpret_cast<double2*>(smraw);
  const int per = G * ACC;
  if (rg < RG) {
#pragma unroll
    for (int t = 0; t < ACC; ++t) red[rg * per + g * ACC + t] = acc[t];
  }
  __syncthreads();
  double2* out = partial + (size_t)cta.x * nout;
  for (int e = tid; e < per; e += blockDim.x) {
    const int o = tile0 + e;
    if (o >= nout) break;
    double2 sum = red[e];
    for (int q = 1; q < RG; ++q) sum = cadd(sum, red[q * per + e]);
    out[o] = sum;
  }
}
template <int ACC>
__global__ void __launch_bounds__(GRAM_THREADS)
gram_partial_x32_kernel(int n, int rows_per_chunk, const double2* __restrict__ X, int ldx, int wx,
                        const double2* __restrict__ Y0, int ldy0, int wy0, const double2* __restrict__ Y1,
                        int ldy1, int wy1, int herm, int nout, int G, int RG, double2* __restrict__ partial,
                        const int* skip) {
  gram_partial_x32_body<ACC>(Cta::hw(), n, rows_per_chunk, X, ldx, wx, Y0, ldy0, wy0, Y1, ldy1, wy1, herm,
      nout, G, RG, partial, skip);
}

// C = sum_b partial[b] (deterministic): one warp per output, lane l adds the chunks
// l, l+32, ... in order, then a fixed xor-shuffle tree.  The output enumeration is
// mapped back to (i, j) of the wx x wy result (row-major, ld = wy); with herm = 1 the
// lower triangle is filled with the conjugate transpose.
constexpr int GRED_WARPS = 8;
// C row stride ldc (>= the row length: wy, or wx for the transposed form), so that a
// product can fill a column block of a wider C.
__device__ __forceinline__ void gram_reduce_body(const Cta& cta, int nchunk, int nout, int wx, int wy, int herm,
                                   const double2* partial, double2* C, int ldc,
                                   const int* skip) {
  if (skip && *skip == 0) return;
  const int lane = threadIdx.x & 31;
  const int o = cta.x * GRED_WARPS + (threadIdx.x >> 5);
  if (o >= nout) return;
  double2 s = make_double2(0.0, 0.0);
  for (int b = lane; b < nchunk; b += 32) s = cadd(s, partial[(size_t)b * nout + o]);
  for (int off = 16; off > 0; off >>= 1) s = cadd(s, shfl_xor2(s, off));
  if (lane == 0) {
    if (herm == 2) {  // the partials hold the transposed product: C(j, i) = conj(partial (i, j))
      const int i = o / wy, j = o - i * wy;
      C[(size_t)j * ldc + i] = make_double2(s.x, -s.y);
      return;
    }
    int i, j;
    gram_index(o, wx, wy, herm, i, j);
    C[(size_t)i * ldc + j] = s;
    if (herm && i != j) C[(size_t)j * ldc + i] = make_double2(s.x, -s.y);
  }
}
__global__ void gram_reduce_kernel(int nchunk, int nout, int wx, int wy, int herm,
                                   const double2* __restrict__ partial, double2* __restrict__ C, int ldc,
                                   const int* skip) {
  gram_reduce_body(Cta::hw(), nchunk, nout, wx, wy, herm, partial, C, ldc, skip);
}

// ---------------------------------------------------------------- combine -----
// Y[r][0:c] = beta * Y[r][0:c] + sum_t alpha_t * (X_t[r][0:w_t] C_t), C_t is w_t x c
// row-major on the device.  Rows are staged in shared memory before any write, so
// Y may alias the rows of any X_t (in-place block transforms such as X <- X R^{-1}).
// Output columns [0, c_split) go to Y, columns [c_split, c_store) to Y2 (column
// c - c_split of Y2), and columns [c_store, c) are not stored: their |.|^2 is summed
// per CTA into normpart[blockIdx.x][col - c_store].  beta applies to stored columns.
// With skip != null and *skip == 0 the kernel does nothing.
constexpr int COMB_MAX_IN = 4;
constexpr int COMB_MAX_NORMS = 128;
struct CombIn {
  const double2* X;
  int ldx;
  int w;
  const double2* C;  // w x c, row stride ldc
  int ldc;
  double2 alpha;
};
struct CombArgs {
  CombIn in[COMB_MAX_IN];
  int nin;
  double2* Y;
  int ldy;
  double2* Y2;
  int ldy2;
  int c;
  int c_split;      // == c_store when there is no second output
  int c_store;      // == c when nothing but stores
  int beta_one;     // 1: Y += ..., 0: Y = ...
  double* normpart; // [gridDim.x][c - c_store] or null
  const int* skip;
  int upper;        // 1: single input whose C is upper triangular (X R^{-1}): sum j <= col
  int rows_tile;    // rows staged per tile (comb_rows_tile, halved on the host while the
                    // staging would not fit in shared memory)
};
constexpr int COMB_THREADS = 256;

// Rows staged per tile (at most).  For the triangular form the tile is 32 rows and
// threads are mapped column-major (a warp = 32 rows of one output column), so the loop
// bound j <= col is uniform across each warp: no predicated-off DFMAs.
__host__ __device__ inline int comb_rows_tile(int c, int upper = 0) {
  if (upper) return 32;
  return c >= COMB_THREADS ? 1 : COMB_THREADS / c;
}

__device__ __forceinline__ double2* comb_out(const CombArgs& a, int r, int cc) {
  return cc < a.c_split ? a.Y + (size_t)r * a.ldy + cc : a.Y2 + (size_t)r * a.ldy2 + (cc - a.c_split);
}

template <typename T = double>
__device__ __forceinline__ void combine_body(const Cta& cta, int n, int rows_per_cta, CombArgs a) {
  if (a.skip && *a.skip == 0) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  using C2 = cplx<T>;
  C2* sm = reinterpret_cast<C2*>(smraw);
  // layout: C_0 .. C_{nin-1} (w_t x c each, pre-scaled by alpha_t), then the staged
  // rows: rows_tile x (sum w_t) X values, then rows_tile x c old Y values (beta = 1)
  int wsum = 0;
  for (int t = 0; t < a.nin; ++t) wsum += a.in[t].w;
  C2* cs = sm;
  C2* xs = cs + wsum * a.c;
  const int rows_tile = a.rows_tile;
  C2* ys = xs + rows_tile * wsum;
  __shared__ double nsum[COMB_MAX_NORMS];
  {
    int off = 0;
    for (int t = 0; t < a.nin; ++t) {
      const int sz = a.in[t].w * a.c;
      for (int e = threadIdx.x; e < sz; e += blockDim.x)
        cs[off + e] = to_t<T>(cmul(a.in[t].alpha, a.in[t].C[(size_t)(e / a.c) * a.in[t].ldc + e % a.c]));
      off += sz;
    }
  }
  const int nnorm = a.c - a.c_store;
  for (int e = threadIdx.x; e < nnorm; e += blockDim.x) nsum[e] = 0.0;
  const int r0 = cta.x * rows_per_cta;
  const int r1 = min(n, r0 + rows_per_cta);
  for (int rb = r0; rb < r1; rb += rows_tile) {
    const int nr = min(rows_tile, r1 - rb);
    __syncthreads();
    int off = 0;
    for (int t = 0; t < a.nin; ++t) {
      const int w = a.in[t].w;
      for (int e = threadIdx.x; e < nr * w; e += blockDim.x) {
        const int rr = e / w, cc = e - rr * w;
        xs[rr * wsum + off + cc] = to_t<T>(a.in[t].X[(size_t)(rb + rr) * a.in[t].ldx + cc]);
      }
      off += w;
    }
    if (a.beta_one) {
      for (int e = threadIdx.x; e < nr * a.c_store; e += blockDim.x) {
        const int rr = e / a.c_store, cc = e - rr * a.c_store;
        ys[rr * a.c + cc] = to_t<T>(*comb_out(a, rb + rr, cc));
      }
    }
    __syncthreads();
    const int nwork = a.upper ? rows_tile * a.c : nr * a.c;
    for (int e = threadIdx.x; e < nwork; e += blockDim.x) {
      int rr, cc;
      if (a.upper) {
        rr = e % rows_tile;
        cc = e / rows_tile;
        if (rr >= nr) continue;
      } else {
        rr = e / a.c;
        cc = e - rr * a.c;
      }
      C2 acc = (a.beta_one && cc < a.c_store) ? ys[rr * a.c + cc] : czero<T>();
      const C2* xr = xs + rr * wsum;
      const int jend = a.upper ? cc + 1 : wsum;
      for (int j = 0; j < jend; ++j) acc = cfma(xr[j], cs[j * a.c + cc], acc);
      if (cc < a.c_store) {
        *comb_out(a, rb + rr, cc) = to_d(acc);
      } else {
        const double2 v = to_d(acc);
        atomicAdd(&nsum[cc - a.c_store], v.x * v.x + v.y * v.y);
      }
    }
  }
  if (a.normpart) {
    __syncthreads();
    for (int e = threadIdx.x; e < nnorm; e += blockDim.x)
      a.normpart[(size_t)cta.x * nnorm + e] = nsum[e];
  }
}
template <typename T = double>
__global__ void combine_kernel(int n, int rows_per_cta, CombArgs a) {
  combine_body<T>(Cta::hw(), n, rows_per_cta, a);
}

// normout[j] = sum_b normpart[b][j]  (fixed order)
// one warp per column, lane-strided then a fixed shuffle tree (deterministic)
__device__ __forceinline__ void norm_reduce_body(const Cta& cta, int nb, int nc, const double* part,
                                   double* out) {
  const int lane = threadIdx.x & 31;
  const int j = cta.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= nc) return;
  double s = 0.0;
  for (int b = lane; b < nb; b += 32) s += part[(size_t)b * nc + j];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) out[j] = s;
}
__global__ void norm_reduce_kernel(int nb, int nc, const double* __restrict__ part,
                                   double* __restrict__ out) {
  norm_reduce_body(Cta::hw(), nb, nc, part, out);
}

// Y = alpha X1 + beta X2 (elementwise, n x w)
__device__ __forceinline__ void axpby_body(const Cta& cta,
    int n, int w, double2 alpha, const double2* X1, int ld1,
                             double2 beta, const double2* X2, int ld2,
                             double2* Y, int ldy) {
  const size_t total = (size_t)n * w;
  for (size_t e = cta.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)cta.gx * blockDim.x) {
    const int r = (int)(e / w), c = (int)(e - (size_t)r * w);
    double2 v = cmul(alpha, X1[(size_t)r * ld1 + c]);
    v = cfma(beta, X2[(size_t)r * ld2 + c], v);
    Y[(size_t)r * ldy + c] = v;
  }
}
__global__ void axpby_kernel(int n, int w, double2 alpha, const double2* __restrict__ X1, int ld1,
                             double2 beta, const double2* __restrict__ X2, int ld2,
                             double2* __restrict__ Y, int ldy) {
  axpby_body(Cta::hw(), n, w, alpha, X1, ld1, beta, X2, ld2, Y, ldy);
}

// Copy an n x w block (any lds)
__device__ __forceinline__ void copy_block_body(const Cta& cta,
    int n, int w, const double2* X, int ldx,
                                  double2* Y, int ldy) {
  const size_t total = (size_t)n * w;
  for (size_t e = cta.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)cta.gx * blockDim.x) {
    const int r = (int)(e / w), c = (int)(e - (size_t)r * w);
    Y[(size_t)r * ldy + c] = X[(size_t)r * ldx + c];
  }
}
__global__ void copy_block_kernel(int n, int w, const double2* __restrict__ X, int ldx,
                                  double2* __restrict__ Y, int ldy) {
  copy_block_body(Cta::hw(), n, w, X, ldx, Y, ldy);
}

// complex128 block -> complex64 block (ld = w), for the FP32 sparse products.
__device__ __forceinline__ void to_c64_body(const Cta& cta,
    int n, int w, const double2* X, int ldx, float2* Y,
                              int ldy) {
  const size_t total = (size_t)n * w;
  for (size_t e = cta.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)cta.gx * blockDim.x) {
    const int r = (int)(e / w), c = (int)(e - (size_t)r * w);
    const double2 v = X[(size_t)r * ldx + c];
    Y[(size_t)r * ldy + c] = make_float2((float)v.x, (float)v.y);
  }
}
__global__ void to_c64_kernel(int n, int w, const double2* __restrict__ X, int ldx, float2* __restrict__ Y,
                              int ldy) {
  to_c64_body(Cta::hw(), n, w, X, ldx, Y, ldy);
}

// Real n x w (row-major, ld = w) to complex block.
__global__ void real_to_complex_kernel(int n, int w, const double* __restrict__ X,
                                       double2* __restrict__ Y, int ldy) {
  const size_t total = (size_t)n * w;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / w), c = (int)(e - (size_t)r * w);
    Y[(size_t)r * ldy + c] = make_double2(X[e], 0.0);
  }
}

// --------------------------------------------------------- preconditioners ----
// Jacobi: Y[r][c] = d[r] X[r][c]
template <typename T = double>
__device__ __forceinline__ void jacobi_body(const Cta& cta,
    int n, int w, const double2* d, const double2* X,
                              int ldx, double2* Y, int ldy) {
  const size_t total = (size_t)n * w;
  for (size_t e = cta.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)cta.gx * blockDim.x) {
    const int r = (int)(e / w), c = (int)(e - (size_t)r * w);
    Y[(size_t)r * ldy + c] = to_d(cmul(to_t<T>(d[r]), to_t<T>(X[(size_t)r * ldx + c])));
  }
}
template <typename T = double>
__global__ void jacobi_kernel(int n, int w, const double2* __restrict__ d, const double2* __restrict__ X,
                              int ldx, double2* __restrict__ Y, int ldy) {
  jacobi_body<T>(Cta::hw(), n, w, d, X, ldx, Y, ldy);
}

// Block-Jacobi: for block b (rows [b bs, b bs + nb_b)), Y_b = Tinv_b X_b with Tinv_b
// stored as bs x bs row-major (a ragged last block is identity-padded).  One CTA
// handles BJ_BLOCKS_PER_CTA consecutive blocks; X rows are staged in shared memory,
// so Y may equal X.
constexpr int BJ_THREADS = 256;
template <typename T = double, typename TT = double2>
__device__ __forceinline__ void block_jacobi_body(const Cta& cta,
    int n, int bs, int w, const TT* Tinv,
                                    const double2* X, int ldx,
                                    double2* Y, int ldy, int blocks_per_cta) {
  extern __shared__ __align__(16) unsigned char smraw[];
  using C2 = cplx<T>;
  C2* xs = reinterpret_cast<C2*>(smraw);  // blocks_per_cta * bs rows x w
  const int nblocks = (n + bs - 1) / bs;
  const int b0 = cta.x * blocks_per_cta;
  const int b1 = min(nblocks, b0 + blocks_per_cta);
  if (b0 >= b1) return;
  const int rstart = b0 * bs;
  const int rend = min(n, b1 * bs);
  const int nrows = rend - rstart;
  for (int e = threadIdx.x; e < nrows * w; e += blockDim.x) {
    const int rr = e / w, cc = e - rr * w;
    xs[rr * w + cc] = to_t<T>(X[(size_t)(rstart + rr) * ldx + cc]);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nrows * w; e += blockDim.x) {
    const int rr = e / w, cc = e - rr * w;
    const int blk = rr / bs, i = rr - blk * bs;
    const int gb = b0 + blk;
    const int rows_in_blk = min(bs, n - gb * bs);
    const TT* Tm = Tinv + (size_t)gb * bs * bs + (size_t)i * bs;
    C2 acc = czero<T>();
    const C2* xb = xs + (size_t)blk * bs * w;
    for (int j = 0; j < rows_in_blk; ++j) acc = cfma(to_t<T>(Tm[j]), xb[j * w + cc], acc);
    Y[(size_t)(rstart + rr) * ldy + cc] = to_d(acc);
  }
}
template <typename T = double, typename TT = double2>
__global__ void block_jacobi_kernel(int n, int bs, int w, const TT* __restrict__ Tinv,
                                    const double2* __restrict__ X, int ldx,
                                    double2* __restrict__ Y, int ldy, int blocks_per_cta) {
  block_jacobi_body<T, TT>(Cta::hw(), n, bs, w, Tinv, X, ldx, Y, ldy, blocks_per_cta);
}

// Setup: extract the diagonal blocks of K = A - sigma B (B = I if hasB = 0) into
// blocks[b] (bs x bs, identity-padded past n).  One thread per row.
template <typename VTA, typename VTB>
__global__ void extract_blocks_kernel(int n, int bs, CsrDev<VTA> A, CsrDev<VTB> B, int hasB,
                                      double2 sigma, double2* __restrict__ blocks, int nblocks) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nblocks * bs) return;
  const int b = r / bs, i = r - b * bs;
  double2* row = blocks + (size_t)b * bs * bs + (size_t)i * bs;
  for (int j = 0; j < bs; ++j) row[j] = make_double2(0.0, 0.0);
  if (r >= n) {
    row[i] = make_double2(1.0, 0.0);
    return;
  }
  const int c0 = b * bs;
  for (int jj = A.rowptr[r]; jj < A.rowptr[r + 1]; ++jj) {
    const int cc = A.col[jj];
    if (cc >= c0 && cc < c0 + bs) row[cc - c0] = vfma(A.val[jj], make_double2(1.0, 0.0), row[cc - c0]);
  }
  const double2 ms = make_double2(-sigma.x, -sigma.y);
  if (hasB) {
    for (int jj = B.rowptr[r]; jj < B.rowptr[r + 1]; ++jj) {
      const int cc = B.col[jj];
      if (cc >= c0 && cc < c0 + bs) {
        double2 v = vfma(B.val[jj], make_double2(1.0, 0.0), make_double2(0.0, 0.0));
        row[cc - c0] = cfma(ms, v, row[cc - c0]);
      }
    }
  } else {
    row[i] = cadd(row[i], ms);
  }
}

// Setup: invert each bs x bs block in place by Gauss-Jordan elimination with partial
// pivoting, one warp per block (bs <= 32) on a [bs][2 bs] shared-memory tableau.
// flag[0] is set to 1 + block index of a block whose pivot vanishes.
__global__ void invert_blocks_kernel(int nblocks, int bs, double2* __restrict__ blocks, int* flag) {
  extern __shared__ double2 sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wpc = blockDim.x >> 5;
  const int b = blockIdx.x * wpc + warp;
  if (b >= nblocks) return;
  double2* tab = sm + (size_t)warp * bs * 2 * bs;
  double2* blk = blocks + (size_t)b * bs * bs;
  const int w2 = 2 * bs;
  for (int e = lane; e < bs * w2; e += 32) {
    const int i = e / w2, j = e - i * w2;
    tab[e] = j < bs ? blk[i * bs + j] : make_double2(j - bs == i ? 1.0 : 0.0, 0.0);
  }
  __syncwarp();
  double scale = 0.0;
  for (int e = 0; e < bs * bs; ++e) scale = fmax(scale, fabs(blk[e].x) + fabs(blk[e].y));
  bool singular = false;
  for (int p = 0; p < bs; ++p) {
    // pivot search (every lane does it: bs <= 32 values)
    int piv = p;
    double best = -1.0;
    for (int i = p; i < bs; ++i) {
      const double v = hypot(tab[i * w2 + p].x, tab[i * w2 + p].y);
      if (v > best) { best = v; piv = i; }
    }
    if (!(best > 1e-300 && best > 1e-14 * scale)) { singular = true; break; }
    if (piv != p) {
      for (int j = lane; j < w2; j += 32) {
        double2 t = tab[p * w2 + j];
        tab[p * w2 + j] = tab[piv * w2 + j];
        tab[piv * w2 + j] = t;
      }
      __syncwarp();
    }
    const double2 d = tab[p * w2 + p];
    const double dd = d.x * d.x + d.y * d.y;
    const double2 inv = make_double2(d.x / dd, -d.y / dd);
    __syncwarp();
    for (int j = lane; j < w2; j += 32) tab[p * w2 + j] = cmul(inv, tab[p * w2 + j]);
    __syncwarp();
    // eliminate column p from all other rows: row i -= tab[i][p] * row p
    for (int i = 0; i < bs; ++i) {
      if (i == p) continue;
      const double2 f = tab[i * w2 + p];
      __syncwarp();
      for (int j = lane; j < w2; j += 32) {
        const double2 v = tab[p * w2 + j];
        tab[i * w2 + j] = csub(tab[i * w2 + j], cmul(f, v));
      }
      __syncwarp();
    }
  }
  if (singular) {
    if (lane == 0) atomicCAS(flag, 0, 1 + b);
    return;
  }
  for (int e = lane; e < bs * bs; e += 32) {
    const int i = e / bs, j = e - i * bs;
    blk[e] = tab[i * w2 + bs + j];
  }
}

// Setup: Jacobi diagonal d[r] = 1 / (A[r][r] - sigma B[r][r]).
template <typename VTA, typename VTB>
__global__ void jacobi_setup_kernel(int n, CsrDev<VTA> A, CsrDev<VTB> B, int hasB, double2 sigma,
                                    double2* __restrict__ d) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  double2 v = make_double2(0.0, 0.0);
  for (int jj = A.rowptr[r]; jj < A.rowptr[r + 1]; ++jj)
    if (A.col[jj] == r) v = vfma(A.val[jj], make_double2(1.0, 0.0), v);
  double2 bv = make_double2(hasB ? 0.0 : 1.0, 0.0);
  if (hasB)
    for (int jj = B.rowptr[r]; jj < B.rowptr[r + 1]; ++jj)
      if (B.col[jj] == r) bv = vfma(B.val[jj], make_double2(1.0, 0.0), bv);
  d[r] = csub(v, cmul(sigma, bv));
}

__global__ void reciprocal_kernel(int n, double2* __restrict__ d) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const double2 v = d[r];
  const double dd = v.x * v.x + v.y * v.y;
  d[r] = make_double2(v.x / dd, -v.y / dd);
}

// ------------------------------------------------------ Cholesky QR helpers ----
// Single-CTA Cholesky of the Hermitian w x w Gram matrix G (row-major) and the
// inverse of its upper triangular factor: G = R^* R, R(j,j) > 0, Rinv = R^{-1}.
// If the factorisation breaks down (a pivot <= eps_rel * max diag), the kernel
// retries once on G + shift I with shift = 11 (n w + w (w+1)) u ||G||_F (the shift of
// shifted Cholesky QR, Fukaya et al. 2020) and sets status[0] = 1 (shift used);
// status[0] = 2 if that fails too.  fallback_counter[0] counts shifted retries and
// fallback_counter[1] final failures.  Rout (may be null) receives R itself.  When `skip_if_zero` is non-null and *skip_if_zero
// is 0, the kernel writes the identity and returns (used for the conditional third
// pass of shifted Cholesky QR).
// 1 / sqrt(a) for a finite a > 0: the exponent is scaled by a power of 4 into [1, 4) in
// the bits (exact), an FP32 seed is refined by two Newton-Raphson steps for the reciprocal
// square root, y <- y (3 - a y^2) / 2 (each step doubles the correct bits: ~23 -> 46 -> 92),
// and the scaling is undone.  Accurate to a few ulp; on GB300 a dependent FP64 operation
// takes ~70 cycles, and this chain is about half as long as sqrt followed by a division.
__device__ __forceinline__ double rsqrt_newton(double a) {
  const long long b = __double_as_longlong(a);
  const int e = (int)((b >> 52) & 0x7FF) - 1023;         // a = f 2^e, f in [1, 2) (normal a)
  const int h = e >> 1;                                   // floor(e / 2)
  const double as = __longlong_as_double(b - ((long long)(2 * h) << 52));  // a 2^(-2h) in [1, 4)
  double y = (double)rsqrtf((float)as);
  const double ha = 0.5 * as;
#pragma unroll
  for (int it = 0; it < 2; ++it) y = y * fma(-ha * y, y, 1.5);
  return __longlong_as_double(__double_as_longlong(y) - ((long long)h << 52));  // y 2^(-h)
}

// work: null = the two w x w work arrays in dynamic shared memory; else 2 w^2 values of
// global memory owned by the caller (the persistent kernel, whose CTAs cannot all hold
// 32 w^2 bytes of shared memory for a wide block).
__device__ __forceinline__ void chol_inv_body(const Cta& cta, int w, int64_t n, const double2* G,
                                double2* Rinv, int* status, const int* skip_if_zero,
                                int* fallback_counter, double2* Rout, double2* work = nullptr) {
  extern __shared__ double2 sm[];
  double2* a = work ? work : sm;  // w x w working copy -> R (upper)
  double2* inv = a + w * w;       // w x w -> R^{-1}
  __shared__ int fail;
  __shared__ double shift, piv_r, piv_ri;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (skip_if_zero && *skip_if_zero == 0) {
    for (int e = tid; e < w * w; e += nt) {
      const int i = e / w, j = e - i * w;
      Rinv[e] = make_double2(i == j ? 1.0 : 0.0, 0.0);
    }
    return;
  }
  // G -> inv (as a staging copy) in parallel; ||G||_F by a block reduction
  __shared__ double red[32];
  double f = 0.0;
  for (int e = tid; e < w * w; e += nt) {
    const double2 v = G[e];
    inv[e] = v;
    f += v.x * v.x + v.y * v.y;
  }
  for (int off = 16; off > 0; off >>= 1) f += __shfl_xor_sync(0xffffffffu, f, off);
  if ((tid & 31) == 0) red[tid >> 5] = f;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int q = 0; q < (nt + 31) / 32; ++q) t += red[q];
    const double u = 1.1102230246251565e-16;
    shift = 11.0 * ((double)n * w + (double)w * (w + 1)) * u * sqrt(t);
    if (status) status[0] = 0;
  }
  for (int attempt = 0; attempt < 2; ++attempt) {
    __syncthreads();
    for (int e = tid; e < w * w; e += nt) {
      const int i = e / w, j = e - i * w;
      double2 v = inv[e];
      if (i == j) v = make_double2(v.x + (attempt ? shift : 0.0), 0.0);
      a[e] = v;
    }
    if (tid == 0) fail = 0;
    __syncthreads();
    double dmax = 0.0;
    if (tid == 0)
      for (int i = 0; i < w; ++i) dmax = fmax(dmax, a[i * w + i].x);
    for (int p = 0; p < w; ++p) {
      // one thread takes the pivot's square root and reciprocal (GB300's FP64 pipe is
      // narrow: the same sequence in every thread costs thousands of cycles per pivot)
      if (tid == 0) {
        const double piv = a[p * w + p].x;
        if (!(piv > 1e-15 * dmax) || !(piv > 0.0) || !(piv <= 1e300) || !(piv >= 1e-300)) {
          fail = 1;
        } else {
          piv_ri = rsqrt_newton(piv);
          piv_r = piv * piv_ri;
        }
      }
      __syncthreads();
      if (fail) break;
      const double rp = piv_r, rpi = piv_ri;
      // scale row p (upper part) by 1/rp
      for (int j = p + tid; j < w; j += nt) {
        double2 v = a[p * w + j];
        a[p * w + j] = j == p ? make_double2(rp, 0.0) : make_double2(v.x * rpi, v.y * rpi);
      }
      __syncthreads();
      // trailing update a[i][j] -= conj(R[p][i]) R[p][j], i, j > p, j >= i
      const int m = w - p - 1;
      for (int e = tid; e < m * m; e += nt) {
        const int i = p + 1 + e / m, j = p + 1 + e % m;
        if (j < i) continue;
        const double2 ri = a[p * w + i], rj = a[p * w + j];
        double2 v = a[i * w + j];
        v = cfmaconj(ri, make_double2(-rj.x, -rj.y), v);
        a[i * w + j] = v;
      }
      __syncthreads();
    }
    if (!fail) break;
    if (attempt == 0 && tid == 0 && status) status[0] = 1;
    if (attempt == 0 && tid == 0 && fallback_counter) atomicAdd(fallback_counter, 1);
    if (attempt == 1 && tid == 0 && status) status[0] = 2;
    if (attempt == 1 && tid == 0 && fallback_counter) atomicAdd(fallback_counter + 1, 1);
  }
  __syncthreads();
  // inverse of the upper triangular R by right-looking back substitution: inv starts as I;
  // for t = w-1 .. 0, row t of inv is final once scaled by 1/R(t,t), and its multiples
  // R(i,t) inv(t, :) are taken from the rows i < t, all entries in parallel (chain depth
  // ~2w dependent operations instead of ~w^2/2 per column).  The staging copy of G in inv
  // is dead from here on.
  for (int e = tid; e < w * w; e += nt) {
    const int i = e / w, j = e - i * w;
    inv[e] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
  __shared__ double dinv[256];
  for (int i = tid; i < w; i += nt) dinv[i] = 1.0 / a[i * w + i].x;
  __syncthreads();
  for (int t = w - 1; t >= 0; --t) {
    for (int c = t + tid; c < w; c += nt) {
      const double2 v = inv[t * w + c];
      inv[t * w + c] = make_double2(v.x * dinv[t], v.y * dinv[t]);
    }
    __syncthreads();
    const int wc = w - t;  // columns t .. w-1
    for (int e = tid; e < t * wc; e += nt) {
      const int i = e / wc, c = t + (e - i * wc);
      inv[i * w + c] = csub(inv[i * w + c], cmul(a[i * w + t], inv[t * w + c]));
    }
    __syncthreads();
  }
  __syncthreads();
  for (int e = tid; e < w * w; e += nt) {
    const int i = e / w, j = e - i * w;
    Rinv[e] = (j >= i) ? inv[e] : make_double2(0.0, 0.0);
    if (Rout) Rout[e] = (j >= i) ? a[e] : make_double2(0.0, 0.0);
  }
}
__global__ void chol_inv_kernel(int w, int64_t n, const double2* __restrict__ G,
                                double2* __restrict__ Rinv, int* status, const int* skip_if_zero,
                                int* fallback_counter, double2* __restrict__ Rout) {
  chol_inv_body(Cta::hw(), w, n, G, Rinv, status, skip_if_zero, fallback_counter, Rout);
}

// ------------------------------------------------------------------ adjoint ----
// Eigenvalue adjoint on the CSR pattern of a matrix M: for nonzero j = (p, q),
//   out[j] = sum_i Y[p][i] conj(X[q][i]) coef[i]
// (Y: left vectors, X: right vectors, paired by column; coef carries
// G_i / conj(y_i^* B x_i), times -conj(lambda_i) for B).  OUT = double keeps the real
// part (real matrices).  One warp per row, lanes over the row's nonzeros.
__device__ __forceinline__ void store_out(double* o, double2 v) { *o = v.x; }
__device__ __forceinline__ void store_out(double2* o, double2 v) { *o = v; }

template <typename OUT>
__global__ void adjoint_scatter_kernel(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                                       const double2* __restrict__ Y, int ldy, const double2* __restrict__ X,
                                       int ldx, int k, const double2* __restrict__ coef, OUT* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int p = warp; p < n; p += nwarps) {
    const double2* yp = Y + (size_t)p * ldy;
    for (int j = rowptr[p] + lane; j < rowptr[p + 1]; j += 32) {
      const double2* xq = X + (size_t)col[j] * ldx;
      double2 acc = make_double2(0.0, 0.0);
      for (int i = 0; i < k; ++i) {
        const double2 t = cmul(yp[i], make_double2(xq[i].x, -xq[i].y));
        acc = cfma(t, coef[i], acc);
      }
      store_out(out + j, acc);
    }
  }
}

// Counter-based Gaussian start block (used when no V0 is given): Box-Muller on
// two uniforms from a 64-bit splitmix of (seed, element index).
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
__global__ void gaussian_block_kernel(int n, int w, uint64_t seed, double2* __restrict__ Y, int ldy) {
  const size_t total = (size_t)n * w;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const uint64_t h1 = splitmix64(seed ^ (2 * e));
    const uint64_t h2 = splitmix64(seed ^ (2 * e + 1));
    const double u1 = ((h1 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    const double u2 = ((h2 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    const double g = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
    const int r = (int)(e / w), c = (int)(e - (size_t)r * w);
    Y[(size_t)r * ldy + c] = make_double2(g, 0.0);
  }
}

}  // namespace gplhr
