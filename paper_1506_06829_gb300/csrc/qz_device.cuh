// Ordered complex QZ of a small pencil on the device: one CTA runs the host QZ's steps
// (qz.cpp) in the same order -- Givens reduction to Hessenberg-triangular form, single-
// shift QZ sweeps (Moler & Stewart), adjacent swaps (Van Dooren's direct swap) and the
// unit-phase scaling that makes RB's diagonal real and non-negative -- so that the
// projected pencil's QZ (footnote to Alg. 2 step 2) can be timed on the device against
// the host.  Every rotation is a chain step: its angle is read from entries the previous
// rotation wrote, so thread 0 forms the angle, a barrier publishes it, and all threads
// apply it (one entry pair of a row, column or accumulator row each), then a barrier ends
// the step.  H and T live split-complex in shared memory (4 s^2 doubles, s <= 80); the
// accumulators Y_L^T, Y_R^T are formed in the output arrays and transposed in place at the
// end.  Every loop is bounded: the sweeps by 60 s (as on the host), the chases and swaps by
// s; a pencil that needs more sweeps sets *status = 1.
#pragma once

#include <cuda_runtime.h>

namespace gplhr {

constexpr int DQZ_THREADS = 128;
constexpr int DQZ_SMAX = 80;

__host__ __device__ constexpr size_t dqz_smem_bytes(int s) { return (size_t)4 * s * s * sizeof(double); }

struct DqzM {  // s x s split-complex, row-major, in shared memory
  double* re;
  double* im;
  int n;
  __device__ double2 get(int i, int j) const { return make_double2(re[i * n + j], im[i * n + j]); }
  __device__ void set(int i, int j, double2 v) const {
    re[i * n + j] = v.x;
    im[i * n + j] = v.y;
  }
};

__device__ __forceinline__ double dqz_abs(double2 z) { return hypot(z.x, z.y); }
__device__ __forceinline__ double dqz_norm(double2 z) { return z.x * z.x + z.y * z.y; }
__device__ __forceinline__ double2 dqz_mul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 dqz_conj(double2 a) { return make_double2(a.x, -a.y); }
// a / b by the plain formula (the host QZ is compiled with limited-range complex division)
__device__ __forceinline__ double2 dqz_div(double2 a, double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
// principal square root
__device__ __forceinline__ double2 dqz_sqrt(double2 z) {
  const double r = hypot(z.x, z.y);
  if (r == 0.0) return make_double2(0.0, 0.0);
  const double t = sqrt(0.5 * (r + fabs(z.x)));
  if (z.x >= 0.0) return make_double2(t, z.y / (2.0 * t));
  return make_double2(fabs(z.y) / (2.0 * t), copysign(t, z.y));
}

// Plane rotation G = [[c, s], [-conj(s), c]], c real >= 0, with G [f; g] = [r; 0]: the
// host QZ's formulas.
__device__ void dqz_givens(double2 f, double2 g, double& c, double2& s, double2& r) {
  const double gr = g.x, gi = g.y, fr = f.x, fi = f.y;
  const double ag2 = gr * gr + gi * gi, af2 = fr * fr + fi * fi;
  const bool plain = ag2 < 1e300 && af2 < 1e300 && (ag2 == 0.0 || ag2 > 1e-300) && (af2 == 0.0 || af2 > 1e-300);
  const double ag = plain ? sqrt(ag2) : hypot(gr, gi);
  if (ag == 0.0) {
    c = 1.0;
    s = make_double2(0.0, 0.0);
    r = f;
    return;
  }
  const double af = plain ? sqrt(af2) : hypot(fr, fi);
  if (af == 0.0) {
    c = 0.0;
    s = make_double2(gr / ag, -gi / ag);
    r = make_double2(ag, 0.0);
    return;
  }
  const double nrm = plain ? sqrt(af2 + ag2) : hypot(af, ag);
  const double iaf = 1.0 / af, inrm = 1.0 / nrm;
  const double phr = fr * iaf, phi = fi * iaf;
  c = af * inrm;
  s = make_double2((phr * gr + phi * gi) * inrm, (phi * gr - phr * gi) * inrm);
  r = make_double2(phr * nrm, phi * nrm);
}

// x' = c x + s y, y' = -conj(s) x + c y on entry pair (x, y)
__device__ __forceinline__ void dqz_rot(double& xr, double& xi, double& yr, double& yi, double c, double sr,
                                        double si) {
  const double ar = xr, ai = xi, br = yr, bi = yi;
  xr = c * ar + sr * br - si * bi;
  xi = c * ai + sr * bi + si * br;
  yr = -sr * ar - si * ai + c * br;
  yi = -sr * ai + si * ar + c * bi;
}

// rows (i1, i2) of M, columns [c0, c1): G M
__device__ void dqz_rot_rows(const DqzM& M, int i1, int i2, double c, double2 s, int c0, int c1) {
  for (int j = c0 + (int)threadIdx.x; j < c1; j += DQZ_THREADS) {
    const int p = i1 * M.n + j, q = i2 * M.n + j;
    dqz_rot(M.re[p], M.im[p], M.re[q], M.im[q], c, s.x, s.y);
  }
}
// columns (j, j + 1) of M, rows [r0, r1): M Zr, Zr = [[c, s], [-conj(s), c]]:
// x' = c x - conj(s) y, y' = s x + c y
__device__ void dqz_rot_cols(const DqzM& M, int j, double c, double2 s, int r0, int r1) {
  for (int i = r0 + (int)threadIdx.x; i < r1; i += DQZ_THREADS) {
    const int p = i * M.n + j, q = p + 1;
    const double xr = M.re[p], xi = M.im[p], yr = M.re[q], yi = M.im[q];
    M.re[p] = c * xr - s.x * yr - s.y * yi;
    M.im[p] = c * xi - s.x * yi + s.y * yr;
    M.re[q] = s.x * xr - s.y * xi + c * yr;
    M.im[q] = s.x * xi + s.y * xr + c * yi;
  }
}
// rows (j, j + 1) of an accumulator held transposed (global, n x n): Yt <- K Yt with
// K = [[c, s'], [-conj(s'), c]]; s' = conj(s) for a left rotation (Y_L <- Y_L G^*),
// -conj(s) for a right one (Y_R <- Y_R Zr)
__device__ void dqz_accum(double2* Yt, int n, int j, double c, double2 sp) {
  for (int e = (int)threadIdx.x; e < n; e += DQZ_THREADS) {
    double2 x = Yt[(size_t)j * n + e], y = Yt[(size_t)(j + 1) * n + e];
    dqz_rot(x.x, x.y, y.x, y.y, c, sp.x, sp.y);
    Yt[(size_t)j * n + e] = x;
    Yt[(size_t)(j + 1) * n + e] = y;
  }
}

struct DqzRot {  // the current rotation, formed by thread 0
  double c;
  double2 s;
  int skip;
};

// Eigenvalue of the 2 x 2 pencil block nearest h22 / t22 (the host's Wilkinson shift).
__device__ double2 dqz_wilkinson(double2 h11, double2 h12, double2 h21, double2 h22, double2 t11, double2 t12,
                                 double2 t22) {
  const double eps = 2.220446049250313e-16;
  const double2 a = dqz_mul(t11, t22);
  const double2 hb = dqz_mul(h11, t22), hc = dqz_mul(h22, t11), hd = dqz_mul(h21, t12);
  const double2 b = make_double2(-(hb.x + hc.x - hd.x), -(hb.y + hc.y - hd.y));
  const double2 p1 = dqz_mul(h11, h22), p2 = dqz_mul(h12, h21);
  const double2 cc = make_double2(p1.x - p2.x, p1.y - p2.y);
  const double scale = dqz_abs(h22) + dqz_abs(h11) + dqz_abs(h21) + dqz_abs(h12);
  const double tsc = dqz_abs(t11) * dqz_abs(t22);
  if (tsc <= eps * eps * fmax(1.0, scale) || dqz_abs(a) == 0.0) return dqz_abs(t22) > 0 ? dqz_div(h22, t22) : h22;
  const double2 bb = dqz_mul(b, b), ac = dqz_mul(a, cc);
  const double2 disc = dqz_sqrt(make_double2(bb.x - 4.0 * ac.x, bb.y - 4.0 * ac.y));
  const double2 a2 = make_double2(2.0 * a.x, 2.0 * a.y);
  const double2 l1 = dqz_div(make_double2(-b.x + disc.x, -b.y + disc.y), a2);
  const double2 l2 = dqz_div(make_double2(-b.x - disc.x, -b.y - disc.y), a2);
  const double2 ref = dqz_abs(t22) > 0 ? dqz_div(h22, t22) : l1;
  return dqz_abs(make_double2(l1.x - ref.x, l1.y - ref.y)) <= dqz_abs(make_double2(l2.x - ref.x, l2.y - ref.y)) ? l1
                                                                                                               : l2;
}

__device__ __forceinline__ double dqz_distance(double2 alpha, double2 beta, double2 sigma) {
  const double ab = dqz_abs(beta);
  if (ab == 0.0) return __longlong_as_double(0x7FF0000000000000ll);
  const double2 sb = dqz_mul(sigma, beta);
  return dqz_abs(make_double2(alpha.x - sb.x, alpha.y - sb.y)) / ab;
}
__device__ bool dqz_key_less(double2 a1, double2 b1, double2 a2, double2 b2, double2 sigma) {
  const double d1 = dqz_distance(a1, b1, sigma), d2 = dqz_distance(a2, b2, sigma);
  if (d1 != d2) return d1 < d2;
  if (!isfinite(d1)) return false;
  const double2 l1 = dqz_div(a1, b1), l2 = dqz_div(a2, b2);
  if (l1.x != l2.x) return l1.x < l2.x;
  return l1.y < l2.y;
}

// One left rotation on rows (i, i + 1) of (P over [p0, s), Q over [q0, s)) accumulated into
// Y_L; thread 0 has formed rot; ends with a barrier.
__device__ __forceinline__ void dqz_left(const DqzM& P, int p0, const DqzM& Q, int q0, double2* YLt, int i,
                                         const DqzRot& rot) {
  dqz_rot_rows(P, i, i + 1, rot.c, rot.s, p0, P.n);
  dqz_rot_rows(Q, i, i + 1, rot.c, rot.s, q0, Q.n);
  dqz_accum(YLt, P.n, i, rot.c, dqz_conj(rot.s));
  __syncthreads();
}
// One right rotation on columns (j, j + 1) of (P over rows [0, pr), Q over [0, qr)) accumulated
// into Y_R; ends with a barrier.
__device__ __forceinline__ void dqz_right(const DqzM& P, int pr, const DqzM& Q, int qr, double2* YRt, int j,
                                          const DqzRot& rot) {
  dqz_rot_cols(P, j, rot.c, rot.s, 0, pr);
  dqz_rot_cols(Q, j, rot.c, rot.s, 0, qr);
  dqz_accum(YRt, P.n, j, rot.c, make_double2(-rot.s.x, rot.s.y));
  __syncthreads();
}

__global__ void __launch_bounds__(DQZ_THREADS, 1)
    ordqz_device_kernel(int n, const double2* __restrict__ Phi, const double2* __restrict__ Psi, double2 sigma,
                        int nsort, double2* __restrict__ RA, double2* __restrict__ RB, double2* __restrict__ YL,
                        double2* __restrict__ YR, int* status) {
  extern __shared__ __align__(16) double dqz_smem[];
  __shared__ DqzRot rot;
  __shared__ int s_tri, s_mode, s_j, s_ilo, s_best;
  __shared__ double2 s_mu;
  __shared__ double s_red[DQZ_THREADS / 32];
  __shared__ double2 s_t[DQZ_SMAX];
  const int tid = threadIdx.x;
  const double eps = 2.220446049250313e-16, dmin = 2.2250738585072014e-308;
  // A triangular Phi is the triangular factor from the start (the host's rule)
  if (tid == 0) s_tri = 1;
  __syncthreads();
  for (int e = tid; e < n * n; e += DQZ_THREADS) {
    const int i = e / n, j = e - i * n;
    if (i > j && (Phi[e].x != 0.0 || Phi[e].y != 0.0)) s_tri = 0;
  }
  __syncthreads();
  const bool tri = s_tri != 0;
  const DqzM H{dqz_smem, dqz_smem + n * n, n}, T{dqz_smem + 2 * n * n, dqz_smem + 3 * n * n, n};
  for (int e = tid; e < n * n; e += DQZ_THREADS) {
    const double2 h = tri ? Psi[e] : Phi[e], t = tri ? Phi[e] : Psi[e];
    H.re[e] = h.x;
    H.im[e] = h.y;
    T.re[e] = t.x;
    T.im[e] = t.y;
    const int i = e / n, j = e - i * n;
    YL[e] = make_double2(i == j ? 1.0 : 0.0, 0.0);  // Y_L^T, Y_R^T
    YR[e] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
  if (tid == 0) *status = 0;
  __syncthreads();

  // ---------------------------------------------------- Hessenberg-triangular --
  if (!tri) {
    for (int j = 0; j < n; ++j)
      for (int i = n - 1; i > j; --i) {
        if (T.re[i * n + j] == 0.0 && T.im[i * n + j] == 0.0) continue;  // uniform: read after a barrier
        __syncthreads();
        if (tid == 0) {
          double2 r;
          dqz_givens(T.get(i - 1, j), T.get(i, j), rot.c, rot.s, r);
        }
        __syncthreads();
        dqz_rot_rows(T, i - 1, i, rot.c, rot.s, j, n);
        dqz_rot_rows(H, i - 1, i, rot.c, rot.s, 0, n);
        dqz_accum(YL, n, i - 1, rot.c, dqz_conj(rot.s));
        __syncthreads();
        if (tid == 0) T.set(i, j, make_double2(0.0, 0.0));
        __syncthreads();
      }
  }
  for (int j = 0; j + 2 < n; ++j)
    for (int i = n - 1; i >= j + 2; --i) {
      if (H.re[i * n + j] == 0.0 && H.im[i * n + j] == 0.0) continue;
      __syncthreads();
      if (tid == 0) {
        double2 r;
        dqz_givens(H.get(i - 1, j), H.get(i, j), rot.c, rot.s, r);
      }
      __syncthreads();
      dqz_left(H, j, T, i - 1, YL, i - 1, rot);
      if (tid == 0) {
        H.set(i, j, make_double2(0.0, 0.0));
        double2 r;
        dqz_givens(T.get(i, i), T.get(i, i - 1), rot.c, rot.s, r);  // right zeroing of T(i, i-1)
      }
      __syncthreads();
      dqz_right(T, i + 1, H, n, YR, i - 1, rot);
      if (tid == 0) T.set(i, i - 1, make_double2(0.0, 0.0));
      __syncthreads();
    }

  // ------------------------------------------------------------- QZ sweeps --
  // norms of the reduced pencil (a block reduction)
  double fh = 0.0, ft = 0.0;
  for (int e = tid; e < n * n; e += DQZ_THREADS) {
    fh += H.re[e] * H.re[e] + H.im[e] * H.im[e];
    ft += T.re[e] * T.re[e] + T.im[e] * T.im[e];
  }
  for (int off = 16; off > 0; off >>= 1) {
    fh += __shfl_xor_sync(0xffffffffu, fh, off);
    ft += __shfl_xor_sync(0xffffffffu, ft, off);
  }
  double normH = 0.0, normT = 0.0;
  if ((tid & 31) == 0) s_red[tid >> 5] = fh;
  __syncthreads();
  for (int q = 0; q < DQZ_THREADS / 32; ++q) normH += s_red[q];
  __syncthreads();
  if ((tid & 31) == 0) s_red[tid >> 5] = ft;
  __syncthreads();
  for (int q = 0; q < DQZ_THREADS / 32; ++q) normT += s_red[q];
  __syncthreads();
  const double atolH = eps * fmax(sqrt(normH), dmin), atolT = eps * fmax(sqrt(normT), dmin);
  int ihi = n - 1, since = 0, total = 0;
  const int max_total = 60 * max(n, 1);
  bool converged = true;
  // every pass either deflates (ihi drops), chases (an infinite eigenvalue deflates at
  // ihi) or sweeps (total grows): at most n + n + max_total passes
  for (int pass = 0; pass < 2 * n + max_total + 1 && ihi > 0; ++pass) {
    if (tid == 0) {
      int ilo = ihi;
      while (ilo > 0) {
        const double h = dqz_abs(H.get(ilo, ilo - 1));
        const double rel = eps * (dqz_abs(H.get(ilo, ilo)) + dqz_abs(H.get(ilo - 1, ilo - 1)));
        if (h <= atolH || h <= rel) {
          H.set(ilo, ilo - 1, make_double2(0.0, 0.0));
          break;
        }
        --ilo;
      }
      s_ilo = ilo;
      if (ilo == ihi) {
        s_mode = 0;  // deflate
      } else {
        s_mode = 2;  // sweep, unless a negligible T(j, j) asks for a chase
        for (int j = ilo; j <= ihi; ++j)
          if (dqz_abs(T.get(j, j)) <= atolT) {
            s_mode = 1;
            s_j = j;
            break;
          }
      }
    }
    __syncthreads();
    const int mode = s_mode, ilo = s_ilo;
    if (mode == 0) {
      --ihi;
      since = 0;
      __syncthreads();
      continue;
    }
    if (mode == 1) {  // move T(j, j) = 0 down to (ihi, ihi) and deflate there
      const int j0 = s_j;
      if (tid == 0) T.set(j0, j0, make_double2(0.0, 0.0));
      __syncthreads();
      for (int i = j0; i < ihi; ++i) {
        if (tid == 0) {
          double2 r;
          dqz_givens(T.get(i, i + 1), T.get(i + 1, i + 1), rot.c, rot.s, r);
        }
        __syncthreads();
        dqz_left(T, i, H, max(i - 1, 0), YL, i, rot);
        if (tid == 0) {
          T.set(i + 1, i + 1, make_double2(0.0, 0.0));
          if (i > 0) {
            double2 r;
            dqz_givens(H.get(i + 1, i), H.get(i + 1, i - 1), rot.c, rot.s, r);
          }
        }
        __syncthreads();
        if (i > 0) {
          dqz_right(H, min(i + 2, n), T, i + 1, YR, i - 1, rot);
          if (tid == 0) H.set(i + 1, i - 1, make_double2(0.0, 0.0));
          __syncthreads();
        }
      }
      if (tid == 0) {
        double2 r;
        dqz_givens(H.get(ihi, ihi), H.get(ihi, ihi - 1), rot.c, rot.s, r);
      }
      __syncthreads();
      dqz_right(H, ihi + 1, T, ihi + 1, YR, ihi - 1, rot);
      if (tid == 0) H.set(ihi, ihi - 1, make_double2(0.0, 0.0));
      __syncthreads();
      continue;
    }
    if (++total > max_total) {
      converged = false;
      break;
    }
    ++since;
    if (tid == 0) {
      if (since % 10 == 0) {
        const double2 q = dqz_div(H.get(ihi, ihi), T.get(ihi, ihi));
        const double f = dqz_abs(H.get(ihi, ihi - 1)) / dqz_abs(T.get(ihi - 1, ihi - 1));
        s_mu = make_double2(q.x + 0.75 * f, q.y + 0.35 * f);
      } else {
        s_mu = dqz_wilkinson(H.get(ihi - 1, ihi - 1), H.get(ihi - 1, ihi), H.get(ihi, ihi - 1), H.get(ihi, ihi),
                             T.get(ihi - 1, ihi - 1), T.get(ihi - 1, ihi), T.get(ihi, ihi));
      }
      const double2 mt = dqz_mul(s_mu, T.get(ilo, ilo)), h = H.get(ilo, ilo);
      double2 r;
      dqz_givens(make_double2(h.x - mt.x, h.y - mt.y), H.get(ilo + 1, ilo), rot.c, rot.s, r);
    }
    __syncthreads();
    dqz_left(H, ilo, T, ilo, YL, ilo, rot);
    for (int j = ilo; j < ihi; ++j) {
      if (tid == 0) {
        double2 r;
        dqz_givens(T.get(j + 1, j + 1), T.get(j + 1, j), rot.c, rot.s, r);  // right zeroing of T(j+1, j)
      }
      __syncthreads();
      dqz_right(T, j + 2, H, min(j + 3, n), YR, j, rot);
      if (tid == 0) {
        T.set(j + 1, j, make_double2(0.0, 0.0));
        if (j + 2 <= ihi) {
          double2 r;
          dqz_givens(H.get(j + 1, j), H.get(j + 2, j), rot.c, rot.s, r);
        }
      }
      __syncthreads();
      if (j + 2 <= ihi) {
        dqz_left(H, j, T, j + 1, YL, j + 1, rot);
        if (tid == 0) H.set(j + 2, j, make_double2(0.0, 0.0));
        __syncthreads();
      }
    }
  }
  if (ihi > 0) converged = false;
  if (!converged) {
    if (tid == 0) *status = 1;
    return;
  }

  // -------------------------------------------------------------- ordering --
  const DqzM& A = tri ? T : H;  // the factor of Phi
  const DqzM& B = tri ? H : T;  // the factor of Psi
  for (int e = tid; e < n * n; e += DQZ_THREADS) {
    const int i = e / n, j = e - i * n;
    if (i > j) {
      A.re[e] = A.im[e] = 0.0;
      B.re[e] = B.im[e] = 0.0;
    }
  }
  __syncthreads();
  const int npos = nsort < 0 ? n - 1 : min(nsort, n - 1);
  for (int pos = 0; pos < npos; ++pos) {
    if (tid == 0) {
      int best = pos;
      for (int j = pos + 1; j < n; ++j)
        if (dqz_key_less(A.get(j, j), B.get(j, j), A.get(best, best), B.get(best, best), sigma)) best = j;
      s_best = best;
    }
    __syncthreads();
    const int best = s_best;
    for (int j = best - 1; j >= pos; --j) {
      // right rotation from the 2 x 2 pencil's eigenvector for (a22, b22)
      if (tid == 0) {
        const double2 a11 = A.get(j, j), a12 = A.get(j, j + 1), a22 = A.get(j + 1, j + 1);
        const double2 b11 = B.get(j, j), b12 = B.get(j, j + 1), b22 = B.get(j + 1, j + 1);
        const double2 u1 = dqz_mul(b22, a12), u2 = dqz_mul(a22, b12);
        const double2 num = make_double2(-(u1.x - u2.x), -(u1.y - u2.y));
        const double2 v1 = dqz_mul(b22, a11), v2 = dqz_mul(a22, b11);
        const double2 den = make_double2(v1.x - v2.x, v1.y - v2.y);
        const double nn = dqz_abs(num), nd = dqz_abs(den);
        rot.skip = (nd == 0.0 && nn == 0.0) ? 1 : 0;
        if (!rot.skip) {
          const double nrm = hypot(nn, nd);
          if (nn == 0.0) {
            rot.c = 0.0;
            rot.s = make_double2(-den.x / nd, den.y / nd);
          } else {
            const double2 ph = make_double2(num.x / nn, num.y / nn);
            rot.c = nn / nrm;
            const double2 pc = dqz_mul(ph, dqz_conj(den));
            rot.s = make_double2(-pc.x / nrm, -pc.y / nrm);
          }
        }
      }
      __syncthreads();
      if (rot.skip) {
        __syncthreads();
        continue;
      }
      dqz_right(A, j + 2, B, j + 2, YR, j, rot);
      if (tid == 0) {
        const double na = dqz_norm(A.get(j, j)) + dqz_norm(A.get(j + 1, j));
        const double nb = dqz_norm(B.get(j, j)) + dqz_norm(B.get(j + 1, j));
        double2 r;
        if (na >= nb)
          dqz_givens(A.get(j, j), A.get(j + 1, j), rot.c, rot.s, r);
        else
          dqz_givens(B.get(j, j), B.get(j + 1, j), rot.c, rot.s, r);
      }
      __syncthreads();
      dqz_left(A, j, B, j, YL, j, rot);
      if (tid == 0) {
        A.set(j + 1, j, make_double2(0.0, 0.0));
        B.set(j + 1, j, make_double2(0.0, 0.0));
      }
      __syncthreads();
    }
  }

  // ------------------------------------------- unit phases and the outputs --
  for (int j = tid; j < n; j += DQZ_THREADS) {
    const double2 bjj = B.get(j, j);
    const double mag = dqz_abs(bjj);
    s_t[j] = mag > 0.0 ? make_double2(bjj.x / mag, -bjj.y / mag) : make_double2(1.0, 0.0);
  }
  __syncthreads();
  for (int e = tid; e < n * n; e += DQZ_THREADS) {
    const int j = e / n, c = e - j * n;
    const double2 t = s_t[j];
    if (c < j) {
      RA[e] = make_double2(0.0, 0.0);
      RB[e] = make_double2(0.0, 0.0);
    } else {
      RA[e] = dqz_mul(A.get(j, c), t);
      RB[e] = c == j ? make_double2(dqz_abs(B.get(j, j)), 0.0) : dqz_mul(B.get(j, c), t);
    }
  }
  // Y_L(i, j) = Y_L^T(j, i) conj(t_j), Y_R(i, j) = Y_R^T(j, i): in-place transposes
  for (int e = tid; e < n * n; e += DQZ_THREADS) {
    const int i = e / n, j = e - i * n;
    if (i > j) continue;
    const size_t p = (size_t)i * n + j, q = (size_t)j * n + i;
    const double2 ap = YL[p], aq = YL[q];
    YL[p] = dqz_mul(aq, dqz_conj(s_t[j]));
    if (i != j) YL[q] = dqz_mul(ap, dqz_conj(s_t[i]));
    const double2 bp = YR[p], bq = YR[q];
    YR[p] = bq;
    if (i != j) YR[q] = bp;
  }
}

}  // namespace gplhr
