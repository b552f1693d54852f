// Host-side complex QZ with reordering, and the k x k Q-free factor algebra.
//
// The sorted QZ of the projected pencil (U^*AZ, U^*BZ) is what the paper's
// harmonic Schur-Rayleigh-Ritz step needs (Sec. 3.4, footnote to Alg. 2 step 2):
// the FULL generalized Schur form, ordered by distance of the eigenvalues to sigma.
// Written from the published algorithms:
//   * reduction to Hessenberg-triangular form by Givens rotations and the
//     single-shift implicit QZ sweep of Moler & Stewart (1973);
//   * reordering by swapping adjacent 1x1 diagonal blocks with one right and one
//     left plane rotation (Van Dooren's direct swap for triangular pencils);
//   * a final unit-phase scaling that makes the diagonal of RB real non-negative.
// When Phi is upper triangular (the projected pencil in factored form), the QZ runs on
// (Psi, Phi): Phi is then the triangular factor from the start, and the QR half of the
// Hessenberg-triangular reduction is skipped.
#include "qz.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>

namespace gplhr {

namespace {

const double kEps = std::numeric_limits<double>::epsilon();

// Plane rotation G = [[c, s], [-conj(s), c]] with c real >= 0 such that
// G [f; g] = [r; 0].
void givens(cd f, cd g, double& c, cd& s, cd& r) {
  const double gr = g.real(), gi = g.imag(), fr = f.real(), fi = f.imag();
  const double ag2 = gr * gr + gi * gi, af2 = fr * fr + fi * fi;
  // squares of moduli far from over- and underflow: the plain formulas are exact to
  // rounding; otherwise the scaled library moduli
  const bool plain = ag2 < 1e300 && af2 < 1e300 && (ag2 == 0.0 || ag2 > 1e-300) && (af2 == 0.0 || af2 > 1e-300);
  const double ag = plain ? std::sqrt(ag2) : std::abs(g);
  if (ag == 0.0) {
    c = 1.0;
    s = 0.0;
    r = f;
    return;
  }
  const double af = plain ? std::sqrt(af2) : std::abs(f);
  if (af == 0.0) {
    c = 0.0;
    s = std::conj(g) / ag;
    r = ag;
    return;
  }
  const double nrm = plain ? std::sqrt(af2 + ag2) : std::hypot(af, ag);
  const double iaf = 1.0 / af, inrm = 1.0 / nrm;
  const double phr = fr * iaf, phi = fi * iaf;  // f / |f|
  c = af * inrm;
  s = cd((phr * gr + phi * gi) * inrm, (phi * gr - phr * gi) * inrm);  // ph conj(g) / nrm
  r = cd(phr * nrm, phi * nrm);
}

// Matrices of the QZ are held split-complex (separate real and imaginary planes, row-major)
// so that every plane rotation is a loop of real multiply-adds over contiguous doubles,
// which the compiler vectorises.  The accumulators are held transposed (Yt(j, i) = Y(i, j))
// so that a rotation of two columns of Y runs over two contiguous rows.
struct ZMat {
  int n = 0;
  std::vector<double> re, im;
  explicit ZMat(int n_ = 0) : n(n_), re((size_t)n_ * n_, 0.0), im((size_t)n_ * n_, 0.0) {}
  cd get(int i, int j) const { return cd(re[(size_t)i * n + j], im[(size_t)i * n + j]); }
  void set(int i, int j, cd v) {
    re[(size_t)i * n + j] = v.real();
    im[(size_t)i * n + j] = v.imag();
  }
  double* R(int i) { return re.data() + (size_t)i * n; }
  double* I(int i) { return im.data() + (size_t)i * n; }
};

// Two split-complex rows x, y of length len: x' = c x + s y, y' = -conj(s) x + c y.
void rot_pair(double* __restrict ar, double* __restrict ai, double* __restrict br, double* __restrict bi, int len,
              double c, double sr, double si) {
  for (int j = 0; j < len; ++j) {
    const double xr = ar[j], xi = ai[j], yr = br[j], yi = bi[j];
    ar[j] = c * xr + sr * yr - si * yi;
    ai[j] = c * xi + sr * yi + si * yr;
    br[j] = -sr * xr - si * xi + c * yr;
    bi[j] = -sr * xi + si * xr + c * yi;
  }
}

// M <- G M on rows (i1, i2), columns [c0, c1): x' = c x + s y, y' = -conj(s) x + c y.
void rot_rows(ZMat& M, int i1, int i2, double c, cd s, int c0, int c1) {
  if (c1 > c0) rot_pair(M.R(i1) + c0, M.I(i1) + c0, M.R(i2) + c0, M.I(i2) + c0, c1 - c0, c, s.real(), s.imag());
}

// The plane rotations of the reduction, each on adjacent indices (j, j + 1), in the order
// they were applied to the pencil.  The Schur-vector accumulators are products of them;
// only the leading columns the caller needs are formed, at the end (form_columns).
// Left: YL <- YL K, K = [[c, -s], [conj(s), c]] (= G^*, so that YL (G M) = YL_old M);
// right: YR <- YR Zr, Zr = [[c, s], [-conj(s), c]].  Both are logged as (j, c, s') with
// K or Zr = [[c, s'], [-conj(s'), c]]: s' = -s on the left, s on the right.
struct RotLog {
  std::vector<int> j;
  std::vector<double> c, sr, si;
  void add(int jj, double cc, cd s) {
    j.push_back(jj);
    c.push_back(cc);
    sr.push_back(s.real());
    si.push_back(s.imag());
  }
};

// Y <- Y G^* on columns (j1, j1 + 1): logged.
void rot_left_accum(RotLog& YL, int j1, double c, cd s) { YL.add(j1, c, -s); }

// M <- M Zr on columns (j, j + 1), rows [r0, r1), Zr = [[c, s], [-conj(s), c]]:
// x' = c x - conj(s) y, y' = s x + c y.  The two columns' entries of a row are adjacent,
// so a row is one pair of real parts R = (xr, yr) and one of imaginary parts I = (xi, yi):
// R' = c R + (-sr, sr) swap(R) - si swap(I), I' = c I + (-sr, sr) swap(I) + si swap(R)
// (generic two-lane vectors of the compiler, no target intrinsics).
void rot_cols(ZMat& M, int j, double c, cd s, int r0, int r1) {
  typedef double v2d __attribute__((vector_size(16)));
  const double sr = s.real(), si = s.imag();
  const int n = M.n;
  double* __restrict re = M.re.data();
  double* __restrict im = M.im.data();
  const v2d vc = {c, c}, va = {-sr, sr}, vs = {si, si};
  for (int i = r0; i < r1; ++i) {
    const size_t p = (size_t)i * n + j;
    v2d R, I;
    std::memcpy(&R, re + p, sizeof R);
    std::memcpy(&I, im + p, sizeof I);
    const v2d Rs = __builtin_shufflevector(R, R, 1, 0), Is = __builtin_shufflevector(I, I, 1, 0);
    const v2d Rn = vc * R + va * Rs - vs * Is;
    const v2d In = vc * I + va * Is + vs * Rs;
    std::memcpy(re + p, &Rn, sizeof Rn);
    std::memcpy(im + p, &In, sizeof In);
  }
}

// YR <- YR Zr on columns (j1, j1 + 1): logged.
void rot_right_accum(RotLog& YR, int j1, double c, cd s) { YR.add(j1, c, s); }

// E (n x nc, split-complex rows) = M_1 M_2 ... M_m I(:, 0:nc) for the logged rotations
// M_i = [[c, s'], [-conj(s'), c]] on rows (j, j + 1): applied to E from the last one; rows
// below the highest one a rotation has reached so far are zero and are skipped.
void form_columns(const RotLog& L, int n, int nc, std::vector<double>& er, std::vector<double>& ei) {
  er.assign((size_t)n * nc, 0.0);
  ei.assign((size_t)n * nc, 0.0);
  for (int j = 0; j < nc; ++j) er[(size_t)j * nc + j] = 1.0;
  int hi = nc - 1;
  for (size_t t = L.j.size(); t-- > 0;) {
    const int j = L.j[t];
    if (j > hi) continue;  // both rows zero
    if (j + 1 > hi) hi = j + 1;
    rot_pair(er.data() + (size_t)j * nc, ei.data() + (size_t)j * nc, er.data() + (size_t)(j + 1) * nc,
             ei.data() + (size_t)(j + 1) * nc, nc, L.c[t], L.sr[t], L.si[t]);
  }
}

// Right rotation on columns (j1, j2) that zeroes the entry x = M(i, j1) against
// y = M(i, j2): with (c, s, r) = givens(y, x), [x y] Zr = [0 r].
void right_zeroing(cd x, cd y, double& c, cd& s) {
  cd r;
  givens(y, x, c, s, r);
}

// |z| from the sum of squares while that stays far from over- and underflow, else the
// library modulus
double cabs_fast(cd z) {
  const double t = z.real() * z.real() + z.imag() * z.imag();
  return (t < 1e300 && (t > 1e-300 || t == 0.0)) ? std::sqrt(t) : std::abs(z);
}

double fro(const ZMat& M) {
  double t = 0.0;
  for (size_t i = 0; i < M.re.size(); ++i) t += M.re[i] * M.re[i] + M.im[i] * M.im[i];
  return std::sqrt(t);
}
double fro(const SqMat& M) {
  double t = 0.0;
  for (const cd& v : M.a) t += std::norm(v);
  return std::sqrt(t);
}

// Eigenvalue of the 2x2 upper-Hessenberg/triangular pencil (H2, T2) nearest h22/t22.
cd wilkinson_shift(cd h11, cd h12, cd h21, cd h22, cd t11, cd t12, cd t22) {
  // det(H2 - l T2) = a l^2 + b l + c
  const cd a = t11 * t22;
  const cd b = -(h11 * t22 + h22 * t11 - h21 * t12);
  const cd c = h11 * h22 - h12 * h21;
  const double scale = std::abs(h22) + std::abs(h11) + std::abs(h21) + std::abs(h12);
  const double tsc = std::abs(t11) * std::abs(t22);
  if (tsc <= kEps * kEps * std::max(1.0, scale) || std::abs(a) == 0.0) {
    return std::abs(t22) > 0 ? h22 / t22 : h22;
  }
  const cd disc = std::sqrt(b * b - 4.0 * a * c);
  const cd l1 = (-b + disc) / (2.0 * a);
  const cd l2 = (-b - disc) / (2.0 * a);
  const cd ref = std::abs(t22) > 0 ? h22 / t22 : l1;
  return std::abs(l1 - ref) <= std::abs(l2 - ref) ? l1 : l2;
}

// Reduce (H, T) to upper Hessenberg / upper triangular form, accumulating YL, YR.
// t_triangular: T is upper triangular already (the QR phase is skipped).
void hessenberg_triangular(ZMat& H, ZMat& T, RotLog& YL, RotLog& YR, bool t_triangular) {
  const int n = H.n;
  if (!t_triangular) {
    // T -> upper triangular by left rotations (a Givens QR).
    for (int j = 0; j < n; ++j) {
      for (int i = n - 1; i > j; --i) {
        if (T.get(i, j) == cd(0.0)) continue;
        double c;
        cd s, r;
        givens(T.get(i - 1, j), T.get(i, j), c, s, r);
        rot_rows(T, i - 1, i, c, s, j, n);
        rot_rows(H, i - 1, i, c, s, 0, n);
        rot_left_accum(YL, i - 1, c, s);
        T.set(i, j, 0.0);
      }
    }
  }
  // H -> upper Hessenberg, keeping T triangular.
  for (int j = 0; j + 2 < n; ++j) {
    for (int i = n - 1; i >= j + 2; --i) {
      if (H.get(i, j) == cd(0.0)) continue;
      double c;
      cd s, r;
      givens(H.get(i - 1, j), H.get(i, j), c, s, r);
      rot_rows(H, i - 1, i, c, s, j, n);
      rot_rows(T, i - 1, i, c, s, i - 1, n);
      rot_left_accum(YL, i - 1, c, s);
      H.set(i, j, 0.0);
      // fill T(i, i-1): zero it from the right on columns (i-1, i)
      right_zeroing(T.get(i, i - 1), T.get(i, i), c, s);
      rot_cols(T, i - 1, c, s, 0, i + 1);
      rot_cols(H, i - 1, c, s, 0, n);
      rot_right_accum(YR, i - 1, c, s);
      T.set(i, i - 1, 0.0);
    }
  }
}

// Move a negligible T(j, j) (ilo <= j <= ihi) down to T(ihi, ihi) and deflate an
// infinite eigenvalue by zeroing H(ihi, ihi-1).
void chase_zero_down(ZMat& H, ZMat& T, RotLog& YL, RotLog& YR, int j, int ihi) {
  const int n = H.n;
  T.set(j, j, 0.0);
  for (int i = j; i < ihi; ++i) {
    double c;
    cd s, r;
    givens(T.get(i, i + 1), T.get(i + 1, i + 1), c, s, r);
    rot_rows(T, i, i + 1, c, s, i, n);
    rot_rows(H, i, i + 1, c, s, std::max(i - 1, 0), n);
    rot_left_accum(YL, i, c, s);
    T.set(i + 1, i + 1, 0.0);
    if (i > 0) {
      // H(i+1, i-1) filled: zero it from the right on columns (i-1, i)
      right_zeroing(H.get(i + 1, i - 1), H.get(i + 1, i), c, s);
      rot_cols(H, i - 1, c, s, 0, std::min(i + 2, n));
      rot_cols(T, i - 1, c, s, 0, i + 1);
      rot_right_accum(YR, i - 1, c, s);
      H.set(i + 1, i - 1, 0.0);
    }
  }
  if (ihi > 0) {
    double c;
    cd s;
    right_zeroing(H.get(ihi, ihi - 1), H.get(ihi, ihi), c, s);
    rot_cols(H, ihi - 1, c, s, 0, ihi + 1);
    rot_cols(T, ihi - 1, c, s, 0, ihi + 1);
    rot_right_accum(YR, ihi - 1, c, s);
    H.set(ihi, ihi - 1, 0.0);
  }
}

// Single-shift QZ iterations until (H, T) is upper triangular.
bool qz_iterate(ZMat& H, ZMat& T, RotLog& YL, RotLog& YR) {
  const int n = H.n;
  const double normH = fro(H), normT = fro(T);
  const double atolH = kEps * std::max(normH, std::numeric_limits<double>::min());
  const double atolT = kEps * std::max(normT, std::numeric_limits<double>::min());
  int ihi = n - 1;
  int since_deflation = 0;
  int total = 0;
  const int max_total = 60 * std::max(n, 1);
  while (ihi > 0) {
    // find the start of the active unreduced block
    int ilo = ihi;
    while (ilo > 0) {
      const double h = cabs_fast(H.get(ilo, ilo - 1));
      const double rel = kEps * (cabs_fast(H.get(ilo, ilo)) + cabs_fast(H.get(ilo - 1, ilo - 1)));
      if (h <= atolH || h <= rel) {
        H.set(ilo, ilo - 1, 0.0);
        break;
      }
      --ilo;
    }
    if (ilo == ihi) {
      --ihi;
      since_deflation = 0;
      continue;
    }
    // a negligible diagonal entry of T in the active block: infinite eigenvalue
    bool chased = false;
    for (int j = ilo; j <= ihi; ++j) {
      if (cabs_fast(T.get(j, j)) <= atolT) {
        chase_zero_down(H, T, YL, YR, j, ihi);
        chased = true;
        break;
      }
    }
    if (chased) continue;
    if (++total > max_total) return false;
    ++since_deflation;
    cd mu;
    if (since_deflation % 10 == 0) {
      // exceptional shift
      mu = H.get(ihi, ihi) / T.get(ihi, ihi) +
           cd(0.75, 0.35) * std::abs(H.get(ihi, ihi - 1)) / std::abs(T.get(ihi - 1, ihi - 1));
    } else {
      mu = wilkinson_shift(H.get(ihi - 1, ihi - 1), H.get(ihi - 1, ihi), H.get(ihi, ihi - 1), H.get(ihi, ihi),
                           T.get(ihi - 1, ihi - 1), T.get(ihi - 1, ihi), T.get(ihi, ihi));
    }
    // implicit single-shift sweep on [ilo, ihi]
    double c;
    cd s, r;
    givens(H.get(ilo, ilo) - mu * T.get(ilo, ilo), H.get(ilo + 1, ilo), c, s, r);
    rot_rows(H, ilo, ilo + 1, c, s, ilo, n);
    rot_rows(T, ilo, ilo + 1, c, s, ilo, n);
    rot_left_accum(YL, ilo, c, s);
    for (int j = ilo; j < ihi; ++j) {
      // T(j+1, j) is the bulge: zero it from the right on columns (j, j+1)
      right_zeroing(T.get(j + 1, j), T.get(j + 1, j + 1), c, s);
      rot_cols(T, j, c, s, 0, j + 2);
      rot_cols(H, j, c, s, 0, std::min(j + 3, n));
      rot_right_accum(YR, j, c, s);
      T.set(j + 1, j, 0.0);
      if (j + 2 <= ihi) {
        // H(j+2, j) filled: zero it from the left on rows (j+1, j+2)
        givens(H.get(j + 1, j), H.get(j + 2, j), c, s, r);
        rot_rows(H, j + 1, j + 2, c, s, j, n);
        rot_rows(T, j + 1, j + 2, c, s, j + 1, n);
        rot_left_accum(YL, j + 1, c, s);
        H.set(j + 2, j, 0.0);
      }
    }
  }
  return true;
}

// Swap the adjacent 1x1 diagonal pairs at (j, j+1) of the triangular pencil (A, B).
void swap_adjacent(ZMat& A, ZMat& B, RotLog& YL, RotLog& YR, int j) {
  const int n = A.n;
  const cd a11 = A.get(j, j), a12 = A.get(j, j + 1), a22 = A.get(j + 1, j + 1);
  const cd b11 = B.get(j, j), b12 = B.get(j, j + 1), b22 = B.get(j + 1, j + 1);
  // right eigenvector x of the 2x2 pencil for the pair (a22, b22): (b22 A - a22 B) x = 0
  const cd num = -(b22 * a12 - a22 * b12);
  const cd den = b22 * a11 - a22 * b11;
  const double nn = std::abs(num), nd = std::abs(den);
  if (nd == 0.0 && nn == 0.0) return;  // identical pairs: nothing to swap
  const double nrm = std::hypot(nn, nd);
  double c;
  cd s;
  if (nn == 0.0) {
    c = 0.0;
    s = -std::conj(den) / nd;
  } else {
    const cd ph = num / nn;
    c = nn / nrm;
    s = -ph * std::conj(den) / nrm;
  }
  rot_cols(A, j, c, s, 0, j + 2);
  rot_cols(B, j, c, s, 0, j + 2);
  rot_right_accum(YR, j, c, s);
  // first columns of A, B are now parallel in rows (j, j+1): zero row j+1 from the left
  const double na = std::norm(A.get(j, j)) + std::norm(A.get(j + 1, j));
  const double nb = std::norm(B.get(j, j)) + std::norm(B.get(j + 1, j));
  cd r;
  if (na >= nb)
    givens(A.get(j, j), A.get(j + 1, j), c, s, r);
  else
    givens(B.get(j, j), B.get(j + 1, j), c, s, r);
  rot_rows(A, j, j + 1, c, s, j, n);
  rot_rows(B, j, j + 1, c, s, j, n);
  rot_left_accum(YL, j, c, s);
  A.set(j + 1, j, 0.0);
  B.set(j + 1, j, 0.0);
}

bool key_less(cd a1, cd b1, cd a2, cd b2, cd sigma) {
  const double d1 = pair_distance(a1, b1, sigma), d2 = pair_distance(a2, b2, sigma);
  if (d1 != d2) return d1 < d2;
  if (!std::isfinite(d1)) return false;
  const cd l1 = a1 / b1, l2 = a2 / b2;
  if (l1.real() != l2.real()) return l1.real() < l2.real();
  return l1.imag() < l2.imag();
}

}  // namespace

double pair_distance(cd alpha, cd beta, cd sigma) {
  const double ab = std::abs(beta);
  if (ab == 0.0) return std::numeric_limits<double>::infinity();
  return std::abs(alpha - sigma * beta) / ab;
}

bool ordered_qz(const SqMat& Phi, const SqMat& Psi, cd sigma, SqMat& RA, SqMat& RB, SqMat& YL,
                SqMat& YR, int nsort, int nyl, int nyr) {
  const int n = Phi.n;
  if (n == 0) {
    RA = RB = YL = YR = SqMat(0);
    return true;
  }
  // A triangular Phi (the factored projected pencil) is used as the triangular factor
  // from the start: the QZ runs on (H, T) = (Psi, Phi), whose generalized Schur form is
  // that of (Phi, Psi) with the two triangular factors exchanged, and the QR phase of the
  // Hessenberg-triangular reduction is skipped.
  bool phi_tri = true;
  for (int i = 1; i < n && phi_tri; ++i)
    for (int j = 0; j < i; ++j)
      if (Phi(i, j) != cd(0.0)) {
        phi_tri = false;
        break;
      }
  ZMat H(n), T(n);
  RotLog YLt, YRt;
  const SqMat& Hs = phi_tri ? Psi : Phi;
  const SqMat& Ts = phi_tri ? Phi : Psi;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      H.set(i, j, Hs(i, j));
      T.set(i, j, Ts(i, j));
    }
  hessenberg_triangular(H, T, YLt, YRt, phi_tri);
  if (!qz_iterate(H, T, YLt, YRt)) return false;
  ZMat& A = phi_tri ? T : H;  // the factor of Phi
  ZMat& B = phi_tri ? H : T;  // the factor of Psi
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) {
      A.set(i, j, 0.0);
      B.set(i, j, 0.0);
    }
  // selection sort of the leading nsort positions: bring the nearest remaining pair to
  // position pos by adjacent swaps (positions past nsort keep the QZ's order)
  const int npos = nsort < 0 ? n - 1 : std::min(nsort, n - 1);
  for (int pos = 0; pos < npos; ++pos) {
    int best = pos;
    for (int j = pos + 1; j < n; ++j)
      if (key_less(A.get(j, j), B.get(j, j), A.get(best, best), B.get(best, best), sigma)) best = j;
    for (int j = best - 1; j >= pos; --j) swap_adjacent(A, B, YLt, YRt, j);
  }
  // the leading columns of the accumulators, then the unit-phase scaling: RB(j, j) real >= 0
  const int ncl = nyl < 0 ? n : std::min(nyl, n), ncr = nyr < 0 ? n : std::min(nyr, n);
  std::vector<double> lr, li, rr, ri;
  form_columns(YLt, n, ncl, lr, li);
  form_columns(YRt, n, ncr, rr, ri);
  RA = SqMat(n);
  RB = SqMat(n);
  YL = SqMat(n);
  YR = SqMat(n);
  for (int j = 0; j < n; ++j) {
    const cd bjj = B.get(j, j);
    const double mag = std::abs(bjj);
    const cd t = mag > 0.0 ? std::conj(bjj) / mag : cd(1.0);
    for (int c = j; c < n; ++c) {
      RA(j, c) = A.get(j, c) * t;
      RB(j, c) = B.get(j, c) * t;
    }
    if (mag > 0.0) RB(j, j) = mag;
    const cd ct = std::conj(t);
    if (j < ncl)
      for (int i = 0; i < n; ++i) YL(i, j) = cd(lr[(size_t)i * ncl + j], li[(size_t)i * ncl + j]) * ct;
    if (j < ncr)
      for (int i = 0; i < n; ++i) YR(i, j) = cd(rr[(size_t)i * ncr + j], ri[(size_t)i * ncr + j]);
  }
  return true;
}

void m_factors(const SqMat& RA, const SqMat& RB, SqMat& MA, SqMat& MB) {
  const int k = RA.n;
  std::vector<cd> g1(k), g2(k);
  for (int j = 0; j < k; ++j) {
    const cd a = RA(j, j), b = RB(j, j);
    if (std::abs(a) < std::abs(b)) {  // Eqs. G1_fix, G2_fix, tau_j = 0
      g1[j] = 0.0;
      g2[j] = 1.0 / b;
    } else {                          // tau_j = 1
      g1[j] = (1.0 - b) / a;
      g2[j] = 1.0;
    }
  }
  SqMat G(k);
  for (int i = 0; i < k; ++i)
    for (int j = i; j < k; ++j) G(i, j) = RA(i, j) * g1[j] + RB(i, j) * g2[j];
  // X = G^{-1} RA by back substitution (G upper triangular, unit diagonal in exact arithmetic)
  SqMat X(k);
  for (int c = 0; c < k; ++c) {
    for (int i = k - 1; i >= 0; --i) {
      cd acc = RA(i, c);
      for (int t = i + 1; t < k; ++t) acc -= G(i, t) * X(t, c);
      X(i, c) = acc / G(i, i);
    }
  }
  MA = SqMat(k);
  MB = SqMat(k);
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) {
      MA(i, j) = g2[i] * X(i, j);
      MB(i, j) = (i == j ? cd(1.0) : cd(0.0)) - g1[i] * X(i, j);
    }
}

SqMat tri_eigvecs(const SqMat& RA, const SqMat& RB) {
  const int k = RA.n;
  SqMat Zv(k);
  const double nA = fro(RA), nB = fro(RB);
  for (int j = 0; j < k; ++j) {
    const cd a = RA(j, j), b = RB(j, j);
    const double small =
        kEps * std::max(std::abs(b) * nA + std::abs(a) * nB, std::numeric_limits<double>::min());
    Zv(j, j) = 1.0;
    for (int i = j - 1; i >= 0; --i) {
      cd rhs = 0.0;
      for (int t = i + 1; t <= j; ++t) rhs -= (b * RA(i, t) - a * RB(i, t)) * Zv(t, j);
      cd piv = b * RA(i, i) - a * RB(i, i);
      if (std::abs(piv) < small) piv = small;
      Zv(i, j) = rhs / piv;
    }
  }
  return Zv;
}

void least_squares(std::vector<cd>& H, int M, int N, std::vector<cd>& E, int r, std::vector<cd>& Y) {
  std::vector<cd> v(M);
  for (int j = 0; j < N; ++j) {
    // Householder reflector I - 2 v v^* mapping H(j:, j) to a multiple of e_1
    double nx = 0.0;
    for (int i = j; i < M; ++i) nx += std::norm(H[(size_t)i * N + j]);
    nx = std::sqrt(nx);
    if (nx == 0.0) continue;
    const cd x0 = H[(size_t)j * N + j];
    const cd ph = std::abs(x0) > 0.0 ? x0 / std::abs(x0) : cd(1.0, 0.0);
    const cd alpha = -ph * nx;
    double nv = 0.0;
    for (int i = j; i < M; ++i) {
      v[i] = H[(size_t)i * N + j] - (i == j ? alpha : cd(0.0, 0.0));
      nv += std::norm(v[i]);
    }
    nv = std::sqrt(nv);
    if (nv == 0.0) continue;
    for (int i = j; i < M; ++i) v[i] /= nv;
    for (int c = j; c < N; ++c) {
      cd d = 0.0;
      for (int i = j; i < M; ++i) d += std::conj(v[i]) * H[(size_t)i * N + c];
      for (int i = j; i < M; ++i) H[(size_t)i * N + c] -= 2.0 * v[i] * d;
    }
    for (int c = 0; c < r; ++c) {
      cd d = 0.0;
      for (int i = j; i < M; ++i) d += std::conj(v[i]) * E[(size_t)i * r + c];
      for (int i = j; i < M; ++i) E[(size_t)i * r + c] -= 2.0 * v[i] * d;
    }
  }
  double dmax = 0.0;
  for (int j = 0; j < N; ++j) dmax = std::max(dmax, std::abs(H[(size_t)j * N + j]));
  Y.assign((size_t)N * r, cd(0.0, 0.0));
  for (int j = N - 1; j >= 0; --j) {
    const cd d = H[(size_t)j * N + j];
    if (!(std::abs(d) > 1e-14 * dmax)) continue;
    for (int c = 0; c < r; ++c) {
      cd acc = E[(size_t)j * r + c];
      for (int t = j + 1; t < N; ++t) acc -= H[(size_t)j * N + t] * Y[(size_t)t * r + c];
      Y[(size_t)j * r + c] = acc / d;
    }
  }
}

}  // namespace gplhr
