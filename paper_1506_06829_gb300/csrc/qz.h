// Small dense complex algebra on the host for the GPLHR driver.
#pragma once
#include <complex>
#include <vector>

namespace gplhr {

using cd = std::complex<double>;

// Row-major square matrix view.
struct SqMat {
  int n = 0;
  std::vector<cd> a;
  SqMat() = default;
  explicit SqMat(int n_) : n(n_), a((size_t)n_ * n_, cd(0.0, 0.0)) {}
  cd& operator()(int i, int j) { return a[(size_t)i * n + j]; }
  const cd& operator()(int i, int j) const { return a[(size_t)i * n + j]; }
  static SqMat eye(int n_) {
    SqMat m(n_);
    for (int i = 0; i < n_; ++i) m(i, i) = 1.0;
    return m;
  }
};

// Ordered complex QZ (footnote to Alg. 2 step 2): Phi = YL RA YR^*, Psi = YL RB YR^*,
// |RA(j,j)/RB(j,j) - sigma| non-decreasing over the leading nsort positions (< 0: all),
// which hold the nsort pairs nearest sigma; RB(j,j) real >= 0.  Only the leading nyl
// columns of YL and nyr of YR are formed (< 0: all); the others are returned zero.
// Returns false if the QZ iteration did not converge.
bool ordered_qz(const SqMat& Phi, const SqMat& Psi, cd sigma, SqMat& RA, SqMat& RB, SqMat& YL,
                SqMat& YR, int nsort = -1, int nyl = -1, int nyr = -1);

// Theorem 1 with Eqs. G1_fix/G2_fix: MA = G2 G^{-1} RA, MB = I - G1 G^{-1} RA.
void m_factors(const SqMat& RA, const SqMat& RB, SqMat& MA, SqMat& MB);

// Columns z_j of the upper triangular pencil's eigenvectors: (b_j RA - a_j RB) z_j = 0,
// z_j(j) = 1, z_j(i > j) = 0 (safeguarded back substitution).
SqMat tri_eigvecs(const SqMat& RA, const SqMat& RB);

// Distance of the pair (alpha, beta) to sigma: |alpha - sigma beta| / |beta| (inf if beta = 0).
double pair_distance(cd alpha, cd beta, cd sigma);

// Least squares min ||E - H Y||_F for a dense row-major H (M x N, M >= N) and E (M x r),
// by Householder QR; Y (N x r, row-major).  A column whose R diagonal is at most
// 1e-14 times the largest is dropped (its row of Y is zero).  H and E are overwritten.
void least_squares(std::vector<cd>& H, int M, int N, std::vector<cd>& E, int r, std::vector<cd>& Y);

}  // namespace gplhr
