// Dense FP64 linear algebra for the host-side plan builder.
//
// Real nonsymmetric eigendecomposition (Householder reduction to Hessenberg
// form, Francis double-shift QR to real Schur form, back-substitution for the
// eigenvectors) and LU inversion.  Used once per plan on matrices of size
// Nr x Nr; never on the per-step path.
#pragma once
#include <vector>

namespace fdetd {

// Row-major square matrix helper.
struct Mat {
  int n = 0, m = 0;  // rows, cols
  std::vector<double> a;
  Mat() {}
  Mat(int rows, int cols) : n(rows), m(cols), a((size_t)rows * cols, 0.0) {}
  double& operator()(int i, int j) { return a[(size_t)i * m + j]; }
  double operator()(int i, int j) const { return a[(size_t)i * m + j]; }
};

Mat matmul(const Mat& A, const Mat& B);

// Eigen-decomposition of a real matrix whose eigenvalues are expected to be real.
// On success returns 0, eigenvalues in w (ascending), eigenvectors as the columns
// of V (unit 2-norm, largest-magnitude component positive).  Returns nonzero if
// the QR iteration fails to converge or a complex pair with
// |Im| > imag_tol * max|lambda| appears.
int eig_real(const Mat& A, std::vector<double>& w, Mat& V, double imag_tol, double* max_imag);

// Inverse by LU with partial pivoting.  Returns nonzero if singular.
int invert(const Mat& A, Mat& Ainv);

// Solve A x = b (LU with partial pivoting), A square.  Returns nonzero if singular.
int solve(const Mat& A, std::vector<double>& x, const std::vector<double>& b);

}  // namespace fdetd
